"""Benchmark: halo-finding particles/s on one GB300 (3D FoF -> 6D hierarchy -> unbinding ->
halo properties), on a seeded synthetic NFW snapshot.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one pass of the whole path over one snapshot with inputs resident in HBM. Prints one
JSON line (rank 0). For N > 1 (torchrun, one rank per GPU) every rank processes its own
independent snapshot (seed + rank): weak scaling, no data-path collective; the value is all
ranks' particles over the slowest rank's time.

--impl reference times the CPU oracle (the plain definition the CUDA path is checked against)
on a bounded sample of the same workload, on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "halo-finding particles/s on 1 GB300, plain vs batched+surrogate; % of roofline"
UNIT = "particles/s"
DEFAULT_WORKLOAD = "nfw-2^24-L256-sub"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
# fraction of the box side of the cubic sub-volume the CPU oracle is timed on
ORACLE_SUBBOX = 0.5


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(elapsed_s: float, units: float, world_size: int, backend_device="cpu"):
    """Max elapsed and summed units over ranks (identity when world_size == 1)."""
    if world_size <= 1:
        return elapsed_s, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=backend_device)
    u = torch.tensor([units], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def _barrier(world_size):
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        self.path = None
        self.device_index = device_index

    def __enter__(self):
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.device_index).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = []
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # wait for the first sample, so nvidia-smi's start-up (driver queries) is over before
        # the timed region begins and only its steady 200 ms polling overlaps it
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 10.0:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)
        time.sleep(0.25)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
def synth_seed_for_rank(workload, rank):
    """Seed of the independent snapshot rank `rank` processes (weak scaling, no exchange)."""
    from paper_2412_18629_gb300 import synth
    return synth.WORKLOADS[workload].seed + 1000 * rank


def _snapshot(workload, rank):
    import dataclasses

    from paper_2412_18629_gb300 import synth
    spec = dataclasses.replace(synth.WORKLOADS[workload], seed=synth_seed_for_rank(workload, rank))
    return spec, synth.generate(spec)


def _oracle_sample(snap):
    """Bounded sample of the workload for the CPU oracle: the particles in the cubic sub-volume
    [0, f L)^3 of the same snapshot (its halos are cut at the sub-volume's faces)."""
    from paper_2412_18629_gb300 import synth
    keep = np.all(snap["pos"] < np.float32(ORACLE_SUBBOX * snap["box"]), axis=1)
    return synth.subsample(snap, keep)


def time_oracle(snap, threads):
    import oracle
    from paper_2412_18629_gb300 import G_NEWTON
    sub = _oracle_sample(snap)
    t0 = time.perf_counter()
    lab = oracle.fof3d_grid(sub["pos"], sub["ids"], sub["box"], sub["link_length"])
    h = oracle.hierarchy(sub["pos"], sub["vel"], sub["ids"], lab, sub["box"], threads=threads)
    ub = oracle.unbind(h["member_off"], h["member_idx"], sub["pos"], sub["vel"], sub["box"],
                       sub["softening"], G_NEWTON, sub["particle_mass"], threads=threads,
                       want_phi=False)
    oracle.props(h["member_off"], h["member_idx"], sub["pos"], sub["vel"], ub["bound"],
                 ub["is_halo"], sub["box"], sub["particle_mass"], len(snap["ids"]), threads=threads)
    dt = time.perf_counter() - t0
    return sub["n"], dt


def _hier_work(ctx):
    """Algorithmic pair counts of the hierarchy: sum over nodes of g (g - 1); also the part of
    the nodes above 384 members (the blocked potential kernel's share)."""
    import paper_2412_18629_gb300 as rs
    sizes = rs.rs_fof6d_copy(ctx)["size"].cpu().numpy().astype(np.float64)
    big = sizes[sizes > 384]
    return float((sizes * (sizes - 1)).sum()), float((big * (big - 1)).sum())


# FP32-pipe operations per pair for the two O(n_g^2) kernels (no FMA contraction):
# 6D distance = 6 sub + 6 mul + 4 add + 2 mul (scales) + 1 add, plus the min / compare = 20;
# potential = 3 sub + 3 FMA + 1 add (+ 1 MUFU rsqrt) = 7.
OPS_PER_PAIR = {"k_nn6d": 20.0, "k_link6d": 20.0, "k_potential": 7.0}


def _measure(ctx, pos, vel, ids, n, args, ws, local):
    """Warm up, then time exactly args.steps steps of the whole path on device-resident inputs."""
    import torch
    import paper_2412_18629_gb300 as rs
    stream = torch.cuda.current_stream()

    def step():
        lab, _ = rs.rs_fof3d(ctx, pos, ids)
        rs.rs_fof6d(ctx, pos, vel, ids, lab)
        _, bound, nfb = rs.rs_unbind(ctx, pos, vel, want_potential=False)
        props = rs.rs_halo_props(ctx)
        return nfb

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    pairs, pairs_big = _hier_work(ctx)
    ctx.profile(True)
    l0 = ctx.kernel_launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        _barrier(ws)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            nfb = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        _barrier(ws)
    launches = ctx.kernel_launches - l0
    elapsed = ev0.elapsed_time(ev1) / 1e3
    prof = ctx.profile_totals()
    ctx.profile(False)
    work = None
    if ctx.mode != "plain":  # one untimed step through the counting variants of the 6D kernels
        ctx.count_work(True)
        step()
        work = ctx.count_work(False)
    t_max, units = aggregate(elapsed, float(n) * args.steps, ws, f"cuda:{local}")
    return {"value": units / t_max, "ms_per_step": t_max / args.steps * 1e3, "launches": launches,
            "prof": prof, "pairs": pairs, "pairs_big": pairs_big, "clocks": clk.summary(),
            "fallback": nfb, "work": work, "n": n, "autotune": ctx.tuning()}


def _roofline(prof, pairs, steps, work=None):
    """Roofline entry of the dominant instrumented kernel (largest summed CUDA-event time).
    Brute-force pair kernels: algorithmic operations = pairs x operations per pair. Pruned 6D
    kernels: the d6 evaluations and box lower bounds they perform (tallied in one untimed step
    by the counting variants), 20 FP32 operations each."""
    if not prof:
        return None
    name, (ms, cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    peak_ops = SM_COUNT * FP32_LANES_PER_SM * 2070e6
    base = name.replace("_pruned", "").replace("_blocked", "")
    entry = {"bound": "alu", "kernel": name, "achieved": None, "peak": peak_ops / 1e12,
             "unit": "Tops/s", "frac": None, "traffic": None, "launches": cnt,
             "kernel_ms_per_step": ms / steps,
             "peak_note": "FP32-pipe lane operations at 2070 MHz (152 SMs x 128 lanes)"}
    work_ops = None
    if name.endswith("_pruned") and work:
        key = "nn" if base == "k_nn6d" else "link"
        work_ops = (work[f"{key}_d6"] + work[f"{key}_box"]) * OPS_PER_PAIR["k_nn6d"] * steps
        entry["work"] = {"d6_per_step": work[f"{key}_d6"], "box_tests_per_step": work[f"{key}_box"],
                         "ops_each": OPS_PER_PAIR["k_nn6d"]}
    elif base in OPS_PER_PAIR and not name.endswith("_pruned"):
        pr = pairs if base != "k_link6d" else pairs / 2.0
        work_ops = pr * OPS_PER_PAIR[base] * steps
    if work_ops is not None:
        achieved = work_ops / (ms / 1e3)
        entry.update(achieved=achieved / 1e12, frac=achieved / peak_ops)
    return entry


def _measured_peaks():
    """The machine's measured peaks (HBM copy GB/s, bf16 TFLOP/s), if the file is present."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _stages(r, steps):
    """Per-stage roofline figures of the kernels with a defined algorithmic work: the 3D FoF
    link pass against the measured HBM copy bandwidth (28 B per particle: position, id,
    label), the pair kernels against the FP32-pipe lane rate (brute force: pairs x operations;
    pruned: tallied d6 evaluations and box tests; blocked potential: pairs of the nodes above
    384 members x 7 operations)."""
    prof, out = r["prof"], {}
    peak_ops = SM_COUNT * FP32_LANES_PER_SM * 2070e6
    hbm = _measured_peaks().get("hbm_gbs")

    def ms(k):
        return prof[k][0] / steps / 1e3 if k in prof and prof[k][0] > 0 else None

    if ms("k_fof_link") and hbm:
        gbs = r["n"] * 28.0 / ms("k_fof_link") / 1e9
        out["k_fof_link"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                             "frac": gbs / hbm, "note": "latency-bound union-find; HBM is not its limit"}
    alu = {}
    if ms("k_potential_blocked") and r.get("form") != "surrogate":
        alu["k_potential_blocked"] = r["pairs_big"] * OPS_PER_PAIR["k_potential"]
    for k in ("k_nn6d", "k_link6d"):
        if ms(k):
            alu[k] = r["pairs"] * OPS_PER_PAIR[k] / (2.0 if k == "k_link6d" else 1.0)
    w = r.get("work")
    if w:
        for k, key in (("k_nn6d_pruned", "nn"), ("k_link6d_pruned", "link")):
            if ms(k):
                alu[k] = (w[f"{key}_d6"] + w[f"{key}_box"]) * OPS_PER_PAIR["k_nn6d"]
    for k, ops in alu.items():
        a = ops / ms(k)
        out[k] = {"bound": "alu", "achieved": a / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                  "frac": a / peak_ops, "ms_per_step": ms(k) * 1e3}
    return out


TRAIN_SAMPLES = 1_000_000
TRAIN_EPOCHS = 300


def train_surrogate(ctx, workload, device, samples=None, epochs=None):
    """Train the context's surrogate on the GPU, outside any timed region: exact potentials of
    a snapshot drawn with the same generator and a disjoint seed (100), 10% held out."""
    import dataclasses

    import torch
    import paper_2412_18629_gb300 as rs
    from paper_2412_18629_gb300 import synth
    spec = dataclasses.replace(synth.WORKLOADS[workload], seed=100)
    s = synth.generate(spec)
    tctx = rs.Context(box=s["box"], link_len=s["link_length"], softening=s["softening"],
                      particle_mass=s["particle_mass"], device=device, mode="batched")
    p, v, i = (torch.from_numpy(s[k]).cuda() for k in ("pos", "vel", "ids"))
    lab, _ = rs.rs_fof3d(tctx, p, i)
    rs.rs_fof6d(tctx, p, v, i, lab)
    rs.rs_unbind(tctx, p, v, want_potential=False)
    x, t = rs.rs_surrogate_features(tctx)
    k = min(x.shape[0], samples or TRAIN_SAMPLES)
    sel = torch.randperm(x.shape[0], generator=torch.Generator().manual_seed(100))[:k].cuda()
    x, t = x[sel].contiguous(), t[sel].contiguous()
    t0 = time.perf_counter()
    rs.rs_mlp_set_params(tctx, np.zeros(rs.MLP_PARAMS, np.float32))
    epochs = epochs or TRAIN_EPOCHS
    err_max, mse = rs.rs_mlp_train(tctx, x, t, epochs=epochs, batch=4096, lr=1e-3, seed=100)
    dt = time.perf_counter() - t0
    rs.rs_mlp_set_params(ctx, rs.rs_mlp_get_params(tctx))
    rs.rs_mlp_set_err_max(ctx, err_max)
    tctx.close()
    return {"samples": int(k), "epochs": epochs, "err_max_psi": err_max, "last_batch_mse": mse,
            "train_s": dt,
            "snapshot": f"{workload} generator, seed 100"}


def run_ours(args):
    import torch
    import paper_2412_18629_gb300 as rs
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    spec, snap = _snapshot(args.workload, rank)
    pos = torch.from_numpy(snap["pos"]).cuda()
    vel = torch.from_numpy(snap["vel"]).cuda()
    ids = torch.from_numpy(snap["ids"]).cuda()
    n = len(snap["ids"])
    forms = ("plain", "batched", "surrogate") if args.form == "all" else (args.form,)
    res, ctxs, training = {}, {}, None
    for form in forms:
        ctxs[form] = rs.Context(box=snap["box"], link_len=snap["link_length"],
                                softening=snap["softening"], particle_mass=snap["particle_mass"],
                                device=local, mode=form)
        if form == "surrogate":
            training = train_surrogate(ctxs[form], args.workload, local, args.train_samples,
                                       args.train_epochs)
        res[form] = _measure(ctxs[form], pos, vel, ids, n, args, ws, local)
        if form == "surrogate":
            res[form]["surrogate_stats"] = rs.rs_surrogate_stats(ctxs[form])
    # headline: the fastest form (all forms give identical outputs)
    head = max(res, key=lambda f: res[f]["value"])
    ctx, r = ctxs[head], res[head]
    for f in list(ctxs):  # the other forms' device buffers are released before the e2e timing
        if f != head:
            ctxs.pop(f).close()
    torch.cuda.empty_cache()
    # ---- end to end through the public API with host buffers (headline form)
    pin = {k: torch.from_numpy(snap[k]).pin_memory() for k in ("pos", "vel", "ids")}
    h2d = sum(t.numel() * t.element_size() for t in pin.values())
    e_pos, e_vel, e_ids = (torch.empty_like(pos), torch.empty_like(vel), torch.empty_like(ids))
    out_lab = torch.empty(n, dtype=torch.int64).pin_memory()
    out_bound = torch.empty(ctx.n_members, dtype=torch.uint8).pin_memory()
    out_props = torch.empty((ctx.n_nodes, 8 * rs.PROPS_FIELDS), dtype=torch.uint8).pin_memory()
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()

    def e2e_step():
        # pos and ids feed the 3D FoF; vel (needed from the 6D split on) is copied on a side
        # stream meanwhile, and the labels go back on it while the 6D hierarchy is built
        e_pos.copy_(pin["pos"], non_blocking=True)
        e_ids.copy_(pin["ids"], non_blocking=True)
        side.wait_stream(main)
        with torch.cuda.stream(side):
            e_vel.copy_(pin["vel"], non_blocking=True)
            vel_ready = side.record_event()
        lab, _ = rs.rs_fof3d(ctx, e_pos, e_ids)
        side.wait_stream(main)
        with torch.cuda.stream(side):
            out_lab.copy_(lab, non_blocking=True)
            lab.record_stream(side)
        main.wait_event(vel_ready)
        rs.rs_fof6d(ctx, e_pos, e_vel, e_ids, lab)
        _, bound, _ = rs.rs_unbind(ctx, e_pos, e_vel, want_potential=False)
        props = rs.rs_halo_props(ctx)
        b_h = out_bound[:bound.numel()]
        p_h = out_props[:props.shape[0]]
        b_h.copy_(bound, non_blocking=True)
        p_h.copy_(props, non_blocking=True)
        torch.cuda.synchronize()
        return b_h.numel() + p_h.numel() + out_lab.numel() * 8

    e2e_step()
    torch.cuda.synchronize()
    _barrier(ws)
    e0 = time.perf_counter()
    d2h = 0
    for _ in range(args.steps):
        d2h = e2e_step()
    torch.cuda.synchronize()
    e_el = time.perf_counter() - e0
    e_max, e_units = aggregate(e_el, float(n) * args.steps, ws, f"cuda:{local}")
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        ns, dt = time_oracle(snap, threads)
        cpu = {"value": ns / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"particles in the sub-volume [0, {ORACLE_SUBBOX} L)^3 of the same "
                         f"snapshot ({ns} particles, {dt:.1f} s): FoF, hierarchy, unbinding, props"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "box": snap["box"], "seed": spec.seed,
                       "form": head, "nodes": int(ctx.n_nodes), "members": int(ctx.n_members),
                       "pairs": r["pairs"], "l2": "inputs and hierarchy larger than L2 (no flush)",
                       "parallelism": f"independent snapshots x{ws}"},
            "roofline": _roofline(r["prof"], r["pairs"], args.steps, r["work"]), "cpu_baseline": cpu,
            "e2e": {"value": e_units / e_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": r["launches"], "clocks": r["clocks"], "surrogate_training": training,
            "forms": {f: {"value": v["value"], "ms_per_step": v["ms_per_step"],
                          "gpu_launches": v["launches"], "fallback_members": v["fallback"],
                          "kernels_ms_per_step": {k: t[0] / args.steps for k, t in v["prof"].items()},
                          "roofline": _roofline(v["prof"], v["pairs"], args.steps, v["work"]),
                          "stages": _stages(dict(v, form=f), args.steps),
                          "clocks": v["clocks"],
                          "autotune": v.get("autotune"),
                          "surrogate_stats": v.get("surrogate_stats")}
                      for f, v in res.items()},
        }
        print(json.dumps(line), flush=True)
    for c in ctxs.values():
        c.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    spec, snap = _snapshot(args.workload, 0)
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        time_oracle(snap, threads)
    tot_n, tot_t = 0, 0.0
    for _ in range(args.steps):
        ns, dt = time_oracle(snap, threads)
        tot_n += ns
        tot_t += dt
    value = tot_n / tot_t
    sample = (f"particles in the sub-volume [0, {ORACLE_SUBBOX} L)^3 of the same snapshot "
              f"({tot_n // max(args.steps, 1)} per step)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "form": "oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", choices=("plain", "batched", "surrogate", "all"), default="all")
    ap.add_argument("--train-samples", type=int, default=1_000_000)
    ap.add_argument("--train-epochs", type=int, default=TRAIN_EPOCHS)
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Benchmark: halo-finding particles/s on one GB300 (3D FoF -> 6D hierarchy -> unbinding ->
halo properties), on a seeded synthetic NFW snapshot (default: 2^27 particles in a 512 Mpc/h
box, halos up to 2e6 particles with three levels of subhalos).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one pass of the whole path over one snapshot with inputs resident in HBM. The
headline is the batched + surrogate form timed over exactly K steps after W warm-up steps; the
plain and batched forms are timed beside it with their own (stated) step counts, and every
form's outputs are checked identical. Prints one JSON line (rank 0). For N > 1 (torchrun, one
rank per GPU) every rank processes its own independent snapshot (seed + 1000 rank): weak
scaling, no data-path collective; the value is all ranks' particles over the slowest rank's
time.

--impl reference times the CPU oracle (the plain definition the CUDA path is checked against)
on a bounded sample of the same workload, on this machine's host cores.
"""
from __future__ import annotations

import argparse
import hashlib
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
DEFAULT_WORKLOAD = "nfw-2^27-L512-sub3"
SM_COUNT = 152
FP32_LANES_PER_SM = 128


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


ORACLE_CUBES = 8    # the sample cubes' side is L / ORACLE_CUBES
ORACLE_SAMPLE = 5   # cubes the CPU baseline times (the median-load cube and its neighbours in load)


def _oracle_cubes(snap, count=ORACLE_SAMPLE):
    """Indices (ix, iy, iz) of the sample cubes: of the ORACLE_CUBES^3 cubes of side
    L / ORACLE_CUBES, ranked by the sum of squared particle counts of the catalogued top-level
    halos centred in them (the oracle's cost is dominated by sum n^2), the `count` cubes around
    the median (ties: lowest index first)."""
    L = float(snap["box"])
    k = ORACLE_CUBES
    w = np.zeros(k ** 3)
    for depth, cnt, _, centre, _, _ in snap["catalogue"]:
        if depth != 0:
            continue
        c = np.floor(np.mod(np.asarray(centre, dtype=np.float64), L) / (L / k)).astype(int) % k
        w[(c[0] * k + c[1]) * k + c[2]] += float(cnt) ** 2
    order = np.argsort(w, kind="stable")
    mid = len(order) // 2
    pick = order[max(0, mid - count // 2): max(0, mid - count // 2) + count]
    return [(int(i) // (k * k), (int(i) // k) % k, int(i) % k) for i in pick]


def _oracle_sample(snap, cube):
    """The particles of cube `cube` (side L / ORACLE_CUBES) of the same snapshot: a bounded
    sample of the workload for the CPU oracle (its halos are cut at the cube's faces)."""
    from paper_2412_18629_gb300 import synth
    side = float(snap["box"]) / ORACLE_CUBES
    lo = np.array(cube, dtype=np.float64) * side
    p = snap["pos"].astype(np.float64)
    keep = np.all((p >= lo) & (p < lo + side), axis=1)
    return synth.subsample(snap, keep)


def time_oracle(snap, threads, cube):
    """Run the oracle over one sample cube: 3D FoF, hierarchy, unbinding, properties. Returns
    (particles, seconds)."""
    import oracle
    from paper_2412_18629_gb300 import G_NEWTON
    sub = _oracle_sample(snap, cube)
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


# ---------------------------------------------------------------------------------------------
# Algorithmic work per kernel (the per-unit figures of the roofline) and the peaks.
FP32_PEAK_OPS = SM_COUNT * FP32_LANES_PER_SM * 2070e6   # FP32-pipe lane operations per second
FOF_BYTES_PER_PARTICLE = 28.0   # position 12 + id 8 + label 8
SORT_BYTES_PER_KEY_PASS = 24.0  # key 8 + value 4, read and written
NODE_BYTES_PER_MEMBER = 40.0    # 6D level: u 12 + v 12 + id 8 + label 8 per member and level
OPS_D6 = 20.0                   # 6D distance: 6 sub, 6 mul, 4 add, 2 scale mul, 1 add, 1 compare
OPS_PAIR = 7.0                  # potential pair: 3 sub, 3 FMA, 1 add (+ 1 MUFU rsqrt)
OPS_EXPANSION = 50.0            # tree walk: one quadrupole expansion with its bound and test
TREE_MIN_DEFAULT = 16384        # the library's default smallest node of the tree bound


def _measured_peaks():
    """The machine's measured peaks (HBM copy GB/s, bf16 TFLOP/s), if the file is present."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


HBM_FALLBACK_GBS = 6800.0


def _hbm_peak():
    p = _measured_peaks().get("hbm_gbs")
    return (float(p), "measured") if p else (HBM_FALLBACK_GBS, "fallback")


def _sizes_work(sizes, form, tree_min):
    """Pair counts of the direct-sum kernels from the node sizes: k_potential (nodes up to 384
    members) and the blocked / tiled kernel (larger nodes handled by the direct sum in this
    form: below the surrogate's 1024 members or the tree's threshold); brute-force 6D pairs."""
    g = np.asarray(sizes, dtype=np.float64)
    pairs = g * (g - 1.0)
    small = pairs[g <= 384].sum()
    if form == "plain":
        lim = np.inf
    elif form == "surrogate":
        lim = 1024.0
    else:
        lim = float(tree_min) if tree_min > 0 else np.inf
    big = pairs[(g > 384) & (g < lim)].sum()
    return {"pairs_all": float(pairs.sum()), "pairs_small": float(small), "pairs_blocked": float(big)}


def kernel_work(r):
    """{kernel: (bound, algorithmic units per step, unit, note)} for the kernels with a defined
    work figure, from the form's measured tallies r: n, members, sort key-passes per step,
    pair counts from node sizes, the pruned kernels' d6 tallies and the tree's counters.
    Bytes for HBM-bound kernels, FP32-pipe operations for ALU-bound ones."""
    out = {}
    out["k_fof_link"] = ("hbm", r["n"] * FOF_BYTES_PER_PARTICLE, "B", "28 B per particle")
    if r.get("sort_keypasses"):
        out["k_sort"] = ("hbm", r["sort_keypasses"] * SORT_BYTES_PER_KEY_PASS, "B",
                         "24 B per key and 8-bit pass (k_sort_hist + k_sort_scatter)")
    # the batched forms run the brute-force pair kernels only on small levels (a few thousand
    # members), which the per-member figure does not separate: they get no stage entry there
    six = ("k_nn6d", "k_link6d") if r.get("form") == "plain" else ("k_nn6d_pruned", "k_link6d_pruned")
    for k in six:
        out[k] = ("hbm", r["members"] * NODE_BYTES_PER_MEMBER, "B", "40 B per member and level")
    w = r.get("pairs", {})
    out["k_potential"] = ("alu", w.get("pairs_small", 0.0) * OPS_PAIR, "ops", "7 per ordered pair")
    for k in ("k_potential_blocked", "k_potential_tiled"):
        out[k] = ("alu", w.get("pairs_blocked", 0.0) * OPS_PAIR, "ops", "7 per ordered pair")
    t = r.get("tree") or {}
    if t.get("list_pairs"):
        out["k_potential_list"] = ("alu", t["list_pairs"] * OPS_PAIR, "ops", "7 per listed pair")
    if t.get("expansions") or t.get("direct_pairs"):
        out["k_tree_walk"] = ("alu", t["expansions"] * OPS_EXPANSION + t["direct_pairs"] * OPS_PAIR,
                              "ops", "50 per expansion + 7 per direct pair")
    return out


def _alu_d6(r, k):
    """FP32-pipe figure of a 6D kernel counting d6 evaluations only (box bounds as overhead)."""
    wk = r.get("work")
    if k.endswith("_pruned"):
        if not wk:
            return None
        d6 = wk["nn_d6" if k.startswith("k_nn6d") else "link_d6"]
    else:
        pa = r["pairs"]["pairs_all"]
        d6 = pa if k == "k_nn6d" else pa / 2.0
    return d6 * OPS_D6


def stages(r, traffic=None):
    """Per-kernel roofline figures of one form from its profiled step (CUDA events per launch):
    achieved = algorithmic work per step / kernel time per step, against the measured HBM copy
    bandwidth or the FP32-pipe lane rate; with the ncu DRAM traffic per launch where captured
    (and, for HBM-bound kernels, the algorithmic bytes per launch beside it)."""
    prof = dict(r["prof"])
    if "k_sort_hist" in prof or "k_sort_scatter" in prof:
        a, b = prof.get("k_sort_hist", (0.0, 0)), prof.get("k_sort_scatter", (0.0, 0))
        prof["k_sort"] = (a[0] + b[0], a[1] + b[1])
    hbm, hbm_src = _hbm_peak()
    out = {}
    for k, (bound, units, unit, note) in kernel_work(r).items():
        if k not in prof or prof[k][0] <= 0 or units <= 0:
            continue
        sec = prof[k][0] / 1e3
        e = {"bound": bound, "ms_per_step": prof[k][0], "launches": prof[k][1], "work_note": note}
        if bound == "hbm":
            e.update(achieved=units / sec / 1e9, peak=hbm, unit="GB/s", frac=units / sec / 1e9 / hbm,
                     peak_source=hbm_src)
        else:
            e.update(achieved=units / sec / 1e12, peak=FP32_PEAK_OPS / 1e12, unit="Tops/s",
                     frac=units / sec / FP32_PEAK_OPS, peak_source="FP32 lanes x 2070 MHz")
        if traffic and traffic.get(k):
            e["traffic"] = traffic[k]
            if bound == "hbm":
                e["algorithmic_bytes_per_launch"] = units / max(prof[k][1], 1)
        if k.startswith(("k_nn6d", "k_link6d")):
            ops = _alu_d6(r, k)
            if ops:
                e["alu_d6_only"] = {"achieved": ops / sec / 1e12, "peak": FP32_PEAK_OPS / 1e12,
                                    "unit": "Tops/s", "frac": ops / sec / FP32_PEAK_OPS}
        out[k] = e
    return out


def roofline(r, traffic=None):
    """The roofline entry of the dominant kernel (largest time in the profiled step among the
    kernels with a work figure); launches and average duration per launch."""
    st = stages(r, traffic)
    if not st:
        return None
    k = max(st, key=lambda x: st[x]["ms_per_step"])
    e = dict(st[k])
    e["kernel"] = k
    e["ms_per_launch"] = e["ms_per_step"] / max(e["launches"], 1)
    e["traffic"] = (traffic or {}).get(k)
    return e


def _traffic_table():
    """DRAM bytes (read + write) per launch of the profiled kernels, from one ncu capture of the
    bench command (profiles/dram_traffic.json, written from that capture; the summary beside it
    gives the command): {workload: {kernel: bytes per launch}}. A kernel changed since its
    capture has no entry."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return {}
    return {w: {k: v for k, v in e.items() if not k.startswith("_")} for w, e in t.items()}


# ---------------------------------------------------------------------------------------------
def _digest(ctx, lab, bound, props):
    """SHA-256 of a form's outputs: 3D labels, hierarchy arrays, bound flags, properties."""
    import paper_2412_18629_gb300 as rs
    hsh = hashlib.sha256()
    hsh.update(lab.cpu().numpy().tobytes())
    for k, v in sorted(rs.rs_fof6d_copy(ctx).items()):
        hsh.update(k.encode())
        hsh.update(v.cpu().numpy().tobytes())
    hsh.update(bound.cpu().numpy().tobytes())
    hsh.update(props.cpu().numpy().tobytes())
    return hsh.hexdigest()


def _measure(ctx, pos, vel, ids, n, steps, warmup, ws, local, form):
    """W warm-up steps, then exactly `steps` steps timed with CUDA events on the launching
    stream between barriers (no per-kernel instrumentation), clocks sampled meanwhile; then one
    untimed profiled step (CUDA events around each dominant kernel) and, for the batched forms,
    one untimed step through the counting variants of the pruned 6D kernels."""
    import torch
    import paper_2412_18629_gb300 as rs
    stream = torch.cuda.current_stream()
    last = {}

    def step():
        lab, _ = rs.rs_fof3d(ctx, pos, ids)
        rs.rs_fof6d(ctx, pos, vel, ids, lab)
        _, bound, nfb = rs.rs_unbind(ctx, pos, vel, want_potential=False)
        props = rs.rs_halo_props(ctx)
        last.update(lab=lab, bound=bound, props=props, nfb=nfb)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    l0 = ctx.kernel_launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        _barrier(ws)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        _barrier(ws)
    launches = ctx.kernel_launches - l0
    elapsed = ev0.elapsed_time(ev1) / 1e3
    digest = _digest(ctx, last["lab"], last["bound"], last["props"])
    tree = rs.rs_tree_stats(ctx)
    sur = rs.rs_surrogate_stats(ctx) if form.startswith("surrogate") else None
    bound_host = last["bound"].cpu().numpy()
    sizes = rs.rs_fof6d_copy(ctx)["size"].cpu().numpy()
    # one profiled step (kernel shares), untimed
    k0 = ctx.sort_keypasses
    ctx.profile(True)
    step()
    torch.cuda.synchronize()
    prof = ctx.profile_totals()
    ctx.profile(False)
    keypasses = ctx.sort_keypasses - k0
    pot_pairs = rs.rs_potential_pairs(ctx)
    work = None
    if form != "plain":
        ctx.count_work(True)
        step()
        work = ctx.count_work(False)
    t_max, units = aggregate(elapsed, float(n) * steps, ws, f"cuda:{local}")
    r = {"form": form, "value": units / t_max, "ms_per_step": t_max / steps * 1e3, "steps": steps,
         "warmup": warmup, "launches": launches, "launches_per_step": launches / max(steps, 1),
         "prof": prof, "clocks": clk.summary(), "fallback": last["nfb"], "work": work, "n": n,
         "members": int(ctx.n_members), "nodes": int(ctx.n_nodes), "digest": digest,
         "tree": tree, "surrogate_stats": sur, "sort_keypasses": keypasses,
         "autotune": ctx.tuning(), "bound_host": bound_host}
    tm = int(ctx.cfg.tree_min_members)
    r["pairs"] = _sizes_work(sizes, "surrogate" if form.startswith("surrogate") else form,
                             0 if form == "plain" or tm < 0 else (tm or TREE_MIN_DEFAULT))
    # the direct sums' own pair tallies (they include the nodes the surrogate sends whole to
    # the exact sum, which node sizes alone do not show)
    r["pairs"]["pairs_small"], r["pairs"]["pairs_blocked"] = map(float, pot_pairs)
    return r


TRAIN_SAMPLES = 1_000_000
TRAIN_EPOCHS = 300
TRAIN_WORKLOAD = "nfw-2^24-L256-sub"


def train_surrogate(ctx, workload, device, samples=None, epochs=None):
    """Train the context's surrogate on the GPU, outside any timed region: exact potentials of
    a snapshot drawn with the generator of `workload` and a disjoint seed (100), 10% held out."""
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
    rs.rs_unbind(tctx, p, v, want_potential=True)  # targets need every member's potential
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
    del p, v, i
    torch.cuda.empty_cache()
    return {"samples": int(k), "epochs": epochs, "err_max_psi": err_max, "last_batch_mse": mse,
            "train_s": dt, "snapshot": f"{workload} generator, seed 100"}


STREAM_BASE = "nfw-2^24-L256-sub"   # the batched stream: this snapshot plus STREAM_COUNT others
STREAM_COUNT = 64


def _gen_stream(k):
    """Snapshot k of the stream (k = -1: the base snapshot); runs in a spawned worker."""
    from paper_2412_18629_gb300 import synth
    spec = synth.WORKLOADS[STREAM_BASE] if k < 0 else synth.stream_spec(k)
    s = synth.generate(spec)
    return {key: s[key] for key in ("pos", "vel", "ids", "box", "link_length", "softening",
                                    "particle_mass")}


def _stream_snapshots(count):
    import multiprocessing as mp
    ks = [-1] + list(range(count))
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        return pool.map(_gen_stream, ks, chunksize=1)


def measure_stream(args, local):
    """The batched form over the stream of independent snapshots (the 2^24 snapshot plus 64 of
    2^18..2^22 particles at unit spacing): one context running the four calls snapshot after
    snapshot, against rs_run_batched's concurrent lanes; identical outputs required."""
    import torch
    import paper_2412_18629_gb300 as rs
    t0 = time.perf_counter()
    host = _stream_snapshots(args.stream_count)
    gen_s = time.perf_counter() - t0
    dev = [dict(pos=torch.from_numpy(h["pos"]).cuda(), vel=torch.from_numpy(h["vel"]).cuda(),
                ids=torch.from_numpy(h["ids"]).cuda(), box=h["box"], link_length=h["link_length"],
                softening=h["softening"]) for h in host]
    sizes = [h["pos"].shape[0] for h in host]
    n_tot = int(sum(sizes))
    mk = dict(softening=host[0]["softening"], particle_mass=host[0]["particle_mass"], device=local,
              mode="batched")
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps

    # sequential: the four calls snapshot after snapshot on one stream, one context per box
    # (the box is part of a context's configuration)
    by_box = {}
    for d in dev:
        key = (d["box"], d["link_length"])
        if key not in by_box:
            by_box[key] = rs.Context(box=d["box"], link_len=d["link_length"], **mk)
    seq_ctx = list(by_box.values())
    ctx_of = [by_box[(d["box"], d["link_length"])] for d in dev]
    seq_out = {}

    def sequential():
        for k, (c, d) in enumerate(zip(ctx_of, dev)):
            lab, _ = rs.rs_fof3d(c, d["pos"], d["ids"])
            rs.rs_fof6d(c, d["pos"], d["vel"], d["ids"], lab)
            rs.rs_unbind(c, d["pos"], d["vel"], want_potential=False)
            seq_out[k] = (lab, rs.rs_halo_props(c))

    l0 = sum(c.kernel_launches for c in seq_ctx)
    t_seq = timed(sequential, args.stream_steps, 1)
    seq_launches = (sum(c.kernel_launches for c in seq_ctx) - l0) / (args.stream_steps + 1)
    seq_digest = hashlib.sha256()
    for k in range(len(dev)):
        seq_digest.update(seq_out[k][0].cpu().numpy().tobytes())
        seq_digest.update(seq_out[k][1].cpu().numpy().tobytes())
    for c in seq_ctx:
        c.close()
    torch.cuda.empty_cache()
    bctx = rs.Context(box=dev[0]["box"], link_len=dev[0]["link_length"], **mk)
    cap = [max(n // 4, 16) for n in sizes]
    out = rs.BatchOutputs(sizes, cap, local, deepest=False)
    counts = rs.rs_run_batched(bctx, dev, out, lanes=args.stream_lanes)   # sizes the lanes
    l0 = bctx.kernel_launches
    t_bat = timed(lambda: rs.rs_run_batched(bctx, dev, out, lanes=args.stream_lanes),
                  args.stream_steps, 1)
    bat_launches = (bctx.kernel_launches - l0) / (args.stream_steps + 1)
    bat_digest = hashlib.sha256()
    for k in range(len(dev)):
        bat_digest.update(out.labels[k].cpu().numpy().tobytes())
        bat_digest.update(out.props[k][:counts[k][1]].cpu().numpy().tobytes())
    bctx.close()
    del dev, out
    torch.cuda.empty_cache()
    return {"workload": f"{STREAM_BASE} + {args.stream_count} snapshots of 2^18..2^22 "
                        "(n = 2^(18 + seed mod 5), unit spacing, seeds 0..)",
            "snapshots": len(sizes), "particles": n_tot, "form": "batched",
            "sequential": {"value": n_tot / t_seq, "ms_per_pass": t_seq * 1e3,
                           "launches_per_pass": seq_launches},
            "lanes": {"value": n_tot / t_bat, "ms_per_pass": t_bat * 1e3, "lanes": args.stream_lanes,
                      "launches_per_pass": bat_launches},
            "unit": UNIT, "steps": args.stream_steps, "warmup": 1,
            "identical_outputs": seq_digest.hexdigest() == bat_digest.hexdigest(),
            "nodes": int(counts[:, 1].sum()), "generation_s": gen_s}


def _form_entry(r, traffic):
    traffic = traffic if r["form"] == "surrogate" else None  # captured on the headline form
    return {"value": r["value"], "ms_per_step": r["ms_per_step"], "steps": r["steps"],
            "warmup": r["warmup"], "gpu_launches": r["launches"],
            "launches_per_step": r["launches_per_step"], "fallback_members": r["fallback"],
            "kernels_ms_profiled_step": {k: t[0] for k, t in r["prof"].items()},
            "roofline": roofline(r, traffic), "stages": stages(r, traffic), "clocks": r["clocks"],
            "autotune": r["autotune"], "tree_stats": r["tree"], "work_tallies": r["work"],
            "sort_keypasses_per_step": r["sort_keypasses"],
            "surrogate_stats": r["surrogate_stats"], "output_digest": r["digest"]}


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
    traffic = _traffic_table().get(args.workload, {})
    mk = dict(box=snap["box"], link_len=snap["link_length"], softening=snap["softening"],
              particle_mass=snap["particle_mass"], device=local)
    res, training = {}, None
    # headline: batched + surrogate at the requested step counts
    ctx = rs.Context(mode="surrogate", **mk)
    if args.weights:
        rs.rs_surrogate_load(ctx, args.weights)
        training = {"loaded": args.weights}
    else:
        training = train_surrogate(ctx, args.train_workload, local, args.train_samples,
                                   args.train_epochs)
        if args.save_weights and rank == 0:
            rs.rs_surrogate_save(ctx, args.save_weights)
    res["surrogate"] = _measure(ctx, pos, vel, ids, n, args.steps, args.warmup, ws, local, "surrogate")
    # the other forms, each with its own stated step counts: batched (exact flags), the
    # surrogate with the per-node calibrated gate (opt-in), plain
    others = [] if args.form == "surrogate" else [
        ("batched", args.batched_steps, args.batched_warmup),
        ("surrogate_calibrated", args.calibrated_steps, 1),
        ("plain", args.plain_steps, args.plain_warmup)]
    for form, k, w in others:
        if k <= 0:
            continue
        if form == "surrogate_calibrated":
            c = rs.Context(mode="surrogate", surrogate_gate=1, **mk)
            rs.rs_mlp_set_params(c, rs.rs_mlp_get_params(ctx))
            rs.rs_mlp_set_err_max(c, rs.rs_mlp_get_err_max(ctx))
        else:
            c = rs.Context(mode=form, **mk)
        res[form] = _measure(c, pos, vel, ids, n, k, w, ws, local, form)
        c.close()
        torch.cuda.empty_cache()
    r = res["surrogate"]
    # ---- end to end through the public API with host buffers (headline form): every step
    # copies its inputs from pinned host memory and reads its results back; the copy of the
    # next step's inputs runs on a copy stream while this step computes (two device input sets)
    pin = {k: torch.from_numpy(snap[k]).pin_memory() for k in ("pos", "vel", "ids")}
    h2d = sum(t.numel() * t.element_size() for t in pin.values())
    bufs = [tuple(torch.empty_like(t) for t in (pos, vel, ids)) for _ in range(2)]
    out_lab = torch.empty(n, dtype=torch.int64).pin_memory()
    out_bound = torch.empty(r["members"] + 1, dtype=torch.uint8).pin_memory()
    out_props = torch.empty((r["nodes"] + 1, 8 * rs.PROPS_FIELDS), dtype=torch.uint8).pin_memory()
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    copy_s = torch.cuda.Stream()
    ready, freed = [None, None], [None, None]

    def issue_copy(k):
        with torch.cuda.stream(copy_s):
            if freed[k % 2] is not None:  # the step that last read this input set is done
                copy_s.wait_event(freed[k % 2])
            for t, key in zip(bufs[k % 2], ("pos", "vel", "ids")):
                t.copy_(pin[key], non_blocking=True)
            ready[k % 2] = copy_s.record_event()

    def e2e_step(k, last):
        if not last:
            issue_copy(k + 1)
        e_pos, e_vel, e_ids = bufs[k % 2]
        main.wait_event(ready[k % 2])
        lab, _ = rs.rs_fof3d(ctx, e_pos, e_ids)
        side.wait_stream(main)
        with torch.cuda.stream(side):  # the labels go back while the hierarchy is built
            out_lab.copy_(lab, non_blocking=True)
            lab.record_stream(side)
        rs.rs_fof6d(ctx, e_pos, e_vel, e_ids, lab)
        _, bound, _ = rs.rs_unbind(ctx, e_pos, e_vel, want_potential=False)
        props = rs.rs_halo_props(ctx)
        freed[k % 2] = main.record_event()
        b_h = out_bound[:bound.numel()]
        p_h = out_props[:props.shape[0]]
        b_h.copy_(bound, non_blocking=True)
        p_h.copy_(props, non_blocking=True)
        torch.cuda.synchronize()
        return b_h.numel() + p_h.numel() + out_lab.numel() * 8

    issue_copy(0)
    e2e_step(0, True)
    torch.cuda.synchronize()
    e_steps = max(1, min(args.steps, int(args.e2e_seconds * 1e3 / max(r["ms_per_step"], 1e-3))))
    _barrier(ws)
    e0 = time.perf_counter()
    d2h = 0
    issue_copy(0)
    for k in range(e_steps):
        d2h = e2e_step(k, k == e_steps - 1)
    torch.cuda.synchronize()
    e_el = time.perf_counter() - e0
    e_max, e_units = aggregate(e_el, float(n) * e_steps, ws, f"cuda:{local}")
    ctx.close()
    del bufs
    torch.cuda.empty_cache()
    stream_res = measure_stream(args, local) if args.stream_steps > 0 else None
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        tot_n, tot_t = 0, 0.0
        cubes = _oracle_cubes(snap)
        for cube in cubes:
            ns, dt = time_oracle(snap, threads, cube)
            tot_n += ns
            tot_t += dt
        cpu = {"value": tot_n / tot_t, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{len(cubes)} cubes of side L/{ORACLE_CUBES} of the same snapshot "
                         f"(those around the median halo load sum n^2), {tot_n} particles, "
                         f"{tot_t:.1f} s: FoF, hierarchy, unbinding, props"}
    if rank == 0:
        ident = {f: v["digest"] == r["digest"] for f, v in res.items()}
        exact = res.get("batched")
        mism = ({f: int(np.count_nonzero(v["bound_host"] != exact["bound_host"]))
                 for f, v in res.items() if f.startswith("surrogate")} if exact else None)
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "box": snap["box"], "seed": spec.seed,
                       "form": "surrogate (batched + surrogate)", "nodes": r["nodes"],
                       "members": r["members"], "pairs": r["pairs"]["pairs_all"],
                       "l2": "inputs and hierarchy larger than L2 (no flush)",
                       "parallelism": f"independent snapshots x{ws}"},
            "roofline": roofline(r, traffic), "cpu_baseline": cpu,
            "e2e": {"value": e_units / e_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e_steps,
                    "copies": "pinned host buffers; the next step's inputs copied on a second "
                              "stream during this step's compute; results read back every step"},
            "gpu_launches": r["launches"], "clocks": r["clocks"],
            "plain_ms_per_step": res["plain"]["ms_per_step"] if "plain" in res else None,
            "plain_value": res["plain"]["value"] if "plain" in res else None,
            "batched_ms_per_step": res["batched"]["ms_per_step"] if "batched" in res else None,
            "identical_outputs": ident,
            "surrogate_flag_mismatches_vs_batched": mism,
            "surrogate_training": training,
            "stream": stream_res,
            "forms": {f: _form_entry(v, traffic) for f, v in res.items()},
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, one sample cube of the workload per step
    (cycling through the median-load cubes), on this machine's host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    spec, snap = _snapshot(args.workload, 0)
    threads = os.cpu_count() or 1
    cubes = _oracle_cubes(snap)
    for i in range(args.warmup):
        time_oracle(snap, threads, cubes[i % len(cubes)])
    tot_n, tot_t = 0, 0.0
    for i in range(args.steps):
        ns, dt = time_oracle(snap, threads, cubes[i % len(cubes)])
        tot_n += ns
        tot_t += dt
    value = tot_n / tot_t
    sample = (f"one cube of side L/{ORACLE_CUBES} of the same snapshot per step, cycling through "
              f"the {len(cubes)} cubes around the median halo load ({tot_n // max(args.steps, 1)} "
              f"particles per step on average)")
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
    ap.add_argument("--form", choices=("surrogate", "all"), default="all",
                    help="surrogate: time the headline form only")
    ap.add_argument("--batched-steps", type=int, default=2)
    ap.add_argument("--batched-warmup", type=int, default=1)
    ap.add_argument("--calibrated-steps", type=int, default=2)
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--plain-warmup", type=int, default=1)
    ap.add_argument("--e2e-seconds", type=float, default=30.0,
                    help="end-to-end timing: as many steps (at most --steps) as fit in this time")
    ap.add_argument("--stream-steps", type=int, default=2,
                    help="passes over the batched snapshot stream (0: skip it)")
    ap.add_argument("--stream-count", type=int, default=STREAM_COUNT)
    ap.add_argument("--stream-lanes", type=int, default=4)
    ap.add_argument("--train-workload", default=TRAIN_WORKLOAD)
    ap.add_argument("--weights", default=None,
                    help="load the surrogate from this checkpoint (rs_surrogate_save) instead of training")
    ap.add_argument("--save-weights", default=None, help="save the trained surrogate here")
    ap.add_argument("--train-samples", type=int, default=TRAIN_SAMPLES)
    ap.add_argument("--train-epochs", type=int, default=TRAIN_EPOCHS)
    args = ap.parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

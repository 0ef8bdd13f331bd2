"""Shared helpers for the parity tests: run the CUDA path through the C ABI and the oracle on
the same seeded inputs, and compare."""
import numpy as np

import oracle
from paper_2412_18629_gb300 import G_NEWTON, synth


def gpu_ctx(snap, **kw):
    import paper_2412_18629_gb300 as rs
    return rs.Context(box=snap["box"], link_len=snap["link_length"], softening=snap["softening"],
                      particle_mass=snap["particle_mass"], **kw)


def to_dev(snap):
    import torch
    return (torch.from_numpy(snap["pos"]).cuda(), torch.from_numpy(snap["vel"]).cuda(),
            torch.from_numpy(snap["ids"]).cuda())


def gpu_pipeline(snap, ctx=None, stages=("fof3d", "fof6d", "unbind", "props"), mode="plain"):
    """Run the requested stages on cuda:0; return host numpy results."""
    import torch
    import paper_2412_18629_gb300 as rs
    ctx = ctx or gpu_ctx(snap, mode=mode)
    pos, vel, ids = to_dev(snap)
    out = {}
    lab, ng = rs.rs_fof3d(ctx, pos, ids)
    out["labels"], out["n_groups"] = lab.cpu().numpy(), ng
    if "fof6d" in stages:
        nn, nm = rs.rs_fof6d(ctx, pos, vel, ids, lab)
        h = rs.rs_fof6d_copy(ctx)
        out["hier"] = {k: v.cpu().numpy() for k, v in h.items()}
        out["n_nodes"], out["n_members"] = nn, nm
    if "unbind" in stages:
        phi, bound, nfb = rs.rs_unbind(ctx, pos, vel)
        out["phi"], out["bound"], out["n_fallback"] = phi.cpu().numpy(), bound.cpu().numpy(), nfb
    if "props" in stages:
        out["props"] = rs.props_to_float64(rs.rs_halo_props(ctx)).cpu().numpy()
    torch.cuda.synchronize()
    return out


def oracle_pipeline(snap, labels=None, stages=("fof3d", "fof6d", "unbind", "props"), threads=None):
    out = {}
    pos, vel, ids, box = snap["pos"], snap["vel"], snap["ids"], snap["box"]
    lab = oracle.fof3d(pos, ids, box, snap["link_length"]) if labels is None else labels
    out["labels"] = lab
    if "fof6d" in stages:
        out["hier"] = oracle.hierarchy(pos, vel, ids, lab, box, threads=threads)
    if "unbind" in stages:
        h = out["hier"]
        out["unbind"] = oracle.unbind(h["member_off"], h["member_idx"], pos, vel, box,
                                      snap["softening"], G_NEWTON, snap["particle_mass"],
                                      threads=threads)
    if "props" in stages:
        h, u = out["hier"], out["unbind"]
        out["props"] = oracle.props(h["member_off"], h["member_idx"], pos, vel, u["bound"],
                                    u["is_halo"], box, snap["particle_mass"], len(ids),
                                    threads=threads)
    return out


def small_snapshot(n, box, seed, n_max=3000, sub_levels=1):
    return synth.generate(synth.SnapshotSpec(n=n, box=box, seed=seed, n_max=n_max,
                                             sub_levels=sub_levels))


def assert_hier_equal(g, o):
    for k in ("parent", "level", "min_id", "size", "member_off", "member_idx", "deepest"):
        a, b = np.asarray(g[k]), np.asarray(o[k])
        assert a.shape == b.shape, (k, a.shape, b.shape)
        if not np.array_equal(a, b):
            bad = np.flatnonzero(a != b)
            raise AssertionError(f"{k}: {len(bad)} mismatches, first at {bad[:5]}: "
                                 f"gpu {a[bad[:5]]} oracle {b[bad[:5]]}")

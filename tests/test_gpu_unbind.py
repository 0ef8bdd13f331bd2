"""rs_unbind / rs_halo_props (CUDA) vs the oracle: bound flags, bound counts and halo decisions
bit for bit; float32 potential within 1e-5 relative of the float64 definition; properties
(float64 canonical-order sums) bit for bit except r_vir (cube root, within 4 ulp)."""
import numpy as np
import pytest

import oracle
from helpers import gpu_ctx, gpu_pipeline, oracle_pipeline, small_snapshot, to_dev
from paper_2412_18629_gb300 import G_NEWTON, synth

pytestmark = pytest.mark.gpu

POT_RTOL = 1e-5


def _compare(g, o):
    ub = o["unbind"]
    assert np.array_equal(g["bound"], ub["bound"])
    rel = np.abs(g["phi"].astype(np.float64) - ub["phi"]) / np.abs(ub["phi"])
    assert rel.max() <= POT_RTOL, rel.max()
    P, Q = g["props"], o["props"]
    assert np.array_equal(P[:, 1], ub["n_bound"].astype(np.float64))
    assert np.array_equal(P[:, 2], ub["is_halo"].astype(np.float64))
    assert np.array_equal(P[:, 3], ub["m_bound"])
    exact = [c for c in range(20) if c != 12]
    assert np.array_equal(P[:, exact], Q[:, exact]), np.argwhere(P[:, exact] != Q[:, exact])[:5]
    np.testing.assert_allclose(P[:, 12], Q[:, 12], rtol=4 * 2.0 ** -52, atol=0)


@pytest.mark.parametrize("mode", ("plain", "batched"))
@pytest.mark.parametrize("n,box,seed,n_max", [(1 << 13, 20.0, 31, 1500), (1 << 15, 32.0, 32, 5000)])
def test_unbind_props_small(n, box, seed, n_max, mode):
    s = small_snapshot(n, box, seed, n_max=n_max)
    g = gpu_pipeline(s, mode=mode)
    o = oracle_pipeline(s)
    _compare(g, o)


@pytest.mark.parametrize("mode", ("plain", "batched"))
def test_unbind_props_2e18_workload(mode):
    s = synth.generate(synth.WORKLOADS["nfw-2^18-L64"])
    g = gpu_pipeline(s, mode=mode)
    o = oracle_pipeline(s, labels=g["labels"])
    assert np.array_equal(g["labels"], oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"]))
    _compare(g, o)


def test_energy_shifted_members_take_the_exact_path():
    """Velocities of some members are set so that KE = -phi (1 +- 1e-7) in their node's frame:
    the float32 potential cannot decide them, so the exact float64 path must, and flags must
    still match the definition."""
    s = small_snapshot(1 << 13, 20.0, 33, n_max=1500)
    o = oracle_pipeline(s, stages=("fof3d", "fof6d", "unbind"))
    h, ub = o["hier"], o["unbind"]
    q = int(np.argmax(h["size"]))                       # a level-0 node (FoF group)
    lo, hi = h["member_off"][q], h["member_off"][q + 1]
    mem = h["member_idx"][lo:hi]
    rng = np.random.default_rng(0)
    pick = rng.choice(len(mem), size=min(64, len(mem) // 8), replace=False)
    phi = ub["phi"][lo:hi][pick]
    sgn = np.where(rng.random(len(pick)) < 0.5, 1.0 - 1e-7, 1.0 + 1e-7)
    speed = np.sqrt(-2.0 * phi * sgn)
    d = rng.normal(size=(len(pick), 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    vel = s["vel"].copy()
    for _ in range(8):                                   # settle the node's bulk velocity
        vb = vel[mem].astype(np.float64).mean(0)
        vel[mem[pick]] = (vb + d * speed[:, None]).astype(np.float32)
    s2 = dict(s)
    s2["vel"] = vel
    g = gpu_pipeline(s2, mode="batched")
    o2 = oracle_pipeline(s2, labels=g["labels"])
    assert g["n_fallback"] >= len(pick) // 2
    _compare(g, o2)


def test_autotuner_picks_a_candidate_and_keeps_the_sums():
    """On a call with >= 2^20 members the autotuner times 2, 4 and 8 members per thread for the
    blocked potential and keeps the fastest; the potentials of the tuning call and of a later
    call with the kept choice are bit-identical."""
    import paper_2412_18629_gb300 as rs
    s = synth.generate(synth.WORKLOADS["nfw-2^21-L128-sub"])
    ctx = gpu_ctx(s, mode="batched")
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    assert ctx.n_members >= 1 << 20
    assert ctx.tuning()["blocked_potential"]["members_per_thread"] == 0
    phi1, b1, _ = rs.rs_unbind(ctx, pos, vel, want_potential=True)
    t = ctx.tuning()["blocked_potential"]
    assert t["members_per_thread"] in (2, 4, 8) and all(v > 0 for v in t["ms"].values()), t
    phi1, b1 = phi1.cpu().numpy(), b1.cpu().numpy()
    phi2, b2, _ = rs.rs_unbind(ctx, pos, vel, want_potential=True)
    assert np.array_equal(phi1, phi2.cpu().numpy()) and np.array_equal(b1, b2.cpu().numpy())


@pytest.mark.parametrize("mode,tree_min", (("plain", 0), ("batched", 0), ("batched", 2048)))
def test_direct_sum_pair_tallies(mode, tree_min):
    """rs_potential_pairs counts exactly the ordered pairs g (g - 1) of the nodes each direct-sum
    kernel ran on: nodes up to 384 members in [0], larger ones in [1] (below the tree's
    threshold when the tree bound is on), whatever the autotuner did first."""
    import paper_2412_18629_gb300 as rs
    s = small_snapshot(1 << 16, 40.3, 33, n_max=8000)
    ctx = gpu_ctx(s, mode=mode, tree_min=tree_min)
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    g = rs.rs_fof6d_copy(ctx)["size"].cpu().numpy().astype(np.int64)
    rs.rs_unbind(ctx, pos, vel, want_potential=False)
    small, big = rs.rs_potential_pairs(ctx)
    lim = tree_min if (mode == "batched" and tree_min > 0) else np.inf
    p = g * (g - 1)
    assert small == int(p[g <= 384].sum())
    assert big == int(p[(g > 384) & (g < lim)].sum())
    assert big > 0 and (lim == np.inf or (g >= lim).any())

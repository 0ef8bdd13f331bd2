"""Parity at the benchmarked size: the 2^24-particle workload bench.py times, in its launch
configuration (batched form; batched + surrogate form). FoF labels are compared in full with the
oracle; per sampled node, the 6D split (metric scales, l2 and children), the float32 potential,
the bound flags, bound count, halo decision and properties against the oracle's per-node
functions run on the same member lists; and the surrogate form's flags against the certified
exact flags of the batched form for every member of every node."""
import numpy as np
import pytest

import oracle
from helpers import gpu_ctx, to_dev
from paper_2412_18629_gb300 import G_NEWTON, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

WORKLOAD = "nfw-2^24-L256-sub"
POT_RTOL = 1e-5


def _wrap(d, L):
    hL = np.float32(0.5) * L
    d = np.where(d > hL, d - L, d)
    return np.where(d < -hL, d + L, d).astype(np.float32)


@pytest.fixture(scope="module")
def run():
    import paper_2412_18629_gb300 as rs
    s = synth.generate(synth.WORKLOADS[WORKLOAD])
    ctx = gpu_ctx(s, mode="batched")
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    phi, bound, _ = rs.rs_unbind(ctx, pos, vel, want_potential=True)
    props = rs.props_to_float64(rs.rs_halo_props(ctx)).cpu().numpy()
    h = {k: v.cpu().numpy() for k, v in rs.rs_fof6d_copy(ctx).items()}
    prm = rs.rs_fof6d_node_params(ctx).cpu().numpy()
    out = dict(snap=s, labels=lab.cpu().numpy(), hier=h, params=prm, phi=phi.cpu().numpy(),
               bound=bound.cpu().numpy(), props=props)
    ctx.close()
    return out


def _sample_nodes(h, rng, k_random, g_max):
    size = h["size"]
    ok = np.flatnonzero(size <= g_max)
    big = ok[np.argsort(-size[ok], kind="stable")[:3]]
    deep = ok[h["level"][ok] >= 1]
    pick = np.unique(np.r_[big, rng.choice(ok, k_random, replace=False),
                           rng.choice(deep, min(k_random, len(deep)), replace=False)])
    return pick


def test_fof3d_labels_full(run):
    s = run["snap"]
    lab = oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"])
    assert np.array_equal(run["labels"], lab)


def test_sampled_node_splits(run):
    """Metric scales, l2 and the children of sampled nodes, from the oracle's split of the
    node's own members."""
    s, h, prm = run["snap"], run["hier"], run["params"]
    L = np.float32(s["box"])
    rng = np.random.default_rng(24)
    off, mem, par = h["member_off"], h["member_idx"], h["parent"]
    checked = 0
    for q in _sample_nodes(h, rng, 12, 16000):
        m = mem[off[q]:off[q + 1]]
        g = len(m)
        u = _wrap((s["pos"][m] - s["pos"][m[0]]).astype(np.float32), L)
        isx, isv, l2, _, comp = oracle.split_node(u, s["vel"][m].astype(np.float32))
        assert (np.float32(isx), np.float32(isv), np.float32(l2)) == tuple(prm[q, :3]), q
        labels, counts = np.unique(comp, return_counts=True)
        want = {frozenset(m[comp == c]) for c, k in zip(labels, counts) if 10 <= k < g}
        kids = np.flatnonzero(par == q)
        got = {frozenset(mem[off[c]:off[c + 1]]) for c in kids}
        assert got == want, q
        checked += 1
    assert checked >= 10


def test_sampled_node_unbinding_and_props(run):
    """Potential, flags, bound counts, halo decisions and properties of sampled nodes."""
    s, h = run["snap"], run["hier"]
    rng = np.random.default_rng(25)
    off, mem = h["member_off"], h["member_idx"]
    pick = _sample_nodes(h, rng, 16, 12000)
    sub_off = np.r_[0, np.cumsum(off[pick + 1] - off[pick])]
    sub_idx = np.concatenate([mem[off[q]:off[q + 1]] for q in pick])
    pos_csr = np.concatenate([np.arange(off[q], off[q + 1]) for q in pick])
    ub = oracle.unbind(sub_off, sub_idx, s["pos"], s["vel"], s["box"], s["softening"], G_NEWTON,
                       s["particle_mass"])
    assert np.array_equal(run["bound"][pos_csr], ub["bound"])
    rel = np.abs(run["phi"][pos_csr].astype(np.float64) - ub["phi"]) / np.abs(ub["phi"])
    assert rel.max() <= POT_RTOL, rel.max()
    P = run["props"][pick]
    assert np.array_equal(P[:, 1], ub["n_bound"].astype(np.float64))
    assert np.array_equal(P[:, 2], ub["is_halo"].astype(np.float64))
    Q = oracle.props(sub_off, sub_idx, s["pos"], s["vel"], ub["bound"], ub["is_halo"], s["box"],
                     s["particle_mass"], len(s["ids"]))
    exact = [c for c in range(20) if c != 12]
    assert np.array_equal(P[:, exact], Q[:, exact])
    np.testing.assert_allclose(P[:, 12], Q[:, 12], rtol=4 * 2.0 ** -52, atol=0)


@pytest.mark.parametrize("gate", (0, 1))
def test_surrogate_form_flags_equal_exact_flags_everywhere(run, gate):
    """The batched + surrogate form, with a network trained on another snapshot, gives the
    same flag as the certified exact path for every (node, member) of the 2^24 workload, with
    the held-out-maximum gate (0) and the calibrated gate (1); the calibrated gate decides a
    real share of the large nodes' members."""
    import paper_2412_18629_gb300 as rs
    from test_gpu_surrogate import _train
    spec = synth.SnapshotSpec(n=1 << 20, box=float(np.cbrt(2.0 ** 20)), seed=100, n_max=3.0e4,
                              sub_levels=1)
    params, err_max, _ = _train(synth.generate(spec))
    s = run["snap"]
    ctx = gpu_ctx(s, mode="surrogate", surrogate_gate=gate)
    rs.rs_mlp_set_params(ctx, params)
    rs.rs_mlp_set_err_max(ctx, err_max)
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    _, bound, _ = rs.rs_unbind(ctx, pos, vel, want_potential=False)
    props = rs.props_to_float64(rs.rs_halo_props(ctx)).cpu().numpy()
    stats = rs.rs_surrogate_stats(ctx)
    assert int(np.sum(bound.cpu().numpy() != run["bound"])) == 0
    assert np.array_equal(props, run["props"])
    if gate == 1:
        assert stats["surrogate_decided"] > 0.3 * stats["surrogate_members"], stats

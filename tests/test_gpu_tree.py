"""The certified tree bound of the potential (batched forms of rs_unbind called without a
potential output) against the oracle: every recorded interval [S_lo, S_hi] holds the oracle's
float64 sum S_i = -phi_i / (G m), and the bound flags, bound counts, halo decisions and
properties equal the oracle's bit for bit, for several opening angles, with the tree forced
onto small nodes so that most nodes and levels of a snapshot go through it."""
import numpy as np
import pytest

from helpers import gpu_ctx, oracle_pipeline, small_snapshot, to_dev
from paper_2412_18629_gb300 import G_NEWTON, synth

pytestmark = pytest.mark.gpu


def _run(s, tree_min, theta=0.0, record=True, mode="batched", want_potential=False):
    import paper_2412_18629_gb300 as rs
    ctx = gpu_ctx(s, mode=mode, tree_min=tree_min, tree_theta=theta)
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    if record:
        rs.rs_tree_record(ctx, True)
    phi, bound, nfb = rs.rs_unbind(ctx, pos, vel, want_potential=want_potential)
    out = {"labels": lab.cpu().numpy(), "bound": bound.cpu().numpy(), "stats": rs.rs_tree_stats(ctx),
           "hier": {k: v.cpu().numpy() for k, v in rs.rs_fof6d_copy(ctx).items()},
           "props": rs.props_to_float64(rs.rs_halo_props(ctx)).cpu().numpy()}
    if record and not want_potential:
        lo, hi = rs.rs_tree_bounds(ctx)
        out["lo"], out["hi"] = lo.cpu().numpy(), hi.cpu().numpy()
    ctx.close()
    return out


def _check_against_oracle(s, g):
    o = oracle_pipeline(s, labels=g["labels"])
    for k in ("member_off", "member_idx"):
        assert np.array_equal(g["hier"][k], o["hier"][k])
    ub = o["unbind"]
    assert np.array_equal(g["bound"], ub["bound"])
    P, Q = g["props"], o["props"]
    assert np.array_equal(P[:, 1], ub["n_bound"].astype(np.float64))
    assert np.array_equal(P[:, 2], ub["is_halo"].astype(np.float64))
    exact = [c for c in range(20) if c != 12]
    assert np.array_equal(P[:, exact], Q[:, exact])
    return o


def _check_intervals(s, g, o):
    S = -o["unbind"]["phi"] / (G_NEWTON * s["particle_mass"])
    rec = np.isfinite(g["lo"])
    assert rec.sum() == g["stats"]["decided_by_bound"] + g["stats"]["exact_path"]
    assert np.all(g["lo"][rec] <= S[rec]) and np.all(S[rec] <= g["hi"][rec])
    return rec


@pytest.mark.parametrize("theta", (0.3, 0.5, 0.7, 0.9))
def test_tree_flags_and_intervals_small_nodes(theta):
    s = small_snapshot(1 << 16, 40.0, 41, n_max=5000)
    g = _run(s, tree_min=128, theta=theta)
    st = g["stats"]
    assert st["tree_nodes"] > 10 and st["decided_by_bound"] > 0, st
    o = _check_against_oracle(s, g)
    rec = _check_intervals(s, g, o)
    assert rec.sum() == st["tree_members"]


def test_tree_interval_width_shrinks_with_theta():
    """A smaller opening angle gives narrower intervals and decides more members."""
    s = small_snapshot(1 << 16, 40.0, 42, n_max=5000)
    a = _run(s, tree_min=256, theta=0.3)
    b = _run(s, tree_min=256, theta=0.8)
    assert np.array_equal(a["bound"], b["bound"])
    rec = np.isfinite(a["lo"])
    wa = np.median((a["hi"] - a["lo"])[rec] / a["hi"][rec])
    wb = np.median((b["hi"] - b["lo"])[rec] / b["hi"][rec])
    assert wa < wb
    assert a["stats"]["decided_by_bound"] >= b["stats"]["decided_by_bound"]
    assert a["stats"]["expansions"] + a["stats"]["direct_pairs"] > 0


def test_tree_default_threshold_matches_direct_flags_2e20():
    """Default threshold (16384 members) on a 2^20-particle snapshot with halos up to 3e4: the
    flags of the tree path equal those of the exact direct sums (potential requested), member
    for member, and the tree decided most members of its nodes."""
    spec = synth.SnapshotSpec(n=1 << 20, box=101.6, seed=43, n_max=3.0e4, sub_levels=1)
    s = synth.generate(spec)
    t = _run(s, tree_min=0, record=False)
    d = _run(s, tree_min=0, record=False, want_potential=True)
    assert t["stats"]["tree_nodes"] >= 1, t["stats"]
    assert d["stats"]["tree_nodes"] == 0
    assert np.array_equal(t["bound"], d["bound"])
    assert np.array_equal(t["props"], d["props"])
    st = t["stats"]
    assert st["decided_by_bound"] >= 0.8 * st["tree_members"], st

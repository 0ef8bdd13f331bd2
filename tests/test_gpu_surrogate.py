"""Batched + surrogate form: the MLP is trained on the GPU from exact potentials of one
snapshot, then gates the unbinding of another. Flags, bound counts and halo decisions must be
identical to the oracle's (no mismatch), the surrogate must classify a real share of the
members of large nodes, and the exact work it saves is reported (the gain)."""
import numpy as np
import pytest

import oracle
from helpers import gpu_ctx, oracle_pipeline, to_dev
from paper_2412_18629_gb300 import synth

pytestmark = pytest.mark.gpu


def _train(train_snap):
    import paper_2412_18629_gb300 as rs
    ctx = gpu_ctx(train_snap, mode="batched")
    pos, vel, ids = to_dev(train_snap)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    rs.rs_unbind(ctx, pos, vel, want_potential=True)  # targets need every member's potential
    x, t = rs.rs_surrogate_features(ctx)
    assert x.shape[0] > 10000
    err_max, mse = rs.rs_mlp_train(ctx, x.contiguous(), t.contiguous(), epochs=12, batch=4096,
                                   lr=1e-3, seed=1)
    return rs.rs_mlp_get_params(ctx), err_max, mse


@pytest.fixture(scope="module")
def trained():
    spec = synth.SnapshotSpec(n=1 << 20, box=float(np.cbrt(2.0 ** 20)), seed=100, n_max=3.0e4,
                              sub_levels=1)
    return _train(synth.generate(spec))


def _run_surrogate(s, params, err_max, **kw):
    import paper_2412_18629_gb300 as rs
    ctx = gpu_ctx(s, mode="surrogate", **kw)
    rs.rs_mlp_set_params(ctx, params)
    rs.rs_mlp_set_err_max(ctx, err_max)
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    _, bound, _ = rs.rs_unbind(ctx, pos, vel, want_potential=False)
    props = rs.props_to_float64(rs.rs_halo_props(ctx)).cpu().numpy()
    sizes = rs.rs_fof6d_copy(ctx)["size"].cpu().numpy()
    return lab.cpu().numpy(), bound.cpu().numpy(), props, rs.rs_surrogate_stats(ctx), sizes


@pytest.fixture(scope="module")
def workload_2e18():
    s = synth.generate(synth.WORKLOADS["nfw-2^18-L64"])
    return s


@pytest.mark.parametrize("gate", (0, 1))
def test_surrogate_flags_match_oracle(trained, workload_2e18, gate):
    """With the trained network, every flag, bound count and halo decision equals the oracle's,
    for the held-out-maximum gate (0) and the calibrated gate (1); the counters account for
    every member of the large nodes exactly once."""
    params, err_max, _ = trained
    s = workload_2e18
    lab, bound, props, stats, _ = _run_surrogate(s, params, err_max, surrogate_gate=gate)
    o = oracle_pipeline(s, labels=lab, stages=("fof3d", "fof6d", "unbind"))
    ub = o["unbind"]
    assert int(np.sum(bound != ub["bound"])) == 0
    assert np.array_equal(props[:, 1], ub["n_bound"].astype(np.float64))
    assert np.array_equal(props[:, 2], ub["is_halo"].astype(np.float64))
    assert stats["surrogate_members"] > 0
    accounted = (stats["surrogate_decided"] + stats["exact_member_path"] + stats["spot_checked"]
                 + stats["rerun_members"] + stats["whole_node_members"])
    assert accounted == stats["surrogate_members"], stats


@pytest.mark.parametrize("gate", (0, 1))
def test_surrogate_gain(trained, workload_2e18, gate):
    """What the trained network gains over the method without it: the share of the large
    nodes' members whose flag it decides (no O(g) exact sum for them), with zero flag
    mismatches against the oracle. The held-out-maximum gate (0) is reported (it decides few
    members: four times the maximum error of the training's hold-out is a wide margin); the
    calibrated gate (1) must decide a real share."""
    params, err_max, _ = trained
    s = workload_2e18
    lab, bound, props, stats, sizes = _run_surrogate(s, params, err_max, surrogate_gate=gate)
    o = oracle_pipeline(s, labels=lab, stages=("fof3d", "fof6d", "unbind"))
    assert int(np.sum(bound != o["unbind"]["bound"])) == 0
    big = sizes[sizes >= 1024].astype(np.float64)
    decided_share = stats["surrogate_decided"] / stats["surrogate_members"]
    print("surrogate gain on the 2^18 workload: decided", stats["surrogate_decided"], "of",
          stats["surrogate_members"], f"large-node members ({decided_share:.1%}); exact sums for",
          stats["exact_member_path"] + stats["spot_checked"] + stats["rerun_members"],
          "members;", stats, "err_max", err_max, "large-node pairs", float((big * big).sum()))
    if gate == 1:
        assert stats["surrogate_decided"] > 0.1 * stats["surrogate_members"], stats


def test_overconfident_surrogate_is_caught_by_spot_checks(trained, workload_2e18):
    """With a gate far below its calibrated error (margin factor 0.05 instead of 4), wrong
    predictions get through the gate; the spot checks must notice (nodes fail and their gated
    members are recomputed exactly)."""
    params, err_max, _ = trained
    lab, bound, props, stats, _ = _run_surrogate(workload_2e18, params, err_max, margin_factor=0.05)
    assert stats["gated"] > 0
    assert stats["failed_nodes"] > 0 and stats["rerun_members"] > 0, stats
    assert stats["spot_mismatches"] > 0, stats
    o = oracle_pipeline(workload_2e18, labels=lab, stages=("fof3d", "fof6d", "unbind"))
    assert int(np.sum(bound != o["unbind"]["bound"])) == 0


def test_surrogate_requires_weights_and_null_potential():
    import paper_2412_18629_gb300 as rs
    s = synth.generate(synth.SnapshotSpec(n=1 << 14, box=25.0, seed=7, n_max=2000, sub_levels=1))
    ctx = gpu_ctx(s, mode="surrogate")
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    with pytest.raises(rs.RSError, match="RS_ERR_STATE"):
        rs.rs_unbind(ctx, pos, vel, want_potential=False)
    rs.rs_mlp_set_params(ctx, np.zeros(rs.MLP_PARAMS, np.float32))
    with pytest.raises(rs.RSError, match="RS_ERR_INVALID_ARG"):
        rs.rs_unbind(ctx, pos, vel, want_potential=True)

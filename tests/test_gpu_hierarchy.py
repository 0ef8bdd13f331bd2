"""rs_fof6d (CUDA) vs the oracle's 6D phase-space FoF hierarchy: node table, member lists and
deepest-node map bit for bit (Section "Parallelization": subhalo finding per FoF halo from 6D
phase-space information)."""
import numpy as np
import pytest

import oracle
from helpers import assert_hier_equal, gpu_pipeline, small_snapshot
from paper_2412_18629_gb300 import synth

pytestmark = pytest.mark.gpu
MODES = ("plain", "batched")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,box,seed,n_max", [(1 << 13, 20.0, 21, 1500), (1 << 15, 32.0, 22, 4000),
                                              (1 << 16, 40.0, 23, 12000)])
def test_hierarchy_small(n, box, seed, n_max, mode):
    s = small_snapshot(n, box, seed, n_max=n_max)
    g = gpu_pipeline(s, stages=("fof3d", "fof6d"), mode=mode)
    lab = oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"])
    assert np.array_equal(g["labels"], lab)
    o = oracle.hierarchy(s["pos"], s["vel"], s["ids"], lab, s["box"])
    assert_hier_equal(g["hier"], o)
    assert o["level"].max() >= 1


@pytest.mark.parametrize("mode", MODES)
def test_hierarchy_2e18_workload(mode):
    s = synth.generate(synth.WORKLOADS["nfw-2^18-L64"])
    g = gpu_pipeline(s, stages=("fof3d", "fof6d"), mode=mode)
    lab = oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"])
    assert np.array_equal(g["labels"], lab)
    assert_hier_equal(g["hier"], oracle.hierarchy(s["pos"], s["vel"], s["ids"], lab, s["box"]))


@pytest.mark.parametrize("mode", MODES)
def test_no_groups_and_tiny_groups(mode):
    rng = np.random.default_rng(3)
    n = 2000
    snap = {"pos": rng.uniform(0, 100, (n, 3)).astype(np.float32),
            "vel": rng.normal(0, 10, (n, 3)).astype(np.float32),
            "ids": rng.permutation(n).astype(np.int64), "box": 100.0, "link_length": 0.05,
            "softening": 0.01, "particle_mass": 1e10}
    g = gpu_pipeline(snap, stages=("fof3d", "fof6d"), mode=mode)
    assert g["n_nodes"] == 0 and g["n_members"] == 0 and np.all(g["hier"]["deepest"] == -1)


@pytest.mark.parametrize("mode", MODES)
def test_velocity_scaling_invariance_on_gpu(mode):
    s = small_snapshot(1 << 14, 25.0, 24)
    a = gpu_pipeline(s, stages=("fof3d", "fof6d"), mode=mode)
    s2 = dict(s)
    s2["vel"] = s["vel"] * np.float32(2.0)
    b = gpu_pipeline(s2, stages=("fof3d", "fof6d"), mode=mode)
    assert_hier_equal(a["hier"], b["hier"])


def test_plain_and_batched_identical_on_large_groups():
    """Large nodes (thousands of members, many buckets) exercise the pruning: both forms must
    produce the same hierarchy, and it must equal the oracle's."""
    s = small_snapshot(1 << 17, 50.0, 25, n_max=30000)
    a = gpu_pipeline(s, stages=("fof3d", "fof6d"), mode="plain")
    b = gpu_pipeline(s, stages=("fof3d", "fof6d"), mode="batched")
    assert_hier_equal(a["hier"], b["hier"])
    assert a["hier"]["size"].max() > 5000
    o = oracle.hierarchy(s["pos"], s["vel"], s["ids"], a["labels"], s["box"])
    assert_hier_equal(b["hier"], o)


def test_work_counting_variant_gives_the_same_hierarchy():
    """The counting variants of the pruned kernels (instrumentation for the roofline) leave the
    hierarchy unchanged and tally fewer d6 evaluations than the brute-force pair count."""
    import paper_2412_18629_gb300 as rs
    from helpers import gpu_ctx, to_dev
    s = small_snapshot(1 << 16, 40.0, 23, n_max=12000)
    ref = gpu_pipeline(s, stages=("fof3d", "fof6d"), mode="batched")
    ctx = gpu_ctx(s, mode="batched")
    pos, vel, ids = to_dev(s)
    ctx.count_work(True)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    w = ctx.count_work(False)
    got = {k: v.cpu().numpy() for k, v in rs.rs_fof6d_copy(ctx).items()}
    assert_hier_equal(got, ref["hier"])
    sizes = got["size"].astype(np.float64)
    assert 0 < w["nn_d6"] < (sizes * (sizes - 1)).sum()
    assert w["nn_box"] > 0 and w["link_d6"] > 0 and w["link_box"] > 0


@pytest.mark.parametrize("mode", MODES)
def test_sparse_ids_give_the_same_hierarchy(mode):
    """Level 0 groups particles by a count per label when the labels are dense (at most about
    2 n) and by a sort of (label, id) keys otherwise; ids spread up to ~2^31 take the second
    path, and the hierarchy must still equal the oracle's."""
    s = small_snapshot(1 << 15, 32.0, 22, n_max=4000)
    rng = np.random.default_rng(7)
    s = dict(s)
    s["ids"] = (rng.permutation(len(s["ids"])).astype(np.int64) * 65521 + 977).astype(np.int64)
    g = gpu_pipeline(s, stages=("fof3d", "fof6d"), mode=mode)
    lab = oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"])
    assert np.array_equal(g["labels"], lab)
    assert lab.max() > 4 * len(lab)
    assert_hier_equal(g["hier"], oracle.hierarchy(s["pos"], s["vel"], s["ids"], lab, s["box"]))

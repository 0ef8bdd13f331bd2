"""Bounded nearest-neighbour searches of the batched form (nodes of at least 4096 members):
a sample of each large node's buckets is searched exactly, its order statistics bound the
adaptive link length, and the other members are searched only as far as those bounds need.
The hierarchy (node table, member lists, deepest nodes, split parameters including l2) must be
bit-identical to the plain form's brute-force searches and to the oracle, both with the default
bounds and when every bounded node is forced through the exact fallback (empty bounds)."""
import numpy as np
import pytest

import oracle
from helpers import assert_hier_equal, gpu_ctx, small_snapshot, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snap():
    # halos up to 6e4 particles: several level-0 nodes and subnodes above 4096 members
    return small_snapshot(1 << 18, 64.0, 77, n_max=6.0e4)


def _hierarchy(s, mode, margin=None, min_members=0):
    import paper_2412_18629_gb300 as rs
    ctx = gpu_ctx(s, mode=mode)
    if margin is not None or min_members:
        ctx.nn_bounds(1.0 if margin is None else margin, min_members)
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    if mode != "plain":
        ctx.count_work(True)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    work = ctx.count_work(False) if mode != "plain" else None
    h = {k: v.cpu().numpy() for k, v in rs.rs_fof6d_copy(ctx).items()}
    params = rs.rs_fof6d_node_params(ctx).cpu().numpy()
    ctx.close()
    return lab.cpu().numpy(), h, params, work


@pytest.fixture(scope="module")
def plain(snap):
    return _hierarchy(snap, "plain")


def test_bounded_search_matches_plain_and_oracle(snap, plain):
    lab, h, params, work = _hierarchy(snap, "batched")
    assert work["bounded_nodes"] >= 2, work
    _, hp, pp, _ = plain
    assert_hier_equal(h, hp)
    assert np.array_equal(params.view(np.uint32), pp.view(np.uint32))
    sizes = np.diff(h["member_off"])
    assert (sizes >= 4096).sum() >= 2
    o = oracle.hierarchy(snap["pos"], snap["vel"], snap["ids"], lab, snap["box"])
    assert_hier_equal(h, o)
    assert np.array_equal(params[:, :3].view(np.uint32), o["params"][:, :3].view(np.uint32))


def test_forced_fallback_gives_the_same_hierarchy(snap, plain):
    lab, h, params, work = _hierarchy(snap, "batched", margin=-1.0)
    assert work["bounded_nodes"] >= 2 and work["bound_failures"] == work["bounded_nodes"], work
    _, hp, pp, _ = plain
    assert_hier_equal(h, hp)
    assert np.array_equal(params.view(np.uint32), pp.view(np.uint32))


def test_tight_margin_still_exact(snap, plain):
    """A margin of zero (bounds at the sample's own quantile +- 8 ranks) fails more often; the
    fallback keeps every result exact whatever the sample gave."""
    lab, h, params, work = _hierarchy(snap, "batched", margin=0.0)
    _, hp, pp, _ = plain
    assert_hier_equal(h, hp)
    assert np.array_equal(params.view(np.uint32), pp.view(np.uint32))


def test_smaller_bounded_nodes(snap, plain):
    """Bounds down to 2048-member nodes (samples of every 1st-2nd bucket there): still exact."""
    lab, h, params, work = _hierarchy(snap, "batched", min_members=2048)
    assert work["bounded_nodes"] > 10, work
    _, hp, pp, _ = plain
    assert_hier_equal(h, hp)
    assert np.array_equal(params.view(np.uint32), pp.view(np.uint32))


def test_forced_fallback_of_small_bounded_nodes(snap, plain):
    """Bounded nodes of 2048-4096 members take the warp-level selection: when all of them fail
    (empty bounds), that selection runs again on them and the hierarchy stays exact."""
    lab, h, params, work = _hierarchy(snap, "batched", margin=-1.0, min_members=2048)
    assert work["bounded_nodes"] > 10 and work["bound_failures"] == work["bounded_nodes"], work
    sizes = np.diff(h["member_off"])
    assert ((sizes >= 2048) & (sizes <= 4096)).sum() >= 1
    _, hp, pp, _ = plain
    assert_hier_equal(h, hp)
    assert np.array_equal(params.view(np.uint32), pp.view(np.uint32))

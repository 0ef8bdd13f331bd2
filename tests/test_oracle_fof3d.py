"""Pins for the oracle's 3D friends-of-friends (Section "Parallelization": each process runs 3D
FoF over its particles). The oracle is checked against things other than itself: a hand-derived
golden case, lattice and periodic special cases, its own brute force vs its grid, and SciPy's
periodic k-d tree plus graph components."""
import os

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components
from scipy.spatial import cKDTree

import oracle
from paper_2412_18629_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _min_id_labels(n, pairs, ids):
    if len(pairs):
        g = coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
    else:
        g = coo_matrix((n, n))
    _, comp = connected_components(g, directed=False)
    mins = np.full(comp.max() + 1, np.iinfo(np.int64).max)
    np.minimum.at(mins, comp, ids)
    return mins[comp]


def _pair_slack(box, ll, wrapped):
    """Relative error bound of the float32 periodic distance vs the exact one: a few ulps of the
    distance itself, or ~u L / ll when the coordinate difference is rounded before the wrap."""
    u = 2.0 ** -24
    return np.where(wrapped, 4 * u * box / ll, 8 * u)


def _scipy_labels(pos, ids, box, ll):
    """Labels from SciPy's periodic k-d tree (float64 distances). Pairs whose float64 distance is
    within float32 rounding of ll are ambiguous; returns the labels with all of them unlinked
    and with all of them linked (the float32 result must match one when there is at most one)."""
    p64 = pos.astype(np.float64)
    tree = cKDTree(p64, boxsize=box)
    pairs = tree.query_pairs(r=ll * 1.001, output_type="ndarray")
    d = p64[pairs[:, 0]] - p64[pairs[:, 1]]
    wrapped = np.any(np.abs(d) > box / 2, axis=1)
    d -= box * np.round(d / box)
    r = np.sqrt((d * d).sum(1))
    amb = np.abs(r - ll) / ll <= _pair_slack(box, ll, wrapped)
    sure = pairs[(r <= ll) & ~amb]
    lo = _min_id_labels(len(ids), sure, ids)
    hi = _min_id_labels(len(ids), np.concatenate([sure, pairs[amb]]), ids)
    return lo, hi, int(amb.sum())


def _matches(lab, lo, hi, n_amb):
    assert n_amb <= 1
    return np.array_equal(lab, lo) or np.array_equal(lab, hi)


def test_golden_chain():
    rows = np.loadtxt(os.path.join(GOLDEN, "fof3d_chain.txt"))
    pos = rows[:, :3].astype(np.float32)
    ids = rows[:, 3].astype(np.int64)
    want = rows[:, 4].astype(np.int64)
    assert np.array_equal(oracle.fof3d_brute(pos, ids, 10.0, 1.0), want)
    assert np.array_equal(oracle.fof3d_grid(pos, ids, 10.0, 1.0), want)


@pytest.mark.parametrize("spacing,ll,expect_one", [(0.5, 0.5, True), (0.5, 0.49, False)])
def test_periodic_lattice(spacing, ll, expect_one):
    k = 8
    g = (np.arange(k) * spacing).astype(np.float32)
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    ids = np.random.default_rng(1).permutation(len(pos)).astype(np.int64)
    box = k * spacing
    for fn in (oracle.fof3d_brute, oracle.fof3d_grid):
        lab = fn(pos, ids, box, ll)
        if expect_one:
            assert np.all(lab == 0)
        else:
            assert np.array_equal(lab, ids)


def test_periodic_pair_and_empty():
    pos = np.array([[0.05, 3, 3], [9.95, 3, 3.1]], np.float32)
    ids = np.array([5, 2], np.int64)
    for fn in (oracle.fof3d_brute, oracle.fof3d_grid):
        assert list(fn(pos, ids, 10.0, 0.2)) == [2, 2]
        assert list(fn(pos, ids, 10.0, 0.05)) == [5, 2]
        assert len(fn(np.zeros((0, 3), np.float32), np.zeros(0, np.int64), 10.0, 0.2)) == 0


def test_adversarial_grid_equals_brute():
    rng = np.random.default_rng(7)
    box, ll = 6.0, 0.3
    c = box / np.floor(box / (1.01 * ll))
    on_faces = (rng.integers(0, 20, (300, 3)) * c).astype(np.float32) % np.float32(box)
    dup = np.repeat(rng.uniform(0, box, (40, 3)), 3, axis=0).astype(np.float32)
    one_cell = (2.0 + rng.uniform(0, 0.2, (200, 3))).astype(np.float32)
    near_edge = np.where(rng.random((300, 3)) < 0.5, rng.uniform(0, 0.3, (300, 3)),
                         rng.uniform(box - 0.3, box, (300, 3))).astype(np.float32)
    pos = np.concatenate([on_faces, dup, one_cell, near_edge])
    pos[pos >= np.float32(box)] = 0
    ids = rng.permutation(len(pos)).astype(np.int64)
    a = oracle.fof3d_brute(pos, ids, box, ll)
    b = oracle.fof3d_grid(pos, ids, box, ll)
    assert np.array_equal(a, b)


def test_random_vs_scipy_components():
    rng = np.random.default_rng(3)
    n, box, ll = 3000, 12.0, 0.55
    pos = rng.uniform(0, box, (n, 3)).astype(np.float32)
    ids = rng.permutation(n).astype(np.int64) * 3 + 11
    lo, hi, n_amb = _scipy_labels(pos, ids, box, ll)
    assert _matches(oracle.fof3d_brute(pos, ids, box, ll), lo, hi, n_amb)
    assert _matches(oracle.fof3d_grid(pos, ids, box, ll), lo, hi, n_amb)


def test_clustered_snapshot_vs_scipy_and_invariants():
    spec = synth.SnapshotSpec(n=1 << 15, box=32.0, seed=11, n_max=3000, sub_levels=1)
    s = synth.generate(spec)
    pos, ids, box, ll = s["pos"], s["ids"], s["box"], s["link_length"]
    lab = oracle.fof3d_grid(pos, ids, box, ll)
    lo, hi, n_amb = _scipy_labels(pos, ids, box, ll)
    assert _matches(lab, lo, hi, n_amb)
    # invariants: each label is the id of one of its members, and the smallest one
    uniq, first = np.unique(lab, return_index=True)
    order = np.lexsort((ids, lab))
    starts = np.r_[0, np.flatnonzero(np.diff(lab[order])) + 1]
    assert np.array_equal(ids[order][starts], uniq)
    assert np.bincount(np.searchsorted(uniq, lab)).sum() == len(ids)
    assert (np.bincount(np.searchsorted(uniq, lab)) >= 20).sum() > 10

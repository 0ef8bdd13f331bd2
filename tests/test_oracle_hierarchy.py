"""Pins for the oracle's 6D phase-space FoF hierarchy (Section "Parallelization": subhalo finding
inside each FoF halo from 6D phase-space information; Rockstar's metric
d^2 = |dx|^2/sigma_x^2 + |dv|^2/sigma_v^2, linked fraction f = 0.7, recursion). The paper prints
no worked example, so the pins are an independent k-d tree nearest-neighbour and component
search, the defining property of the adaptive link length, structural invariants, exact
invariance under power-of-two velocity scaling and two-population special cases."""
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components
from scipy.spatial import cKDTree

import oracle
from paper_2412_18629_gb300 import synth


def _node(rng, g, blobs=1, dv=0.0, dx=0.0):
    u = rng.normal(0, 1.0, (g, 3))
    v = rng.normal(0, 1.0, (g, 3))
    lab = np.arange(g) % blobs
    v[:, 0] += lab * dv
    u[:, 0] += lab * dx
    return u.astype(np.float32), v.astype(np.float32), lab


def _variance(a):
    a = a.astype(np.float64)
    return float(np.var(a, axis=0).sum())


@pytest.mark.parametrize("g", [10, 57, 400, 1500])
def test_split_node_vs_kdtree(g):
    rng = np.random.default_rng(g)
    u, v, _ = _node(rng, g)
    isx, isv, l2, nn2, comp = oracle.split_node(u, v)
    # sigma from CRO moments agrees with NumPy's float64 variance
    assert isx == pytest.approx(1.0 / _variance(u), rel=1e-6)
    assert isv == pytest.approx(1.0 / _variance(v), rel=1e-6)
    # nearest neighbours in the scaled 6D space (float64 k-d tree)
    w = np.hstack([u.astype(np.float64) * np.sqrt(isx), v.astype(np.float64) * np.sqrt(isv)])
    tree = cKDTree(w)
    d, _ = tree.query(w, k=2)
    np.testing.assert_allclose(nn2, d[:, 1] ** 2, rtol=2e-6)
    # adaptive link length: the k-th smallest nn2, k = ceil(0.7 g) - 1
    k = -(-7 * g // 10) - 1
    assert l2 == np.sort(nn2)[k]
    assert (nn2 <= l2).sum() >= k + 1
    # components of the link graph d6 <= l2
    pairs = tree.query_pairs(r=np.sqrt(l2) * (1 + 1e-5), output_type="ndarray")
    dd = ((w[pairs[:, 0]] - w[pairs[:, 1]]) ** 2).sum(1)
    border = np.abs(dd - l2) <= 1e-5 * l2
    assert np.all(dd[~border] < l2)  # nothing in the ambiguous band except pairs at l2 itself
    adj = coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(g, g))
    _, cc = connected_components(adj, directed=False)
    # same partition; oracle labels each component by its smallest member position
    first = {}
    want = np.array([first.setdefault(c, i) for i, c in enumerate(cc)])
    assert np.array_equal(comp, want)


def test_velocity_scaling_by_two_is_exact():
    spec = synth.SnapshotSpec(n=1 << 14, box=25.0, seed=4, n_max=2500, sub_levels=1)
    s = synth.generate(spec)
    lab = oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"])
    a = oracle.hierarchy(s["pos"], s["vel"], s["ids"], lab, s["box"])
    b = oracle.hierarchy(s["pos"], s["vel"] * np.float32(2.0), s["ids"], lab, s["box"])
    for k in a:
        if k != "params":
            assert np.array_equal(a[k], b[k]), k
    # the velocity variance scales by exactly 4, the 6D distances and l2 not at all
    assert np.array_equal(a["params"][:, 0], b["params"][:, 0])
    assert np.array_equal(a["params"][:, 1], b["params"][:, 1] * np.float32(4.0))
    assert np.array_equal(a["params"][:, 2], b["params"][:, 2])
    assert a["level"].max() >= 1


def test_two_velocity_populations_never_share_a_child():
    rng = np.random.default_rng(9)
    u, v, blob = _node(rng, 600, blobs=2, dv=60.0)
    _, _, _, _, comp = oracle.split_node(u, v)
    for c in np.unique(comp):
        assert len(np.unique(blob[comp == c])) == 1
    sizes = {b: max(np.sum(comp == c) for c in np.unique(comp[blob == b])) for b in (0, 1)}
    assert min(sizes.values()) >= 10


def test_two_position_clumps_split_into_children():
    rng = np.random.default_rng(10)
    g = 800
    u, v, blob = _node(rng, g, blobs=2, dx=40.0)
    ids = np.arange(g, dtype=np.int64)
    pos = (u + np.float32(50.0)).astype(np.float32)
    h = oracle.hierarchy(pos, v, ids, np.zeros(g, np.int64), 200.0)
    kids = np.flatnonzero(h["parent"] == 0)
    assert len(kids) >= 2
    for q in kids:
        mem = h["member_idx"][h["member_off"][q]:h["member_off"][q + 1]]
        assert len(np.unique(blob[mem])) == 1


def test_hierarchy_structure_invariants():
    spec = synth.SnapshotSpec(n=1 << 15, box=32.0, seed=12, n_max=4000, sub_levels=1)
    s = synth.generate(spec)
    ids = s["ids"]
    lab = oracle.fof3d(s["pos"], ids, s["box"], s["link_length"])
    h = oracle.hierarchy(s["pos"], s["vel"], ids, lab, s["box"])
    off, mem = h["member_off"], h["member_idx"]
    n_nodes = len(h["size"])
    assert n_nodes > 0 and h["level"].max() >= 2
    # level 0 = FoF groups with >= 10 members, ascending label
    ul, cnt = np.unique(lab, return_counts=True)
    roots = np.flatnonzero(h["level"] == 0)
    assert np.array_equal(h["min_id"][roots], ul[cnt >= 10])
    assert np.all(h["parent"][roots] == -1)
    prev = (-1, -1, -1)
    for q in range(n_nodes):
        m = mem[off[q]:off[q + 1]]
        assert len(m) == h["size"][q] >= 10
        assert np.all(np.diff(ids[m]) > 0)          # ascending id
        assert h["min_id"][q] == ids[m[0]]
        key = (h["level"][q], h["parent"][q], h["min_id"][q])
        assert key > prev                            # BFS order: (level, parent, min id)
        prev = key
        p = h["parent"][q]
        if p >= 0:
            pm = mem[off[p]:off[p + 1]]
            assert h["level"][q] == h["level"][p] + 1
            assert len(m) < len(pm) and np.all(np.isin(m, pm))
    for p in range(n_nodes):                          # children of a node are disjoint
        kids = np.flatnonzero(h["parent"] == p)
        if len(kids) > 1:
            allm = np.concatenate([mem[off[q]:off[q + 1]] for q in kids])
            assert len(np.unique(allm)) == len(allm)
    # deepest node: the last (deepest) node holding each particle, -1 outside every node
    deep = np.full(len(ids), -1)
    for q in range(n_nodes):
        deep[mem[off[q]:off[q + 1]]] = q
    assert np.array_equal(deep, h["deepest"])

"""Pins for the oracle's large-node paths: the exactly pruned k-d tree 6D search must give the
all-pairs search's nearest-neighbour distances, link length and components bit for bit (on
clustered, duplicated, lattice and zero-dispersion inputs, single- and multi-threaded), and the
sampled unbinding must equal the whole-node unbinding at the sampled members."""
import numpy as np
import pytest

import oracle
from helpers import small_snapshot
from paper_2412_18629_gb300 import G_NEWTON


def _both(u, v, threads=4):
    a = oracle.split_node(u, v, pruned=0)
    b = oracle.split_node(u, v, pruned=1, threads=threads)
    assert a[:3] == b[:3]
    assert np.array_equal(a[3], b[3])
    assert np.array_equal(a[4], b[4])
    return a


def _blobs(rng, g, k=3):
    c = rng.normal(0, 3, (k, 3))
    w = rng.normal(0, 50, (k, 3))
    lab = rng.integers(0, k, g)
    u = (c[lab] + rng.normal(0, 0.3, (g, 3))).astype(np.float32)
    v = (w[lab] + rng.normal(0, 20, (g, 3))).astype(np.float32)
    return u, v


@pytest.mark.parametrize("g,seed", [(2, 0), (17, 1), (300, 2), (2500, 3)])
def test_pruned_equals_all_pairs_on_clustered_nodes(g, seed):
    rng = np.random.default_rng(seed)
    u, v = _blobs(rng, g)
    _both(u, v)


def test_pruned_equals_all_pairs_with_duplicates_and_ties():
    rng = np.random.default_rng(5)
    u, v = _blobs(rng, 800)
    u[400:500] = u[300:400]            # exact duplicates in position and velocity
    v[400:500] = v[300:400]
    lat = np.stack(np.meshgrid(*(np.arange(6.0),) * 3, indexing="ij"), -1).reshape(-1, 3)
    u2 = np.concatenate([u, lat.astype(np.float32)])
    v2 = np.concatenate([v, np.zeros_like(lat, dtype=np.float32)])
    _both(u2, v2)


def test_pruned_equals_all_pairs_with_zero_velocity_dispersion():
    rng = np.random.default_rng(6)
    u = rng.normal(0, 1, (1500, 3)).astype(np.float32)
    v = np.full((1500, 3), 7.0, np.float32)   # sigma_v = 0: the velocity term drops out
    isx, isv, l2, nn2, comp = _both(u, v)
    assert isv == 0.0


def test_pruned_thread_count_does_not_change_results():
    rng = np.random.default_rng(7)
    u, v = _blobs(rng, 5000, k=5)
    a = oracle.split_node(u, v, pruned=1, threads=1)
    b = oracle.split_node(u, v, pruned=1, threads=8)
    c = oracle.split_node(u, v)        # by size: 5000 > 4096 takes the tree
    for x in (b, c):
        assert a[:3] == x[:3] and np.array_equal(a[3], x[3]) and np.array_equal(a[4], x[4])


def test_unbind_sample_equals_whole_node_unbinding():
    s = small_snapshot(1 << 14, 25.0, 9, n_max=3000)
    lab = oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"])
    h = oracle.hierarchy(s["pos"], s["vel"], s["ids"], lab, s["box"])
    ub = oracle.unbind(h["member_off"], h["member_idx"], s["pos"], s["vel"], s["box"],
                       s["softening"], G_NEWTON, s["particle_mass"])
    rng = np.random.default_rng(0)
    for q in np.argsort(-h["size"])[:4]:
        lo, hi = h["member_off"][q], h["member_off"][q + 1]
        mem = h["member_idx"][lo:hi]
        pick = rng.choice(len(mem), min(50, len(mem)), replace=False)
        phi, bound = oracle.unbind_sample(mem, s["pos"], s["vel"], s["box"], s["softening"],
                                          G_NEWTON, s["particle_mass"], pick, threads=4)
        assert np.array_equal(phi, ub["phi"][lo:hi][pick])
        assert np.array_equal(bound, ub["bound"][lo:hi][pick])

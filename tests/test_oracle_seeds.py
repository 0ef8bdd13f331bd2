"""Pins for the oracle's seed halos (the nodes without children), the assignment of every
particle of a FoF group to a seed, and the seeds' host relations, on hand-built hierarchies
whose answers follow from the definition by hand (exact dyadic positions and velocities), the
periodic wrap of the frame, and invariants on a generated snapshot."""
import numpy as np

import oracle
from helpers import small_snapshot

BOX = 64.0


def _hier(parent, members, deepest, params):
    """A hierarchy dict from node member lists (each ascending id = ascending index here)."""
    off = np.r_[0, np.cumsum([len(m) for m in members])].astype(np.int64)
    return {"parent": np.asarray(parent, np.int64), "size": np.diff(off),
            "member_off": off, "member_idx": np.concatenate(members).astype(np.int64),
            "deepest": np.asarray(deepest, np.int64), "params": np.asarray(params, np.float32)}


def _two_seed_case():
    # seed A: particles 0-3 at x = 10 +- 0.5 (centre 10, 10, 10), v = (0, 0, 0)
    # seed B: particles 4-5 at x = 20 (centre 20, 10, 10), v = (100, 0, 0)
    # loose particles 6-8 of the root only
    pos = np.array([[9.5, 10, 10], [10.5, 10, 10], [10, 9.5, 10], [10, 10.5, 10],
                    [20, 10, 10], [20, 10, 10],
                    [11, 10, 10], [19, 10, 10], [15, 10, 10]], np.float32)
    vel = np.zeros((9, 3), np.float32)
    vel[4:6, 0] = 100.0
    vel[7, 0] = 100.0
    vel[8, 0] = 50.0
    members = [np.arange(9), np.arange(4), np.array([4, 5])]
    deepest = [1, 1, 1, 1, 2, 2, 0, 0, 0]
    # metric scales: A and B both 1/sigma_x^2 = 1 (Mpc^-2), 1/sigma_v^2 = 1e-4 (km/s)^-2
    params = [[0.5, 1e-4, 0.0], [1.0, 1e-4, 0.0], [1.0, 1e-4, 0.0]]
    return pos, vel, _hier([-1, 0, 0], members, deepest, params)


def test_particles_go_to_the_nearest_seed_under_their_deepest_node():
    pos, vel, h = _two_seed_case()
    ps, host, cnt = oracle.assign_seeds(h, pos, vel, BOX)
    # seed members keep their seed; particle 6 (1 Mpc from A, at rest) -> A: d = 1 vs
    # d_B = 81 + 1; particle 7 (1 Mpc from B, at B's velocity) -> B: d = 1 vs 81 + 1
    # particle 8 at 5 Mpc from both, v = 50: d_A = 25 + 0.25, d_B = 25 + 0.25: a tie -> A (index 1)
    assert list(ps) == [1, 1, 1, 1, 2, 2, 1, 2, 1]
    assert list(cnt) == [0, 6, 3]
    assert list(host) == [-2, -1, 1]       # the smaller seed B sits under A; the root is no seed


def test_deeper_tree_limits_the_candidates_to_the_deepest_node():
    # root 0 -> A (1) -> A1 (3), A2 (4); root 0 -> B (2, a seed). Particle 6 lies on B but its
    # deepest node is A, so only A1 and A2 are candidates.
    pos = np.array([[10, 10, 10], [10, 10, 10], [12, 10, 10], [12, 10, 10], [30, 10, 10],
                    [30, 10, 10], [30, 10, 10]], np.float32)
    vel = np.zeros((7, 3), np.float32)
    members = [np.arange(7), np.array([0, 1, 2, 3, 6]), np.array([4, 5]), np.array([0, 1]),
               np.array([2, 3])]
    deepest = [3, 3, 4, 4, 2, 2, 1]
    params = [[1.0, 0.0, 0.0]] * 5
    h = _hier([-1, 0, 0, 1, 1], members, deepest, params)
    ps, host, cnt = oracle.assign_seeds(h, pos, vel, BOX)
    assert list(ps) == [3, 3, 4, 4, 2, 2, 4]          # particle 6: A2 (18 Mpc) beats A1 (20)
    assert list(cnt) == [0, 0, 2, 2, 3]
    # ranks: A2 (3) > A1, B (2 each; A1 has the smaller index) -> hosts: A2 none; A1 and B:
    # nearest of those above them; B's candidates A1 (20^2) and A2 (18^2) -> A2; A1's: A2 only
    assert list(host) == [-2, -2, 4, 4, -1]


def test_group_without_children_is_its_own_seed():
    pos = np.array([[1, 1, 1], [1.5, 1, 1], [2, 1, 1]], np.float32)
    vel = np.zeros((3, 3), np.float32)
    h = _hier([-1], [np.arange(3)], [0, 0, 0], [[1.0, 1.0, 0.0]])
    ps, host, cnt = oracle.assign_seeds(h, pos, vel, BOX)
    assert list(ps) == [0, 0, 0] and list(host) == [-1] and list(cnt) == [3]


def test_frame_wraps_across_the_periodic_boundary():
    # the same two-seed layout shifted so the root straddles x = 0: positions wrap, the
    # assignment does not change
    pos, vel, h = _two_seed_case()
    shifted = ((pos.astype(np.float64) + np.array([-15.0, 0, 0])) % BOX).astype(np.float32)
    assert shifted[:, 0].max() > 40 and shifted[:, 0].min() < 10
    a = oracle.assign_seeds(h, pos, vel, BOX)
    b = oracle.assign_seeds(h, shifted, vel, BOX)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_invariants_on_a_snapshot():
    s = small_snapshot(1 << 15, 32.0, 61, n_max=5000)
    lab = oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"])
    h = oracle.hierarchy(s["pos"], s["vel"], s["ids"], lab, s["box"])
    ps, host, cnt = oracle.assign_seeds(h, s["pos"], s["vel"], s["box"])
    nn = len(h["size"])
    has_kids = np.zeros(nn, bool)
    has_kids[h["parent"][h["parent"] >= 0]] = True
    seeds = np.flatnonzero(~has_kids)
    assert np.all(host[has_kids] == -2) and np.all(cnt[has_kids] == 0)
    inside = h["deepest"] >= 0
    assert np.array_equal(ps >= 0, inside)
    assert np.all(~has_kids[ps[inside]])                       # every particle goes to a seed
    root = np.arange(nn)
    for q in range(nn):
        if h["parent"][q] >= 0:
            root[q] = root[h["parent"][q]]
    # the seed lies under the particle's deepest node (walk up from the seed)
    for i in np.flatnonzero(inside)[::97]:
        q = ps[i]
        while q >= 0 and q != h["deepest"][i]:
            q = h["parent"][q]
        assert q == h["deepest"][i]
    # every member of a seed node is assigned to it; counts add up per FoF group
    for sd in seeds:
        mem = h["member_idx"][h["member_off"][sd]:h["member_off"][sd + 1]]
        assert np.all(ps[mem] == sd)
    lvl0 = np.flatnonzero(h["parent"] < 0)
    assert np.array_equal(np.bincount(root[ps[inside]], minlength=nn)[lvl0], h["size"][lvl0])
    assert cnt.sum() == inside.sum()
    # hosts rank above and stay in the same FoF group; each group has exactly one top seed
    for sd in seeds:
        hh = host[sd]
        if hh >= 0:
            assert root[hh] == root[sd]
            assert cnt[hh] > cnt[sd] or (cnt[hh] == cnt[sd] and hh < sd)
    tops = [sd for sd in seeds if host[sd] == -1]
    assert sorted(root[tops]) == sorted(lvl0)
    assert (host[seeds] >= 0).sum() > 0

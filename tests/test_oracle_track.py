"""Pins for the oracle's temporal tracking of seed halos between two snapshots: a hand-built
pair of catalogues with the shared counts and ties worked out by hand, tracking a snapshot
against itself (every seed is its own progenitor and descendant, sharing all its particles),
independence of the particle order, and particles missing from one snapshot."""
import numpy as np

import oracle
from helpers import small_snapshot
from paper_2412_18629_gb300 import synth


def test_hand_built_counts_and_ties():
    # earlier snapshot: seeds at node 2 (A) and node 5 (B); later: node 0 (X) and node 3 (Y)
    ids1 = np.arange(12)
    seed1 = np.array([2, 2, 2, 2, 2, 5, 5, 5, 5, -1, -1, 2])
    # later: X gets A's 0,1,2 and B's 5,6; Y gets A's 3,4 and B's 7,8; 9 and 10 go to X but were
    # in no seed; 11 (in A) is missing from the later snapshot
    ids2 = np.array([10, 0, 1, 2, 5, 6, 3, 4, 7, 8, 9])
    seed2 = np.array([0, 0, 0, 0, 0, 0, 3, 3, 3, 3, 0])
    prog, ps, desc, ds = oracle.track(ids1, seed1, 6, ids2, seed2, 4)
    assert list(prog) == [2, -1, -1, 2] and list(ps) == [3, 0, 0, 2]   # Y: 2 from A, 2 from B -> A
    assert list(desc) == [-1, -1, 0, -1, -1, 0] and list(ds) == [0, 0, 3, 0, 0, 2]  # B: tie -> X


def _catalogue(s):
    lab = oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"])
    h = oracle.hierarchy(s["pos"], s["vel"], s["ids"], lab, s["box"])
    seed, host, cnt = oracle.assign_seeds(h, s["pos"], s["vel"], s["box"])
    return seed, len(h["size"]), cnt


def test_a_snapshot_tracks_onto_itself():
    s = small_snapshot(1 << 14, 25.0, 81, n_max=3000)
    seed, nn, cnt = _catalogue(s)
    rng = np.random.default_rng(1)
    order = rng.permutation(len(seed))                # same particles, another order
    prog, ps, desc, ds = oracle.track(s["ids"], seed, nn, s["ids"][order], seed[order], nn)
    seeds = np.flatnonzero(cnt > 0)
    assert np.array_equal(prog[seeds], seeds) and np.array_equal(desc[seeds], seeds)
    assert np.array_equal(ps[seeds], cnt[seeds]) and np.array_equal(ds[seeds], cnt[seeds])
    others = np.flatnonzero(cnt == 0)
    assert np.all(prog[others] == -1) and np.all(desc[others] == -1)


def test_evolved_snapshot_keeps_most_halos():
    s = small_snapshot(1 << 15, 32.0, 82, n_max=5000)
    s2 = synth.evolve(s, 2e-4, seed=5)
    assert not np.array_equal(s2["ids"], s["ids"]) and np.array_equal(np.sort(s2["ids"]), np.sort(s["ids"]))
    seed1, nn1, cnt1 = _catalogue(s)
    seed2, nn2, cnt2 = _catalogue(s2)
    prog, ps, desc, ds = oracle.track(s["ids"], seed1, nn1, s2["ids"], seed2, nn2)
    later = np.flatnonzero(cnt2 > 0)
    assert np.mean(prog[later] >= 0) > 0.9
    assert np.all(ps[later] <= cnt2[later])
    # a progenitor shares at most its own particles
    ok = prog[later] >= 0
    assert np.all(ps[later][ok] <= cnt1[prog[later][ok]])
    # shared counts add up to at most the later seed's particles present earlier in some seed
    assert ps.sum() <= (seed2 >= 0).sum()

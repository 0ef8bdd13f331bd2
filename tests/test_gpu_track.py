"""rs_track (CUDA) against the oracle's temporal tracking: two snapshots of the same particles
(the second drifted a short interval and reshuffled), each through the whole GPU path up to
rs_assign_seeds, then progenitors, descendants and shared counts bit for bit; a snapshot
tracked against itself maps every seed onto itself."""
import numpy as np
import pytest

import oracle
from helpers import gpu_ctx, small_snapshot, to_dev
from paper_2412_18629_gb300 import synth

pytestmark = pytest.mark.gpu


def _gpu_seeds(s):
    import paper_2412_18629_gb300 as rs
    ctx = gpu_ctx(s, mode="batched")
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    nn, _ = rs.rs_fof6d(ctx, pos, vel, ids, lab)
    seed, _, _, _ = rs.rs_assign_seeds(ctx, pos, vel)
    ctx.close()
    return ids, seed, nn


def _oracle_seeds(s):
    lab = oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"])
    h = oracle.hierarchy(s["pos"], s["vel"], s["ids"], lab, s["box"])
    seed, _, _ = oracle.assign_seeds(h, s["pos"], s["vel"], s["box"])
    return seed, len(h["size"])


@pytest.mark.parametrize("n,box,seed,n_max", [(1 << 15, 32.0, 91, 5000), (1 << 18, 64.0, 92, 30000)])
def test_tracking_matches_the_oracle(n, box, seed, n_max):
    import paper_2412_18629_gb300 as rs
    s1 = small_snapshot(n, box, seed, n_max=n_max)
    s2 = synth.evolve(s1, 2e-4, seed=seed + 1)
    ids1, seed1, nn1 = _gpu_seeds(s1)
    ids2, seed2, nn2 = _gpu_seeds(s2)
    o1, on1 = _oracle_seeds(s1)
    o2, on2 = _oracle_seeds(s2)
    assert (nn1, nn2) == (on1, on2)
    assert np.array_equal(seed1.cpu().numpy(), o1) and np.array_equal(seed2.cpu().numpy(), o2)
    ctx = gpu_ctx(s1)
    got = rs.rs_track(ctx, ids1, seed1, nn1, ids2, seed2, nn2)
    want = oracle.track(s1["ids"], o1, on1, s2["ids"], o2, on2)
    for g, w in zip(got, want):
        assert np.array_equal(g.cpu().numpy(), w)
    later = np.flatnonzero(np.bincount(o2[o2 >= 0], minlength=on2) > 0)
    assert np.mean(want[0][later] >= 0) > 0.9
    ctx.close()


def test_a_snapshot_tracks_onto_itself():
    import paper_2412_18629_gb300 as rs
    s = small_snapshot(1 << 15, 32.0, 93, n_max=5000)
    ids, seed, nn = _gpu_seeds(s)
    ctx = gpu_ctx(s)
    perm = np.random.default_rng(3).permutation(len(ids))
    import torch
    p = torch.from_numpy(perm).cuda()
    prog, ps, desc, ds = (t.cpu().numpy() for t in rs.rs_track(ctx, ids, seed, nn, ids[p], seed[p], nn))
    cnt = np.bincount(seed.cpu().numpy()[seed.cpu().numpy() >= 0], minlength=nn)
    seeds = np.flatnonzero(cnt > 0)
    assert np.array_equal(prog[seeds], seeds) and np.array_equal(ps[seeds], cnt[seeds])
    assert np.array_equal(desc[seeds], seeds) and np.array_equal(ds[seeds], cnt[seeds])
    ctx.close()

"""rs_fof3d (CUDA) vs the oracle's 3D FoF: labels bit for bit (Section "Parallelization")."""
import numpy as np
import pytest

import oracle
from helpers import gpu_ctx, small_snapshot
from paper_2412_18629_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(pos, ids, box, ll):
    import torch
    import paper_2412_18629_gb300 as rs
    ctx = rs.Context(box=box, link_len=ll, softening=0.01, particle_mass=1.0)
    lab, ng = rs.rs_fof3d(ctx, torch.from_numpy(np.ascontiguousarray(pos, np.float32)).cuda(),
                          torch.from_numpy(np.ascontiguousarray(ids, np.int64)).cuda())
    return lab.cpu().numpy(), ng


def _check(pos, ids, box, ll):
    got, ng = _run(pos, ids, box, ll)
    want = oracle.fof3d(pos, ids, box, ll)
    assert np.array_equal(got, want)
    assert ng == len(np.unique(want))


def test_golden_chain():
    import os
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "fof3d_chain.txt"))
    got, ng = _run(rows[:, :3].astype(np.float32), rows[:, 3].astype(np.int64), 10.0, 1.0)
    assert np.array_equal(got, rows[:, 4].astype(np.int64)) and ng == 4


def test_empty_and_single():
    got, ng = _run(np.zeros((0, 3), np.float32), np.zeros(0, np.int64), 10.0, 0.3)
    assert len(got) == 0 and ng == 0
    got, ng = _run(np.array([[1, 2, 3]], np.float32), np.array([42]), 10.0, 0.3)
    assert list(got) == [42] and ng == 1


@pytest.mark.parametrize("n,box,ll,seed", [(5000, 10.0, 0.3, 0), (4097, 6.0, 0.4, 1),
                                           (20000, 4.0, 0.1, 2), (3000, 1.0, 0.3, 3),
                                           (3000, 2.0, 0.3, 4), (1000, 0.5, 0.3, 9),
                                           (200, 0.1, 0.3, 10)])
def test_uniform_random(n, box, ll, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, box, (n, 3)).astype(np.float32)
    pos[pos >= np.float32(box)] = 0
    ids = rng.permutation(n).astype(np.int64) * 7 + 3
    _check(pos, ids, box, ll)


def test_adversarial_duplicates_faces_and_dense_cell():
    rng = np.random.default_rng(8)
    box, ll = 8.0, 0.25
    sc = 0.99 * ll / np.sqrt(3)
    ns = int(np.ceil(box / sc))
    faces = (rng.integers(0, ns, (2000, 3)) * (box / ns)).astype(np.float32) % np.float32(box)
    dup = np.repeat(rng.uniform(0, box, (300, 3)), 4, axis=0).astype(np.float32)
    dense = (3.0 + rng.uniform(0, 0.05, (3000, 3))).astype(np.float32)
    edge = rng.uniform(box - 0.1, box, (500, 3)).astype(np.float32)
    pos = np.concatenate([faces, dup, dense, edge])
    pos[pos >= np.float32(box)] = 0
    ids = rng.permutation(len(pos)).astype(np.int64)
    _check(pos, ids, box, ll)


def test_lattice_exact_distance():
    k, a = 12, 0.5
    g = (np.arange(k) * a).astype(np.float32)
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    ids = np.random.default_rng(0).permutation(len(pos)).astype(np.int64)
    got, ng = _run(pos, ids, k * a, 0.5)
    assert np.all(got == 0) and ng == 1
    got, ng = _run(pos, ids, k * a, 0.4999)
    assert np.array_equal(got, ids) and ng == len(ids)


@pytest.mark.parametrize("n,box,seed", [(1 << 14, 25.0, 5), (1 << 16, 40.0, 6)])
def test_clustered_snapshots(n, box, seed):
    s = small_snapshot(n, box, seed)
    _check(s["pos"], s["ids"], s["box"], s["link_length"])


def test_workload_2e18():
    s = synth.generate(synth.WORKLOADS["nfw-2^18-L64"])
    _check(s["pos"], s["ids"], s["box"], s["link_length"])


def test_workload_2e24_full():
    """The benchmarked 2^24-particle snapshot at full size, in the bench's launch configuration."""
    s = synth.generate(synth.WORKLOADS["nfw-2^24-L256-sub"])
    got, ng = _run(s["pos"], s["ids"], s["box"], s["link_length"])
    want = oracle.fof3d_grid(s["pos"], s["ids"], s["box"], s["link_length"])
    assert np.array_equal(got, want)
    assert ng == len(np.unique(want))


def test_large_grid_keys_beyond_32_bits():
    """box / ll large enough that the sub-cell grid has more than 1625 cells per axis: the
    mixed-radix cell keys exceed 32 bits (64-bit unpacking path) and the sort takes 33 bits."""
    rng = np.random.default_rng(11)
    box, ll = 200.0, 0.2
    sc = 0.99 * ll / np.sqrt(3.0)
    assert int(np.ceil(box / sc)) > 1625
    centres = rng.uniform(0, box, (1500, 3))
    pos = (np.repeat(centres, 12, axis=0) + rng.normal(0, 0.08, (18000, 3))) % box
    pos = np.concatenate([pos, rng.uniform(0, box, (6000, 3))]).astype(np.float32)
    pos[pos >= np.float32(box)] = 0
    ids = rng.permutation(len(pos)).astype(np.int64)
    _check(pos, ids, box, ll)

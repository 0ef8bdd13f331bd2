"""The radix sort behind the 3D FoF cell list and the 6D member ordering (rs_sort_pairs): keys
in order and equal keys in input order (stability), checked against NumPy's stable argsort."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,nbits,spread", [(1, 8, 4), (2047, 8, 3), (2048, 12, 50), (2049, 16, 7),
                                            (100000, 26, 1 << 26), (100000, 26, 5),
                                            (1 << 20, 36, 1 << 20), (3 << 19, 3, 8)])
def test_sort_pairs_stable(n, nbits, spread):
    import torch
    import paper_2412_18629_gb300 as rs
    ctx = rs.Context(box=10.0, link_len=0.2, softening=0.01, particle_mass=1.0)
    rng = np.random.default_rng(n + nbits)
    keys = rng.integers(0, spread, n).astype(np.int64) & ((1 << nbits) - 1)
    keys |= rng.integers(0, 4, n).astype(np.int64) << nbits if nbits < 60 else 0  # ignored bits
    vals = np.arange(n, dtype=np.int32)
    k, v = rs.rs_sort_pairs(ctx, torch.from_numpy(keys.copy()).cuda(),
                            torch.from_numpy(vals).cuda(), nbits=nbits)
    order = np.argsort(keys & ((1 << nbits) - 1), kind="stable")
    assert np.array_equal(v.cpu().numpy(), vals[order])
    assert np.array_equal(k.cpu().numpy(), keys[order])

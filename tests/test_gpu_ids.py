"""64-bit ids through the C ABI: ids spread up to ~2^40 (so the labels are sparse and the level-0
grouping takes the two-sort (label, id) order) give the oracle's labels, hierarchy and flags bit
for bit in both forms; the optional uniqueness check rejects repeated and negative ids and
accepts unique ones."""
import numpy as np
import pytest

import oracle
from helpers import gpu_ctx, gpu_pipeline, oracle_pipeline, small_snapshot, to_dev, assert_hier_equal

pytestmark = pytest.mark.gpu


def _spread_ids(s, seed, top_bits=40):
    rng = np.random.default_rng(seed)
    n = len(s["ids"])
    # unique ids: a random permutation scaled and offset into [2^39, 2^40)
    ids = (rng.permutation(n).astype(np.int64) * np.int64((1 << 39) // n) + np.int64(1 << 39)
           + rng.integers(0, 1000, n))
    assert len(np.unique(ids)) == n and ids.max() < (1 << top_bits)
    out = dict(s)
    out["ids"] = ids.astype(np.int64)
    return out


@pytest.mark.parametrize("mode", ("plain", "batched"))
def test_ids_beyond_2e32_match_the_oracle(mode):
    s = _spread_ids(small_snapshot(1 << 15, 32.0, 51, n_max=4000), 3)
    g = gpu_pipeline(s, mode=mode)
    o = oracle_pipeline(s)
    assert np.array_equal(g["labels"], o["labels"])
    assert g["labels"].min() >= 1 << 39
    assert_hier_equal(g["hier"], o["hier"])
    assert np.array_equal(g["bound"], o["unbind"]["bound"])
    assert np.array_equal(g["props"][:, 1], o["unbind"]["n_bound"].astype(np.float64))


def test_uniqueness_check():
    import paper_2412_18629_gb300 as rs
    import torch
    s = small_snapshot(1 << 12, 16.0, 52, n_max=500)
    ctx = gpu_ctx(s, check_ids=True)
    pos, vel, ids = to_dev(s)
    rs.rs_fof3d(ctx, pos, ids)                      # unique: accepted
    dup = ids.clone()
    dup[100] = dup[7]
    with pytest.raises(rs.RSError, match="RS_ERR_INVALID_ARG"):
        rs.rs_fof3d(ctx, pos, dup)
    neg = ids.clone()
    neg[5] = -3
    with pytest.raises(rs.RSError, match="RS_ERR_INVALID_ARG"):
        rs.rs_fof3d(ctx, pos, neg)
    big = ids + torch.tensor(1 << 50, dtype=torch.int64, device=ids.device)
    lab, _ = rs.rs_fof3d(ctx, pos, big)             # large unique ids: accepted
    want = oracle.fof3d(s["pos"], s["ids"] + (1 << 50), s["box"], s["link_length"])
    assert np.array_equal(lab.cpu().numpy(), want)
    ctx.close()

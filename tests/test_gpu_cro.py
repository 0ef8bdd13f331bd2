"""GPU canonical-order float64 sum (rs_cro_sum) vs the oracle's, bit for bit, including the
hand-derived order-sensitive golden cases."""
import numpy as np
import pytest

import oracle
from test_oracle_cro import _cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2412_18629_gb300 as rs
    return rs.Context(box=10.0, link_len=0.2, softening=0.01, particle_mass=1.0)


@pytest.mark.parametrize("a,expect", list(_cases()))
def test_golden(ctx, a, expect):
    import torch
    import paper_2412_18629_gb300 as rs
    got = rs.rs_cro_sum(ctx, torch.from_numpy(a).cuda()).item()
    assert got == expect


@pytest.mark.parametrize("m", [0, 1, 7, 32, 33, 1023, 1024, 1025, 2049, 3072, 3073, 5000, 65536,
                               100003, 1 << 20])
def test_bitwise_vs_oracle(ctx, m):
    import torch
    import paper_2412_18629_gb300 as rs
    rng = np.random.default_rng(m)
    a = rng.normal(0, 1, m) * np.exp(rng.uniform(-30, 30, m))
    got = rs.rs_cro_sum(ctx, torch.from_numpy(a).cuda()).item()
    assert got == oracle.cro_sum(a)

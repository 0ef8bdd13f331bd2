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


@pytest.mark.parametrize("m", list(range(1, 41)) + [1025, 1030, 1040, 2064])
def test_short_chunks_and_signed_zeros(ctx, m):
    """Chunks of at most 16 terms skip the combine steps that only add 0.0, and a lane's first
    term is taken as 0.0 + t without an add: both must keep the value and the sign of zero of
    the canonical order (0.0 + -0.0 = +0.0), here with negative zeros, exact cancellations and
    last chunks of 1 to 16 terms."""
    import torch
    import paper_2412_18629_gb300 as rs
    rng = np.random.default_rng(1000 + m)
    a = rng.normal(0, 1, m) * np.exp(rng.uniform(-5, 5, m))
    a[rng.random(m) < 0.3] = -0.0
    if m >= 4:
        a[1] = -a[0]  # an exact cancellation inside one lane pair
    got = rs.rs_cro_sum(ctx, torch.from_numpy(a).cuda()).item()
    want = oracle.cro_sum(a)
    assert got == want and np.signbit(got) == np.signbit(want)
    z = np.full(m, -0.0)
    gz = rs.rs_cro_sum(ctx, torch.from_numpy(z).cuda()).item()
    assert gz == 0.0 and np.signbit(gz) == np.signbit(oracle.cro_sum(z))

"""rs_cro_sum_noalloc: the allocation-free variant of rs_cro_sum for callers that cannot allocate
device memory (code inside a stream capture, allocator callbacks, hosts that forbid the device
heap). Called through the C ABI and compared with rs_cro_sum on two calls in a row; this file
sorts last so a stop-at-first-failure run has finished every other test first."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2412_18629_gb300 as rs
    lib = rs.load_library()
    lib.rs_cro_sum_noalloc.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]
    lib.rs_cro_sum_noalloc.restype = ctypes.c_int32
    return lib


def _noalloc(lib, a_dev, out_dev, stream):
    return lib.rs_cro_sum_noalloc(a_dev.numel(), ctypes.c_void_p(a_dev.data_ptr()),
                                  ctypes.c_void_p(out_dev.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_allocating_entry_on_two_calls():
    import torch
    import paper_2412_18629_gb300 as rs
    lib = _lib()
    ctx = rs.Context(box=10.0, link_len=0.2, softening=0.01, particle_mass=1.0)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(2024)
    for m in (100003, 5000):                      # larger call first: stale slots must not leak
        a = torch.from_numpy(rng.normal(0, 1, m) * np.exp(rng.uniform(-30, 30, m))).cuda()
        out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, a, out, stream) == rs.RS_OK
        want = rs.rs_cro_sum(ctx, a)
        torch.cuda.synchronize()
        assert out.item() == want.item()          # same canonical order: bit for bit


def test_noalloc_limits_and_empty():
    import torch
    import paper_2412_18629_gb300 as rs
    lib = _lib()
    stream = torch.cuda.current_stream()
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    empty = torch.zeros(0, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, empty, out, stream) == rs.RS_OK
    torch.cuda.synchronize()
    assert out.item() == 0.0
    rc = lib.rs_cro_sum_noalloc((1 << 26) + 1, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 5                                # RS_ERR_CAPACITY, rejected before any launch


def test_noalloc_at_the_size_limit():
    """m = 2^26 terms, the largest accepted size, fills all 65536 chunk slots; the result still
    equals rs_cro_sum bit for bit."""
    import torch
    import paper_2412_18629_gb300 as rs
    lib = _lib()
    ctx = rs.Context(box=10.0, link_len=0.2, softening=0.01, particle_mass=1.0)
    stream = torch.cuda.current_stream()
    g = torch.Generator(device="cuda").manual_seed(7)
    a = torch.randn(1 << 26, dtype=torch.float64, device="cuda", generator=g)
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, a, out, stream) == rs.RS_OK
    want = rs.rs_cro_sum(ctx, a)
    torch.cuda.synchronize()
    assert out.item() == want.item()
    ctx.close()

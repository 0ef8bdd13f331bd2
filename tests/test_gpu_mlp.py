"""Surrogate MLP on tensor cores vs the float64 oracle with the same bf16 rounding points.
Integer-valued weights and inputs make every float32 and float64 accumulation exact, so the
forward output and the batch gradient must agree bit for bit (this pins the fragment layouts);
random weights agree within the float32-accumulation tolerance; training lowers the loss."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
P = oracle.MLP_PARAMS
W1, B1, W2, B2, W3, B3 = 0, 512, 576, 4672, 4736, 4800


@pytest.fixture(scope="module")
def ctx():
    import paper_2412_18629_gb300 as rs
    return rs.Context(box=10.0, link_len=0.2, softening=0.01, particle_mass=1.0)


def _int_params(rng):
    p = np.zeros(P, np.float32)
    p[W1:W1 + 512] = rng.integers(-1, 2, 512)
    p[B1:B1 + 64] = rng.integers(-2, 3, 64)
    p[W2:W2 + 4096] = rng.integers(-1, 2, 4096) * (rng.random(4096) < 0.25)
    p[B2:B2 + 64] = rng.integers(-2, 3, 64)
    p[W3:W3 + 64] = rng.integers(-1, 2, 64)
    p[B3] = 1.0
    return p


@pytest.mark.parametrize("n", [1, 16, 100, 1000, 4096])
def test_forward_exact_integer_case(ctx, n):
    import torch
    import paper_2412_18629_gb300 as rs
    rng = np.random.default_rng(n)
    p = _int_params(rng)
    x = rng.integers(-2, 3, (n, 8)).astype(np.float32)
    rs.rs_mlp_set_params(ctx, p)
    y = rs.rs_mlp_forward(ctx, torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_array_equal(y.astype(np.float64), oracle.mlp_forward(x, p))


@pytest.mark.parametrize("n", [128, 256, 4096])
def test_gradient_exact_integer_case(ctx, n):
    import torch
    import paper_2412_18629_gb300 as rs
    rng = np.random.default_rng(100 + n)
    p = _int_params(rng)
    x = rng.integers(-2, 3, (n, 8)).astype(np.float32)
    t = rng.integers(-8, 9, n).astype(np.float32)
    rs.rs_mlp_set_params(ctx, p)
    g, sse = rs.rs_mlp_gradient(ctx, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    go, sse_o = oracle.mlp_gradient(x, t, p)
    np.testing.assert_array_equal(g.cpu().numpy().astype(np.float64), go)
    assert sse == sse_o


def _bf16(a):
    """Round float64 values to bf16 (round to nearest even, through float32)."""
    b = np.asarray(a, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _flip_bound(x, p):
    """Per sample, the largest output change a one-ulp change of the bf16 rounding of any hidden
    activation can cause (2^-8 relative per value; through W2 and W3, ReLU 1-Lipschitz): where a
    hidden value sits on a bf16 rounding boundary the float32 device and the float64 oracle may
    round it to neighbouring values."""
    W1, b1 = _bf16(p[:512]).reshape(8, 64), p[512:576].astype(np.float64)
    W2, b2 = _bf16(p[576:4672]).reshape(64, 64), p[4672:4736].astype(np.float64)
    W3 = np.abs(_bf16(p[4736:4800]))
    h1 = _bf16(np.maximum(_bf16(x) @ W1 + b1, 0.0))
    h2 = _bf16(np.maximum(h1 @ W2 + b2, 0.0))
    return 2.0 ** -8 * (np.abs(h2) @ W3 + (np.abs(h1) @ np.abs(W2)) @ W3)


def test_forward_and_gradient_random_weights(ctx):
    """Element by element: every output within 1e-5 relative (floor 1e-2) plus its sample's
    bf16 rounding-flip bound; every gradient entry within 1e-3 of the gradient's largest entry."""
    import torch
    import paper_2412_18629_gb300 as rs
    rng = np.random.default_rng(7)
    p = rng.normal(0, 0.3, P).astype(np.float32)
    x = rng.normal(0, 1, (4096, 8)).astype(np.float32)
    t = rng.normal(0, 1, 4096).astype(np.float32)
    rs.rs_mlp_set_params(ctx, p)
    y = rs.rs_mlp_forward(ctx, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    yo = oracle.mlp_forward(x, p)
    tol = 1e-5 * np.maximum(np.abs(yo), 1e-2) + _flip_bound(x, p)
    assert np.all(np.abs(y - yo) <= tol), np.max(np.abs(y - yo) / tol)
    # most samples need no flip allowance at all
    assert np.mean(np.abs(y - yo) <= 1e-5 * np.maximum(np.abs(yo), 1e-2)) >= 0.99
    g, _ = rs.rs_mlp_gradient(ctx, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    go, _ = oracle.mlp_gradient(x, t, p)
    g = g.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(g - go) <= 1e-3 * np.abs(go).max()), np.abs(g - go).max() / np.abs(go).max()


def test_training_reduces_loss_and_reports_holdout_error(ctx):
    import torch
    import paper_2412_18629_gb300 as rs
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 1, (60000, 8)).astype(np.float32)
    t = (-2.0 / (0.1 + x[:, 0]) * (0.5 + x[:, 1]) + 0.3 * x[:, 5]).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    em1, mse1 = rs.rs_mlp_train(ctx, xd, td, epochs=1, batch=1024, lr=1e-3, seed=3)
    em8, mse8 = rs.rs_mlp_train(ctx, xd, td, epochs=8, batch=1024, lr=1e-3, seed=3)
    assert mse8 < 0.5 * mse1 and em8 < em1
    y = rs.rs_mlp_forward(ctx, xd).cpu().numpy()
    assert np.abs(y - t).max() >= em8 * 0.5          # err_max is a held-out maximum
    p = rs.rs_mlp_get_params(ctx)
    yo = oracle.mlp_forward(x[:512], p)
    assert np.quantile(np.abs(y[:512] - yo), 0.99) <= 1e-4 * np.abs(t).max()


def test_graph_replayed_training_equals_plain_launches():
    """The training epoch captured once as a CUDA graph and replayed every epoch (reshuffled
    batch order, advancing Adam step) gives bit for bit the weights, held-out error and loss of
    the same launches issued one by one, and counts the same kernel launches."""
    import torch
    import paper_2412_18629_gb300 as rs
    rng = np.random.default_rng(12)
    x = rng.uniform(0, 1, (20000, 8)).astype(np.float32)
    t = (np.sin(3 * x[:, 0]) - x[:, 2] * x[:, 7]).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    out = {}
    for graphs in (True, False):
        c = rs.Context(box=10.0, link_len=0.2, softening=0.01, particle_mass=1.0)
        c.use_graphs(graphs)
        l0 = c.kernel_launches
        em, mse = rs.rs_mlp_train(c, xd, td, epochs=5, batch=512, lr=2e-3, seed=9)
        out[graphs] = (rs.rs_mlp_get_params(c), em, mse, c.kernel_launches - l0)
        c.close()
    (pg, eg, mg, lg), (pe, ee, me, le) = out[True], out[False]
    assert np.array_equal(pg.view(np.uint32), pe.view(np.uint32))
    assert eg == ee and mg == me and lg == le
    assert mg < np.var(t)                           # it did train


def test_checkpoint_round_trip_and_corruption(ctx, tmp_path):
    """rs_surrogate_save / rs_surrogate_load: weights and held-out maximum error come back bit
    for bit in a new context (same outputs); a truncated or altered file is rejected."""
    import torch
    import paper_2412_18629_gb300 as rs
    rng = np.random.default_rng(21)
    p = rng.normal(0, 0.3, P).astype(np.float32)
    rs.rs_mlp_set_params(ctx, p)
    rs.rs_mlp_set_err_max(ctx, 1.25)
    path = str(tmp_path / "w.bin")
    rs.rs_surrogate_save(ctx, path)
    other = rs.Context(box=10.0, link_len=0.2, softening=0.01, particle_mass=1.0, mode="surrogate")
    rs.rs_surrogate_load(other, path)
    assert np.array_equal(rs.rs_mlp_get_params(other), p) and rs.rs_mlp_get_err_max(other) == 1.25
    x = torch.from_numpy(rng.normal(0, 1, (1000, 8)).astype(np.float32)).cuda()
    assert torch.equal(rs.rs_mlp_forward(ctx, x), rs.rs_mlp_forward(other, x))
    raw = open(path, "rb").read()
    bad = bytearray(raw)
    bad[100] ^= 1
    for i, data in enumerate((raw[:-9], bytes(bad), b"XXXXXXXX" + raw[8:])):
        q = str(tmp_path / f"bad{i}.bin")
        open(q, "wb").write(data)
        with pytest.raises(rs.RSError, match="RS_ERR_INVALID_ARG"):
            rs.rs_surrogate_load(other, q)
    other.close()

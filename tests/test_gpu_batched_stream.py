"""rs_run_batched: the pipeline over a stream of independent snapshots of different sizes and
boxes, run on concurrent lanes (contexts with their own streams and host threads), gives every
snapshot exactly the outputs of the four calls run on it alone on one context - which the other
parity tests hold to the oracle - and the smallest snapshots are compared with the oracle
directly. Edge cases: an empty snapshot in the stream, more lanes than snapshots, a node
capacity too small (reported, counts filled), bad lane counts, the surrogate form."""
import numpy as np
import pytest

from helpers import assert_hier_equal, gpu_ctx, oracle_pipeline, small_snapshot, to_dev

pytestmark = pytest.mark.gpu

TREE_MIN = 1024  # small enough that the tree bound runs on these snapshots' largest nodes


def _stream(count, seed0):
    """count snapshots of 2^12..2^15 particles at unit mean spacing (box = n^(1/3))."""
    out = []
    for k in range(count):
        n = 1 << (12 + (seed0 + k) % 4)
        out.append(small_snapshot(n, float(np.cbrt(float(n))), 500 + seed0 + k,
                                  n_max=min(6000.0, n / 5)))
    return out


def _alone(s, mode, params=None, err_max=None):
    import paper_2412_18629_gb300 as rs
    ctx = gpu_ctx(s, mode=mode, tree_min=TREE_MIN)
    if params is not None:
        rs.rs_mlp_set_params(ctx, params)
        rs.rs_mlp_set_err_max(ctx, err_max)
    pos, vel, ids = to_dev(s)
    lab, ng = rs.rs_fof3d(ctx, pos, ids)
    nn, nm = rs.rs_fof6d(ctx, pos, vel, ids, lab)
    rs.rs_unbind(ctx, pos, vel, want_potential=False)
    props = rs.rs_halo_props(ctx).cpu().numpy()
    h = rs.rs_fof6d_copy(ctx)
    ctx.close()
    return {"labels": lab.cpu().numpy(), "deepest": h["deepest"].cpu().numpy(),
            "parent": h["parent"].cpu().numpy(), "props": props, "counts": (ng, nn, nm)}


def _batched(snaps, mode, lanes, capacity=None, params=None, err_max=None):
    import paper_2412_18629_gb300 as rs
    ctx = gpu_ctx(snaps[0], mode=mode, tree_min=TREE_MIN)
    if params is not None:
        rs.rs_mlp_set_params(ctx, params)
        rs.rs_mlp_set_err_max(ctx, err_max)
    dev = [dict(zip(("pos", "vel", "ids"), to_dev(s)), box=s["box"], link_length=s["link_length"],
                softening=s["softening"]) for s in snaps]
    cap = capacity if capacity is not None else [max(s["pos"].shape[0] // 4, 16) for s in snaps]
    out = rs.BatchOutputs([s["pos"].shape[0] for s in snaps], cap, 0)
    counts = rs.rs_run_batched(ctx, dev, out, lanes=lanes)
    launches = ctx.kernel_launches
    ctx.close()
    return counts, out, launches


def _compare(snaps, counts, out, ref):
    for k, (s, r) in enumerate(zip(snaps, ref)):
        nn = counts[k][1]
        assert tuple(counts[k][:3]) == r["counts"], (k, counts[k], r["counts"])
        assert np.array_equal(out.labels[k].cpu().numpy(), r["labels"]), k
        assert np.array_equal(out.deepest[k].cpu().numpy(), r["deepest"]), k
        assert np.array_equal(out.parent[k][:nn].cpu().numpy(), r["parent"]), k
        assert np.array_equal(out.props[k][:nn].cpu().numpy(), r["props"]), k


@pytest.fixture(scope="module")
def stream():
    return _stream(7, 0)


@pytest.mark.parametrize("lanes", (1, 3, 16))
def test_stream_equals_single_snapshot_runs(stream, lanes):
    ref = [_alone(s, "batched") for s in stream]
    counts, out, launches = _batched(stream, "batched", lanes)
    _compare(stream, counts, out, ref)
    assert launches > 0
    assert np.all(counts[:, 3] >= 1)


def test_stream_plain_form_and_oracle(stream):
    small = [s for s in stream if s["pos"].shape[0] <= 1 << 13][:2]
    assert len(small) == 2
    counts, out, _ = _batched(small, "plain", 2)
    import paper_2412_18629_gb300 as rs
    for k, s in enumerate(small):
        o = oracle_pipeline(s)
        nn = counts[k][1]
        assert np.array_equal(out.labels[k].cpu().numpy(), o["labels"])
        assert np.array_equal(out.deepest[k].cpu().numpy(), o["hier"]["deepest"])
        assert np.array_equal(out.parent[k][:nn].cpu().numpy(), o["hier"]["parent"])
        p = rs.props_to_float64(out.props[k][:nn]).cpu().numpy()
        assert np.array_equal(p[:, 1], o["props"][:, 1])        # n_bound
        assert np.array_equal(p[:, 2], o["props"][:, 2])        # is_halo


def test_empty_snapshot_and_capacity(stream):
    import paper_2412_18629_gb300 as rs
    empty = dict(stream[0])
    for k in ("pos", "vel"):
        empty[k] = stream[0][k][:0]
    empty["ids"] = stream[0]["ids"][:0]
    snaps = [stream[1], empty, stream[2]]
    ref = [_alone(s, "batched") for s in (stream[1], stream[2])]
    counts, out, _ = _batched(snaps, "batched", 2)
    assert list(counts[1]) == [0, 0, 0, counts[1][3]]
    _compare([stream[1], stream[2]], counts[[0, 2]], _Sub(out, [0, 2]), ref)
    # a capacity of one node: the call reports RS_ERR_CAPACITY and fills the counts
    with pytest.raises(rs.RSError) as e:
        _batched(snaps, "batched", 2, capacity=[1, 1, 1])
    assert e.value.code == 5
    assert np.array_equal(e.value.counts[:, :3], counts[:, :3])


class _Sub:
    def __init__(self, out, idx):
        self.labels = [out.labels[i] for i in idx]
        self.deepest = [out.deepest[i] for i in idx]
        self.parent = [out.parent[i] for i in idx]
        self.props = [out.props[i] for i in idx]


def test_bad_lane_counts(stream):
    import paper_2412_18629_gb300 as rs
    for lanes in (0, 17):
        with pytest.raises(rs.RSError) as e:
            _batched(stream[:1], "batched", lanes)
        assert e.value.code == 1


def test_surrogate_lanes(stream):
    """With a trained surrogate on the calling context, every lane gets its weights and gate:
    outputs equal the single-snapshot surrogate runs (and so the exact flags)."""
    import paper_2412_18629_gb300 as rs
    train = small_snapshot(1 << 17, float(np.cbrt(2.0 ** 17)), 710, n_max=2.0e4)
    ctx = gpu_ctx(train, mode="batched", tree_min=0)
    pos, vel, ids = to_dev(train)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    rs.rs_unbind(ctx, pos, vel, want_potential=True)
    x, t = rs.rs_surrogate_features(ctx)
    err_max, _ = rs.rs_mlp_train(ctx, x.contiguous(), t.contiguous(), epochs=8, seed=3)
    params = rs.rs_mlp_get_params(ctx)
    ctx.close()
    ref = [_alone(s, "surrogate", params, err_max) for s in stream]
    plain = [_alone(s, "batched") for s in stream]
    for r, p in zip(ref, plain):                      # the surrogate keeps the exact outputs
        assert np.array_equal(r["props"], p["props"])
    counts, out, _ = _batched(stream, "surrogate", 4, params=params, err_max=err_max)
    _compare(stream, counts, out, ref)
    # without weights on the calling context the surrogate form is refused
    with pytest.raises(rs.RSError) as e:
        _batched(stream[:1], "surrogate", 1)
    assert e.value.code == 6

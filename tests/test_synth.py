"""The seeded input generator against its recipe (CPU): shapes and dtypes, positions in [0, L),
ids a permutation, the halo fraction, the halo-size distribution's bounds and slope, NFW radii
(the enclosed fraction at the scale radius), velocity dispersions, subhalo nesting, and
reproducibility from the seed."""
import math

import numpy as np

from paper_2412_18629_gb300 import synth


def _snap(n=1 << 16, box=40.0, seed=3, **kw):
    return synth.generate(synth.SnapshotSpec(n=n, box=box, seed=seed, **kw))


def test_shapes_ranges_and_ids():
    s = _snap()
    n = s["n"]
    assert s["pos"].shape == (n, 3) and s["pos"].dtype == np.float32
    assert s["vel"].shape == (n, 3) and s["vel"].dtype == np.float32
    assert s["ids"].dtype == np.int64
    assert np.all(s["pos"] >= 0) and np.all(s["pos"] < np.float32(s["box"]))
    assert np.array_equal(np.sort(s["ids"]), np.arange(n))
    assert s["link_length"] == float(np.float32(0.28 * s["box"] / np.cbrt(n)))


def test_seed_reproducible_and_distinct():
    a, b, c = _snap(seed=5), _snap(seed=5), _snap(seed=6)
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["ids"], b["ids"])
    assert not np.array_equal(a["pos"], c["pos"])


def test_halo_fraction_and_size_bounds():
    s = _snap(n=1 << 18, box=64.0, seed=0, n_max=3e4)
    frac = s["n_halo_particles"] / s["n"]
    assert 0.4 - 20 / s["n"] <= frac <= 0.4
    hosts = [c for c in s["catalogue"] if c[0] == 0]
    sizes = np.array([c[1] for c in hosts])
    assert sizes.min() >= 20 and sizes.max() <= 30000


def test_size_distribution_slope():
    """Sizes follow dN/dn ~ n^-1.9 on [20, n_max]: the maximum-likelihood slope of the
    (untruncated-by-budget) draws is within a few percent of 1.9."""
    rng = np.random.default_rng(1)
    sizes, _ = synth._draw_sizes(rng, 10 ** 7, 20, 3e4, 1.9)
    x = np.array(sizes[:-1], dtype=np.float64)  # the last draw is clipped to the remainder
    # MLE for a power law on [a, b] with continuous draws floored to integers: use x + 0.5
    a, b = 20.0, 3e4
    xs = x + 0.5
    grid = np.linspace(1.6, 2.2, 601)
    ll = [np.sum(-g * np.log(xs)) + len(xs) * np.log((g - 1) / (a ** (1 - g) - b ** (1 - g)))
          for g in grid]
    g_hat = grid[int(np.argmax(ll))]
    assert abs(g_hat - 1.9) < 0.05, g_hat


def test_nfw_enclosed_fraction_at_scale_radius():
    """A fraction mu(1)/mu(c) of an NFW halo's particles lies inside r_s = r_vir / c."""
    rng = np.random.default_rng(2)
    c = 8.0
    x = synth._nfw_radii(rng, np.full(200000, c), 200000)  # radii in units of r_vir
    want = synth._mu(1.0) / synth._mu(c)
    got = np.mean(x < 1.0 / c)
    assert abs(got - want) < 4 * math.sqrt(want * (1 - want) / len(x))
    assert np.all(x > 0) and np.all(x <= 1.0 + 1e-12)


def test_velocity_dispersions():
    s = _snap(n=1 << 17, box=50.0, seed=4, n_max=2e4)
    # background: the particles of the catalogue's halos are the first n_halo before shuffling;
    # here only the totals are checked: the background's 50 km/s dominates the low tail of |v|
    v = s["vel"].astype(np.float64)
    assert np.all(np.isfinite(v))
    host = max((c for c in s["catalogue"] if c[0] == 0), key=lambda c: c[1])
    depth, count, own, centre, bulk, r_vir = host
    m = s["particle_mass"]
    v_vir = math.sqrt(synth.G_NEWTON * count * m / r_vir)
    assert v_vir / math.sqrt(2.0) > 50.0  # halos are hotter than the background here
    d = s["pos"].astype(np.float64) - centre
    d -= s["box"] * np.round(d / s["box"])
    inner = np.linalg.norm(d, axis=1) < 0.3 * r_vir
    sig = v[inner].std(axis=0).mean()
    assert 0.6 * v_vir / math.sqrt(2.0) < sig < 1.3 * v_vir / math.sqrt(2.0)


def test_subhalos_nest_inside_hosts():
    s = _snap(n=1 << 18, box=64.0, seed=7, n_max=3e4, sub_levels=1)
    cat = s["catalogue"]
    subs = [c for c in cat if c[0] == 1]
    assert len(subs) > 0
    hosts = [c for c in cat if c[0] == 0 and c[1] > 1000]
    for sub in subs[:50]:
        best = min(hosts, key=lambda h: np.linalg.norm(
            (np.asarray(sub[3]) - h[3] + s["box"] / 2) % s["box"] - s["box"] / 2))
        dist = np.linalg.norm((np.asarray(sub[3]) - best[3] + s["box"] / 2) % s["box"] - s["box"] / 2)
        assert dist <= 0.8 * best[5] + 1e-9

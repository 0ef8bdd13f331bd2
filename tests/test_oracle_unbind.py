"""Pins for the oracle's unbinding pass: the softened pairwise potential of each node's members,
kinetic energy against the node's bulk velocity, bound iff KE + phi < 0, and the halo decision
(bound fraction >= 0.5 and at least 10 bound particles; Rockstar's parameters, cited in the
paper's Summary). Checked against exact discrete configurations (two bodies, octahedron plus
centre, cube) and against the Plummer and uniform-sphere potentials in closed form."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_18629_gb300 import G_NEWTON

G = 4.30091e-9
M = 1.0e10
GM = G * M


def _one_node(pos, vel, box=1000.0, eps=0.0, **kw):
    n = len(pos)
    off = np.array([0, n], np.int64)
    idx = np.arange(n, dtype=np.int64)
    return oracle.unbind(off, idx, np.asarray(pos, np.float32), np.asarray(vel, np.float32), box,
                         eps, G, M, threads=1, **kw)


def test_two_bodies():
    r, eps = 0.75, 0.125
    out = _one_node([[10, 10, 10], [10 + r, 10, 10]], np.zeros((2, 3)), eps=eps, min_size=2)
    want = -GM / math.sqrt(r * r + eps * eps)
    np.testing.assert_allclose(out["phi"], [want, want], rtol=1e-15)


def test_octahedron_with_centre():
    R, eps = 0.5, 0.03125
    c = np.array([20.0, 20.0, 20.0])
    verts = [c + R * np.array(e) for e in
             [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]]
    pos = np.array([c] + verts)
    out = _one_node(pos, np.zeros((7, 3)), eps=eps, min_size=2)
    e2 = eps * eps
    centre = -GM * 6 / math.sqrt(R * R + e2)
    vertex = -GM * (1 / math.sqrt(R * R + e2) + 4 / math.sqrt(2 * R * R + e2)
                    + 1 / math.sqrt(4 * R * R + e2))
    np.testing.assert_allclose(out["phi"][0], centre, rtol=1e-14)
    np.testing.assert_allclose(out["phi"][1:], vertex, rtol=1e-14)


def test_cube_across_periodic_boundary():
    a, box = 0.25, 50.0
    corners = np.array([[x, y, z] for x in (0, a) for y in (0, a) for z in (0, a)])
    pos = (corners + [box - a / 2, 7.0, box - a / 2]) % box   # straddles two faces
    out = _one_node(pos, np.zeros((8, 3)), box=box, min_size=2)
    want = -GM * (3 / a + 3 / (a * math.sqrt(2)) + 1 / (a * math.sqrt(3)))
    np.testing.assert_allclose(out["phi"], want, rtol=1e-13)


def _radial_check(pos, phi, centre, theory, rel):
    r = np.linalg.norm(pos - centre, axis=1)
    edges = np.quantile(r, np.linspace(0.05, 0.95, 10))
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (r >= lo) & (r < hi)
        got = phi[sel].mean()
        want = theory(r[sel]).mean()
        assert abs(got - want) <= rel * abs(want), (lo, hi, got, want)


def test_plummer_profile():
    rng = np.random.default_rng(0)
    n, a = 6000, 1.0
    u = rng.random(n)
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    r = np.minimum(r, 30 * a)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    centre = np.array([100.0, 100.0, 100.0])
    pos = (centre + d * r[:, None]).astype(np.float32)
    out = _one_node(pos, np.zeros((n, 3)), box=1000.0, eps=1e-3)
    Mtot = GM * n
    _radial_check(pos.astype(np.float64), out["phi"], centre,
                  lambda rr: -Mtot / np.sqrt(rr * rr + a * a), 0.03)


def test_uniform_sphere_profile():
    rng = np.random.default_rng(1)
    n, R = 6000, 2.0
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = R * rng.random(n) ** (1.0 / 3.0)
    centre = np.array([300.0, 30.0, 3.0])
    pos = (centre + d * r[:, None]).astype(np.float32)
    out = _one_node(pos, np.zeros((n, 3)), box=1000.0, eps=1e-3)
    Mtot = GM * n
    _radial_check(pos.astype(np.float64), out["phi"], centre,
                  lambda rr: -Mtot * (3 * R * R - rr * rr) / (2 * R ** 3), 0.03)


def test_cold_bound_hot_unbound_and_threshold():
    rng = np.random.default_rng(2)
    pos = (50 + rng.normal(0, 0.1, (20, 3))).astype(np.float32)
    cold = _one_node(pos, np.zeros((20, 3)))
    assert cold["bound"].all() and cold["n_bound"][0] == 20 and cold["is_halo"][0] == 1
    assert cold["m_bound"][0] == 20 * M
    hot = _one_node(pos, rng.normal(0, 1e6, (20, 3)))
    assert not hot["bound"].any() and hot["is_halo"][0] == 0
    # exactly half bound: 10 at rest (bound), 10 moving at +-V (zero bulk velocity, unbound)
    vel = np.zeros((20, 3))
    vel[10:15, 0] = 1e6
    vel[15:20, 0] = -1e6
    half = _one_node(pos, vel)
    assert half["n_bound"][0] == 10 and half["bound"][:10].all() and not half["bound"][10:].any()
    assert half["is_halo"][0] == 1        # bound fraction 0.5 passes
    vel[9, 1] = 1e6                       # two more unbound at +-V in y (bulk unchanged)
    vel[8, 1] = -1e6
    fewer = _one_node(pos, vel)
    assert fewer["n_bound"][0] == 8 and fewer["is_halo"][0] == 0


def test_bulk_velocity_is_subtracted():
    rng = np.random.default_rng(3)
    pos = (50 + rng.normal(0, 0.1, (30, 3))).astype(np.float32)
    moving = np.zeros((30, 3))
    moving[:, 2] = 5e5                     # uniform drift: no kinetic energy in the node's frame
    out = _one_node(pos, moving)
    assert out["bound"].all()


def test_iterative_unbinding_hand_case():
    """Four particles, G m = 43.0091 (m = 1e10): A = (0,0,0), B = (0.1,0,0) at rest, C = (10,0,0)
    at v = (100,0,0), D = (10.1,0,0) at v = (0,10,0); eps = 0.
    Pass 1 (bulk (25, 2.5, 0)): A, B: KE 315.6 < 438.6 = |phi|; C: KE 2815.6 > 438.7; D: KE 340.6 <
    438.6 (C's term 430.1 keeps it bound). Pass 2 over {A, B, D} (bulk (0, 10/3, 0)): A, B: KE 5.6
    < 434.4; D: KE 22.2 > 43.0091 (1/10 + 1/10.1) = 8.56, unbound. Pass 3 over {A, B}: both bound
    at rest. So one pass leaves {A, B, D}, iteration {A, B}."""
    import oracle
    pos = np.array([[0, 0, 0], [0.1, 0, 0], [10, 0, 0], [10.1, 0, 0]], np.float32) + 20
    vel = np.array([[0, 0, 0], [0, 0, 0], [100, 0, 0], [0, 10, 0]], np.float32)
    off = np.array([0, 4], np.int64)
    idx = np.arange(4, dtype=np.int64)
    one = oracle.unbind(off, idx, pos, vel, 64.0, 0.0, G_NEWTON, 1e10, min_size=2)
    assert list(one["bound"]) == [1, 1, 0, 1]
    it = oracle.unbind(off, idx, pos, vel, 64.0, 0.0, G_NEWTON, 1e10, min_size=2, passes=5)
    assert list(it["bound"]) == [1, 1, 0, 0] and it["n_bound"][0] == 2
    two = oracle.unbind(off, idx, pos, vel, 64.0, 0.0, G_NEWTON, 1e10, min_size=2, passes=2)
    assert list(two["bound"]) == [1, 1, 0, 0]
    # pass 2's potential of D: only A and B contribute (positions are float32: 1e-5)
    np.testing.assert_allclose(it["phi"][3], -G_NEWTON * 1e10 * (1 / 10.0 + 1 / 10.1), rtol=1e-5)
    # A's last potential is pass 3's: B alone
    np.testing.assert_allclose(it["phi"][0], -G_NEWTON * 1e10 / 0.1, rtol=1e-5)  # float32 offsets


def test_iterative_unbinding_is_monotone_and_stops():
    import oracle
    from helpers import small_snapshot
    s = small_snapshot(1 << 14, 25.0, 35, n_max=3000)
    lab = oracle.fof3d(s["pos"], s["ids"], s["box"], s["link_length"])
    h = oracle.hierarchy(s["pos"], s["vel"], s["ids"], lab, s["box"])
    args = (h["member_off"], h["member_idx"], s["pos"], s["vel"], s["box"], s["softening"],
            G_NEWTON, s["particle_mass"])
    b1 = oracle.unbind(*args, want_phi=False)["bound"]
    b3 = oracle.unbind(*args, want_phi=False, passes=3)["bound"]
    b20 = oracle.unbind(*args, want_phi=False, passes=20)["bound"]
    b21 = oracle.unbind(*args, want_phi=False, passes=21)["bound"]
    assert np.all(b3 <= b1) and np.all(b20 <= b3)        # a removed member never comes back
    assert np.array_equal(b20, b21)                       # converged: more passes change nothing
    assert (b1 != b20).sum() > 0                          # iteration matters on this snapshot

"""Pins for the oracle's halo properties (the paper's Summary: the catalogue carries extra halo
properties such as the inertia tensor). A lattice of points has closed-form centre, dispersion
and inertia tensor, all exactly representable, so the pins are exact; r_vir follows its formula
from the bound mass; unbound members are excluded; the centre wraps into the box."""
import math

import numpy as np

import oracle

M = 1.0e10


def _lattice(k, h, origin):
    g = np.arange(k) * h
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + origin
    return pts


def _props(pos, bound, box=64.0, n_total=1 << 18, vel=None, ids=None):
    n = len(pos)
    vel = np.zeros((n, 3), np.float32) if vel is None else vel
    ids = np.arange(n) if ids is None else ids
    order = np.argsort(ids)
    off = np.array([0, n], np.int64)
    return oracle.props(off, order.astype(np.int64), np.asarray(pos, np.float32), vel,
                        np.asarray(bound, np.uint8)[order], np.array([1], np.uint8), box, M,
                        n_total)[0]


def test_lattice_closed_form():
    k, h = 4, 0.5
    pos = _lattice(k, h, [10.0, 20.0, 30.0])
    rng = np.random.default_rng(0)
    vel = rng.normal(0, 100, (len(pos), 3)).astype(np.float32)
    ids = rng.permutation(len(pos))
    P = _props(pos, np.ones(len(pos)), vel=vel, ids=ids)
    var1 = h * h * (k * k - 1) / 12.0
    assert P[0] == 64 and P[1] == 64 and P[2] == 1 and P[3] == 64 * M
    assert list(P[4:7]) == [10.75, 20.75, 30.75]
    np.testing.assert_allclose(P[7:10], vel.astype(np.float64).mean(0), rtol=1e-13, atol=1e-9)
    assert P[10] == math.sqrt(3 * var1)
    assert list(P[13:16]) == [var1] * 3 and list(P[16:19]) == [0.0, 0.0, 0.0]
    rho_bar = (1 << 18) * M / 64.0 ** 3
    np.testing.assert_allclose(P[12], (3 * 64 * M / (4 * math.pi * 200 * rho_bar)) ** (1 / 3),
                               rtol=1e-15)


def test_only_bound_members_count():
    pos = _lattice(4, 0.5, [5.0, 5.0, 5.0])
    bound = (pos[:, 0] < 5.6).astype(np.uint8)     # the two x-planes 5.0 and 5.5
    P = _props(pos, bound)
    assert P[1] == 32 and P[3] == 32 * M
    assert list(P[4:7]) == [5.25, 5.75, 5.75]
    assert P[13] == 0.0625 and P[14] == 0.3125 and P[15] == 0.3125


def test_centre_wraps_into_box():
    box = 64.0
    pos = (_lattice(2, 0.5, [box - 0.5, 1.0, 1.0]) % box).astype(np.float32)  # x in {63.5, 0}
    P = _props(pos, np.ones(len(pos)), box=box, ids=np.arange(len(pos)))
    assert P[4] == 63.75
    pos2 = pos.copy()
    ids2 = np.array([4, 5, 6, 7, 0, 1, 2, 3])                                  # reference at x = 0
    P2 = _props(pos2, np.ones(len(pos)), box=box, ids=ids2)
    assert P2[4] == 63.75


def test_no_bound_members():
    pos = _lattice(2, 0.5, [1.0, 1.0, 1.0])
    P = _props(pos, np.zeros(len(pos)))
    assert P[0] == 8 and P[1] == 0 and np.all(P[3:] == 0)


def _sheared_case(k=4, h=0.5):
    """A k^3 lattice sheared by the dyadic matrix A = [[1, 1/2, 1/4], [0, 1, 1/2], [0, 0, 1]]
    with dyadic velocities v = (16 j - 24, 32 l, 8 i + 4 j) at lattice index (i, j, l).
    The lattice coordinates are independent and uniform on {0, h, .., (k-1) h}, each with
    variance s = h^2 (k^2 - 1) / 12, so the position covariance is s A A^T (non-zero
    off-diagonal terms, all different) and every moment is a short dyadic fraction: the oracle's
    float64 sums are exact and the pins below are equalities."""
    idx = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij"),
                   -1).reshape(-1, 3).astype(np.float64)
    A = np.array([[1.0, 0.5, 0.25], [0.0, 1.0, 0.5], [0.0, 0.0, 1.0]])
    pos = (idx * h) @ A.T + np.array([10.0, 20.0, 30.0])
    i, j, l = idx[:, 0], idx[:, 1], idx[:, 2]
    vel = np.stack([16 * j - 24, 32 * l, 8 * i + 4 * j], axis=1)
    s = h * h * (k * k - 1) / 12.0
    cov = s * (A @ A.T)
    return pos.astype(np.float32), vel.astype(np.float32), s, cov, A


def test_sheared_lattice_inertia_and_velocity_dispersion():
    pos, vel, s, cov, A = _sheared_case()
    assert np.array_equal(pos.astype(np.float64), np.asarray(pos, np.float64))  # exact in float32
    rng = np.random.default_rng(7)
    ids = rng.permutation(len(pos))
    P = _props(pos, np.ones(len(pos)), vel=vel, ids=ids)
    # centre: origin + A (mean lattice offset); mean offset is h (k - 1) / 2 = 0.75 per axis
    centre = np.array([10.0, 20.0, 30.0]) + A @ np.full(3, 0.75)
    assert list(P[4:7]) == list(centre)
    # bulk velocity: (16 * 1.5 - 24, 32 * 1.5, 8 * 1.5 + 4 * 1.5)
    assert list(P[7:10]) == [0.0, 48.0, 18.0]
    # sigma_x^2 = trace(cov); sigma_v^2 = 256 v1 + 1024 v1 + (64 + 16) v1, v1 = var of {0..3}
    assert P[10] == math.sqrt(np.trace(cov))
    v1 = 15.0 / 12.0
    assert P[11] == math.sqrt((256 + 1024 + 80) * v1)
    # inertia xx yy zz xy xz yz = the covariance entries, each different
    want = [cov[0, 0], cov[1, 1], cov[2, 2], cov[0, 1], cov[0, 2], cov[1, 2]]
    assert len(set(want)) == 6
    assert list(P[13:19]) == want


def test_sheared_lattice_bound_subset():
    """Only the bound half (lattice index i < 2) enters: its lattice x-coordinate takes two
    values, variance h^2 / 4, the other two axes keep s; the covariance is A diag(h^2/4, s, s)
    A^T and the velocity z-component loses the i-spread."""
    pos, vel, s, cov, A = _sheared_case()
    h = 0.5
    idx = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij"),
                   -1).reshape(-1, 3)
    bound = (idx[:, 0] < 2).astype(np.uint8)
    P = _props(pos, bound, vel=vel)
    assert P[1] == 32
    c = A @ np.diag([h * h / 4.0, s, s]) @ A.T
    assert list(P[13:19]) == [c[0, 0], c[1, 1], c[2, 2], c[0, 1], c[0, 2], c[1, 2]]
    v1 = 15.0 / 12.0
    # v = (16 j - 24, 32 l, 8 i + 4 j) with i in {0, 1}: var(i) = 1/4
    assert P[11] == math.sqrt(256 * v1 + 1024 * v1 + (64 * 0.25 + 16 * v1))
    assert list(P[7:10]) == [0.0, 48.0, 8 * 0.5 + 4 * 1.5]

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

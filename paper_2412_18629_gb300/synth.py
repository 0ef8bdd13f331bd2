"""Seeded synthetic N-body snapshots: NFW halos (with nested subhalos) on a uniform background.

This module only draws inputs. It holds none of the halo-finding arithmetic (no linking, no
6D metric, no potential); both the CUDA path and the CPU oracle read its arrays.

Recipe (the stand-in for the cosmological snapshots the paper analyses, Section
"Parallelization": 1024^3 particles in 250 Mpc/h, 2560^3 in 400 Mpc/h, ...):

* ``halo_frac`` (40%) of the particles sit in NFW halos. Halo particle counts are drawn one by
  one from dN/dn ~ n^-1.9 on [20, n_max] by inverse CDF until the budget is used; the last draw
  is clipped to the remainder, and a remainder below 20 goes to the background.
* Concentration c = 10 (n/1e4)^-0.1; r_vir = (3 n m / (4 pi 200 rho_bar))^(1/3) with
  rho_bar = n_total m / L^3. Radii invert mu(x)/mu(c), mu(x) = ln(1+x) - x/(1+x), in float64.
* Velocities: isotropic Gaussian with sigma_1D = V_vir / sqrt(2), V_vir = sqrt(G M / r_vir).
* Subhalos (``sub_levels`` >= 1): every halo with n > 1e3 gets U{0..10} subhalos, each holding
  U(1%, 10%) of the host's particles (taken from the host), centred at a radius U(0, 0.8 r_vir)
  in an isotropic direction, with a bulk velocity offset N(0, sigma_host) per component.
  ``sub_levels`` = 3 repeats this inside subhalos down to three levels.
* The rest is uniform background with sigma_v = 50 km/s per component.
* ids are a random permutation of 0..n-1 (int64), and the particle order is shuffled.
* Positions are float32 in [0, L): wrapped in float64, rounded, and a value that rounds to L
  becomes 0.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

G_NEWTON = 4.30091e-9  # Mpc (km/s)^2 / Msun
LINK_B = 0.28          # 3D linking length in units of the mean interparticle spacing


@dataclasses.dataclass(frozen=True)
class SnapshotSpec:
    n: int
    box: float
    seed: int
    n_max: float = 3.0e4
    n_min: int = 20
    slope: float = 1.9
    halo_frac: float = 0.4
    particle_mass: float = 1.0e10
    sub_levels: int = 0
    bg_sigma_v: float = 50.0

    @property
    def spacing(self) -> float:
        return self.box / float(np.cbrt(float(self.n)))

    @property
    def link_length(self) -> float:
        """3D linking length b * mean spacing, rounded once to float32 (passed to both sides)."""
        return float(np.float32(LINK_B * self.spacing))

    @property
    def softening(self) -> float:
        """Plummer softening: 1% of the mean interparticle spacing, float32."""
        return float(np.float32(0.01 * self.spacing))


# The five workloads: sizes, boxes and halo ranges of the configurations this build is measured on.
WORKLOADS = {
    "nfw-2^18-L64": SnapshotSpec(n=1 << 18, box=64.0, seed=0, n_max=3.0e4, sub_levels=0),
    "nfw-2^21-L128-sub": SnapshotSpec(n=1 << 21, box=128.0, seed=5, n_max=3.0e4, sub_levels=1),
    "nfw-2^24-L256-sub": SnapshotSpec(n=1 << 24, box=256.0, seed=1, n_max=3.0e4, sub_levels=1),
    "nfw-2^25-L320-sub": SnapshotSpec(n=1 << 25, box=320.0, seed=2, n_max=5.0e5, sub_levels=1),
    "nfw-2^27-L512-sub3": SnapshotSpec(n=1 << 27, box=512.0, seed=3, n_max=2.0e6, sub_levels=3),
}


def stream_spec(seed: int) -> SnapshotSpec:
    """One of the 64 independent snapshots of the batched stream: n = 2^(18 + seed mod 5), s = 1."""
    n = 1 << (18 + seed % 5)
    return SnapshotSpec(n=n, box=float(np.cbrt(float(n))), seed=seed, n_max=2.0e5, sub_levels=1)


def _draw_sizes(rng, budget, n_min, n_max, slope):
    a = 1.0 - slope  # < 0
    lo, hi = n_min ** a, n_max ** a
    sizes = []
    left = budget
    while left >= n_min:
        u = rng.random()
        s = int((lo + u * (hi - lo)) ** (1.0 / a))
        s = max(n_min, min(s, int(n_max)))
        if s > left:
            s = left
        sizes.append(s)
        left -= s
    return sizes, left


def _mu(x):
    return np.log1p(x) - x / (1.0 + x)


def _nfw_radii(rng, c, count):
    """Radii in units of r_vir for `count` particles of an NFW halo with concentration c."""
    target = rng.random(count) * _mu(c)
    lo = np.zeros(count)
    hi = np.broadcast_to(np.asarray(c, dtype=np.float64), (count,)).copy()
    for _ in range(16):
        mid = 0.5 * (lo + hi)
        below = _mu(mid) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    x = 0.5 * (lo + hi)
    for _ in range(3):  # Newton polish inside the bracket: mu'(x) = x / (1 + x)^2
        step = (_mu(x) - target) * (1.0 + x) ** 2 / np.maximum(x, 1e-300)
        x = np.clip(x - step, lo, hi)
    return x / c


def _directions(rng, count):
    z = rng.uniform(-1.0, 1.0, count)
    phi = rng.uniform(0.0, 2.0 * np.pi, count)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def _r_vir(count, m, rho_bar):
    return (3.0 * count * m / (4.0 * np.pi * 200.0 * rho_bar)) ** (1.0 / 3.0)


def _halo(rng, count, centre, bulk_v, m, rho_bar, levels, plan, depth):
    """Plan one NFW halo (and its nested subhalos): append (own count, c, r_vir, centre, bulk, sigma)."""
    r_vir = _r_vir(count, m, rho_bar)
    v_vir = math.sqrt(G_NEWTON * count * m / r_vir)
    sigma = v_vir / math.sqrt(2.0)
    own = count
    if levels > 0 and count > 1000:
        for _ in range(int(rng.integers(0, 11))):
            sub = int(count * rng.uniform(0.01, 0.10))
            if sub < 20 or own - sub < count // 2:
                continue
            own -= sub
            sub_centre = centre + _directions(rng, 1)[0] * rng.uniform(0.0, 0.8 * r_vir)
            sub_bulk = bulk_v + rng.normal(0.0, sigma, 3)
            _halo(rng, sub, sub_centre, sub_bulk, m, rho_bar, levels - 1, plan, depth + 1)
    conc = 10.0 * (count / 1.0e4) ** -0.1
    plan.append((depth, count, own, conc, r_vir, centre.copy(), bulk_v.copy(), sigma))


def generate(spec: SnapshotSpec) -> dict:
    """Draw one snapshot. Returns pos/vel float32 [n][3], ids int64 [n] and the halo catalogue."""
    rng = np.random.default_rng(spec.seed)
    n, L, m = spec.n, float(spec.box), spec.particle_mass
    rho_bar = n * m / L ** 3
    sizes, _ = _draw_sizes(rng, int(spec.halo_frac * n), spec.n_min, spec.n_max, spec.slope)
    plan = []
    for count in sizes:
        centre = rng.uniform(0.0, L, 3)
        _halo(rng, count, centre, np.zeros(3), m, rho_bar, spec.sub_levels, plan, 0)
    own = np.array([p[2] for p in plan], dtype=np.int64)
    n_halo = int(own.sum())
    if n_halo:
        conc = np.repeat(np.array([p[3] for p in plan]), own)
        r_vir = np.repeat(np.array([p[4] for p in plan]), own)
        centre = np.repeat(np.array([p[5] for p in plan]).reshape(-1, 3), own, axis=0)
        bulk = np.repeat(np.array([p[6] for p in plan]).reshape(-1, 3), own, axis=0)
        sigma = np.repeat(np.array([p[7] for p in plan]), own)
        r = _nfw_radii(rng, conc, n_halo) * r_vir
        halo_pos = centre + _directions(rng, n_halo) * r[:, None]
        halo_vel = bulk + rng.normal(0.0, 1.0, (n_halo, 3)) * sigma[:, None]
    else:
        halo_pos = np.zeros((0, 3))
        halo_vel = np.zeros((0, 3))
    n_bg = n - n_halo
    pos64 = np.concatenate([halo_pos, rng.uniform(0.0, L, (n_bg, 3))])
    vel64 = np.concatenate([halo_vel, rng.normal(0.0, spec.bg_sigma_v, (n_bg, 3))])
    pos64 = np.mod(pos64, L)
    pos = pos64.astype(np.float32)
    pos[pos >= np.float32(L)] = 0.0
    vel = vel64.astype(np.float32)
    order = rng.permutation(n)
    pos = np.ascontiguousarray(pos[order])
    vel = np.ascontiguousarray(vel[order])
    ids = rng.permutation(n).astype(np.int64)
    catalogue = [(p[0], p[1], p[2], p[5], p[6], p[4]) for p in plan]
    return {
        "pos": pos, "vel": vel, "ids": ids, "box": L, "n": n,
        "link_length": spec.link_length, "softening": spec.softening,
        "particle_mass": m, "n_halo_particles": n_halo, "catalogue": catalogue,
    }


MPC_PER_GYR_PER_KMS = 1.0227  # 1 km/s sustained for 1 Gyr covers 1.0227 Mpc


def evolve(snap: dict, dt_gyr: float, seed: int, kick_kms: float = 5.0) -> dict:
    """The same particles a short time later, for temporal tracking: positions drifted
    ballistically by v dt (no forces; h taken as 1 in the unit conversion), wrapped into the box;
    velocities given a Gaussian kick of kick_kms per component; particle order reshuffled (each
    id follows its particle). A stand-in for the next output of a simulation."""
    rng = np.random.default_rng(seed)
    L = float(snap["box"])
    pos64 = snap["pos"].astype(np.float64) + snap["vel"].astype(np.float64) * (MPC_PER_GYR_PER_KMS * dt_gyr)
    pos64 = np.mod(pos64, L)
    pos = pos64.astype(np.float32)
    pos[pos >= np.float32(L)] = 0.0
    vel = (snap["vel"].astype(np.float64) + rng.normal(0.0, kick_kms, snap["vel"].shape)).astype(np.float32)
    order = rng.permutation(len(pos))
    out = dict(snap)
    out["pos"] = np.ascontiguousarray(pos[order])
    out["vel"] = np.ascontiguousarray(vel[order])
    out["ids"] = np.ascontiguousarray(snap["ids"][order])
    return out


def subsample(snap: dict, keep: np.ndarray) -> dict:
    """A snapshot restricted to the particles selected by the boolean mask `keep`."""
    out = dict(snap)
    for k in ("pos", "vel", "ids"):
        out[k] = np.ascontiguousarray(snap[k][keep])
    out["n"] = int(keep.sum())
    return out

"""CPU oracle for the halo-finding path (3D FoF, 6D FoF hierarchy, unbinding, halo properties).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may import this package. The product path (``paper_2412_18629_gb300``) never does.

The arithmetic lives in ``rs_oracle.cpp`` (plain C++17, built with -ffp-contract=off); this
module compiles it with g++ on first use and wraps it with ctypes. Every function takes and
returns NumPy arrays on the host.

Parity status per function (what pins each one to something other than itself is listed in the
tests named here):
* fof3d_brute / fof3d_grid: brute force vs grid, SciPy k-d tree components, lattice, periodic
  and exact-distance special cases (tests/test_oracle_fof3d.py).
* cro_sum: exactly rounded sums (math.fsum) within the recursive-summation bound, hand-derived
  order-sensitive cases (tests/test_oracle_cro.py).
* split_node / hierarchy: invariants (linked fraction, subsets, disjointness, sizes), exact
  velocity-scaling invariance, two-blob special cases, SciPy k-d tree nearest neighbours; the
  exactly pruned k-d tree search of large nodes against the all-pairs search, bit for bit
  (tests/test_oracle_hierarchy.py, tests/test_oracle_pruned.py).
* unbind: two-body, centre-of-sphere and cube closed forms, Plummer and uniform-sphere profiles,
  bound/unbound limits (tests/test_oracle_unbind.py); unbind_sample equals unbind at the sampled
  members (tests/test_oracle_pruned.py).
* props: lattice moments and inertia in closed form, centre wrapping (tests/test_oracle_props.py).
* mlp_forward / mlp_gradient: finite differences of the float64 form, zero-weight and linear
  special cases, bf16 rounding of exactly representable values (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_rs.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-pthread"]


def build(force: bool = False) -> str:
    """Compile the oracle library with g++ (no-op when it is newer than its source)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["g++", *CFLAGS, _SRC, "-o", tmp], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, f32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_double
        lib.or_fof3d_brute.argtypes = [i64, P, P, f32, f32, P]
        lib.or_fof3d_grid.argtypes = [i64, P, P, f32, f32, P]
        lib.or_cro_sum.argtypes = [P, i64]
        lib.or_cro_sum.restype = f64
        lib.or_split_node.argtypes = [i64, P, P, i32, i32, P, P, P]
        lib.or_split_node_ex.argtypes = [i64, P, P, i32, i32, i32, i32, P, P, P]
        lib.or_unbind_sample.argtypes = [i64, P, P, P, f32, f32, f64, f64, i64, P, i32, P, P]
        lib.or_hierarchy.argtypes = [i64, P, P, P, P, f32, i32, i32, i32, i32,
                                     ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.or_hierarchy.restype = P
        lib.or_hierarchy_copy.argtypes = [P, P, P, P, P, P, P, P]
        lib.or_hierarchy_free.argtypes = [P]
        lib.or_hierarchy_params.argtypes = [P, P]
        lib.or_assign_seeds.argtypes = [i64, P, P, f32, i64, P, P, P, P, P, i32, P, P, P]
        lib.or_track.argtypes = [i64, P, P, i64, i64, P, P, i64, P, P, P, P]
        lib.or_unbind.argtypes = [i64, P, P, P, P, f32, f32, f64, f64, i32, i32, i32, i32,
                                  P, P, P, P, P]
        lib.or_unbind_iter.argtypes = [i64, P, P, P, P, f32, f32, f64, f64, i32, i32, i32, i32,
                                       i32, P, P, P, P, P]
        lib.or_props.argtypes = [i64, P, P, P, P, P, P, f32, f64, i64, i32, P]
        lib.or_mlp_forward.argtypes = [i64, P, P, i32, P]
        lib.or_mlp_gradient.argtypes = [i64, P, P, P, i32, P, ctypes.POINTER(f64)]
        _lib = lib
        return lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _threads(threads):
    return int(threads) if threads else (os.cpu_count() or 1)


def fof3d_brute(pos, ids, box, ll):
    pos, ids = _c(pos, np.float32), _c(ids, np.int64)
    out = np.empty(len(ids), np.int64)
    rc = _load().or_fof3d_brute(len(ids), _p(pos), _p(ids), box, ll, _p(out))
    assert rc == 0
    return out


def fof3d_grid(pos, ids, box, ll):
    pos, ids = _c(pos, np.float32), _c(ids, np.int64)
    out = np.empty(len(ids), np.int64)
    rc = _load().or_fof3d_grid(len(ids), _p(pos), _p(ids), box, ll, _p(out))
    assert rc == 0
    return out


def fof3d(pos, ids, box, ll):
    """3D FoF labels (smallest id of each particle's group)."""
    return fof3d_brute(pos, ids, box, ll) if len(ids) <= 2048 else fof3d_grid(pos, ids, box, ll)


def cro_sum(a):
    a = _c(a, np.float64)
    return float(_load().or_cro_sum(_p(a), len(a)))


def split_node(u, v, f_num=7, f_den=10, pruned=-1, threads=1):
    """One 6D FoF level on a single node: (inv_sx2, inv_sv2, l2, nn2[g], comp[g]).
    pruned: 0 all pairs, 1 the exactly pruned k-d tree search, -1 by size (tree above 4096
    members); threads: the tree search's member loops."""
    u, v = _c(u, np.float32), _c(v, np.float32)
    g = len(u)
    scal = np.empty(3, np.float32)
    nn2 = np.empty(g, np.float32)
    comp = np.empty(g, np.int64)
    rc = _load().or_split_node_ex(g, _p(u), _p(v), f_num, f_den, int(pruned), _threads(threads),
                                  _p(scal), _p(nn2), _p(comp))
    assert rc == 0
    return float(scal[0]), float(scal[1]), float(scal[2]), nn2, comp


def hierarchy(pos, vel, ids, fof_label, box, f_num=7, f_den=10, min_size=10, threads=None):
    """6D FoF hierarchy. Returns a dict of node arrays, member CSR, per-particle deepest node
    and each node's split parameters (params: inv_sx2, inv_sv2, l2)."""
    pos, vel = _c(pos, np.float32), _c(vel, np.float32)
    ids, lab = _c(ids, np.int64), _c(fof_label, np.int64)
    lib = _load()
    nn, nm = ctypes.c_int64(0), ctypes.c_int64(0)
    h = lib.or_hierarchy(len(ids), _p(pos), _p(vel), _p(ids), _p(lab), box, f_num, f_den,
                         min_size, _threads(threads), ctypes.byref(nn), ctypes.byref(nm))
    assert h
    try:
        n_nodes, n_mem = nn.value, nm.value
        out = {
            "parent": np.empty(n_nodes, np.int64), "level": np.empty(n_nodes, np.int32),
            "min_id": np.empty(n_nodes, np.int64), "size": np.empty(n_nodes, np.int64),
            "member_off": np.empty(n_nodes + 1, np.int64),
            "member_idx": np.empty(n_mem, np.int64), "deepest": np.empty(len(ids), np.int64),
        }
        rc = lib.or_hierarchy_copy(h, *(_p(out[k]) for k in (
            "parent", "level", "min_id", "size", "member_off", "member_idx", "deepest")))
        assert rc == 0
        out["params"] = np.empty((n_nodes, 3), np.float32)
        assert lib.or_hierarchy_params(h, _p(out["params"])) == 0
    finally:
        lib.or_hierarchy_free(h)
    return out


def assign_seeds(hier, pos, vel, box, threads=None):
    """Seed halos (nodes without children), each particle's seed and each seed's host, for a
    hierarchy dict from hierarchy(): (particle_seed [n], node_host [n_nodes], node_count
    [n_nodes]); -1 = no seed / no host, node_host -2 for nodes that are not seeds."""
    pos, vel = _c(pos, np.float32), _c(vel, np.float32)
    nn = len(hier["size"])
    par, off = _c(hier["parent"], np.int64), _c(hier["member_off"], np.int64)
    idx, deep = _c(hier["member_idx"], np.int64), _c(hier["deepest"], np.int64)
    prm = _c(hier["params"], np.float32)
    ps = np.empty(len(pos), np.int64)
    host = np.empty(nn, np.int64)
    cnt = np.empty(nn, np.int64)
    rc = _load().or_assign_seeds(len(pos), _p(pos), _p(vel), box, nn, _p(par), _p(off), _p(idx),
                                 _p(deep), _p(prm), _threads(threads), _p(ps), _p(host), _p(cnt))
    assert rc == 0
    return ps, host, cnt


def track(ids1, seed1, nn1, ids2, seed2, nn2):
    """Progenitors and descendants of seed halos between two snapshots matched by id:
    (prog [nn2], prog_shared [nn2], desc [nn1], desc_shared [nn1])."""
    ids1, seed1 = _c(ids1, np.int64), _c(seed1, np.int64)
    ids2, seed2 = _c(ids2, np.int64), _c(seed2, np.int64)
    prog, ps = np.empty(nn2, np.int64), np.empty(nn2, np.int64)
    desc, ds = np.empty(nn1, np.int64), np.empty(nn1, np.int64)
    rc = _load().or_track(len(ids1), _p(ids1), _p(seed1), nn1, len(ids2), _p(ids2), _p(seed2), nn2,
                          _p(prog), _p(ps), _p(desc), _p(ds))
    assert rc == 0
    return prog, ps, desc, ds


def unbind(member_off, member_idx, pos, vel, box, eps, G, m, min_size=10, bf_num=1, bf_den=2,
           threads=None, want_phi=True, passes=1):
    """Potential (float64 per member), bound flags, and per-node n_bound / is_halo / m_bound;
    passes > 1: iterative unbinding over the members still bound (or_unbind_iter)."""
    off, idx = _c(member_off, np.int64), _c(member_idx, np.int64)
    pos, vel = _c(pos, np.float32), _c(vel, np.float32)
    n_nodes, n_mem = len(off) - 1, int(off[-1]) if len(off) else 0
    phi = np.empty(n_mem, np.float64) if want_phi else None
    bound = np.empty(n_mem, np.uint8)
    nb = np.empty(n_nodes, np.int64)
    halo = np.empty(n_nodes, np.uint8)
    mb = np.empty(n_nodes, np.float64)
    rc = _load().or_unbind_iter(n_nodes, _p(off), _p(idx), _p(pos), _p(vel), box, eps, G, m,
                                min_size, bf_num, bf_den, int(passes), _threads(threads), _p(phi),
                                _p(bound), _p(nb), _p(halo), _p(mb))
    assert rc == 0
    return {"phi": phi, "bound": bound, "n_bound": nb, "is_halo": halo, "m_bound": mb}


def unbind_sample(mem, pos, vel, box, eps, G, m, sample, threads=None):
    """Potential (float64) and bound flag of the members sample[k] (positions in mem) of the
    node whose particles are mem (ascending id), by or_unbind's definition."""
    mem, sample = _c(mem, np.int64), _c(sample, np.int64)
    pos, vel = _c(pos, np.float32), _c(vel, np.float32)
    phi = np.empty(len(sample), np.float64)
    bound = np.empty(len(sample), np.uint8)
    rc = _load().or_unbind_sample(len(mem), _p(mem), _p(pos), _p(vel), box, eps, G, m,
                                  len(sample), _p(sample), _threads(threads), _p(phi), _p(bound))
    assert rc == 0
    return phi, bound


def props(member_off, member_idx, pos, vel, bound, is_halo, box, m, n_total, threads=None):
    """Halo properties: float64 [n_nodes][20] (layout in rs_oracle.cpp, or_props)."""
    off, idx = _c(member_off, np.int64), _c(member_idx, np.int64)
    pos, vel = _c(pos, np.float32), _c(vel, np.float32)
    bound, is_halo = _c(bound, np.uint8), _c(is_halo, np.uint8)
    out = np.empty((len(off) - 1, 20), np.float64)
    rc = _load().or_props(len(off) - 1, _p(off), _p(idx), _p(pos), _p(vel), _p(bound),
                          _p(is_halo), box, m, n_total, _threads(threads), _p(out))
    assert rc == 0
    return out


MLP_PARAMS = 4801


def mlp_forward(x, params, round_bf16=True):
    """Surrogate MLP output (float64 [n]) for features x [n][8] and the parameter vector."""
    x, params = _c(x, np.float32), _c(params, np.float32)
    y = np.empty(len(x), np.float64)
    rc = _load().or_mlp_forward(len(x), _p(x), _p(params), 1 if round_bf16 else 0, _p(y))
    assert rc == 0
    return y


def mlp_gradient(x, t, params, round_bf16=True):
    """Gradient (float64 [4801]) of the mean squared error and the sum of squared errors."""
    x, t, params = _c(x, np.float32), _c(t, np.float32), _c(params, np.float32)
    g = np.empty(MLP_PARAMS, np.float64)
    sse = ctypes.c_double(0.0)
    rc = _load().or_mlp_gradient(len(x), _p(x), _p(t), _p(params), 1 if round_bf16 else 0, _p(g),
                                 ctypes.byref(sse))
    assert rc == 0
    return g, sse.value

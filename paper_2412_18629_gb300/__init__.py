"""Python binding of librs_gb300.so, the GB300 halo-finding core (C ABI in include/rs_gb300.h).

Argument marshalling only: every step of the path runs in the library's CUDA kernels. Tensors
are PyTorch CUDA tensors (PyTorch supplies device memory and streams); functions carry the C
ABI's names and fail loudly when the library is missing, since there is no fallback.

    ctx = Context(box=256.0, link_len=0.28, softening=0.01, particle_mass=1e10)
    labels, n_groups = rs_fof3d(ctx, pos, ids)
    n_nodes, n_members = rs_fof6d(ctx, pos, vel, ids, labels)
    phi, bound, n_fallback = rs_unbind(ctx, pos, vel)
    props = rs_halo_props(ctx)
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librs_gb300.so")
G_NEWTON = 4.30091e-9

RS_OK = 0
_ERRORS = {1: "RS_ERR_INVALID_ARG", 2: "RS_ERR_CUDA", 3: "RS_ERR_OOM", 4: "RS_ERR_TIMEOUT",
           5: "RS_ERR_CAPACITY", 6: "RS_ERR_STATE"}

# rs_halo_props_t: n, n_bound, is_halo (int64) then 17 float64 = 20 eight-byte fields.
PROPS_FIELDS = 20

_lock = threading.Lock()
_lib = None


class RSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class rs_config(ctypes.Structure):
    _fields_ = [
        ("box_L", ctypes.c_float), ("link_len", ctypes.c_float), ("softening", ctypes.c_float),
        ("margin_factor", ctypes.c_float), ("particle_mass", ctypes.c_double),
        ("G", ctypes.c_double), ("f_num", ctypes.c_int32), ("f_den", ctypes.c_int32),
        ("min_halo_particles", ctypes.c_int32), ("bound_num", ctypes.c_int32),
        ("bound_den", ctypes.c_int32), ("batched", ctypes.c_int32),
        ("use_surrogate", ctypes.c_int32), ("spot_check", ctypes.c_int32),
        ("tree_min_members", ctypes.c_int32), ("tree_theta", ctypes.c_float),
        ("surrogate_gate", ctypes.c_int32), ("check_ids", ctypes.c_int32),
        ("unbind_passes", ctypes.c_int32),
    ]


class rs_snapshot(ctypes.Structure):
    """One snapshot of rs_run_batched (include/rs_gb300.h)."""
    _fields_ = [("n", ctypes.c_int64), ("box_L", ctypes.c_float), ("link_len", ctypes.c_float),
                ("softening", ctypes.c_float), ("reserved", ctypes.c_float),
                ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("ids", ctypes.c_void_p),
                ("label_out", ctypes.c_void_p), ("deepest_out", ctypes.c_void_p),
                ("node_capacity", ctypes.c_int64), ("node_parent_out", ctypes.c_void_p),
                ("props_out", ctypes.c_void_p)]


def load_library():
    """Load librs_gb300.so (built by __graft_entry__.build() / build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.rs_ctx_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(rs_config), ctypes.c_int]
        lib.rs_ctx_destroy.argtypes = [P]
        lib.rs_last_error.argtypes = [P]
        lib.rs_last_error.restype = ctypes.c_char_p
        lib.rs_kernel_launches.argtypes = [P]
        lib.rs_kernel_launches.restype = i64
        lib.rs_sort_keypasses.argtypes = [P]
        lib.rs_sort_keypasses.restype = i64
        lib.rs_fof3d.argtypes = [P, i64, P, P, P, ctypes.POINTER(i64), P]
        lib.rs_fof6d.argtypes = [P, i64, P, P, P, P, ctypes.POINTER(i64), ctypes.POINTER(i64), P]
        lib.rs_fof6d_copy.argtypes = [P, P, P, P, P, P, P, P, P]
        lib.rs_fof6d_node_params.argtypes = [P, P, P]
        lib.rs_unbind.argtypes = [P, P, P, P, P, ctypes.POINTER(i64), P]
        lib.rs_halo_props.argtypes = [P, P, P]
        lib.rs_assign_seeds.argtypes = [P, P, P, P, P, P, ctypes.POINTER(i64), P]
        lib.rs_track.argtypes = [P, i64, P, P, i64, i64, P, P, i64, P, P, P, P, P]
        lib.rs_unbind_passes.argtypes = [P]
        lib.rs_run_batched.argtypes = [P, i32, ctypes.POINTER(rs_snapshot), i32, P, P]
        lib.rs_use_graphs.argtypes = [P, ctypes.c_int]
        lib.rs_potential_pairs.argtypes = [P, P]
        lib.rs_nn_bounds.argtypes = [P, ctypes.c_float, i64]
        lib.rs_cro_sum.argtypes = [P, i64, P, P, P]
        lib.rs_sort_pairs.argtypes = [P, i64, ctypes.c_int, P, P, P]
        lib.rs_mlp_set_params.argtypes = [P, P]
        lib.rs_mlp_get_params.argtypes = [P, P]
        lib.rs_mlp_set_err_max.argtypes = [P, ctypes.c_float]
        lib.rs_mlp_get_err_max.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
        lib.rs_surrogate_save.argtypes = [P, ctypes.c_char_p]
        lib.rs_surrogate_load.argtypes = [P, ctypes.c_char_p]
        lib.rs_mlp_forward.argtypes = [P, i64, P, P, P]
        lib.rs_mlp_gradient.argtypes = [P, i64, P, P, P, ctypes.POINTER(ctypes.c_double), P]
        lib.rs_mlp_train.argtypes = [P, i64, P, P, i32, i32, ctypes.c_float, ctypes.c_uint64, i32,
                                     i32, ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(ctypes.c_double), P]
        for name in ("rs_mlp_set_params", "rs_mlp_get_params", "rs_mlp_set_err_max",
                     "rs_surrogate_save", "rs_surrogate_load", "rs_mlp_get_err_max",
                     "rs_mlp_forward", "rs_mlp_gradient", "rs_mlp_train"):
            getattr(lib, name).restype = i32
        lib.rs_cro_sum_noalloc.argtypes = [i64, P, P, P]
        lib.rs_tree_stats.argtypes = [P, P]
        lib.rs_tree_record.argtypes = [P, ctypes.c_int]
        lib.rs_tree_bounds.argtypes = [P, P, P, P]
        lib.rs_profile.argtypes = [P, ctypes.c_int]
        lib.rs_count_work.argtypes = [P, ctypes.c_int, P]
        lib.rs_tuning.argtypes = [P, P, P]
        lib.rs_profile_get.argtypes = [P, ctypes.c_int, ctypes.c_char_p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
        for name in ("rs_ctx_create", "rs_ctx_destroy", "rs_fof3d", "rs_fof6d", "rs_fof6d_copy",
                     "rs_fof6d_node_params", "rs_unbind", "rs_halo_props", "rs_cro_sum", "rs_profile",
                     "rs_profile_get", "rs_sort_pairs", "rs_cro_sum_noalloc", "rs_count_work", "rs_tuning",
                     "rs_tree_stats", "rs_tree_record", "rs_tree_bounds",
                     "rs_assign_seeds", "rs_track", "rs_unbind_passes", "rs_run_batched",
                     "rs_use_graphs", "rs_potential_pairs", "rs_nn_bounds"):
            getattr(lib, name).restype = i32
        _lib = lib
        return lib


def _torch():
    import torch
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_dev(t, dtype, shape_tail=None, name="tensor"):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} must have shape [n, {shape_tail}]")


class Context:
    """An rs_ctx: configuration plus the library-owned scratch and hierarchy state."""

    def __init__(self, box, link_len, softening, particle_mass, G=G_NEWTON, f=(7, 10),
                 min_halo_particles=10, bound_frac=(1, 2), device=0, mode="plain",
                 margin_factor=4.0, spot_check=32, tree_min=0, tree_theta=0.0, surrogate_gate=0,
                 check_ids=False, unbind_passes=1):
        self.lib = load_library()
        cfg = rs_config()
        cfg.box_L, cfg.link_len, cfg.softening = float(box), float(link_len), float(softening)
        cfg.particle_mass, cfg.G = float(particle_mass), float(G)
        cfg.f_num, cfg.f_den = int(f[0]), int(f[1])
        cfg.min_halo_particles = int(min_halo_particles)
        cfg.bound_num, cfg.bound_den = int(bound_frac[0]), int(bound_frac[1])
        if mode not in ("plain", "batched", "surrogate"):
            raise ValueError("mode must be 'plain', 'batched' or 'surrogate'")
        cfg.batched = 0 if mode == "plain" else 1
        cfg.use_surrogate = 1 if mode == "surrogate" else 0
        cfg.margin_factor = float(margin_factor)
        cfg.spot_check = int(spot_check)
        cfg.tree_min_members = int(tree_min)
        cfg.tree_theta = float(tree_theta)
        if surrogate_gate not in (0, 1):
            raise ValueError("surrogate_gate must be 0 (held-out maximum) or 1 (calibrated per node)")
        cfg.surrogate_gate = int(surrogate_gate)
        cfg.check_ids = 1 if check_ids else 0
        cfg.unbind_passes = int(unbind_passes)
        self.mode = mode
        self.cfg = cfg
        self.device = int(device)
        h = ctypes.c_void_p()
        rc = self.lib.rs_ctx_create(ctypes.byref(h), ctypes.byref(cfg), self.device)
        if rc != RS_OK:
            raise RSError(rc, "rs_ctx_create failed")
        self.handle = h

    def check(self, rc):
        if rc != RS_OK:
            raise RSError(rc, self.lib.rs_last_error(self.handle).decode())

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.rs_kernel_launches(self.handle))

    @property
    def sort_keypasses(self) -> int:
        """Keys moved by radix-sort passes since the context was created."""
        return int(self.lib.rs_sort_keypasses(self.handle))

    def nn_bounds(self, margin_scale=1.0, min_members=0):
        """Margin scale and smallest node of the sampled nearest-neighbour bounds (tuning and
        test instrumentation; 0 members = the default)."""
        self.check(self.lib.rs_nn_bounds(self.handle, float(margin_scale), int(min_members)))

    def use_graphs(self, enable=True):
        """CUDA graphs for static launch sequences (the surrogate's training epoch) on or off."""
        self.check(self.lib.rs_use_graphs(self.handle, 1 if enable else 0))

    def profile(self, enable=True):
        """Start (clearing totals) or stop CUDA-event timing of the dominant kernels."""
        self.check(self.lib.rs_profile(self.handle, 1 if enable else 0))

    def count_work(self, enable=True):
        """Enable (clearing) or disable the counting variants of the pruned 6D kernels; on
        disable returns {nn_d6, nn_box, link_d6, link_box, bounded_nodes, bound_failures}
        accumulated since the enable."""
        import numpy as np
        out = np.zeros(6, np.int64)
        self.check(self.lib.rs_count_work(self.handle, 1 if enable else 0,
                                          None if enable else out.ctypes.data))
        if not enable:
            return dict(zip(("nn_d6", "nn_box", "link_d6", "link_box", "bounded_nodes",
                             "bound_failures"), map(int, out)))
        return None

    def tuning(self):
        """Autotuner choices: members per thread of the blocked and list potential sums (0 =
        not tuned yet) and the candidates' times in ms (2, 4, 8 each)."""
        import numpy as np
        ch = np.zeros(2, np.int32)
        ms = np.zeros(6, np.float32)
        self.check(self.lib.rs_tuning(self.handle, ch.ctypes.data, ms.ctypes.data))
        return {"blocked_potential": {"members_per_thread": int(ch[0]),
                                      "ms": dict(zip((2, 4, 8), map(float, ms[:3])))},
                "list_potential": {"members_per_thread": int(ch[1]),
                                   "ms": dict(zip((2, 4, 8), map(float, ms[3:])))}}

    def profile_totals(self):
        """{kernel: (total_ms, launches)} recorded since profile(True)."""
        out = {}
        buf = ctypes.create_string_buffer(128)
        ms, cnt = ctypes.c_double(0), ctypes.c_int64(0)
        k = 0
        while self.lib.rs_profile_get(self.handle, k, buf, 128, ctypes.byref(ms),
                                      ctypes.byref(cnt)) == RS_OK:
            out[buf.value.decode()] = (ms.value, cnt.value)
            k += 1
        return out

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rs_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rs_fof3d(ctx, pos, ids, label_out=None, stream=None):
    """3D FoF labels (smallest id per group, int64 [n]) and the number of groups."""
    torch = _torch()
    _check_dev(pos, torch.float32, (3,), "pos")
    _check_dev(ids, torch.int64, None, "ids")
    n = pos.shape[0]
    if label_out is None:
        label_out = torch.empty(n, dtype=torch.int64, device=pos.device)
    ng = ctypes.c_int64(0)
    ctx.check(ctx.lib.rs_fof3d(ctx.handle, n, _ptr(pos), _ptr(ids), _ptr(label_out),
                               ctypes.byref(ng), _stream(stream)))
    return label_out, ng.value


def rs_fof6d(ctx, pos, vel, ids, fof_label, stream=None):
    """Build the 6D hierarchy inside the context; returns (n_nodes, n_members)."""
    torch = _torch()
    _check_dev(pos, torch.float32, (3,), "pos")
    _check_dev(vel, torch.float32, (3,), "vel")
    _check_dev(ids, torch.int64, None, "ids")
    _check_dev(fof_label, torch.int64, None, "fof_label")
    nn, nm = ctypes.c_int64(0), ctypes.c_int64(0)
    ctx.check(ctx.lib.rs_fof6d(ctx.handle, pos.shape[0], _ptr(pos), _ptr(vel), _ptr(ids),
                               _ptr(fof_label), ctypes.byref(nn), ctypes.byref(nm),
                               _stream(stream)))
    ctx.n_nodes, ctx.n_members, ctx.n_particles = nn.value, nm.value, pos.shape[0]
    return nn.value, nm.value


def rs_fof6d_copy(ctx, stream=None):
    """Hierarchy arrays as CUDA tensors (parent, level, min_id, size, member_off, member_idx,
    deepest)."""
    torch = _torch()
    dev = torch.device("cuda", ctx.device)
    nn, nm, n = ctx.n_nodes, ctx.n_members, ctx.n_particles
    out = {
        "parent": torch.empty(nn, dtype=torch.int64, device=dev),
        "level": torch.empty(nn, dtype=torch.int32, device=dev),
        "min_id": torch.empty(nn, dtype=torch.int64, device=dev),
        "size": torch.empty(nn, dtype=torch.int64, device=dev),
        "member_off": torch.empty(nn + 1, dtype=torch.int64, device=dev),
        "member_idx": torch.empty(nm, dtype=torch.int64, device=dev),
        "deepest": torch.empty(n, dtype=torch.int64, device=dev),
    }
    ctx.check(ctx.lib.rs_fof6d_copy(ctx.handle, *(_ptr(out[k]) for k in (
        "parent", "level", "min_id", "size", "member_off", "member_idx", "deepest")),
        _stream(stream)))
    return out


def rs_fof6d_node_params(ctx, stream=None):
    """float32 [n_nodes, 4] CUDA tensor: (inv_sx2, inv_sv2, l2, 0) of each node's 6D split."""
    torch = _torch()
    out = torch.empty((ctx.n_nodes, 4), dtype=torch.float32, device=torch.device("cuda", ctx.device))
    ctx.check(ctx.lib.rs_fof6d_node_params(ctx.handle, _ptr(out), _stream(stream)))
    return out


def rs_unbind(ctx, pos, vel, want_potential=True, bound_out=None, stream=None):
    """Per (node, member): float32 potential (or None), uint8 bound flag; and the number of
    members whose flag needed the exact float64 potential."""
    torch = _torch()
    dev = pos.device
    phi = torch.empty(ctx.n_members, dtype=torch.float32, device=dev) if want_potential else None
    if bound_out is None:
        bound_out = torch.empty(ctx.n_members, dtype=torch.uint8, device=dev)
    nfb = ctypes.c_int64(0)
    ctx.check(ctx.lib.rs_unbind(ctx.handle, _ptr(pos), _ptr(vel), _ptr(phi), _ptr(bound_out),
                                ctypes.byref(nfb), _stream(stream)))
    return phi, bound_out, nfb.value


def rs_assign_seeds(ctx, pos, vel, stream=None):
    """Seed halos of the last rs_fof6d hierarchy: (particle_seed [n], node_host [n_nodes],
    node_count [n_nodes]) int64 CUDA tensors and the number of seeds."""
    torch = _torch()
    _check_dev(pos, torch.float32, (3,), "pos")
    _check_dev(vel, torch.float32, (3,), "vel")
    dev = pos.device
    ps = torch.empty(ctx.n_particles, dtype=torch.int64, device=dev)
    host = torch.empty(ctx.n_nodes, dtype=torch.int64, device=dev)
    cnt = torch.empty(ctx.n_nodes, dtype=torch.int64, device=dev)
    ns = ctypes.c_int64(0)
    ctx.check(ctx.lib.rs_assign_seeds(ctx.handle, _ptr(pos), _ptr(vel), _ptr(ps), _ptr(host),
                                      _ptr(cnt), ctypes.byref(ns), _stream(stream)))
    return ps, host, cnt, ns.value


def rs_track(ctx, ids1, seed1, n_nodes1, ids2, seed2, n_nodes2, stream=None):
    """Progenitors (and shared counts) of the later snapshot's seeds, descendants (and shared
    counts) of the earlier snapshot's seeds: four int64 CUDA tensors."""
    torch = _torch()
    for t, nm in ((ids1, "ids1"), (seed1, "seed1"), (ids2, "ids2"), (seed2, "seed2")):
        _check_dev(t, torch.int64, None, nm)
    dev = ids2.device
    prog = torch.empty(n_nodes2, dtype=torch.int64, device=dev)
    ps = torch.empty(n_nodes2, dtype=torch.int64, device=dev)
    desc = torch.empty(n_nodes1, dtype=torch.int64, device=dev)
    ds = torch.empty(n_nodes1, dtype=torch.int64, device=dev)
    ctx.check(ctx.lib.rs_track(ctx.handle, ids1.numel(), _ptr(ids1), _ptr(seed1), int(n_nodes1),
                               ids2.numel(), _ptr(ids2), _ptr(seed2), int(n_nodes2), _ptr(prog),
                               _ptr(ps), _ptr(desc), _ptr(ds), _stream(stream)))
    return prog, ps, desc, ds


def rs_potential_pairs(ctx):
    """Ordered pairs the last rs_unbind's direct sums evaluated: (small nodes, larger nodes)."""
    import numpy as np
    out = np.zeros(2, np.int64)
    ctx.check(ctx.lib.rs_potential_pairs(ctx.handle, out.ctypes.data_as(ctypes.c_void_p)))
    return int(out[0]), int(out[1])


def rs_unbind_passes(ctx):
    """Unbinding passes the last rs_unbind ran."""
    return int(ctx.lib.rs_unbind_passes(ctx.handle))


def rs_halo_props(ctx, props_out=None, stream=None):
    """rs_halo_props_t per node as a uint8 CUDA tensor [n_nodes, 160] (see props_to_float64)."""
    torch = _torch()
    if props_out is None:
        props_out = torch.empty((ctx.n_nodes, 8 * PROPS_FIELDS), dtype=torch.uint8,
                                device=torch.device("cuda", ctx.device))
    ctx.check(ctx.lib.rs_halo_props(ctx.handle, _ptr(props_out), _stream(stream)))
    return props_out


class BatchOutputs:
    """Output buffers of rs_run_batched for a list of snapshots: per snapshot the FoF labels,
    the deepest node of every particle, and (node_capacity rows) the parent of every node and
    its rs_halo_props_t row; reusable across calls on snapshots of the same sizes."""

    def __init__(self, sizes, node_capacity, device, deepest=True, props=True):
        torch = _torch()
        dev = torch.device("cuda", device)
        self.labels = [torch.empty(n, dtype=torch.int64, device=dev) for n in sizes]
        self.deepest = [torch.empty(n, dtype=torch.int64, device=dev) for n in sizes] if deepest else None
        cap = [int(c) for c in node_capacity]
        self.capacity = cap
        self.parent = [torch.empty(c, dtype=torch.int64, device=dev) for c in cap] if props else None
        self.props = ([torch.empty((c, 8 * PROPS_FIELDS), dtype=torch.uint8, device=dev) for c in cap]
                      if props else None)


def rs_run_batched(ctx, snaps, out, lanes=4, stream=None):
    """The pipeline over every snapshot of `snaps` (dicts of CUDA tensors pos, vel, ids and
    floats box, link_length, softening) on `lanes` concurrent lanes, writing into `out`
    (a BatchOutputs). Returns int64 counts [n_snap, 4]: groups, nodes, members, levels.
    Raises RSError (code RS_ERR_CAPACITY) when a snapshot has more nodes than its capacity."""
    import numpy as np
    torch = _torch()
    arr = (rs_snapshot * max(len(snaps), 1))()
    for k, sn in enumerate(snaps):
        _check_dev(sn["pos"], torch.float32, (3,), "pos")
        _check_dev(sn["vel"], torch.float32, (3,), "vel")
        _check_dev(sn["ids"], torch.int64, None, "ids")
        a = arr[k]
        a.n = sn["pos"].shape[0]
        a.box_L, a.link_len, a.softening = (float(sn["box"]), float(sn["link_length"]),
                                            float(sn["softening"]))
        a.pos, a.vel, a.ids = sn["pos"].data_ptr(), sn["vel"].data_ptr(), sn["ids"].data_ptr()
        a.label_out = out.labels[k].data_ptr()
        a.deepest_out = out.deepest[k].data_ptr() if out.deepest is not None else None
        a.node_capacity = out.capacity[k]
        if out.parent is not None:
            a.node_parent_out = out.parent[k].data_ptr() if out.capacity[k] else None
            a.props_out = out.props[k].data_ptr() if out.capacity[k] else None
    counts = np.zeros((len(snaps), 4), np.int64)
    rc = ctx.lib.rs_run_batched(ctx.handle, len(snaps), arr, int(lanes),
                                counts.ctypes.data_as(ctypes.c_void_p), _stream(stream))
    if rc != RS_OK:
        err = RSError(rc, ctx.lib.rs_last_error(ctx.handle).decode(errors="replace"))
        err.counts = counts
        raise err
    return counts


def props_to_float64(raw):
    """rs_halo_props_t rows -> float64 [n, 20]: n, n_bound, is_halo, m_bound, pos[3], vel[3],
    sigma_x, sigma_v, r_vir, inertia[6], reserved."""
    torch = _torch()
    raw = raw.contiguous()
    as_i = raw.view(torch.int64).reshape(-1, PROPS_FIELDS)
    out = raw.view(torch.float64).reshape(-1, PROPS_FIELDS).clone()
    out[:, :3] = as_i[:, :3].to(torch.float64)
    return out


def rs_sort_pairs(ctx, keys, vals, nbits=64, stream=None):
    """Stable in-place sort of (uint64 key as int64 tensor, uint32 value as int32 tensor)."""
    torch = _torch()
    _check_dev(keys, torch.int64, None, "keys")
    _check_dev(vals, torch.int32, None, "vals")
    ctx.check(ctx.lib.rs_sort_pairs(ctx.handle, keys.numel(), int(nbits), _ptr(keys), _ptr(vals),
                                    _stream(stream)))
    return keys, vals


def rs_cro_sum(ctx, a, stream=None):
    """Canonical-order float64 sum of a CUDA float64 tensor (returns a 1-element tensor)."""
    torch = _torch()
    _check_dev(a, torch.float64, None, "a")
    out = torch.empty(1, dtype=torch.float64, device=a.device)
    ctx.check(ctx.lib.rs_cro_sum(ctx.handle, a.numel(), _ptr(a), _ptr(out), _stream(stream)))
    return out


def rs_cro_sum_noalloc(a, out=None, stream=None):
    """rs_cro_sum without a context or any device allocation by the library (for callers that
    cannot allocate); limited to 2^26 terms. Returns the 1-element output tensor."""
    torch = _torch()
    _check_dev(a, torch.float64, None, "a")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=a.device)
    rc = load_library().rs_cro_sum_noalloc(a.numel(), _ptr(a), _ptr(out), _stream(stream))
    if rc != RS_OK:
        raise RSError(rc, "rs_cro_sum_noalloc failed")
    return out


MLP_PARAMS = 4801


def rs_mlp_set_params(ctx, params):
    """Load the surrogate's float32 master parameters (NumPy array of 4801)."""
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != MLP_PARAMS:
        raise ValueError("params must have 4801 entries")
    ctx.check(ctx.lib.rs_mlp_set_params(ctx.handle, ctypes.c_void_p(p.ctypes.data)))


def rs_mlp_get_params(ctx):
    import numpy as np
    p = np.empty(MLP_PARAMS, np.float32)
    ctx.check(ctx.lib.rs_mlp_get_params(ctx.handle, ctypes.c_void_p(p.ctypes.data)))
    return p


def rs_mlp_set_err_max(ctx, err_max):
    ctx.check(ctx.lib.rs_mlp_set_err_max(ctx.handle, float(err_max)))


def rs_mlp_get_err_max(ctx):
    v = ctypes.c_float(0.0)
    ctx.check(ctx.lib.rs_mlp_get_err_max(ctx.handle, ctypes.byref(v)))
    return v.value


def rs_surrogate_save(ctx, path):
    """Write the surrogate's weights and held-out maximum error to `path`."""
    ctx.check(ctx.lib.rs_surrogate_save(ctx.handle, os.fsencode(path)))


def rs_surrogate_load(ctx, path):
    """Load weights and held-out maximum error written by rs_surrogate_save."""
    ctx.check(ctx.lib.rs_surrogate_load(ctx.handle, os.fsencode(path)))


def rs_mlp_forward(ctx, x, stream=None):
    """Surrogate output y [n] for features x [n, 8] (CUDA float32)."""
    torch = _torch()
    _check_dev(x, torch.float32, (8,), "x")
    y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    ctx.check(ctx.lib.rs_mlp_forward(ctx.handle, x.shape[0], _ptr(x), _ptr(y), _stream(stream)))
    return y


def rs_mlp_gradient(ctx, x, t, stream=None):
    """(grad [4801] CUDA float32, sum of squared errors) of the batch mean squared error."""
    torch = _torch()
    _check_dev(x, torch.float32, (8,), "x")
    _check_dev(t, torch.float32, None, "t")
    g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device)
    sse = ctypes.c_double(0.0)
    ctx.check(ctx.lib.rs_mlp_gradient(ctx.handle, x.shape[0], _ptr(x), _ptr(t), _ptr(g),
                                      ctypes.byref(sse), _stream(stream)))
    return g, sse.value


def rs_mlp_train(ctx, x, t, epochs=20, batch=4096, lr=1e-3, seed=0, holdout=(1, 10), stream=None):
    """Train the surrogate on (x [n, 8], t [n]); returns (held-out max |y - t|, last batch MSE)."""
    torch = _torch()
    _check_dev(x, torch.float32, (8,), "x")
    _check_dev(t, torch.float32, None, "t")
    em, mse = ctypes.c_float(0.0), ctypes.c_double(0.0)
    ctx.check(ctx.lib.rs_mlp_train(ctx.handle, x.shape[0], _ptr(x), _ptr(t), int(epochs),
                                   int(batch), float(lr), ctypes.c_uint64(int(seed)),
                                   int(holdout[0]), int(holdout[1]), ctypes.byref(em),
                                   ctypes.byref(mse), _stream(stream)))
    return em.value, mse.value


def rs_surrogate_features(ctx, with_targets=True, stream=None):
    """(features [k, 8], psi targets [k] or None) of the members of nodes with >= 1024 members,
    from the last rs_unbind (CUDA float32 tensors)."""
    torch = _torch()
    lib = ctx.lib
    lib.rs_surrogate_features.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_void_p]
    lib.rs_surrogate_features.restype = ctypes.c_int32
    dev = torch.device("cuda", ctx.device)
    feat = torch.empty((max(ctx.n_members, 1), 8), dtype=torch.float32, device=dev)
    psi = torch.empty(max(ctx.n_members, 1), dtype=torch.float32, device=dev) if with_targets else None
    n = ctypes.c_int64(0)
    ctx.check(lib.rs_surrogate_features(ctx.handle, _ptr(feat), _ptr(psi), ctypes.byref(n),
                                        _stream(stream)))
    k = n.value
    return feat[:k], (psi[:k] if psi is not None else None)


TREE_STATS = ("tree_nodes", "tree_members", "decided_by_bound", "exact_path", "expansions",
              "direct_pairs", "list_pairs", "reserved")


def rs_tree_stats(ctx):
    """Counters of the certified tree bound in the last rs_unbind (see TREE_STATS)."""
    arr = (ctypes.c_int64 * 8)()
    ctx.check(ctx.lib.rs_tree_stats(ctx.handle, ctypes.cast(arr, ctypes.c_void_p)))
    return dict(zip(TREE_STATS, list(arr)))


def rs_tree_record(ctx, enable=True):
    """Record each bounded member's interval of the potential sum in later rs_unbind calls."""
    ctx.check(ctx.lib.rs_tree_record(ctx.handle, 1 if enable else 0))


def rs_tree_bounds(ctx, stream=None):
    """(lo, hi) float64 CUDA tensors [n_members]: the recorded interval of each member's sum
    S_i = sum_{j != i} (|u_j - u_i|^2 + eps^2)^(-1/2) (NaN where the flag came from elsewhere)."""
    torch = _torch()
    dev = torch.device("cuda", ctx.device)
    lo = torch.empty(ctx.n_members, dtype=torch.float64, device=dev)
    hi = torch.empty(ctx.n_members, dtype=torch.float64, device=dev)
    ctx.check(ctx.lib.rs_tree_bounds(ctx.handle, _ptr(lo), _ptr(hi), _stream(stream)))
    return lo, hi


SURROGATE_STATS = ("surrogate_members", "gated", "exact_member_path", "spot_checked",
                   "failed_nodes", "fp64_member_path", "fp64_direct", "rerun_members",
                   "whole_node_members", "surrogate_decided", "spot_mismatches")


def rs_surrogate_stats(ctx):
    lib = ctx.lib
    lib.rs_surrogate_stats.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.rs_surrogate_stats.restype = ctypes.c_int32
    arr = (ctypes.c_int64 * 11)()
    ctx.check(lib.rs_surrogate_stats(ctx.handle, ctypes.cast(arr, ctypes.c_void_p)))
    return dict(zip(SURROGATE_STATS, list(arr)))

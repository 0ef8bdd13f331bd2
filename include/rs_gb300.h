/*
 * rs_gb300.h -- C ABI of the GB300 halo-finding core (librs_gb300.so).
 *
 * The library runs, on one GPU, the data-parallel core of the Rockstar halo finder that
 * MPI-Rockstar parallelises (arXiv:2412.18629, Section "Parallelization": per-process 3D
 * friends-of-friends, then subhalo finding inside every FoF halo from 6D phase-space
 * information; Summary: halo properties such as the inertia tensor):
 *
 *   rs_fof3d      periodic 3D FoF over a snapshot -> per-particle group labels
 *   rs_fof6d      recursive 6D phase-space FoF inside every FoF group -> node hierarchy
 *   rs_unbind     potential + kinetic energy per (node, member) -> bound flags, halo decision
 *   rs_halo_props per-node properties over bound members (centre, velocity, dispersions,
 *                 r_vir, inertia tensor)
 *
 * Conventions for every call:
 *   - Return value: RS_OK (0) or one of the RS_ERR_* codes below; rs_last_error(ctx) then
 *     returns a message owned by the context (valid until the next call on it). No call throws.
 *   - Array arguments are DEVICE pointers owned by the caller, unless a comment says "host".
 *     Positions and velocities are float32 [n][3] (x, y, z contiguous per particle); ids are
 *     int64 [n], non-negative and unique (any value up to 2^63 - 1; uniqueness is verified
 *     only with rs_config.check_ids, a repeated id otherwise gives undefined groupings).
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL = legacy default
 *     stream). Calls that return host-visible counts synchronise that stream before returning.
 *   - The context owns its scratch memory and the hierarchy built by rs_fof6d; those stay
 *     valid until the next rs_fof6d on the same context or rs_ctx_destroy. A context is used
 *     by one host thread at a time.
 *   - Results are deterministic and identical to the CPU oracle's definitions: 3D labels,
 *     6D memberships, bound flags and halo decisions bit for bit; potentials within 1e-5
 *     relative of the float64 value.
 */
#ifndef RS_GB300_H
#define RS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RS_OK 0
#define RS_ERR_INVALID_ARG 1 /* a pointer, size or configuration value is out of range */
#define RS_ERR_CUDA 2        /* a CUDA runtime call or kernel launch failed */
#define RS_ERR_OOM 3         /* device scratch memory could not be allocated */
#define RS_ERR_TIMEOUT 4     /* a bounded device-side wait ran out (status word set) */
#define RS_ERR_CAPACITY 5    /* a fixed-size buffer is too small for this input */
#define RS_ERR_STATE 6       /* the call needs an earlier call on this context first */

/* Parameters shared by every call of a context.
 * box_L, link_len and softening are the float32 values the float32 arithmetic uses; the
 * caller rounds them once (link_len = float(b * L / n^(1/3)), b = 0.28). */
typedef struct rs_config {
  float box_L;                /* periodic box side (Mpc/h); positions must lie in [0, box_L) */
  float link_len;             /* 3D linking length ll; pairs with d^2 <= ll*ll are linked */
  float softening;            /* Plummer softening eps of the potential (Mpc/h) */
  float margin_factor;        /* surrogate gate: classify iff |E_pred| > margin_factor *
                                 err * G M / r_vir (4); err is the surrogate's held-out maximum
                                 error (or the per-node calibrated one, surrogate_gate = 1) */
  double particle_mass;       /* m (Msun/h), equal for all particles */
  double G;                   /* gravitational constant, 4.30091e-9 Mpc (km/s)^2 / Msun */
  int32_t f_num, f_den;       /* linked fraction f = f_num / f_den of the 6D FoF (7, 10) */
  int32_t min_halo_particles; /* minimum node size and minimum bound count (10) */
  int32_t bound_num, bound_den; /* halo iff bound_den * N_bound >= bound_num * n (1, 2) */
  int32_t batched;            /* 0 = plain form (brute-force pair kernels); 1 = batched form
                                 (exactly pruned 6D searches, blocked potential); identical
                                 outputs */
  int32_t use_surrogate;      /* 1: rs_unbind gates members of nodes with >= 1024 members by
                                 the trained MLP (batched + surrogate form) */
  int32_t spot_check;         /* gated members per node re-checked exactly (32) */
  int32_t tree_min_members;   /* batched forms: nodes with at least this many members get their
                                 flags from the certified tree bound (see rs_tree_stats) when
                                 rs_unbind is asked for no potential; 0 = 16384, < 0 = never */
  float tree_theta;           /* opening angle of that bound (0 = 0.45; at most 0.9) */
  int32_t surrogate_gate;     /* 0: the error in the gate is the held-out maximum error of the
                                 training (rs_mlp_set_err_max); 1: per node, calibrated on 64
                                 members evaluated exactly, floored at err_max / 8 */
  int32_t check_ids;          /* 1: rs_fof3d first verifies that the ids are unique and
                                 non-negative (one 64-bit sort), RS_ERR_INVALID_ARG otherwise */
  int32_t unbind_passes;      /* 0 or 1: one unbinding pass; P > 1: iterative unbinding, up to P
                                 passes (see rs_unbind); plain and batched forms only */
} rs_config;

/* Per-node halo properties written by rs_halo_props (all over the node's BOUND members). */
typedef struct rs_halo_props_t {
  int64_t n;          /* members of the node */
  int64_t n_bound;    /* bound members */
  int64_t is_halo;    /* 1 if the node passes the halo decision */
  double m_bound;     /* n_bound * particle_mass */
  double pos[3];      /* centre: reference member + mean offset, wrapped into [0, box_L) */
  double vel[3];      /* bulk velocity */
  double sigma_x;     /* sqrt of the total (3D) position variance */
  double sigma_v;     /* sqrt of the total (3D) velocity variance */
  double r_vir;       /* (3 m_bound / (4 pi 200 rho_bar))^(1/3), rho_bar = n_total m / L^3 */
  double inertia[6];  /* second moments about the centre / n_bound: xx yy zz xy xz yz */
  double reserved;
} rs_halo_props_t;

typedef struct rs_ctx rs_ctx;

/* Create a context on CUDA device `device` with a copy of *cfg. Validates cfg: box_L > 0,
 * link_len > 0 (rs_fof3d rejects a box of more than 4096 sub-cells per axis), softening >= 0,
 * particle_mass > 0, G > 0, 0 < f_num <= f_den, min_halo_particles >= 2, bound_num >= 0,
 * bound_den > 0, 0 <= tree_theta <= 0.9, surrogate_gate 0 or 1, spot_check >= 0,
 * unbind_passes >= 0.
 * out: host pointer receiving the context. No device memory is allocated yet. */
int rs_ctx_create(rs_ctx** out, const rs_config* cfg, int device);

/* Free the context and all device memory it owns. NULL is accepted. */
int rs_ctx_destroy(rs_ctx* ctx);

/* Message for the last failed call on ctx (empty string after success). */
const char* rs_last_error(rs_ctx* ctx);

/* Number of kernels this context has launched since it was created (host counter). */
int64_t rs_kernel_launches(rs_ctx* ctx);

/* Keys moved by radix-sort passes (one pass = one 8-bit digit over n keys) since the context
 * was created (host counter; instrumentation for the sort's bandwidth figure). */
int64_t rs_sort_keypasses(rs_ctx* ctx);

/* CUDA graphs for the context's static launch sequences (1, the default) or plain launches (0);
 * results are identical either way. A sequence is static when its launches and their
 * arguments do not depend on values read back from the device: the surrogate's training
 * epoch (rs_mlp_train) is captured once and replayed for every epoch. */
int rs_use_graphs(rs_ctx* ctx, int enable);

/* 3D friends-of-friends (Section "Parallelization"). Particles i and j are linked iff
 *   d = x_j - x_i (float32, per dimension), wrapped once: d > L/2 -> d - L, d < -L/2 -> d + L;
 *   (dx*dx + dy*dy) + dz*dz <= link_len*link_len, all float32, no fused multiply-add.
 * Groups are the connected components of the link graph.
 * n:            particles (0 <= n < 2^32 - 1).
 * pos:          float32 [n][3], device, in [0, box_L).
 * ids:          int64 [n], device, unique and >= 0.
 * label_out:    int64 [n], device: the smallest id of the particle's group (input order).
 * n_groups_out: host; number of groups (singletons included). May be NULL.
 * Synchronises `stream` when n_groups_out is not NULL.
 * Errors: RS_ERR_INVALID_ARG (null pointer with n > 0; box_L / link_len beyond the 4096-cell
 * grid; with check_ids, a repeated or negative id), RS_ERR_OOM, RS_ERR_CUDA. */
int rs_fof3d(rs_ctx* ctx, int64_t n, const float* pos, const int64_t* ids, int64_t* label_out,
             int64_t* n_groups_out, void* stream);

/* 6D phase-space FoF hierarchy inside every FoF group (Section "Parallelization"; metric,
 * f = 0.7 and recursion from Rockstar). Level 0 = FoF groups (by fof_label) with at least
 * min_halo_particles members. For a node with members in ascending id order and reference
 * member r (smallest id):
 *   u_i = wrapped x_i - x_r (float32, rs_fof3d's wrap); sigma_x^2, sigma_v^2 = total variances
 *   from float64 sums in the canonical reduction order; inv = float(1/sigma^2), 0 if sigma^2<=0;
 *   d6(i,j) = fl(|u_j-u_i|^2 * inv_sx2) + fl(|v_j-v_i|^2 * inv_sv2) (float32, no FMA);
 *   l2 = the k-th smallest nearest-neighbour d6, k = ceil(f_num*g/f_den) - 1 (0-based);
 *   i ~ j iff d6(i,j) <= l2; children = components with >= min_halo_particles and < g
 *   members, each split again with its own sigmas.
 * Node order: level, then parent index, then smallest id (breadth first).
 * n, pos, ids:   as rs_fof3d; vel float32 [n][3] device.
 * fof_label:     int64 [n] device, a 3D FoF labelling (label = smallest id of the group).
 * n_nodes_out, n_members_out: host, may be NULL; total nodes and total (node, member) pairs.
 * Synchronises `stream`. Errors: RS_ERR_INVALID_ARG, RS_ERR_OOM, RS_ERR_CUDA. */
int rs_fof6d(rs_ctx* ctx, int64_t n, const float* pos, const float* vel, const int64_t* ids,
             const int64_t* fof_label, int64_t* n_nodes_out, int64_t* n_members_out,
             void* stream);

/* Copy the hierarchy of the last rs_fof6d out (device pointers; each may be NULL to skip):
 * node_parent int64 [n_nodes] (-1 for level 0), node_level int32 [n_nodes], node_min_id int64,
 * node_size int64, member_offsets int64 [n_nodes + 1], member_idx int64 [n_members] (particle
 * indices, ascending id within each node), particle_deepest_node int64 [n] (-1 if none).
 * Errors: RS_ERR_STATE if no hierarchy exists, RS_ERR_CUDA. */
int rs_fof6d_copy(rs_ctx* ctx, int64_t* node_parent, int32_t* node_level, int64_t* node_min_id,
                  int64_t* node_size, int64_t* member_offsets, int64_t* member_idx,
                  int64_t* particle_deepest_node, void* stream);

/* Per-node parameters of the 6D split of the last rs_fof6d: float32 [n_nodes][4] device =
 * (inv_sx2, inv_sv2, l2, 0): the inverse total position and velocity variances of the node and
 * its adaptive squared link length. Errors: RS_ERR_STATE, RS_ERR_CUDA. */
int rs_fof6d_node_params(rs_ctx* ctx, float* params_out, void* stream);

/* Unbinding of every node of the last rs_fof6d hierarchy (pos, vel: the same arrays).
 * phi_i = -G m sum_{j != i} 1 / sqrt(|u_j - u_i|^2 + eps^2) over the node's members;
 * KE_i = 0.5 |v_i - v_bulk|^2 (float64, v_bulk = mean member velocity); bound iff
 * KE_i + phi_i < 0 with phi the float64 canonical-order sum; halo iff
 * N_bound >= min_halo_particles and bound_den * N_bound >= bound_num * n.
 * The potential is computed in float32 with a certified error bound; members whose energy
 * is within that bound of zero are recomputed exactly in float64, so flags are exact.
 * Iterative unbinding (rs_config.unbind_passes = P > 1; the paper's Rockstar unbinds in
 * passes, the build offers it as an option): pass p > 1 recomputes v_bulk (canonical-order sum
 * over the members still bound, the others contributing 0.0, divided by their count) and the
 * potential of every member still bound over the members still bound only (the others
 * contributing 0.0 like the self term), re-flags them and leaves the others unbound; it stops
 * after P passes or when a pass removes nobody (rs_unbind_passes tells how many ran). Every
 * pass's flags are exact. Not with the surrogate (RS_ERR_INVALID_ARG).
 * potential_out: float32 [n_members] device (member CSR order) or NULL; with passes, each
 * member's potential from the last pass that evaluated it.
 * bound_out:     uint8 [n_members] device (member CSR order), 1 = bound.
 * n_fallback_out: host, may be NULL: members recomputed in float64.
 * Synchronises `stream`. Errors: RS_ERR_STATE (no hierarchy), RS_ERR_INVALID_ARG,
 * RS_ERR_CUDA. */
int rs_unbind(rs_ctx* ctx, const float* pos, const float* vel, float* potential_out,
              uint8_t* bound_out, int64_t* n_fallback_out, void* stream);

/* Unbinding passes the last rs_unbind ran (1 without iterative unbinding). */
int rs_unbind_passes(rs_ctx* ctx);

/* Ordered pairs (i, j != i) the float32 direct sums of the last rs_unbind evaluated, host int64
 * [2]: [0] nodes of at most 384 members (one-block kernel), [1] larger nodes (register-blocked
 * or, in the plain form, tiled kernel), every node those kernels ran on counted once per pass
 * (nodes the surrogate sends whole to the exact sum included; the tree walk and the exact list
 * sums are counted by rs_tree_stats). Instrumentation for the kernels' work figures. */
int rs_potential_pairs(rs_ctx* ctx, int64_t* pairs_out);

/* Seed halos and the assignment of every FoF-group particle to one of them (Section
 * "Parallelization": subhalo finding inside every FoF halo; the step after the hierarchy). The
 * paper gives no formulas; the reading implemented (the CPU oracle's, bit for bit):
 *   seeds: the nodes of the last rs_fof6d hierarchy without children;
 *   frame: u = wrapped offset (rs_fof3d's wrap) from the level-0 node's smallest-id member;
 *   seed s: centre c_s = float(double(wrapped x_{r_s} - x_{r0}) + S_u / g_s), S_u the
 *     canonical-order sum of the offsets from s's own smallest-id member r_s; bulk velocity
 *     w_s = float(S_v / g_s); metric scales inv_sx2_s, inv_sv2_s of s's own 6D split;
 *   distance: fl(|u - c_s|^2 inv_sx2_s) + fl(|v - w_s|^2 inv_sv2_s) (float32, d6's order);
 *   particle: the seed holding it when its deepest node is a seed, else the nearest seed under
 *     its deepest node (ties: smaller node index);
 *   host of seed s: among the other seeds of s's level-0 node ranking above s (more assigned
 *     particles; equal counts: smaller node index), the nearest by the candidate's metric at
 *     (c_s, w_s); -1 when none ranks above.
 * pos, vel: the arrays given to rs_fof6d (others are re-gathered).
 * particle_seed: int64 [n] device: node index of the particle's seed, -1 outside every node.
 * node_host, node_count: int64 [n_nodes] device or NULL: host seed (-2 for nodes that are not
 * seeds), particles assigned (0 for nodes that are not seeds).
 * n_seeds_out: host, may be NULL (synchronises the stream). Errors: RS_ERR_STATE (no
 * hierarchy), RS_ERR_INVALID_ARG, RS_ERR_OOM, RS_ERR_CUDA. */
int rs_assign_seeds(rs_ctx* ctx, const float* pos, const float* vel, int64_t* particle_seed,
                    int64_t* node_host, int64_t* node_count, int64_t* n_seeds_out, void* stream);

/* Temporal tracking of seed halos between two snapshots of the same particles (the paper's
 * Summary names temporal tracking among Rockstar's features; the reading, the CPU oracle's bit
 * for bit): particles are matched by id; the progenitor of a seed h2 of the later snapshot is
 * the seed h1 of the earlier one holding the most of h2's particles (ties: the smaller index;
 * -1 when none is in a seed earlier); the descendant of h1 is the seed h2 receiving the most of
 * h1's particles (ties: the smaller index). Particles missing from one snapshot or in no seed
 * are ignored; ids must be unique and non-negative within each snapshot.
 * n1, ids1, seed1: the earlier snapshot (int64 [n1] device; seed1 = rs_assign_seeds'
 * particle_seed, node indices or -1); n_nodes1 its node count; likewise n2, ids2, seed2,
 * n_nodes2 for the later one.
 * progenitor, prog_shared: int64 [n_nodes2] device (-1 / 0 for nodes without progenitor);
 * descendant, desc_shared: int64 [n_nodes1] device. Work on `stream`; synchronises it.
 * Errors: RS_ERR_INVALID_ARG (sizes >= 2^32 - 1, null pointers), RS_ERR_OOM, RS_ERR_CUDA. */
int rs_track(rs_ctx* ctx, int64_t n1, const int64_t* ids1, const int64_t* seed1, int64_t n_nodes1,
             int64_t n2, const int64_t* ids2, const int64_t* seed2, int64_t n_nodes2,
             int64_t* progenitor, int64_t* prog_shared, int64_t* descendant,
             int64_t* desc_shared, void* stream);

/* Halo properties of every node of the hierarchy over its bound members (last rs_unbind),
 * float64 sums in the canonical reduction order over members in ascending id order with
 * unbound members contributing 0.
 * props_out: rs_halo_props_t [n_nodes] device. Errors: RS_ERR_STATE, RS_ERR_CUDA. */
int rs_halo_props(rs_ctx* ctx, rs_halo_props_t* props_out, void* stream);

/* ---- Batched snapshot stream ------------------------------------------------------------
 * The whole pipeline (rs_fof3d, rs_fof6d, rs_unbind with no potential output, rs_halo_props)
 * over many independent snapshots in one call (Section "Parallelization": independent units of
 * work - there FoF halos over OpenMP threads - keep every core busy; here independent snapshots
 * keep the GPU busy). Snapshots are taken largest first by `lanes` worker lanes, each a
 * context of its own with its own CUDA stream and host thread, so one lane's kernels fill the
 * GPU while another waits on a count it reads back. Every snapshot's outputs are identical to
 * running the four calls on it alone with the same configuration.
 * One snapshot of the batch; every pointer is a device pointer owned by the caller. */
typedef struct rs_snapshot {
  int64_t n;                  /* particles (< 2^32 - 1) */
  float box_L;                /* this snapshot's box side, link length and softening; the */
  float link_len;             /*   other parameters are the calling context's */
  float softening;
  float reserved;
  const float* pos;           /* float32 [n][3] */
  const float* vel;           /* float32 [n][3] */
  const int64_t* ids;         /* int64 [n], unique, non-negative */
  int64_t* label_out;         /* int64 [n]: 3D FoF label (smallest id of the group); required */
  int64_t* deepest_out;       /* int64 [n] or NULL: deepest hierarchy node of each particle, -1 */
  int64_t node_capacity;      /* entries available in node_parent_out and props_out */
  int64_t* node_parent_out;   /* int64 [node_capacity] or NULL: parent node, -1 at level 0 */
  rs_halo_props_t* props_out; /* [node_capacity] or NULL: rs_halo_props of every node */
} rs_snapshot;

/* Runs the pipeline over snaps[0 .. n_snap) with `lanes` lanes (1 .. 16). The lanes' contexts
 * copy ctx's configuration (with each snapshot's box_L, link_len, softening) and, with
 * use_surrogate, ctx's trained surrogate; they are created at the first call and kept, with
 * their scratch memory, until rs_ctx_destroy(ctx).
 * counts_out: host int64 [n_snap][4] or NULL: FoF groups, hierarchy nodes, hierarchy members,
 * hierarchy levels of each snapshot.
 * The lanes wait for the work already enqueued on `stream`; the call returns when every
 * snapshot is done (it synchronises the lanes). Errors: RS_ERR_INVALID_ARG (a bad snapshot or
 * lane count), RS_ERR_STATE (use_surrogate without a trained surrogate on ctx),
 * RS_ERR_CAPACITY (a snapshot has more nodes than node_capacity while node_parent_out or
 * props_out is given; every other snapshot is still processed and counts_out is filled, so the
 * caller can resize), or the first error of a lane (its message in rs_last_error(ctx)). */
int rs_run_batched(rs_ctx* ctx, int32_t n_snap, const rs_snapshot* snaps, int32_t lanes,
                   int64_t* counts_out, void* stream);

/* ---- Certified tree bound of the potential (batched forms) ---------------------------------
 * For nodes with at least tree_min_members members, rs_unbind (called with potential_out NULL)
 * decides most flags from a certified interval of each member's potential sum
 * S_i = sum_{j != i} (|u_j - u_i|^2 + eps^2)^(-1/2) instead of the O(g) direct sum: a
 * Barnes-Hut walk over a Hilbert-ordered tree of the node (leaves of 32 members, 8 children per
 * cell) takes a cell as its quadrupole expansion when its radius bound a is at most tree_theta
 * times the softened distance R', and adds the rigorous truncation bound (n/R') h^3 / (1 - h),
 * h = a / R' (Legendre expansion of the softened kernel, |P_l| <= 1); float32 rounding is
 * covered by a 1e-5 relative slack. A member is decided when the whole interval of
 * E = KE - G m S lies on one side of zero; the others take the exact path (blocked float32 sum
 * with its certified bound, then the float64 canonical-order potential). Flags are therefore
 * identical to the direct sum's. The paper computes the exact potential; this is the build's
 * O(g log g) potential for nodes of 10^5 - 10^6 members (the next step after the exact kernel).
 *
 * rs_tree_stats: host int64 [8] of the last rs_unbind: tree nodes, their members, members
 * decided by the bound, members sent to the exact path, cell expansions evaluated, direct pair
 * terms evaluated by the walk, pair terms of the exact list sums (tree and surrogate paths), 0.
 * rs_tree_record(ctx, 1): later rs_unbind calls also record every bounded member's interval;
 * rs_tree_bounds then copies them out: lo_out, hi_out float64 [n_members] device (member CSR
 * order), NaN for members whose flag did not come from the bound walk. Errors: RS_ERR_STATE when
 * the last rs_unbind recorded nothing. Instrumentation for tests, not part of the method. */
int rs_tree_stats(rs_ctx* ctx, int64_t* stats_out);
int rs_tree_record(rs_ctx* ctx, int enable);
int rs_tree_bounds(rs_ctx* ctx, double* lo_out, double* hi_out, void* stream);

/* Float64 sum of a[0..m) in the canonical reduction order every float64 sum of the path uses
 * (chunks of 1024; lane l of a chunk adds terms l, l+32, ... in order; lanes combine by the
 * halving tree; chunk totals by the level-by-level pairwise tree, odd element carried up).
 * a: float64 [m] device; out: float64 [1] device. Exposed so the order can be checked alone.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_CUDA. */
int rs_cro_sum(rs_ctx* ctx, int64_t m, const double* a, double* out, void* stream);

/* rs_cro_sum without any device allocation, for callers that cannot allocate: code running
 * while a stream is being captured into a CUDA graph, allocator or memory-pool callbacks, or
 * hosts that forbid the library from using the device heap. The paper has no counterpart; this
 * is a library convenience. Same result as rs_cro_sum, bit for bit, with no context.
 * Scratch: a file-scope device array of 65536 float64 chunk totals (512 KiB, held on every GPU
 * that loads the library until the process exits), so m is limited to 2^26 terms.
 * The first call on a device (with that device current) looks up the array's device address;
 * make that first call before any stream capture. The address is cached per device ordinal for
 * the life of the process: after cudaDeviceReset (or anything else that destroys and recreates
 * the device's primary context) it is stale, so a process that resets a device must not call
 * rs_cro_sum_noalloc on it again. Calls share the array and keep the last call's contents:
 * calls whose kernels overlap on the GPU race and must be serialised.
 * a: float64 [m] device; out: float64 [1] device; stream: cudaStream_t as void*.
 * Errors: RS_ERR_INVALID_ARG (m < 0, null pointer), RS_ERR_CAPACITY (m > 2^26), RS_ERR_CUDA. */
int rs_cro_sum_noalloc(int64_t m, const double* a, double* out, void* stream);

/* ---- Learned surrogate of the binding energy (batched form) --------------------------------
 * A small MLP predicts psi = phi r_vir / (G M_node) from 8 per-member features; members whose
 * predicted energy clears a margin are classified without the O(n^2) potential, the rest (and
 * any node failing a spot check) take the exact path. The paper has no learned component; this
 * is the build's batched + surrogate form. Per node with >= 1024 members, rs_unbind gates
 * |E_pred| > margin_factor * err * G M / r_vir with err = err_max, the held-out maximum error of
 * the training (surrogate_gate = 0), or err = max(max |psi_hat - psi| over 64 evenly spaced
 * members evaluated exactly, err_max / 8) (surrogate_gate = 1). It then re-checks exactly the
 * spot_check gated members of smallest margin plus about spot_check more sampled at every
 * margin, and recomputes the whole node exactly if one flag differs or one error exceeds
 * margin_factor / 2 * err. Zero flag mismatches is measured on held-out snapshots, not
 * guaranteed.
 * Network (8 -> 64 -> 64 -> 1, ReLU), bf16 weights and hidden activations, float32
 * accumulation on tensor cores:
 *   z1 = b1 + W1^T bf16(x); h1 = bf16(relu(z1)); z2 = b2 + W2^T h1; h2 = bf16(relu(z2));
 *   y = b3 + sum_k bf16(W3)[k] h2[k] (float32; four partial sums combined pairwise).
 * Parameters: float32 vector of RS_MLP_PARAMS = 4801 entries: W1 [8][64] at 0, b1 [64] at 512,
 * W2 [64][64] at 576 (row = input), b2 [64] at 4672, W3 [64] at 4736, b3 at 4800. */
#define RS_MLP_PARAMS 4801

/* Load (host float32 [4801]) or read back the context's float32 master parameters. */
int rs_mlp_set_params(rs_ctx* ctx, const float* params_host);
int rs_mlp_get_params(rs_ctx* ctx, float* params_host);
/* Held-out maximum |psi_hat - psi| from training (set by rs_mlp_train, or by the caller): the
 * error of the default gate (and err_max / 8 the floor of the calibrated gate's node error). */
int rs_mlp_set_err_max(rs_ctx* ctx, float err_max);
int rs_mlp_get_err_max(rs_ctx* ctx, float* err_max_out);

/* Surrogate checkpoint (host file I/O): rs_surrogate_save writes the context's float32 master
 * parameters and held-out maximum error to `path` (little endian: magic "RSMLPv01", uint32
 * 4801, uint32 0, float32 err_max, float32 params[4801], uint64 FNV-1a hash of the params'
 * bytes); rs_surrogate_load reads such a file into the context (weights and err_max), so a
 * network trained once serves later runs. Errors: RS_ERR_INVALID_ARG (unopenable, truncated or
 * corrupt file: bad magic, count or hash), RS_ERR_STATE (save without weights), RS_ERR_CUDA. */
int rs_surrogate_save(rs_ctx* ctx, const char* path);
int rs_surrogate_load(rs_ctx* ctx, const char* path);

/* Inference: x float32 [n][8] device -> y float32 [n] device. */
int rs_mlp_forward(rs_ctx* ctx, int64_t n, const float* x, float* y, void* stream);

/* Gradient of L = (1/n) sum (y - t)^2 over one batch: grad float32 [4801] device; sse_out host
 * (sum of squared errors) may be NULL. Deterministic. */
int rs_mlp_gradient(rs_ctx* ctx, int64_t n, const float* x, const float* t, float* grad,
                    double* sse_out, void* stream);

/* Train from a seeded He-uniform start with Adam (beta 0.9/0.999, eps 1e-8) on float32 masters:
 * samples x float32 [n][8], t float32 [n] (device); a seeded permutation holds out the last
 * holdout_num/holdout_den; minibatches of `batch` (a partial last batch is left out of the
 * epoch); `epochs` passes, each reshuffled; with graphs on (rs_use_graphs) one epoch's
 * launches are a CUDA graph replayed every epoch. Outputs (host, may be NULL):
 * held-out max |y - t| (also stored as the gate's error) and the last batch's mean squared
 * error. Errors: RS_ERR_INVALID_ARG, RS_ERR_OOM, RS_ERR_CUDA. */
int rs_mlp_train(rs_ctx* ctx, int64_t n, const float* x, const float* t, int32_t epochs,
                 int32_t batch, float lr, uint64_t seed, int32_t holdout_num, int32_t holdout_den,
                 float* err_max_out, double* train_mse_out, void* stream);

/* Surrogate features of the members of every node with >= 1024 members, after rs_unbind:
 * feat_out float32 [n_members][8] device (room for all members; the first *n_out rows are
 * written, node after node, members in id order): r/r_vir (r from the node's mean position),
 * fractions of the node's members with radius below 0.5 r, r, 2 r and 4 r, |v - v_bulk| /
 * sigma_v,1D, log10 g, and psi_mp (the node's potential at the member from the radially split
 * multipole expansion to quadrupole order, in units of G g m / r_vir).
 * psi_out float32 [n_members] device or NULL: training target
 * psi = phi r_vir / (G g m) from the last rs_unbind's float32 potential (that rs_unbind must
 * have computed every member's potential: no surrogate, and potential_out given so that the
 * certified tree bound was not used). n_out: host. Errors: RS_ERR_STATE, RS_ERR_OOM,
 * RS_ERR_CUDA. */
int rs_surrogate_features(rs_ctx* ctx, float* feat_out, float* psi_out, int64_t* n_out,
                          void* stream);

/* Counters of the last rs_unbind (host int64 [11]): members of surrogate nodes, gated by the
 * surrogate, evaluated exactly (calibration members and the members outside the gate, in
 * nodes not sent whole), spot-checked, nodes failing the spot check, float64 fallbacks in the
 * surrogate path, float64 fallbacks of the direct sums, gated members recomputed because their
 * node failed, members of nodes sent whole to the exact path (at most 1/20 of their members
 * gated), members whose flag the surrogate decided, spot-checked members whose surrogate flag
 * differed from the exact one. Members = decided + exact + spot-checked + recomputed +
 * whole-node (the calibration members are counted in exact). */
int rs_surrogate_stats(rs_ctx* ctx, int64_t* stats_out);

/* Stable LSD radix sort of (key, value) pairs by key bits [0, nbits), in place: the sort that
 * orders particles by cell key for the 3D FoF cell list and members by (group, id) for the 6D
 * hierarchy. keys: uint64 [n] device; vals: uint32 [n] device (moved with their keys; equal
 * keys keep their input order). Uses the context's scratch. Errors: RS_ERR_INVALID_ARG
 * (n >= 2^32 - 1, nbits > 64), RS_ERR_OOM, RS_ERR_CUDA. */
int rs_sort_pairs(rs_ctx* ctx, int64_t n, int nbits, uint64_t* keys, uint32_t* vals, void* stream);

/* Per-kernel CUDA-event timing of the dominant kernels (k_fof_link, k_sort_*, k_nn6d,
 * k_link6d, k_select_l2, k_potential, k_fallback). rs_profile(ctx, 1) clears the totals and
 * starts recording events on each launch's stream; rs_profile(ctx, 0) stops. The paper reports
 * whole-run wall times only; this is instrumentation, not part of the method.
 * rs_profile_get: totals of entry `index` (0-based, in first-seen order): kernel name (host
 * buffer of name_cap bytes), summed milliseconds and launch count (host). Waits for the
 * recorded events. Errors: RS_ERR_CAPACITY when index is past the last entry. */
int rs_profile(rs_ctx* ctx, int enable);

/* Work counting of the batched form's pruned 6D kernels (instrumentation, not part of the
 * method): while enabled, k_nn6d_pruned and k_link6d_pruned run a variant that tallies, per
 * query lane, the d6 evaluations it performs and the box lower bounds it computes (bucket,
 * sub-bucket and superbucket tests; box-box tests counted once per warp); the results are
 * unchanged. rs_count_work(ctx, 1, NULL) clears the tallies and enables counting;
 * rs_count_work(ctx, 0, counts) disables it. counts_out (host int64 [6], may be NULL) receives,
 * after a device synchronisation: NN d6 evaluations, NN box tests, link d6 evaluations, link
 * box tests, nodes whose nearest-neighbour search ran with sampled bounds, and those of them
 * whose l2 fell outside the bounds (searched exactly again), accumulated since the last
 * enable. Errors: RS_ERR_OOM, RS_ERR_CUDA. */
int rs_count_work(rs_ctx* ctx, int enable, int64_t* counts_out);

/* The batched form's sampled nearest-neighbour bounds (see rs_fof6d): the scale of their
 * margin (1 = the default) and the smallest node searched with them (0 = the default, 4096
 * members). Tuning and test instrumentation; the results do not depend on either: a negative
 * scale gives every such node empty bounds, so each one fails the check after the selection and
 * is searched again exactly. Errors: RS_ERR_INVALID_ARG (NaN scale, negative size). */
int rs_nn_bounds(rs_ctx* ctx, float margin_scale, int64_t min_members);

/* Autotuner choices of the context (host outputs; either may be NULL). The members per thread
 * of the register-blocked potential sums (rs_unbind's direct sum; the surrogate path's sums for
 * members outside its gate) are picked among 2, 4 and 8 on the first call whose input is large
 * enough (2^20 members, resp. surrogate members): each candidate is timed with CUDA events on
 * that call's own data (the sums are bit-identical for every candidate) and the fastest is kept
 * for the context's later calls. choice_out int32 [2]: blocked potential, list potential (0 =
 * not tuned yet); ms_out float [6]: the candidates' times (2, 4, 8) for each. Build-time
 * choice, not part of the method. Errors: RS_ERR_INVALID_ARG. */
int rs_tuning(rs_ctx* ctx, int32_t* choice_out, float* ms_out);
int rs_profile_get(rs_ctx* ctx, int index, char* name, int name_cap, double* total_ms,
                   int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* RS_GB300_H */

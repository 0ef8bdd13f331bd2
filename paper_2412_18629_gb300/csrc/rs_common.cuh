// Internal definitions shared by the library's translation units: the context, scratch
// buffers, error handling, and small device helpers (exact float32/float64 arithmetic,
// union-find, warp reductions in the canonical order).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/rs_gb300.h"

namespace rs {

// ------------------------------------------------------------------------------------------
// Scratch buffers: grow-only device allocations owned by the context, one per slot.
enum Slot : int {
  // rs_fof3d
  S_KEY_A, S_KEY_B, S_VAL_A, S_VAL_B, S_SORT_HIST, S_POS_SORTED, S_ROW_START, S_CELL_END,
  S_PARENT, S_MINID, S_COUNTER,
  // rs_fof6d (level work)
  S_GKEY_A, S_GKEY_B, S_GVAL_A, S_GVAL_B, S_NN2, S_UF, S_ROOT_CNT, S_CHILD_IDX, S_FLAGS,
  S_SCAN_TMP, S_CHUNK_OFF, S_CHUNK_SUM, S_NODE_TMP, S_SELECT,
  // hierarchy state (persists until the next rs_fof6d)
  S_H_MEM, S_H_MNODE, S_H_U, S_H_V, S_H_NODE_OFF, S_H_NODE_SIZE, S_H_NODE_PARENT,
  S_H_NODE_LEVEL, S_H_NODE_MINID, S_H_NODE_REF, S_H_NODE_INV, S_H_DEEPEST, S_H_DEEPPOS, S_H_WORK,
  S_H_NODE_MOM,
  // rs_unbind / rs_halo_props state
  S_U_PHI, S_U_BOUND, S_U_NB, S_U_VBULK, S_U_AMBIG, S_U_FLAGS, S_U_TILEBIG,
  S_U_TILEPERM, S_U_OKEY_A, S_U_OKEY_B, S_U_OVAL_A, S_U_OVAL_B, S_U_FBMAX, S_U_FBCHUNK,
  // batched form: pruned 6D searches
  S_P_MEANU, S_P_MEANV, S_P_US, S_P_VS, S_P_SP, S_P_BOFF, S_P_BUCKET, S_P_BOX, S_P_SUB,
  S_P_SBOFF, S_P_SBOX, S_P_ORDER, S_P_QCTR, S_P_WORK, S_P_NSTART, S_P_NCNT, S_P_APOS,
  S_P_USA, S_P_VSA, S_P_SPA, S_P_QKEY_A, S_P_QKEY_B, S_P_QVAL_A, S_P_QVAL_B, S_P_QFS, S_P_QFR,
  S_P_QS, S_P_QR, S_P_QCOUNT, S_P_BOUNDS, S_P_FAILED,
  // surrogate MLP
  S_MLP_DEV, S_MLP_W, S_MLP_PART, S_MLP_SSE, S_MLP_M, S_MLP_G, S_MLP_IDX, S_MLP_BIDX, S_MLP_XH,
  S_MLP_YH, S_MLP_CORR, S_MLP_STEP,
  // surrogate gating in rs_unbind
  S_SUR_OFF, S_SUR_RANK, S_SUR_STAT, S_SUR_MEM, S_SUR_BIG, S_SUR_FEAT, S_SUR_PSI, S_SUR_MARGIN,
  S_SUR_SFLAG, S_SUR_CHECKED, S_SUR_SX, S_SUR_LIST_A, S_SUR_LIST_B, S_SUR_GCOUNT, S_SUR_TAU,
  S_SUR_FAIL, S_SUR_COUNTERS, S_SUR_FIX, S_SUR_SPOS, S_SUR_PSISPH, S_SUR_ECOUNT, S_SUR_FULL,
  S_SUR_MP, S_SUR_ERRN, S_SUR_LIST_C, S_SUR_LSCAN, S_SUR_LOFS, S_SUR_TILES, S_SUR_WANT,
  // certified tree bound of the potential (rs_tree.cu)
  S_T_OFF, S_T_RANK, S_T_COFF, S_T_NODES, S_T_BOX, S_T_KA, S_T_KB, S_T_VA, S_T_VB, S_T_X, S_T_POS,
  S_T_CELL, S_T_ORDER, S_T_WF, S_T_WL, S_T_WR, S_T_UF, S_T_LIST, S_T_LR, S_T_SX, S_T_REC,
  S_T_WANT,
  // seed halos (rs_seeds.cu)
  S_SEED_KIDS, S_SEED_ROOT, S_SEED_UCNT, S_SEED_UOFF, S_SEED_CEN, S_SEED_SUMS, S_SEED_SEG,
  S_SEED_COUNT, S_SEED_LIST,
  // temporal tracking (rs_track.cu)
  S_TRK_HEAD, S_TRK_RSTART, S_TRK_RKEY, S_TRK_KA, S_TRK_KB, S_TRK_VA, S_TRK_VB, S_TRK_H1,
  S_TRK_FLAG,
  // iterative unbinding (rs_unbind.cu)
  S_U_PREV, S_U_UM, S_U_PCNT,
  // batched snapshot stream (rs_batch.cu): a lane's bound flags
  S_BATCH_BOUND,
  S_NUM_SLOTS
};

// Nodes with at least this many members are unbound through the surrogate when it is enabled.
constexpr int64_t kSurrogateMinMembers = 1024;
// Default smallest node unbound through the certified tree bound (batched form) and its
// opening angle (a cell is expanded when its radius bound is at most theta times the distance).
constexpr int64_t kTreeMinDefault = 16384;
constexpr float kTreeThetaDefault = 0.45f;

struct Buffer {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace rs

struct rs_ctx {
  rs_config cfg;
  int device = 0;
  char err[512] = {0};
  rs::Buffer buf[rs::S_NUM_SLOTS];
  int64_t launches = 0;
  // host pinned mailbox for small device->host results
  int64_t* host_box = nullptr;
  // hierarchy state
  bool have_hier = false;
  int64_t n_particles = 0;
  int64_t n_nodes = 0;
  int64_t n_members = 0;
  int32_t n_levels = 0;
  bool have_unbind = false;
  bool have_mlp = false;        // surrogate weights loaded or trained
  float mlp_err_max = 0.f;      // held-out max |psi_hat - psi| of the surrogate
  const float* h_pos = nullptr;  // arrays the hierarchy's U, V were gathered from
  const float* h_vel = nullptr;
  // surrogate path of the last rs_unbind
  bool last_unbind_surrogate = false;
  int64_t sur_members = 0;
  int64_t sur_nbig = 0;
  const uint64_t* sur_rkeys = nullptr;
  int64_t sur_stats[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  // certified tree bound (batched form): smallest node, opening angle, state of the last build
  int64_t tree_min = 0;         // 0: the tree bound is off
  float tree_theta = 0.5f;
  int64_t tree_nt = 0, tree_T = 0, tree_C = 0;
  bool tree_record = false;     // record each member's interval (rs_tree_record)
  bool tree_recorded = false;
  int64_t tree_stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int32_t unbind_passes_run = 0;  // passes the last rs_unbind ran (iterative unbinding)
  int64_t pot_pairs[2] = {0, 0};  // ordered pairs the direct sums evaluated (last rs_unbind)
  float nn_bound_margin = 1.f;    // scale of the sampled nearest-neighbour bounds' margin
  int64_t nn_bound_min = 0;       // smallest node searched with sampled bounds (0: default)
  bool nn_bounded_level = false;  // the last level's searches used sampled bounds
  // optional per-kernel CUDA-event timing of the dominant kernels (rs_profile)
  bool profile = false;
  bool count_work = false;  // counting variants of the pruned 6D kernels (rs_count_work)
  int sort_blocks = 0;      // radix-sort blocks resident at once on the device (0 = not known yet)
  int64_t sort_keypasses = 0;  // keys moved by radix-sort passes since the context was created
  // autotuner choices (0 = not tuned yet) and the timings they were chosen from
  int tune_blk_r = 0;       // members per thread of the blocked potential (2, 4, 8)
  float tune_blk_ms[3] = {0.f, 0.f, 0.f};
  int tune_list_r = 0;      // members per thread of the surrogate path's list sums (2, 4, 8)
  float tune_list_ms[3] = {0.f, 0.f, 0.f};
  struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_free;
  struct ProfTot {
    std::string name;
    double ms;
    int64_t launches;
  };
  std::vector<ProfTot> prof_tot;
  // lanes of rs_run_batched: contexts with their own streams, created at the first call
  std::vector<rs_ctx*> lanes;
  std::vector<void*> lane_streams;  // cudaStream_t
  void* lane_event = nullptr;       // cudaEvent_t: the caller's stream as the lanes start
  // CUDA graphs for static launch sequences (rs_use_graphs): on by default; the stream graphs
  // are captured on (the caller's may be the legacy default stream, which cannot be captured)
  bool use_graphs = true;
  void* graph_stream = nullptr;     // cudaStream_t
};

namespace rs {

int set_error(rs_ctx* ctx, int code, const char* fmt, ...);

// Device buffer of at least `bytes` for `slot` (contents undefined on growth).
void* scratch(rs_ctx* ctx, int slot, size_t bytes);

template <class T>
T* scratch_t(rs_ctx* ctx, int slot, size_t count) {
  return static_cast<T*>(scratch(ctx, slot, count * sizeof(T)));
}

// Propagates an error code out of the calling entry point.
#define RS_TRY(expr)            \
  do {                          \
    int _rc = (expr);           \
    if (_rc != RS_OK) return _rc; \
  } while (0)

#define RS_CUDA(ctx, expr)                                                            \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess)                                                            \
      return rs::set_error((ctx), RS_ERR_CUDA, "%s: %s (%s:%d)", #expr,               \
                           cudaGetErrorString(_e), __FILE__, __LINE__);               \
  } while (0)

// CUDA-event timing around one launch when profiling is on (records on the launch stream).
struct ProfScope {
  rs_ctx* ctx;
  cudaStream_t st;
  int idx = -1;
  ProfScope(rs_ctx* c, const char* name, cudaStream_t s);
  ~ProfScope();
};

// Check the launch that was just enqueued and count it.
int after_launch(rs_ctx* ctx, const char* name);
#define RS_LAUNCHED(ctx, name) RS_TRY(rs::after_launch((ctx), (name)))

inline unsigned grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 0x7fffffff) g = 0x7fffffff;
  return unsigned(g);
}

// ------------------------------------------------------------------------------------------
// Primitive device algorithms (rs_primitives.cu).
//
// LSD radix sort of (key, value) pairs over bits [0, nbits) of the 64-bit key; stable.
// Sorted output ends in (*keys_out, *vals_out), which point into the given A/B buffers.
int radix_sort_u64(rs_ctx* ctx, int64_t n, int nbits, uint64_t* keys_a, uint32_t* vals_a,
                   uint64_t* keys_b, uint32_t* vals_b, uint64_t** keys_out,
                   uint32_t** vals_out, cudaStream_t st);

// Exclusive prefix sum of int64 values in place; returns the total via *total_dev (device).
int exclusive_scan_i64(rs_ctx* ctx, int64_t n, int64_t* data, int64_t* total_dev,
                       cudaStream_t st);

// Copy `bytes` device -> host mailbox and synchronise the stream.
int read_back(rs_ctx* ctx, const void* dev, size_t bytes, cudaStream_t st);

// Capture the launches `body(stream)` enqueues into an instantiated graph. Nothing runs while
// capturing: body must only enqueue stream work (scratch already sized, no read-backs). The
// launches it counts are returned in *launches and credited at each replay instead.
int begin_capture(rs_ctx* ctx, cudaStream_t* cs);
int end_capture(rs_ctx* ctx, cudaStream_t cs, int body_rc, int64_t launches0, bool profile,
                cudaGraphExec_t* exec, int64_t* launches);

template <class F>
int capture_graph(rs_ctx* ctx, F&& body, cudaGraphExec_t* exec, int64_t* launches) {
  cudaStream_t cs = nullptr;
  RS_TRY(begin_capture(ctx, &cs));
  const bool profile = ctx->profile;
  ctx->profile = false;  // no event records inside a graph
  const int64_t l0 = ctx->launches;
  const int rc = body(cs);
  return end_capture(ctx, cs, rc, l0, profile, exec, launches);
}

// Replay an instantiated graph on `st` (counted as `launches` kernel launches).
int launch_graph(rs_ctx* ctx, cudaGraphExec_t exec, int64_t launches, cudaStream_t st);

// Copy src's trained surrogate (weights and held-out maximum error) to dst (same device).
int mlp_copy(rs_ctx* dst, rs_ctx* src, cudaStream_t st);

// Device arrays of the 6D hierarchy held by a context (valid after rs_fof6d). Members are
// stored node after node, each node's members in ascending id order.
struct Hier {
  uint32_t* mem;       // particle index per (node, member)
  uint32_t* mnode;     // node per member position
  float4* U;           // member offset from the node's reference (smallest-id) member
  float4* V;           // member velocity
  int64_t* node_off;   // [nodes + 1] member offsets
  int64_t* node_size;
  int64_t* node_parent;
  int32_t* node_level;
  int64_t* node_minid;
  float4* inv;         // (inv_sx2, inv_sv2, l2, 0) of the node's 6D split
  float4* mom;         // (mean u, sigma_v,1D) as float, from the same canonical-order moments
  float4* ref;         // reference member position
  int64_t* deepest;    // [n] deepest node per particle, -1 if none
  uint32_t* deepest_pos;  // [n] member position of the particle in its deepest node
};
Hier hier_of(rs_ctx* ctx);

}  // namespace rs

// ------------------------------------------------------------------------------------------
// Device helpers
namespace rsd {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// float32 periodic minimum-image difference b - a, never contracted or reassociated.
__device__ __forceinline__ float wrap_diff(float a, float b, float L, float hL) {
  float d = __fsub_rn(b, a);
  if (d > hL) {
    d = __fsub_rn(d, L);
  } else if (d < -hL) {
    d = __fadd_rn(d, L);
  }
  return d;
}

// (dx*dx + dy*dy) + dz*dz in float32 with every operation rounded separately.
__device__ __forceinline__ float sq3(float dx, float dy, float dz) {
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Union-find over uint32 indices; roots are the smallest index of their set. Parent reads
// bypass L1 (other SMs write them); stale values are still ancestors, so reads stay valid.
__device__ __forceinline__ uint32_t uf_find(uint32_t* parent, uint32_t x) {
  uint32_t p = __ldcg(parent + x);
  while (p != x) {
    const uint32_t gp = __ldcg(parent + p);
    if (gp != p) parent[x] = gp;  // path halving (benign race: gp is an ancestor of x)
    x = p;
    p = gp;
  }
  return x;
}

__device__ __forceinline__ uint32_t uf_find_ro(const uint32_t* parent, uint32_t x) {
  uint32_t p = __ldcg(parent + x);
  while (p != x) {
    x = p;
    p = __ldcg(parent + x);
  }
  return x;
}

// Hook the larger root under the smaller; retries when another thread moved a root first.
__device__ __forceinline__ void uf_unite(uint32_t* parent, uint32_t a, uint32_t b) {
  while (true) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicCAS(parent + a, a, b);
    if (old == a) return;
  }
}

// Size class of a node with g members for size-ordered work queues: 8 floor(log2 g) + the
// next 3 bits of g (monotone in g; 8..254 for 2 <= g < 2^31), so one 8-bit radix pass on
// 255 - class orders the work largest first.
__device__ __forceinline__ uint32_t size_class(int64_t g) {
  const int L = 63 - __clzll(static_cast<unsigned long long>(g));
  const uint32_t f = L >= 3 ? uint32_t((uint64_t(g) >> (L - 3)) & 7u) : uint32_t((uint64_t(g) << (3 - L)) & 7u);
  const uint32_t c = uint32_t(L < 31 ? L : 31) * 8u + f;
  return c > 254u ? 254u : c;
}

// Exact float32 -> float64 conversion on the integer pipe (the float64 pipe of this part runs
// 2 lanes per clock per SM): for normal values the sign, the exponent rebiased by 1023 - 127 and
// the mantissa shifted up by 29 bits; zero, subnormal, infinite and NaN values take the
// hardware conversion. Bit-identical to double(f).
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return double(f);
  const uint64_t bits = (uint64_t(u >> 31) << 63) | (uint64_t(e + 896u) << 52) |
                        (uint64_t(u & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(bits));
}

// Exact float64 square of a float32 value on the integer pipe. A float is m 2^(e-150) (m the
// 24-bit significand with its leading bit, or the subnormal significand with e = 1), so its
// square is the 48-bit integer m^2 times 2^(2e-300): exactly representable in float64, hence
// equal to the rounded FP64 product f2d(f) * f2d(f); the bits are assembled from m^2's leading
// bit position. Zero, infinite and NaN values take the FP64 multiply.
__device__ __forceinline__ double sq_f2d(float f) {
  const uint32_t b = __float_as_uint(f) & 0x7fffffffu;
  uint32_t e = b >> 23, m = b & 0x7fffffu;
  if (b == 0u || e == 0xffu) {
    const double d = double(f);
    return __dmul_rn(d, d);
  }
  if (e == 0u) e = 1u; else m |= 0x800000u;
  const uint64_t mm = uint64_t(m) * uint64_t(m);
  const int top = 63 - __clzll(static_cast<long long>(mm));
  const uint64_t frac = (mm << (52 - top)) & ((uint64_t(1) << 52) - 1u);
  const uint64_t ebits = uint64_t(int64_t(2) * (int64_t(e) - 150) + top + 1023);
  return __longlong_as_double(static_cast<long long>((ebits << 52) | frac));
}

// Warp-aggregated atomics for keys laid out in runs (members in node order, particles in cell
// order): every lane of the warp calls these; a lane with `valid` false contributes nothing and
// ends a run. Each contiguous run of valid lanes with equal keys gets an id (the number of run
// starts up to the lane); a shuffle-down tree combines only lanes of the same run, so the
// run's first lane holds the run's total (sum or minimum) and issues its one atomic.
__device__ __forceinline__ uint32_t run_id(uint32_t key, bool valid, bool& head) {
  const int lane = threadIdx.x & 31;
  const uint32_t kp = __shfl_up_sync(0xffffffffu, key, 1);
  const bool vp = __shfl_up_sync(0xffffffffu, int(valid), 1) != 0;
  const bool start = !valid || lane == 0 || !vp || kp != key;
  head = valid && start;
  const unsigned starts = __ballot_sync(0xffffffffu, start);
  return uint32_t(__popc(starts & (0xffffffffu >> (31 - lane))));
}

template <class T>
__device__ __forceinline__ void warp_run_add(T* base, uint32_t key, bool valid, T v) {
  const int lane = threadIdx.x & 31;
  bool head;
  const uint32_t rid = run_id(key, valid, head);
  v = valid ? v : T(0);
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T o = __shfl_down_sync(0xffffffffu, v, off);
    const uint32_t ro = __shfl_down_sync(0xffffffffu, rid, off);
    if (lane + off < 32 && ro == rid) v += o;
  }
  if (head && v) atomicAdd(base + key, v);
}

__device__ __forceinline__ void warp_run_min(unsigned long long* base, uint32_t key, bool valid,
                                             unsigned long long v) {
  const int lane = threadIdx.x & 31;
  bool head;
  const uint32_t rid = run_id(key, valid, head);
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long o = __shfl_down_sync(0xffffffffu, v, off);
    const uint32_t ro = __shfl_down_sync(0xffffffffu, rid, off);
    if (lane + off < 32 && ro == rid && o < v) v = o;
  }
  if (head) atomicMin(base + key, v);
}

// One atomic per warp for a count of the lanes with `pred`.
__device__ __forceinline__ void warp_count(unsigned long long* ctr, bool pred) {
  const unsigned b = __ballot_sync(0xffffffffu, pred);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(ctr, (unsigned long long)__popc(b));
}

// Canonical-order combination of the 32 lane partial sums of a warp: halving tree
// s[l] += s[l + off], off = 16 .. 1, realised as an xor butterfly (IEEE + commutes, so lane
// 0 ends with exactly the halving-tree value). When only lanes below 2 off0 hold terms (the
// others hold 0.0 and no lane sum is -0.0), the steps above off0 add 0.0 to every sum they
// touch, so starting at off0 gives lane 0 the same value.
__device__ __forceinline__ double warp_cro_combine(double s, int off0 = 16) {
#pragma unroll
  for (int off = off0; off >= 1; off >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, off));
  return s;
}

// acc <- acc + v in a canonical-order lane sum. The first add of a lane (acc = 0.0) is formed
// without the FP64 pipe: 0.0 + v is v, except that -0.0 becomes +0.0 (so a lane sum is never
// -0.0, and adding a lane that holds 0.0 leaves any lane sum unchanged).
template <bool kFirst>
__device__ __forceinline__ void cro_add(double& acc, double v) {
  if (kFirst)
    acc = (__double_as_longlong(v) << 1) == 0 ? 0.0 : v;
  else
    acc = __dadd_rn(acc, v);
}

// Place the 10 low bits of x at bit positions 0, 3, 6, ..., 27.
__device__ __forceinline__ uint32_t spread10(uint32_t x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

// 3D Hilbert index (B <= 10 bits per axis) of quantised coordinates, by Skilling's transform of
// the axes into the transposed Hilbert index (J. Skilling, "Programming the Hilbert curve", AIP
// Conf. Proc. 707, 2004): consecutive indices are face-adjacent cells, so runs of the curve are
// more compact than runs of the Morton order (no long jumps between octants).
template <int B>
__device__ __forceinline__ uint32_t hilbert3(uint32_t x0, uint32_t x1, uint32_t x2) {
  uint32_t X[3] = {x0, x1, x2};
  for (uint32_t q = 1u << (B - 1); q > 1; q >>= 1) {
    const uint32_t p = q - 1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (X[i] & q) {
        X[0] ^= p;  // invert the low bits of axis 0
      } else {      // exchange the low bits of axes 0 and i
        const uint32_t t = (X[0] ^ X[i]) & p;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  X[1] ^= X[0];  // Gray encode
  X[2] ^= X[1];
  uint32_t t = 0;
  for (uint32_t q = 1u << (B - 1); q > 1; q >>= 1)
    if (X[2] & q) t ^= q - 1;
  X[0] ^= t;
  X[1] ^= t;
  X[2] ^= t;
  return spread10(X[2]) | (spread10(X[1]) << 1) | (spread10(X[0]) << 2);  // axis 0 leads
}

}  // namespace rsd

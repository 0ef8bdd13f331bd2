// Certified far-field bounds of the potential for large nodes (batched form of rs_unbind).
//
// A member's flag depends only on the sign of E_i = KE_i - G m S_i, S_i = sum_{j != i}
// (|u_j - u_i|^2 + eps^2)^(-1/2) (the float64 canonical-order sum). For most members of a large
// node |E_i| is a sizeable fraction of G m S_i, so an interval [S_lo, S_hi] that certainly holds
// S_i decides the flag without the O(g) sum; only members whose interval straddles the sign
// change take the exact path (blocked float32 list sum with its certified bound, then the
// float64 canonical-order potential). The flags are therefore identical to the direct sum's.
//
// Interval (a Barnes-Hut walk with a rigorous truncation bound):
//   tree    the node's members sorted by a 30-bit Hilbert key of their offset u inside the
//           node's bounding box; leaf cells are runs of 32 consecutive members, every level up
//           groups 8 consecutive cells; per cell: centre c (the member mean, rounded to float32),
//           count n, dipole p = sum (x_j - c) (small: c is rounded), second moments
//           Q = sum (x_j - c)(x_j - c)^T, and a >= max |x_j - c| (all from float64 sums);
//   expand  with D = t - c, R'^2 = |D|^2 + eps^2, h_j = |x_j - c| / R' and
//           x = (D.(x_j - c)) / (R' |x_j - c|), the softened kernel is
//           (1/R') (1 - 2 h_j x + h_j^2)^(-1/2) = (1/R') sum_l h_j^l P_l(x)
//           (the Legendre generating function; |x| <= |D| / R' <= 1), so summing l <= 2 over
//           the cell gives n/R' + p.D/R'^3 + (3 D^T Q D - tr(Q) R'^2) / (2 R'^5), and since
//           |P_l| <= 1 on [-1, 1] the rest is at most (n/R') h^3 / (1 - h), h = a / R';
//   walk    one warp per 32 consecutive target members (in tree order); a cell is taken as its
//           expansion when a <= theta R' for every lane and it holds none of the warp's
//           targets, a leaf is summed directly (self excluded), otherwise its children are
//           visited;
//   slack   float32 evaluation and summation (per direct term <= ~8u, 32-term leaf blocks
//           summed as two packed halves <= 31u, the target's own term rsqrt(eps^2) taken out of
//           its leaf once <= u of the leaf sum, expansions with FMAs <= ~20u of n/R', Kahan across
//           visits <= 2u) stay below 1e-5 relative; the truncation terms (fast division, <= 2
//           ulp) are summed in float32 and widened by 0.1%:
//           S_lo = S~ (1 - 1e-5) - 1.001 B, S_hi = S~ (1 + 1e-5) + 1.001 B;
//           the float64 sum differs from the exact one by < g 2^-53 relative.
//   decide  bound iff KE - G m S_lo < -tol, unbound iff KE - G m S_hi > tol (tol = 1e-12 G m
//           S_hi covers the rounding of E itself); otherwise the member is listed for the exact
//           path.
// The paper's implementation computes the exact potential (Rockstar's unbinding); this bound is
// the O(g log g) potential the build adds for nodes of 10^5 - 10^6 members, compared against the
// exact flags in the tests.
#include "rs_exact.cuh"

namespace rs {
int unbind_fallback(rs_ctx* ctx, const unsigned long long* n_ambig, const uint32_t* ambig,
                    const double* vbulk, uint8_t* bound, cudaStream_t st, float* phi_out = nullptr);
int tree_build(rs_ctx* ctx, cudaStream_t st);
int tree_decide(rs_ctx* ctx, const int* only, const uint8_t* want, const double* vbulk,
                uint8_t* bound, unsigned long long* counters, cudaStream_t st);
}  // namespace rs

using namespace rs;

namespace {

constexpr int kT = 256;
constexpr int kLeafBits = 5;   // 32 members per leaf cell
constexpr int kBrBits = 3;     // 8 children per cell
constexpr int kMaxLevels = 10;  // enough for g < 2^32
constexpr int kStack = 64;      // (kMaxLevels - 1) * 7 + 1 pending cells at most
constexpr double kSlack = 1e-5;
constexpr double kBoundWiden = 1.001;

struct Cell {
  float4 ca;  // centre (x, y, z) and radius bound a
  float4 np;  // count n, dipole (px, py, pz)
  float4 q0;  // Qxx, Qyy, Qzz, Qxy
  float4 q1;  // Qxz, Qyz, tr Q, 0
};

__host__ __device__ __forceinline__ int64_t cells_at(int64_t g, int lev) {
  const int sh = kLeafBits + kBrBits * lev;
  return (g + (int64_t(1) << sh) - 1) >> sh;
}

__host__ __device__ __forceinline__ int levels_of(int64_t g) {
  int l = 0;
  while (cells_at(g, l) > 1) ++l;
  return l + 1;
}

__host__ __device__ __forceinline__ int64_t level_off(int64_t g, int lev) {
  int64_t o = 0;
  for (int l = 0; l < lev; ++l) o += cells_at(g, l);
  return o;
}

// Order-preserving map of a float to uint32 (for atomic min / max of floats).
__device__ __forceinline__ uint32_t ord(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unord(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Tree nodes: g >= tmin. Per node q: member count, selection flag and cell count (scanned into
// member offsets, ranks and cell offsets).
__global__ void k_tree_sel(int64_t nn, const int64_t* __restrict__ node_size, int64_t tmin,
                           int64_t* __restrict__ tsz, int64_t* __restrict__ tflag,
                           int64_t* __restrict__ tcells) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nn) return;
  const int64_t g = node_size[q];
  const bool sel = g >= tmin;
  tsz[q] = sel ? g : 0;
  tflag[q] = sel ? 1 : 0;
  tcells[q] = sel ? level_off(g, levels_of(g)) : 0;
}

// Per tree node b (rank order): node index, size, member offset in the tree arrays, cell offset.
__global__ void k_tree_list(int64_t nn, const int64_t* __restrict__ node_size, int64_t tmin,
                            const int64_t* __restrict__ toff, const int64_t* __restrict__ rank,
                            const int64_t* __restrict__ coff, int64_t* __restrict__ tnode,
                            int64_t* __restrict__ tg, int64_t* __restrict__ ttoff,
                            int64_t* __restrict__ tcoff) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nn || node_size[q] < tmin) return;
  const int64_t b = rank[q];
  tnode[b] = q;
  tg[b] = node_size[q];
  ttoff[b] = toff[q];
  tcoff[b] = coff[q];
}

// Bounding box of every tree node's members: warp-aggregated atomic min of the ordered
// encodings (max as the min of the complement). box[6 q + d]: min x, y, z, ~max x, y, z.
__global__ void k_tree_bbox(int64_t m, const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_size,
                            int64_t tmin, const float4* __restrict__ U, unsigned long long* __restrict__ box) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool in = p < m;
  const uint32_t q = in ? mnode[p] : 0u;
  const float4 u = in ? U[p] : make_float4(0, 0, 0, 0);
  // members moved to +inf (removed by an earlier unbinding pass) take no part in the tree
  const bool valid = in && node_size[q] >= tmin && isfinite(u.x);
  const float c[3] = {u.x, u.y, u.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    rsd::warp_run_min(box, uint32_t(6u * q + d), valid, (unsigned long long)ord(c[d]));
    rsd::warp_run_min(box, uint32_t(6u * q + 3 + d), valid, (unsigned long long)(~ord(c[d])));
  }
}

// Sort keys of the tree members: tree rank above a 30-bit Hilbert key of the position inside
// the node's bounding cube (10 bits per axis; runs of the curve make compact cells).
__global__ void k_tree_keys(int64_t m, const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_off,
                            const int64_t* __restrict__ node_size, int64_t tmin,
                            const int64_t* __restrict__ toff, const int64_t* __restrict__ rank,
                            const float4* __restrict__ U, const unsigned long long* __restrict__ box,
                            uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const uint32_t q = mnode[p];
  if (node_size[q] < tmin) return;
  const unsigned long long* B = box + 6 * int64_t(q);
  const float lo[3] = {unord(uint32_t(B[0])), unord(uint32_t(B[1])), unord(uint32_t(B[2]))};
  const float hi[3] = {unord(~uint32_t(B[3])), unord(~uint32_t(B[4])), unord(~uint32_t(B[5]))};
  const float ext = fmaxf(fmaxf(hi[0] - lo[0], hi[1] - lo[1]), fmaxf(hi[2] - lo[2], 1e-30f));
  const float sc = 1023.0f / ext;
  const float4 u = U[p];
  const float c[3] = {u.x, u.y, u.z};
  uint32_t qc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) qc[d] = uint32_t(fminf(fmaxf((c[d] - lo[d]) * sc, 0.f), 1023.f));
  const uint32_t code = rsd::hilbert3<10>(qc[0], qc[1], qc[2]);
  const int64_t k = toff[q] + (p - node_off[q]);
  keys[k] = (uint64_t(rank[q]) << 30) | uint64_t(code);
  vals[k] = uint32_t(p);
}

__global__ void k_tree_gather(int64_t T, const uint32_t* __restrict__ vals, const float4* __restrict__ U,
                              float4* __restrict__ TX, uint32_t* __restrict__ tpos) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= T) return;
  const uint32_t p = vals[s];
  const float4 u = U[p];
  TX[s] = make_float4(u.x, u.y, u.z, 0.f);
  tpos[s] = p;
}

// (tree rank b, level, index j in the level) of global cell c.
__device__ __forceinline__ void cell_decode(int64_t c, int64_t nt, const int64_t* __restrict__ tcoff,
                                            const int64_t* __restrict__ tg, int64_t& b, int& lev,
                                            int64_t& j) {
  b = rsd::upper_bound_i64(tcoff, nt, c) - 1;
  const int64_t g = tg[b];
  int64_t i = c - tcoff[b];
  lev = 0;
  while (i >= cells_at(g, lev)) {
    i -= cells_at(g, lev);
    ++lev;
  }
  j = i;
}

__device__ __forceinline__ float round_up_f(double v) {
  // float >= v (v >= 0), with a relative margin for the float64 rounding of v itself
  return __double2float_ru(v * (1.0 + 1e-12));
}

// Leaf cells (level 0): one warp per cell of the cell array (warps of other levels exit).
__global__ void __launch_bounds__(kT)
k_tree_leaves(int64_t C, int64_t nt, const int64_t* __restrict__ tcoff, const int64_t* __restrict__ tg,
              const int64_t* __restrict__ ttoff, const float4* __restrict__ TX, Cell* __restrict__ cells) {
  const int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= C) return;
  int64_t b, j;
  int lev;
  cell_decode(c, nt, tcoff, tg, b, lev, j);
  if (lev != 0) return;
  const int64_t s0 = ttoff[b] + (j << kLeafBits);
  const int cnt = int(rsd::min64(32, tg[b] - (j << kLeafBits)));
  const float4 xr = lane < cnt ? TX[s0 + lane] : make_float4(0, 0, 0, 0);
  // members moved to +inf (removed by an earlier unbinding pass) are left out of the moments
  const bool valid = lane < cnt && isfinite(xr.x);
  const int nv = __popc(__ballot_sync(0xffffffffu, valid));
  if (nv == 0) {  // an empty cell: contributes nothing
    if (lane == 0) {
      const float4 z = make_float4(0, 0, 0, 0);
      cells[c] = Cell{z, z, z, z};
    }
    return;
  }
  const float4 x = valid ? xr : make_float4(0, 0, 0, 0);
  double sx = x.x, sy = x.y, sz = x.z;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
    sy += __shfl_xor_sync(0xffffffffu, sy, off);
    sz += __shfl_xor_sync(0xffffffffu, sz, off);
  }
  const float cx = float(sx / nv), cy = float(sy / nv), cz = float(sz / nv);
  // offsets from the float32 centre are exact in float64
  const double dx = valid ? double(x.x) - double(cx) : 0.0;
  const double dy = valid ? double(x.y) - double(cy) : 0.0;
  const double dz = valid ? double(x.z) - double(cz) : 0.0;
  double v[10] = {dx, dy, dz, dx * dx, dy * dy, dz * dz, dx * dy, dx * dz, dy * dz,
                  sqrt(dx * dx + dy * dy + dz * dz)};
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
#pragma unroll
    for (int t = 0; t < 9; ++t) v[t] += __shfl_xor_sync(0xffffffffu, v[t], off);
    v[9] = fmax(v[9], __shfl_xor_sync(0xffffffffu, v[9], off));
  }
  if (lane == 0) {
    Cell cl;
    cl.ca = make_float4(cx, cy, cz, round_up_f(v[9]));
    cl.np = make_float4(float(nv), float(v[0]), float(v[1]), float(v[2]));
    cl.q0 = make_float4(float(v[3]), float(v[4]), float(v[5]), float(v[6]));
    cl.q1 = make_float4(float(v[7]), float(v[8]), float(v[3] + v[4] + v[5]), 0.f);
    cells[c] = cl;
  }
}

// Cells of level `lev` >= 1 from their (up to 8) children, moments shifted to the parent's
// float32 centre in float64; the radius bound is max(child a + |child c - c|), rounded up.
__global__ void k_tree_up(int64_t C, int lev, int64_t nt, const int64_t* __restrict__ tcoff,
                          const int64_t* __restrict__ tg, Cell* __restrict__ cells) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int64_t b, j;
  int lv;
  cell_decode(c, nt, tcoff, tg, b, lv, j);
  if (lv != lev) return;
  const int64_t g = tg[b];
  const int64_t c0 = tcoff[b] + level_off(g, lev - 1) + (j << kBrBits);
  const int nch = int(rsd::min64(int64_t(1) << kBrBits, cells_at(g, lev - 1) - (j << kBrBits)));
  double n = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
  for (int k = 0; k < nch; ++k) {
    const Cell ch = cells[c0 + k];
    if (ch.np.x == 0.f) continue;  // empty child
    n += ch.np.x;
    mx += double(ch.np.x) * ch.ca.x + ch.np.y;  // sum of x_j = n c + p
    my += double(ch.np.x) * ch.ca.y + ch.np.z;
    mz += double(ch.np.x) * ch.ca.z + ch.np.w;
  }
  if (n == 0.0) {
    const float4 z = make_float4(0, 0, 0, 0);
    cells[c] = Cell{z, z, z, z};
    return;
  }
  const float cx = float(mx / n), cy = float(my / n), cz = float(mz / n);
  double P[3] = {0.0, 0.0, 0.0}, Q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, a = 0.0;
  for (int k = 0; k < nch; ++k) {
    const Cell ch = cells[c0 + k];
    if (ch.np.x == 0.f) continue;
    const double d[3] = {double(ch.ca.x) - cx, double(ch.ca.y) - cy, double(ch.ca.z) - cz};
    const double nc = ch.np.x;
    const double pc[3] = {ch.np.y, ch.np.z, ch.np.w};
    for (int e = 0; e < 3; ++e) P[e] += pc[e] + nc * d[e];
    // sum (y + d)(y + d)^T over the child's members, y = x - c_child: Q_c + p d^T + d p^T + n d d^T
    const double qc[6] = {ch.q0.x, ch.q0.y, ch.q0.z, ch.q0.w, ch.q1.x, ch.q1.y};
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int t = 0; t < 6; ++t)
      Q[t] += qc[t] + pc[ia[t]] * d[ib[t]] + d[ia[t]] * pc[ib[t]] + nc * d[ia[t]] * d[ib[t]];
    const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * (1.0 + 1e-12);
    a = fmax(a, double(ch.ca.w) + dist);
  }
  Cell cl;
  cl.ca = make_float4(cx, cy, cz, round_up_f(a));
  cl.np = make_float4(float(n), float(P[0]), float(P[1]), float(P[2]));
  cl.q0 = make_float4(float(Q[0]), float(Q[1]), float(Q[2]), float(Q[3]));
  cl.q1 = make_float4(float(Q[4]), float(Q[5]), float(Q[0] + Q[1] + Q[2]), 0.f);
  cells[c] = cl;
}

// Walk order of the tree nodes: largest size class first (stable within a class).
__global__ void k_tree_okeys(int64_t nt, const int64_t* __restrict__ tg, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nt) return;
  keys[b] = 255u - rsd::size_class(tg[b]);
  vals[b] = uint32_t(b);
}

// Wanted flag of every tree member (sorted position s): want[p] if given, else only[q] if given,
// else 1.
__global__ void k_tree_want(int64_t T, const uint32_t* __restrict__ tpos, const uint32_t* __restrict__ mnode,
                            const int* __restrict__ only, const uint8_t* __restrict__ want,
                            int64_t* __restrict__ wf) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= T) return;
  const uint32_t p = tpos[s];
  wf[s] = want ? int64_t(want[p] != 0) : (only ? int64_t(only[mnode[p]] != 0) : 1);
}

__global__ void k_tree_wlist(int64_t T, const int64_t* __restrict__ wf, uint32_t* __restrict__ wl) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= T) return;
  if (wf[s + 1] != wf[s]) wl[wf[s]] = uint32_t(s);
}

// Per node (walk order r): wanted range [wlo, wlo + wcnt) of the wanted list and its warp count.
__global__ void k_tree_items(int64_t nt, const uint32_t* __restrict__ worder, const int64_t* __restrict__ ttoff,
                             const int64_t* __restrict__ tg, const int64_t* __restrict__ wf,
                             int64_t* __restrict__ wlo, int64_t* __restrict__ wcnt,
                             int64_t* __restrict__ items) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= nt) return;
  const int64_t b = worder[r];
  const int64_t a = wf[ttoff[b]], e = wf[ttoff[b] + tg[b]];
  wlo[r] = a;
  wcnt[r] = e - a;
  items[r] = (e - a + 31) / 32;
}

struct WalkArgs {
  int64_t nt;
  const int64_t* item_off;  // [nt + 1], walk order
  const uint32_t* worder;   // walk order -> tree rank
  const int64_t* wlo;       // walk order
  const int64_t* wcnt;      // walk order
  const uint32_t* wl;       // wanted sorted positions
  const float4* TX;
  const uint32_t* tpos;
  const int64_t* ttoff;
  const int64_t* tcoff;
  const int64_t* tg;
  const int64_t* tnode;
  const Cell* cells;
  const float4* V;
  const double* vbulk;
  float eps2, theta2;
  double Gm;
  uint8_t* bound;
  int64_t* und;             // per sorted position: 1 = undecided
  double* rec_lo;           // per member position (optional record of the interval)
  double* rec_hi;
  unsigned long long* counters;  // [0] decided, [1] undecided, [2] expansions, [3] direct pairs
};

// One warp per 32 wanted targets of one node: the certified walk, then the decision. Indices
// inside the walk are 32-bit and relative to the node (its members are [tb, tb + g) of the
// sorted arrays, its cells [cb, cb + cells) of the cell array); a stack entry carries the
// cell's level, its index j within the level and its index within the node's cells.
__global__ void __launch_bounds__(kT)
k_tree_walk(WalkArgs A) {
  __shared__ uint64_t s_stack[kT / 32][kStack];
  __shared__ __align__(16) float s_leaf[kT / 32][3][32];  // a leaf's members in x / y / z rows
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (w >= A.item_off[A.nt]) return;
  const int64_t r = rsd::upper_bound_i64(A.item_off, A.nt, w) - 1;
  const int64_t b = A.worder[r];
  const int64_t it = w - A.item_off[r];
  const int64_t wi = A.wlo[r] + 32 * it + lane;
  const bool valid = 32 * it + lane < A.wcnt[r];
  const int64_t wi0 = A.wlo[r] + 32 * it;  // lane 0's entry: always valid
  const uint32_t s_self = A.wl[valid ? wi : wi0];
  const float4 t = A.TX[s_self];
  const int64_t g = A.tg[b], tb = A.ttoff[b], cb = A.tcoff[b];
  const int nlev = levels_of(g);
  // per-level cell offsets inside the node, lane l holds level l's
  const uint32_t my_lvoff = lane < nlev ? uint32_t(level_off(g, lane)) : 0u;
  const uint32_t g32 = uint32_t(g), self_rel = s_self - uint32_t(tb);
  // the warp's targets as a range of node-relative positions: a cell holds one of them iff
  // its index at its level lies in [lo_rel >> sh, hi_rel >> sh]
  uint32_t lo_rel = self_rel, hi_rel = self_rel;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    lo_rel = min(lo_rel, __shfl_xor_sync(0xffffffffu, lo_rel, off));
    hi_rel = max(hi_rel, __shfl_xor_sync(0xffffffffu, hi_rel, off));
  }
  const Cell* __restrict__ ncell = A.cells + cb;
  const float4* __restrict__ nx = A.TX + tb;
  uint64_t* stk = s_stack[wid];
  float (*leaf)[32] = s_leaf[wid];
  float S = 0.f, Cc = 0.f, Bt = 0.f;
  uint32_t n_exp = 0, n_dir = 0;
  const uint32_t root_off = __shfl_sync(0xffffffffu, my_lvoff, nlev - 1);
  if (lane == 0) stk[0] = (uint64_t(nlev - 1) << 60) | uint64_t(root_off);
  int sp = 1;
  __syncwarp();
  while (sp > 0) {
    --sp;
    const uint64_t e = stk[sp];
    __syncwarp();
    const int lev = int(e >> 60);
    const uint32_t j = uint32_t(e >> 32) & 0x0fffffffu;
    const int sh = kLeafBits + kBrBits * lev;
    const bool overlap = j >= (lo_rel >> sh) && j <= (hi_rel >> sh);
    const Cell cl = ncell[uint32_t(e)];
    if (cl.np.x == 0.f) continue;  // no member left in the cell (iterative unbinding)
    const float dx = t.x - cl.ca.x, dy = t.y - cl.ca.y, dz = t.z - cl.ca.z;
    const float R2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmaf_rn(dz, dz, A.eps2)));
    const bool acc = cl.ca.w * cl.ca.w <= A.theta2 * R2;
    if (!overlap && __all_sync(0xffffffffu, acc)) {
      // quadrupole expansion and its truncation bound; explicit FMAs (the evaluation only has
      // to stay inside the 1e-5 slack, and the library is compiled without contraction)
      const float ri = rsqrtf(R2);
      const float ri2 = ri * ri, ri3 = ri2 * ri;
      const float ax = __fmaf_rn(cl.q1.x + cl.q1.x, dz, __fmaf_rn(cl.q0.w + cl.q0.w, dy, cl.q0.x * dx));
      const float ay = __fmaf_rn(cl.q1.y + cl.q1.y, dz, cl.q0.y * dy);
      const float dqd = __fmaf_rn(ax, dx, __fmaf_rn(ay, dy, cl.q0.z * dz * dz));
      const float pd = __fmaf_rn(cl.np.y, dx, __fmaf_rn(cl.np.z, dy, cl.np.w * dz));
      const float quad = __fmaf_rn(1.5f * dqd, ri2, -0.5f * cl.q1.z);
      const float val = __fmaf_rn(cl.np.x, ri, ri3 * (pd + quad));
      const float h = cl.ca.w * ri;
      const float bnd = __fdividef(cl.np.x * ri * (h * h * h), 1.f - h);
      const float y = __fsub_rn(val, Cc);
      const float tt = __fadd_rn(S, y);
      Cc = __fsub_rn(__fsub_rn(tt, S), y);
      S = tt;
      Bt += bnd;
      ++n_exp;
    } else if (lev == 0) {
      // direct sum over the leaf's members, two per packed float32x2 step; slots past the leaf's
      // count hold +inf, whose term is exactly 0; the target's own term rsqrt(eps^2) is taken
      // out once (or, without softening, skipped per pair)
      const uint32_t c0 = j << kLeafBits;
      const int cnt = int(min(32u, g32 - c0));
      const float inf = __int_as_float(0x7f800000);
      const float4 xm = lane < cnt ? nx[c0 + lane] : make_float4(inf, inf, inf, 0.f);
      leaf[0][lane] = xm.x;
      leaf[1][lane] = xm.y;
      leaf[2][lane] = xm.z;
      __syncwarp();
      float blk;
      if (A.eps2 > 0.f) {
        const float2 ntx = make_float2(-t.x, -t.x), nty = make_float2(-t.y, -t.y),
                     ntz = make_float2(-t.z, -t.z), e2 = make_float2(A.eps2, A.eps2);
        float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int k = 0; k < 32; k += 2) {
          const float2 ex = __fadd2_rn(*reinterpret_cast<const float2*>(&leaf[0][k]), ntx);
          const float2 ey = __fadd2_rn(*reinterpret_cast<const float2*>(&leaf[1][k]), nty);
          const float2 ez = __fadd2_rn(*reinterpret_cast<const float2*>(&leaf[2][k]), ntz);
          const float2 r2 = __ffma2_rn(ex, ex, __ffma2_rn(ey, ey, __ffma2_rn(ez, ez, e2)));
          acc2 = __fadd2_rn(acc2, make_float2(rsqrtf(r2.x), rsqrtf(r2.y)));
        }
        blk = __fadd_rn(acc2.x, acc2.y);
        if ((self_rel >> kLeafBits) == j) blk = __fsub_rn(blk, rsqrtf(A.eps2));
      } else {
        blk = 0.f;
        for (int k = 0; k < cnt; ++k) {
          const float ex = __fsub_rn(leaf[0][k], t.x), ey = __fsub_rn(leaf[1][k], t.y),
                      ez = __fsub_rn(leaf[2][k], t.z);
          const float wv = rsqrtf(__fmaf_rn(ex, ex, __fmaf_rn(ey, ey, __fmaf_rn(ez, ez, A.eps2))));
          blk = __fadd_rn(blk, c0 + uint32_t(k) == self_rel ? 0.f : wv);
        }
      }
      __syncwarp();
      const float y = __fsub_rn(blk, Cc);
      const float tt = __fadd_rn(S, y);
      Cc = __fsub_rn(__fsub_rn(tt, S), y);
      S = tt;
      n_dir += uint32_t(cnt);
    } else {
      const int shc = sh - kBrBits;  // the children's level
      const uint32_t nchild = uint32_t((uint64_t(g32) + (1ull << shc) - 1) >> shc);
      const uint32_t j0 = j << kBrBits;
      const int nch = int(min(1u << kBrBits, nchild - j0));
      const uint32_t lvc = __shfl_sync(0xffffffffu, my_lvoff, lev - 1);
      if (lane < nch)
        stk[sp + lane] = (uint64_t(lev - 1) << 60) | (uint64_t(j0 + lane) << 32) | uint64_t(lvc + j0 + lane);
      sp += nch;
      __syncwarp();
    }
  }
  bool decided = false;
  if (valid) {
    const uint32_t p = A.tpos[s_self];
    const int64_t q = A.tnode[b];
    const double Sd = double(S), Bd = kBoundWiden * double(Bt);
    const double slo = Sd * (1.0 - kSlack) - Bd, shi = Sd * (1.0 + kSlack) + Bd;
    const double ke = kinetic(A.V[p], A.vbulk + 3 * q);
    const double tol = 1e-12 * A.Gm * fabs(shi);
    const double e_hi = ke - A.Gm * slo, e_lo = ke - A.Gm * shi;
    if (slo > 0.0 && e_hi < -tol) {
      A.bound[p] = 1;
      decided = true;
    } else if (e_lo > tol) {
      A.bound[p] = 0;
      decided = true;
    } else {
      A.und[s_self] = 1;
    }
    if (A.rec_lo) {
      A.rec_lo[p] = slo;
      A.rec_hi[p] = shi;
    }
  }
  const unsigned dec = __ballot_sync(0xffffffffu, valid && decided);
  const unsigned und = __ballot_sync(0xffffffffu, valid && !decided);
  unsigned long long n_exp64 = n_exp, n_dir64 = n_dir;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    n_exp64 += __shfl_xor_sync(0xffffffffu, n_exp64, off);
    n_dir64 += __shfl_xor_sync(0xffffffffu, n_dir64, off);
  }
  if (lane == 0) {
    if (dec) atomicAdd(A.counters + 0, (unsigned long long)__popc(dec));
    if (und) atomicAdd(A.counters + 1, (unsigned long long)__popc(und));
    atomicAdd(A.counters + 2, n_exp64);
    atomicAdd(A.counters + 3, n_dir64);
  }
}

__global__ void k_tree_ulist(int64_t T, const int64_t* __restrict__ uf, uint32_t* __restrict__ list,
                             unsigned long long* __restrict__ count) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s == 0) *count = (unsigned long long)uf[T];
  if (s >= T) return;
  if (uf[s + 1] != uf[s]) list[uf[s]] = uint32_t(s);
}

__global__ void k_tree_lranges(int64_t nt, const int64_t* __restrict__ ttoff, const int64_t* __restrict__ tg,
                               const int64_t* __restrict__ uf, int tile, int64_t* __restrict__ lofs,
                               int64_t* __restrict__ lend, int64_t* __restrict__ tiles,
                               unsigned long long* __restrict__ list_pairs) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nt) return;
  const int64_t a = uf[ttoff[b]], e = uf[ttoff[b] + tg[b]];
  lofs[b] = a;
  lend[b] = e;
  tiles[b] = (e - a + tile - 1) / tile;
  if (e > a) atomicAdd(list_pairs, (unsigned long long)((e - a) * tg[b]));
}

__global__ void k_tree_acc(unsigned long long* __restrict__ c, int from, int to) {
  c[to] += c[from];
  c[from] = 0;
}

int bits_for(uint64_t v) {
  int b = 1;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

}  // namespace

// Build the cells of every node with at least ctx->tree_min members (device state kept in the
// context's scratch until the next rs_unbind).
int rs::tree_build(rs_ctx* ctx, cudaStream_t st) {
  ctx->tree_nt = 0;
  ctx->tree_T = 0;
  ctx->tree_C = 0;
  const int64_t tmin = ctx->tree_min;
  if (tmin <= 0) return RS_OK;
  Hier h = hier_of(ctx);
  const int64_t nn = ctx->n_nodes, m = ctx->n_members;
  if (nn == 0) return RS_OK;
  int64_t* tsz = scratch_t<int64_t>(ctx, S_T_OFF, size_t(nn) + 1);
  int64_t* trank = scratch_t<int64_t>(ctx, S_T_RANK, size_t(nn) + 1);
  int64_t* tcells = scratch_t<int64_t>(ctx, S_T_COFF, size_t(nn) + 1);
  if (!tsz || !trank || !tcells) return RS_ERR_OOM;
  k_tree_sel<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_size, tmin, tsz, trank, tcells);
  RS_LAUNCHED(ctx, "k_tree_sel");
  RS_TRY(exclusive_scan_i64(ctx, nn, tsz, tsz + nn, st));
  RS_TRY(exclusive_scan_i64(ctx, nn, trank, trank + nn, st));
  RS_TRY(exclusive_scan_i64(ctx, nn, tcells, tcells + nn, st));
  RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box, tsz + nn, 8, cudaMemcpyDeviceToHost, st));
  RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box + 1, trank + nn, 8, cudaMemcpyDeviceToHost, st));
  RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box + 2, tcells + nn, 8, cudaMemcpyDeviceToHost, st));
  RS_CUDA(ctx, cudaStreamSynchronize(st));
  const int64_t T = ctx->host_box[0], nt = ctx->host_box[1], C = ctx->host_box[2];
  if (nt == 0) return RS_OK;
  int64_t* tn = scratch_t<int64_t>(ctx, S_T_NODES, size_t(nt) * 4 + 4);
  unsigned long long* box = scratch_t<unsigned long long>(ctx, S_T_BOX, size_t(nn) * 6);
  uint64_t* ka = scratch_t<uint64_t>(ctx, S_T_KA, size_t(T));
  uint64_t* kb = scratch_t<uint64_t>(ctx, S_T_KB, size_t(T));
  uint32_t* va = scratch_t<uint32_t>(ctx, S_T_VA, size_t(T));
  uint32_t* vb = scratch_t<uint32_t>(ctx, S_T_VB, size_t(T));
  float4* TX = scratch_t<float4>(ctx, S_T_X, size_t(T));
  uint32_t* tpos = scratch_t<uint32_t>(ctx, S_T_POS, size_t(T));
  Cell* cells = static_cast<Cell*>(scratch(ctx, S_T_CELL, size_t(C) * sizeof(Cell)));
  uint32_t* worder = scratch_t<uint32_t>(ctx, S_T_ORDER, size_t(nt));
  if (!tn || !box || !ka || !kb || !va || !vb || !TX || !tpos || !cells || !worder) return RS_ERR_OOM;
  int64_t *tnode = tn, *tg = tn + nt, *ttoff = tn + 2 * nt, *tcoff = tn + 3 * nt;
  k_tree_list<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_size, tmin, tsz, trank, tcells, tnode, tg, ttoff,
                                              tcoff);
  RS_LAUNCHED(ctx, "k_tree_list");
  RS_CUDA(ctx, cudaMemsetAsync(box, 0xff, sizeof(unsigned long long) * 6 * nn, st));
  k_tree_bbox<<<grid_for(m, kT), kT, 0, st>>>(m, h.mnode, h.node_size, tmin, h.U, box);
  RS_LAUNCHED(ctx, "k_tree_bbox");
  k_tree_keys<<<grid_for(m, kT), kT, 0, st>>>(m, h.mnode, h.node_off, h.node_size, tmin, tsz, trank, h.U,
                                             box, ka, va);
  RS_LAUNCHED(ctx, "k_tree_keys");
  uint64_t* ko;
  uint32_t* vo;
  RS_TRY(radix_sort_u64(ctx, T, 30 + bits_for(uint64_t(nt)), ka, va, kb, vb, &ko, &vo, st));
  k_tree_gather<<<grid_for(T, kT), kT, 0, st>>>(T, vo, h.U, TX, tpos);
  RS_LAUNCHED(ctx, "k_tree_gather");
  {
    ProfScope prof_(ctx, "k_tree_build", st);
    k_tree_leaves<<<grid_for(C * 32, kT), kT, 0, st>>>(C, nt, tcoff, tg, ttoff, TX, cells);
    RS_LAUNCHED(ctx, "k_tree_leaves");
    for (int lev = 1; lev < kMaxLevels; ++lev) {
      k_tree_up<<<grid_for(C, kT), kT, 0, st>>>(C, lev, nt, tcoff, tg, cells);
      RS_LAUNCHED(ctx, "k_tree_up");
    }
  }
  // walk order of the nodes (largest first)
  {
    uint64_t* oka = scratch_t<uint64_t>(ctx, S_U_OKEY_A, size_t(nt));
    uint64_t* okb = scratch_t<uint64_t>(ctx, S_U_OKEY_B, size_t(nt));
    uint32_t* ova = scratch_t<uint32_t>(ctx, S_U_OVAL_A, size_t(nt));
    uint32_t* ovb = scratch_t<uint32_t>(ctx, S_U_OVAL_B, size_t(nt));
    if (!oka || !okb || !ova || !ovb) return RS_ERR_OOM;
    k_tree_okeys<<<grid_for(nt, kT), kT, 0, st>>>(nt, tg, oka, ova);
    RS_LAUNCHED(ctx, "k_tree_okeys");
    uint64_t* oko;
    uint32_t* ovo;
    RS_TRY(radix_sort_u64(ctx, nt, 8, oka, ova, okb, ovb, &oko, &ovo, st));
    RS_CUDA(ctx, cudaMemcpyAsync(worder, ovo, 4 * size_t(nt), cudaMemcpyDeviceToDevice, st));
  }
  ctx->tree_nt = nt;
  ctx->tree_T = T;
  ctx->tree_C = C;
  return RS_OK;
}

// Decide the flags of the wanted members of the tree nodes (want[p] != 0 when `want` is given,
// else the members of the nodes with only[q] != 0 when `only` is given, else every member):
// certified interval walk, then the exact list path (blocked float32 list sums with their
// certified bound, float64 canonical-order potential) for the undecided ones.
// counters: [16] float64 queue of this call, [7] float64 total of the direct sums,
// [12..15] decided by the bound, listed for the exact path, expansions, direct pairs,
// [18] pair terms of the exact list sums.
int rs::tree_decide(rs_ctx* ctx, const int* only, const uint8_t* want, const double* vbulk,
                    uint8_t* bound, unsigned long long* counters, cudaStream_t st) {
  const int64_t nt = ctx->tree_nt, T = ctx->tree_T;
  if (nt == 0 || T == 0) return RS_OK;
  Hier h = hier_of(ctx);
  int64_t* tn = static_cast<int64_t*>(ctx->buf[S_T_NODES].ptr);
  int64_t *tnode = tn, *tg = tn + nt, *ttoff = tn + 2 * nt, *tcoff = tn + 3 * nt;
  const float4* TX = static_cast<const float4*>(ctx->buf[S_T_X].ptr);
  const uint32_t* tpos = static_cast<const uint32_t*>(ctx->buf[S_T_POS].ptr);
  const Cell* cells = static_cast<const Cell*>(ctx->buf[S_T_CELL].ptr);
  const uint32_t* worder = static_cast<const uint32_t*>(ctx->buf[S_T_ORDER].ptr);
  int64_t* wf = scratch_t<int64_t>(ctx, S_T_WF, size_t(T) + 1);
  uint32_t* wl = scratch_t<uint32_t>(ctx, S_T_WL, size_t(T));
  int64_t* wr = scratch_t<int64_t>(ctx, S_T_WR, size_t(nt) * 3 + 3);
  int64_t* uf = scratch_t<int64_t>(ctx, S_T_UF, size_t(T) + 1);
  uint32_t* ulist = scratch_t<uint32_t>(ctx, S_T_LIST, size_t(T));
  int64_t* lr = scratch_t<int64_t>(ctx, S_T_LR, size_t(nt) * 3 + 3);
  float* Sx = scratch_t<float>(ctx, S_T_SX, size_t(T));
  uint32_t* ambig = scratch_t<uint32_t>(ctx, S_U_AMBIG, size_t(ctx->n_members) + 1);
  if (!wf || !wl || !wr || !uf || !ulist || !lr || !Sx || !ambig) return RS_ERR_OOM;
  int64_t *wlo = wr, *wcnt = wr + nt, *items = wr + 2 * nt;
  k_tree_want<<<grid_for(T, kT), kT, 0, st>>>(T, tpos, h.mnode, only, want, wf);
  RS_LAUNCHED(ctx, "k_tree_want");
  RS_TRY(exclusive_scan_i64(ctx, T, wf, wf + T, st));
  k_tree_wlist<<<grid_for(T, kT), kT, 0, st>>>(T, wf, wl);
  RS_LAUNCHED(ctx, "k_tree_wlist");
  k_tree_items<<<grid_for(nt, kT), kT, 0, st>>>(nt, worder, ttoff, tg, wf, wlo, wcnt, items);
  RS_LAUNCHED(ctx, "k_tree_items");
  RS_TRY(exclusive_scan_i64(ctx, nt, items, items + nt, st));
  RS_CUDA(ctx, cudaMemsetAsync(uf, 0, sizeof(int64_t) * (size_t(T) + 1), st));
  // an upper bound of the warps (items): T / 32 + nt
  const int64_t warps_ub = T / 32 + nt + 1;
  WalkArgs A;
  A.nt = nt;
  A.item_off = items;
  A.worder = worder;
  A.wlo = wlo;
  A.wcnt = wcnt;
  A.wl = wl;
  A.TX = TX;
  A.tpos = tpos;
  A.ttoff = ttoff;
  A.tcoff = tcoff;
  A.tg = tg;
  A.tnode = tnode;
  A.cells = cells;
  A.V = h.V;
  A.vbulk = vbulk;
  A.eps2 = ctx->cfg.softening * ctx->cfg.softening;
  A.theta2 = ctx->tree_theta * ctx->tree_theta;
  A.Gm = ctx->cfg.G * ctx->cfg.particle_mass;
  A.bound = bound;
  A.und = uf;
  A.rec_lo = ctx->tree_record ? static_cast<double*>(ctx->buf[S_T_REC].ptr) : nullptr;
  A.rec_hi = A.rec_lo ? A.rec_lo + ctx->n_members : nullptr;
  A.counters = counters + 12;
  {
    ProfScope prof_(ctx, "k_tree_walk", st);
    k_tree_walk<<<grid_for(warps_ub * 32, kT), kT, 0, st>>>(A);
  }
  RS_LAUNCHED(ctx, "k_tree_walk");
  // exact path for the undecided members
  RS_TRY(exclusive_scan_i64(ctx, T, uf, uf + T, st));
  unsigned long long* ucount = counters + 17;
  k_tree_ulist<<<grid_for(T, kT), kT, 0, st>>>(T, uf, ulist, ucount);
  RS_LAUNCHED(ctx, "k_tree_ulist");
  const int R = ctx->tune_list_r ? ctx->tune_list_r : 4;
  int64_t *lofs = lr, *lend = lr + nt, *ltiles = lr + 2 * nt;
  k_tree_lranges<<<grid_for(nt, kT), kT, 0, st>>>(nt, ttoff, tg, uf, kListThreads * R, lofs, lend, ltiles,
                                                  counters + 18);
  RS_LAUNCHED(ctx, "k_tree_lranges");
  RS_TRY(exclusive_scan_i64(ctx, nt, ltiles, ltiles + nt, st));
  const float eps2 = ctx->cfg.softening * ctx->cfg.softening;
  const unsigned grid = grid_for(T / (kListThreads * R) + nt + 1, 1);
  {
    ProfScope prof_(ctx, "k_potential_list", st);
    if (R == 2)
      k_potential_list<2><<<grid, kListThreads, 0, st>>>(nt, ltiles, tnode, lofs, lend, ulist, tpos, h.node_off,
                                                         h.node_size, h.U, eps2, Sx);
    else if (R == 8)
      k_potential_list<8><<<grid, kListThreads, 0, st>>>(nt, ltiles, tnode, lofs, lend, ulist, tpos, h.node_off,
                                                         h.node_size, h.U, eps2, Sx);
    else
      k_potential_list<4><<<grid, kListThreads, 0, st>>>(nt, ltiles, tnode, lofs, lend, ulist, tpos, h.node_off,
                                                         h.node_size, h.U, eps2, Sx);
  }
  RS_LAUNCHED(ctx, "k_potential_list");
  const double Gm = ctx->cfg.G * ctx->cfg.particle_mass;
  k_flags_list<<<grid_for(T, kT), kT, 0, st>>>(ucount, ulist, tpos, h.mnode, h.V, vbulk, eps2, Gm, Sx, bound,
                                              ambig, counters + 16);
  RS_LAUNCHED(ctx, "k_flags_list");
  RS_TRY(unbind_fallback(ctx, counters + 16, ambig, vbulk, bound, st));
  k_tree_acc<<<1, 1, 0, st>>>(counters, 16, 7);
  RS_LAUNCHED(ctx, "k_tree_acc");
  return RS_OK;
}

extern "C" int rs_tree_record(rs_ctx* ctx, int enable) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  ctx->tree_record = enable != 0;
  return RS_OK;
}

extern "C" int rs_tree_bounds(rs_ctx* ctx, double* lo_out, double* hi_out, void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (!ctx->have_unbind || !ctx->tree_recorded)
    return set_error(ctx, RS_ERR_STATE, "no recorded rs_unbind (rs_tree_record(ctx, 1) first)");
  const int64_t m = ctx->n_members;
  if (m > 0 && (!lo_out || !hi_out)) return set_error(ctx, RS_ERR_INVALID_ARG, "null output");
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double* rec = static_cast<const double*>(ctx->buf[S_T_REC].ptr);
  if (m > 0) {
    RS_CUDA(ctx, cudaMemcpyAsync(lo_out, rec, 8 * size_t(m), cudaMemcpyDeviceToDevice, st));
    RS_CUDA(ctx, cudaMemcpyAsync(hi_out, rec + m, 8 * size_t(m), cudaMemcpyDeviceToDevice, st));
  }
  return RS_OK;
}

extern "C" int rs_tree_stats(rs_ctx* ctx, int64_t* stats_out) {
  if (!ctx || !stats_out) return RS_ERR_INVALID_ARG;
  for (int i = 0; i < 8; ++i) stats_out[i] = ctx->tree_stats[i];
  return RS_OK;
}

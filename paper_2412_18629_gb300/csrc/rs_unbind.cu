// Unbinding and halo properties over every node of the 6D hierarchy.
//
// Potential: phi_i = -G m sum_{j != i} (|u_j - u_i|^2 + eps^2)^(-1/2) over the node's members.
//   k_potential   float32 direct sum for nodes up to 384 members: one thread per member, the
//                 node's members read through L1; larger nodes by the register-blocked kernel.
//                 FMA + rsqrt per pair, 32-term blocks added with Kahan compensation.
//                 Certified relative error bound B (see kCertB).
//   k_flags       float64 kinetic energy against the node's bulk velocity (canonical-order sum),
//                 E = KE + phi~. |E| > 2 B |phi~| decides the flag; otherwise the member is queued
//                 for the exact float64 potential.
//   k_fallback_*  the float64 potential of each queued member in the canonical reduction order,
//                 bit-identical to the definition (one warp per 1024-term chunk, chunk totals
//                 combined by the pairwise tree), then the exact flag.
//   k_halo        bound count, halo decision, bound mass per node.
// Properties (rs_halo_props): canonical-order sums over bound members (unbound contribute 0).
#include <cmath>

#include "rs_cro.cuh"

namespace rs {
int gather_members(rs_ctx* ctx, int64_t mb, int64_t me, int64_t nb, int64_t ne, const float* pos,
                   const float* vel, cudaStream_t st);
int surrogate_unbind(rs_ctx* ctx, const double* vbulk, uint8_t* bound, unsigned long long* counters,
                     cudaStream_t st);
int unbind_fallback(rs_ctx* ctx, const unsigned long long* n_ambig, const uint32_t* ambig,
                    const double* vbulk, uint8_t* bound, cudaStream_t st, float* phi_out = nullptr);
int unbind_nodes(rs_ctx* ctx, const int* only, const double* vbulk, uint8_t* bound,
                 uint32_t* ambig, unsigned long long* n_ambig, cudaStream_t st,
                 unsigned long long* counters);
int tree_build(rs_ctx* ctx, cudaStream_t st);
int tree_decide(rs_ctx* ctx, const int* only, const uint8_t* want, const double* vbulk,
                uint8_t* bound, unsigned long long* counters, cudaStream_t st);
}  // namespace rs

using namespace rs;

namespace {

constexpr int kT = 256;
constexpr int kPotTile = 256;

// Relative error bound of the float32 potential sum (all terms positive):
//   per term: operands rounded (3 differences, 3 fused steps, eps^2) <= ~6u relative in r^2, so
//   <= 3u after the square root, plus rsqrt.approx's 2^-22.9 (~2.2u): <= 8u allowing slack;
//   32-term sequential blocks: <= 31u; Kahan-compensated sum of the blocks: <= 2u + O(N u^2).
//   Total <= 41u + 1e-12 with u = 2^-24; the flag test uses twice this.
constexpr double kU = 5.9604644775390625e-08;
constexpr double kCertB = 41.0 * kU + 1e-12;
constexpr int kCounters = 24;  // the unbinding counters (see rs_unbind)

// Nodes up to kBlockedMin members: one thread per member over the flat member list (lanes of
// a warp are consecutive members, mostly of one node), the node's members read through L1 in
// ascending order; the same 32-term blocks and Kahan steps as the blocked kernel. A node is
// selected when its tile count (scanned) is non-zero.
__global__ void __launch_bounds__(kT)
k_potential(int64_t m, const uint32_t* __restrict__ mnode, const int64_t* __restrict__ tile_off,
            const int64_t* __restrict__ node_off, const int64_t* __restrict__ node_size,
            const float4* __restrict__ U, float eps2, float* __restrict__ S_out) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const uint32_t q = mnode[p];
  if (tile_off[q + 1] == tile_off[q]) return;  // not selected for this kernel
  const int64_t base = node_off[q], g = node_size[q];
  const int64_t self = p - base;
  const float4 ui = U[p];
  float S = 0.f, C = 0.f;
  for (int64_t jb = 0; jb < g; jb += 32) {
    const int64_t je = rsd::min64(jb + 32, g);
    float blk = 0.f;
    for (int64_t jj = jb; jj < je; ++jj) {
      const float4 uj = __ldg(U + base + jj);
      const float dx = __fsub_rn(uj.x, ui.x);
      const float dy = __fsub_rn(uj.y, ui.y);
      const float dz = __fsub_rn(uj.z, ui.z);
      const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmaf_rn(dz, dz, eps2)));
      const float w = rsqrtf(r2);
      blk = __fadd_rn(blk, jj == self ? 0.f : w);
    }
    const float y = __fsub_rn(blk, C);
    const float tt = __fadd_rn(S, y);
    C = __fsub_rn(__fsub_rn(tt, S), y);
    S = tt;
  }
  S_out[p] = S;
}

// Register-blocked variant for nodes larger than kBlockedMin: each of the 128 threads of a
// block owns 4 members (i = 512 t + tid + 128 k), processed as two packed pairs with the
// float32x2 add / fma instructions (each half rounded exactly like the scalar operation, so
// the results are bit-identical to the scalar form). Staged members are stored duplicated,
// (x, x, y, y) and (z, z), so a shared load yields the packed operands directly; differences
// are formed as u_j + (-u_i), which equals fl(u_j - u_i). The per-member summation is
// unchanged (32-term sequential blocks, Kahan across blocks), so the certified bound kCertB
// holds as is. The self pair is tested only on the diagonal j-tiles. Blocks are ordered by
// the node's size class, largest first, so the longest blocks start first.
constexpr int kBlkThreads = 128;
// Members per thread (kBlkR) is a template parameter chosen per context by the autotuner among
// 2, 4 and 8 (tiles of 256, 512 or 1024 members); every choice gives bit-identical sums.
constexpr int64_t kBlockedMin = 384;
constexpr int64_t kTuneMinMembers = 1 << 20;  // the autotuner times candidates on inputs this large

// Tiles of the two direct-sum kernels; nodes with >= sur_min members (sur_min > 0) are left to
// the surrogate path. Also the sort key of the blocked tiles' order (size class, descending).
// pairs (if given): ordered pairs g (g - 1) of the selected nodes, [0] small, [1] blocked.
__global__ void k_tiles_split(int64_t nn, const int64_t* __restrict__ node_size, int64_t sur_min,
                              const int* __restrict__ only, int64_t max_g, int blk_tile,
                              int64_t* __restrict__ small, int64_t* __restrict__ big,
                              uint64_t* __restrict__ okey, uint32_t* __restrict__ oval,
                              unsigned long long* __restrict__ pairs) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t g = k < nn ? node_size[k] : 0;
  const bool skip = k >= nn || (only ? (only[k] == 0) : (sur_min > 0 && g >= sur_min)) ||
                    (max_g > 0 && g >= max_g);
  const bool blocked = !skip && g > kBlockedMin;
  if (pairs) {  // warp sums, one atomic per warp and class
    unsigned long long ps = (!skip && !blocked) ? (unsigned long long)(g * (g - 1)) : 0ull;
    unsigned long long pb = blocked ? (unsigned long long)(g * (g - 1)) : 0ull;
    for (int off = 16; off >= 1; off >>= 1) {
      ps += __shfl_xor_sync(0xffffffffu, ps, off);
      pb += __shfl_xor_sync(0xffffffffu, pb, off);
    }
    if ((threadIdx.x & 31) == 0) {
      if (ps) atomicAdd(pairs, ps);
      if (pb) atomicAdd(pairs + 1, pb);
    }
  }
  if (k >= nn) return;
  small[k] = (skip || g > kBlockedMin) ? 0 : (g + kPotTile - 1) / kPotTile;
  big[k] = blocked ? (g + blk_tile - 1) / blk_tile : 0;
  okey[k] = blocked ? uint64_t(63 - __clzll(g)) ^ 63u : 255u;
  oval[k] = uint32_t(k);
}

// Plain form of the direct sum for nodes above kBlockedMin members: one thread per member,
// blocks of 128 members of one node in node order, j-tiles of 128 members staged in shared
// memory; the per-member summation (32-term sequential blocks of the j order, Kahan across
// blocks, self term 0) is the blocked kernel's, so the sums are bit-identical to it.
constexpr int kTileThreads = 128;

__global__ void __launch_bounds__(kTileThreads)
k_potential_tiled(int64_t nn, const int64_t* __restrict__ tile_off, const int64_t* __restrict__ node_off,
                  const int64_t* __restrict__ node_size, const float4* __restrict__ U, float eps2,
                  float* __restrict__ S_out) {
  __shared__ float4 su[kTileThreads];
  const int64_t b = blockIdx.x;
  if (b >= tile_off[nn]) return;
  const int64_t q = rsd::upper_bound_i64(tile_off, nn, b) - 1;
  const int64_t t = b - tile_off[q];
  const int64_t base = node_off[q], g = node_size[q];
  const int64_t i = t * kTileThreads + threadIdx.x;
  const float4 ui = i < g ? U[base + i] : make_float4(0, 0, 0, 0);
  float S = 0.f, C = 0.f;
  for (int64_t j0 = 0; j0 < g; j0 += kTileThreads) {
    if (j0 + threadIdx.x < g) su[threadIdx.x] = U[base + j0 + threadIdx.x];
    __syncthreads();
    const int jn = int(rsd::min64(kTileThreads, g - j0));
    for (int jb = 0; jb < jn; jb += 32) {
      const int je = min(jb + 32, jn);
      float blk = 0.f;
      for (int jj = jb; jj < je; ++jj) {
        const float4 uj = su[jj];
        const float dx = __fsub_rn(uj.x, ui.x);
        const float dy = __fsub_rn(uj.y, ui.y);
        const float dz = __fsub_rn(uj.z, ui.z);
        const float w = rsqrtf(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmaf_rn(dz, dz, eps2))));
        blk = __fadd_rn(blk, j0 + jj == i ? 0.f : w);
      }
      const float y = __fsub_rn(blk, C);
      const float tt = __fadd_rn(S, y);
      C = __fsub_rn(__fsub_rn(tt, S), y);
      S = tt;
    }
    __syncthreads();
  }
  if (i < g) S_out[base + i] = S;
}

__global__ void k_tiles_plain(int64_t nn, const int64_t* __restrict__ node_size, const int* __restrict__ only,
                              int64_t* __restrict__ out) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const int64_t g = node_size[k];
  out[k] = (g > kBlockedMin && (!only || only[k])) ? (g + kTileThreads - 1) / kTileThreads : 0;
}

__global__ void k_perm_tiles(int64_t nn, const uint32_t* __restrict__ perm,
                             const int64_t* __restrict__ big, int64_t* __restrict__ out) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r < nn) out[r] = big[perm[r]];
}

__device__ __forceinline__ void pot_pair(float4 a, float2 zz, float2 nx, float2 ny, float2 nz,
                                         float2 e2, float2& w) {
  const float2 dx = __fadd2_rn(make_float2(a.x, a.y), nx);
  const float2 dy = __fadd2_rn(make_float2(a.z, a.w), ny);
  const float2 dz = __fadd2_rn(zz, nz);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
  w = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
}

template <int kBlkR>
__global__ void __launch_bounds__(kBlkThreads)
k_potential_blocked(int64_t nn, const int64_t* __restrict__ tile_off, const uint32_t* __restrict__ perm,
                    const int64_t* __restrict__ node_off, const int64_t* __restrict__ node_size,
                    const float4* __restrict__ U, float eps2, float* __restrict__ S_out) {
  __shared__ float4 sxy[kBlkThreads];
  __shared__ float2 sz[kBlkThreads];
  const int64_t b = blockIdx.x;
  if (b >= tile_off[nn]) return;
  const int64_t r = rsd::upper_bound_i64(tile_off, nn, b) - 1;
  const int64_t q = perm[r];
  const int64_t t = b - tile_off[r];
  const int64_t base = node_off[q], g = node_size[q];
  float2 nx[kBlkR / 2], ny[kBlkR / 2], nz[kBlkR / 2];
  float S[kBlkR], C[kBlkR];
#pragma unroll
  for (int p = 0; p < kBlkR / 2; ++p) {
    const int64_t i0 = t * (kBlkThreads * kBlkR) + threadIdx.x + kBlkThreads * (2 * p);
    const int64_t i1 = i0 + kBlkThreads;
    const float4 u0 = i0 < g ? U[base + i0] : make_float4(0, 0, 0, 0);
    const float4 u1 = i1 < g ? U[base + i1] : make_float4(0, 0, 0, 0);
    nx[p] = make_float2(-u0.x, -u1.x);
    ny[p] = make_float2(-u0.y, -u1.y);
    nz[p] = make_float2(-u0.z, -u1.z);
  }
#pragma unroll
  for (int k = 0; k < kBlkR; ++k) {
    S[k] = 0.f;
    C[k] = 0.f;
  }
  const float2 e2 = make_float2(eps2, eps2);
  for (int64_t j0 = 0; j0 < g; j0 += kBlkThreads) {
    const int64_t j = j0 + threadIdx.x;
    if (j < g) {
      const float4 u = U[base + j];
      sxy[threadIdx.x] = make_float4(u.x, u.x, u.y, u.y);
      sz[threadIdx.x] = make_float2(u.z, u.z);
    }
    __syncthreads();
    const int jn = int(rsd::min64(kBlkThreads, g - j0));
    const int64_t jt = j0 / kBlkThreads - t * kBlkR;  // diagonal tile for member slot jt
    const bool diag = jt >= 0 && jt < kBlkR;
    for (int jb = 0; jb < jn; jb += 32) {
      const int je = min(jb + 32, jn);
      float2 blk[kBlkR / 2];
#pragma unroll
      for (int p = 0; p < kBlkR / 2; ++p) blk[p] = make_float2(0.f, 0.f);
      if (!diag && je - jb == 32) {
#pragma unroll 8
        for (int jj = jb; jj < jb + 32; ++jj) {
          const float4 a = sxy[jj];
          const float2 zz = sz[jj];
#pragma unroll
          for (int p = 0; p < kBlkR / 2; ++p) {
            float2 w;
            pot_pair(a, zz, nx[p], ny[p], nz[p], e2, w);
            blk[p] = __fadd2_rn(blk[p], w);
          }
        }
      } else {
        for (int jj = jb; jj < je; ++jj) {
          const float4 a = sxy[jj];
          const float2 zz = sz[jj];
          const bool self = diag && jj == int(threadIdx.x);
#pragma unroll
          for (int p = 0; p < kBlkR / 2; ++p) {
            float2 w;
            pot_pair(a, zz, nx[p], ny[p], nz[p], e2, w);
            if (self && jt == 2 * p) w.x = 0.f;
            if (self && jt == 2 * p + 1) w.y = 0.f;
            blk[p] = __fadd2_rn(blk[p], w);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kBlkR; ++k) {
        const float bk = (k & 1) ? blk[k >> 1].y : blk[k >> 1].x;
        const float y = __fsub_rn(bk, C[k]);
        const float tt = __fadd_rn(S[k], y);
        C[k] = __fsub_rn(__fsub_rn(tt, S[k]), y);
        S[k] = tt;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < kBlkR; ++k) {
    const int64_t i = t * (kBlkThreads * kBlkR) + threadIdx.x + kBlkThreads * k;
    if (i < g) S_out[base + i] = S[k];
  }
}

struct VelTerm {
  const float4* V;
  template <bool kFirst>
  __device__ __forceinline__ void add(int64_t, int64_t p, int64_t, double* acc) const {
    const float4 v = V[p];
    rsd::cro_add<kFirst>(acc[0], rsd::f2d(v.x));
    rsd::cro_add<kFirst>(acc[1], rsd::f2d(v.y));
    rsd::cro_add<kFirst>(acc[2], rsd::f2d(v.z));
  }
};

// Iterative unbinding: v of the members still bound, 0.0 for the others (the oracle's order).
struct VelTermMasked {
  const float4* V;
  const uint8_t* in;
  template <bool kFirst>
  __device__ __forceinline__ void add(int64_t, int64_t p, int64_t, double* acc) const {
    const float4 v = V[p];
    const bool keep = in[p] != 0;
    rsd::cro_add<kFirst>(acc[0], keep ? rsd::f2d(v.x) : 0.0);
    rsd::cro_add<kFirst>(acc[1], keep ? rsd::f2d(v.y) : 0.0);
    rsd::cro_add<kFirst>(acc[2], keep ? rsd::f2d(v.z) : 0.0);
  }
};

__global__ void k_vbulk_masked(int64_t nn, const unsigned long long* __restrict__ count,
                               double* __restrict__ v) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= 3 * nn) return;
  const unsigned long long c = count[k / 3];
  v[k] = c ? __ddiv_rn(v[k], double(c)) : 0.0;
}

// Positions of the members still bound; the others moved to +inf, so every pair term with them
// evaluates to exactly 0 (rsqrt(inf) = 1/sqrt(inf) = 0) in every potential kernel.
__global__ void k_mask_u(int64_t m, const float4* __restrict__ U, const uint8_t* __restrict__ in,
                         float4* __restrict__ Um) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const float inf = __int_as_float(0x7f800000);
  Um[p] = in[p] ? U[p] : make_float4(inf, inf, inf, 0.f);
}

// Members a pass removed (bound before, not after); the new flags become the next mask.
__global__ void k_removed(int64_t m, const uint8_t* __restrict__ before, const uint8_t* __restrict__ after,
                          unsigned long long* __restrict__ removed) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  rsd::warp_count(removed, p < m && before[p] && !after[p]);
}

// Bulk velocity of every node, vbulk = (canonical-order sum of v) / g, in place (one float64
// division per node and axis instead of one per member).
__global__ void k_vbulk(int64_t nn, const int64_t* __restrict__ node_size, double* __restrict__ v) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= 3 * nn) return;
  v[k] = __ddiv_rn(v[k], double(node_size[k / 3]));
}

__device__ __forceinline__ double kinetic(float4 v, const double* vb) {
  const double dvx = __dsub_rn(rsd::f2d(v.x), vb[0]);
  const double dvy = __dsub_rn(rsd::f2d(v.y), vb[1]);
  const double dvz = __dsub_rn(rsd::f2d(v.z), vb[2]);
  const double s = __dadd_rn(__dadd_rn(__dmul_rn(dvx, dvx), __dmul_rn(dvy, dvy)), __dmul_rn(dvz, dvz));
  return __dmul_rn(0.5, s);
}

__global__ void k_flags(int64_t m, const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_size,
                        const float4* __restrict__ V, const double* __restrict__ vbulk,
                        const float* __restrict__ S, double Gm, double certB,
                        uint8_t* __restrict__ bound, float* __restrict__ phi_out,
                        uint32_t* __restrict__ ambig, unsigned long long* __restrict__ n_ambig,
                        int64_t sur_min, const int* __restrict__ only, int64_t max_g,
                        const uint8_t* __restrict__ in) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const uint32_t q = mnode[p];
  const int64_t g = node_size[q];
  if ((only ? (only[q] == 0) : (sur_min > 0 && g >= sur_min)) || (max_g > 0 && g >= max_g))
    return;  // other path
  if (in && !in[p]) return;  // removed by an earlier pass: stays unbound
  const double ke = kinetic(V[p], vbulk + 3 * int64_t(q));
  const double ph = -__dmul_rn(Gm, double(S[p]));
  const double e = __dadd_rn(ke, ph);
  if (phi_out) phi_out[p] = __double2float_rn(ph);
  if (fabs(e) > __dmul_rn(2.0 * certB, fabs(ph))) {
    bound[p] = e < 0.0 ? 1 : 0;
  } else {
    bound[p] = 0;
    const unsigned long long k = atomicAdd(n_ambig, 1ull);
    ambig[k] = uint32_t(p);
  }
}

// Exact float64 potential of queued members: the canonical reduction order over j in member
// order with the self term 0.0, spread over the GPU because the float64 pipe runs 2 lanes per
// clock per SM on this part: one warp per chunk of 1024 terms (blocks of 8 chunks of member
// w0 + blockIdx.y) writes the chunk total to chunk_tot[w][c]; k_fallback_finish combines them
// with the pairwise tree and takes the flag.
__global__ void k_fallback_max_chunks(const unsigned long long* __restrict__ n_ambig,
                                      const uint32_t* __restrict__ ambig, const uint32_t* __restrict__ mnode,
                                      const int64_t* __restrict__ node_size,
                                      unsigned long long* __restrict__ out) {
  const unsigned long long total = *n_ambig;
  for (unsigned long long w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < total;
       w += int64_t(gridDim.x) * blockDim.x)
    atomicMax(out, (unsigned long long)((node_size[mnode[ambig[w]]] + 1023) / 1024));
}

__global__ void __launch_bounds__(kT)
k_fallback_chunks(int64_t w0, const uint32_t* __restrict__ ambig, const uint32_t* __restrict__ mnode,
                  const int64_t* __restrict__ node_off, const int64_t* __restrict__ node_size,
                  const float4* __restrict__ U, double eps2, int64_t max_chunks,
                  double* __restrict__ chunk_tot) {
  const int lane = threadIdx.x & 31;
  const int64_t w = w0 + blockIdx.y;
  const int64_t c = int64_t(blockIdx.x) * (kT / 32) + (threadIdx.x >> 5);
  const uint32_t p = ambig[w];
  const uint32_t q = mnode[p];
  const int64_t base = node_off[q], g = node_size[q];
  if (c * 1024 >= g) return;
  const int64_t i = int64_t(p) - base;
  const float4 ui = U[p];
  const double xi = ui.x, yi = ui.y, zi = ui.z;
  double acc = 0.0;
  for (int k = 0; k < 32; ++k) {
    const int64_t j = c * 1024 + lane + 32 * k;
    if (j < g) {
      double term = 0.0;
      if (j != i) {
        const float4 uj = U[base + j];
        const double dx = __dsub_rn(rsd::f2d(uj.x), xi);
        const double dy = __dsub_rn(rsd::f2d(uj.y), yi);
        const double dz = __dsub_rn(rsd::f2d(uj.z), zi);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        term = __ddiv_rn(1.0, __dsqrt_rn(__dadd_rn(r2, eps2)));
      }
      acc = __dadd_rn(acc, term);
    }
  }
  acc = rsd::warp_cro_combine(acc);
  if (lane == 0) chunk_tot[w * max_chunks + c] = acc;
}

__global__ void k_fallback_finish(int64_t n, const uint32_t* __restrict__ ambig,
                                  const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_size,
                                  const float4* __restrict__ V, const double* __restrict__ vbulk, double Gm,
                                  int64_t max_chunks, const double* __restrict__ chunk_tot,
                                  uint8_t* __restrict__ bound, float* __restrict__ phi_out) {
  const int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= n) return;
  const uint32_t p = ambig[w], q = mnode[p];
  const int64_t nc = (node_size[q] + 1023) / 1024;
  rsd::CroTree tree;
  for (int64_t c = 0; c < nc; ++c) tree.push(chunk_tot[w * max_chunks + c]);
  const double ph = -__dmul_rn(Gm, tree.result());
  const double ke = kinetic(V[p], vbulk + 3 * int64_t(q));
  bound[p] = __dadd_rn(ke, ph) < 0.0 ? 1 : 0;
  if (phi_out) phi_out[p] = __double2float_rn(ph);
}

__global__ void k_bound_count(int64_t m, const uint32_t* __restrict__ mnode, const uint8_t* __restrict__ bound,
                              unsigned long long* __restrict__ nb) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool valid = p < m && bound[p];
  rsd::warp_run_add(nb, valid ? mnode[p] : 0u, valid, 1ull);
}

__global__ void k_copy_u8(int64_t n, const uint8_t* __restrict__ a, uint8_t* __restrict__ b) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

// ---------------------------------------------------------------------------------------------
// Properties
struct PropTerm1 {  // bound-masked u, u^2, v, v^2
  const float4* U;
  const float4* V;
  const uint8_t* bound;
  template <bool kFirst>
  __device__ __forceinline__ void add(int64_t, int64_t p, int64_t, double* acc) const {
    if (!bound[p]) {
#pragma unroll
      for (int s = 0; s < 12; ++s) rsd::cro_add<kFirst>(acc[s], 0.0);
      return;
    }
    const float4 u = U[p], v = V[p];
    const double a[3] = {rsd::f2d(u.x), rsd::f2d(u.y), rsd::f2d(u.z)};
    const double b[3] = {rsd::f2d(v.x), rsd::f2d(v.y), rsd::f2d(v.z)};
    const float uc[3] = {u.x, u.y, u.z}, vc[3] = {v.x, v.y, v.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      rsd::cro_add<kFirst>(acc[d], a[d]);
      rsd::cro_add<kFirst>(acc[3 + d], rsd::sq_f2d(uc[d]));  // == a[d] * a[d], exactly
      rsd::cro_add<kFirst>(acc[6 + d], b[d]);
      rsd::cro_add<kFirst>(acc[9 + d], rsd::sq_f2d(vc[d]));
    }
  }
};

struct PropTerm2 {  // bound-masked second moments about the bound mean
  const float4* U;
  const uint8_t* bound;
  const double* mean;  // [node][3]
  template <bool kFirst>
  __device__ __forceinline__ void add(int64_t q, int64_t p, int64_t, double* acc) const {
    if (!bound[p]) {
#pragma unroll
      for (int s = 0; s < 6; ++s) rsd::cro_add<kFirst>(acc[s], 0.0);
      return;
    }
    const float4 u = U[p];
    const double* mu = mean + 3 * q;
    const double d[3] = {__dsub_rn(rsd::f2d(u.x), mu[0]), __dsub_rn(rsd::f2d(u.y), mu[1]),
                         __dsub_rn(rsd::f2d(u.z), mu[2])};
    rsd::cro_add<kFirst>(acc[0], __dmul_rn(d[0], d[0]));
    rsd::cro_add<kFirst>(acc[1], __dmul_rn(d[1], d[1]));
    rsd::cro_add<kFirst>(acc[2], __dmul_rn(d[2], d[2]));
    rsd::cro_add<kFirst>(acc[3], __dmul_rn(d[0], d[1]));
    rsd::cro_add<kFirst>(acc[4], __dmul_rn(d[0], d[2]));
    rsd::cro_add<kFirst>(acc[5], __dmul_rn(d[1], d[2]));
  }
};

__global__ void k_prop_means(int64_t nn, const unsigned long long* __restrict__ nb,
                             const double* __restrict__ s1, double* __restrict__ mean) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nn) return;
  const double c = double(nb[q]);
  for (int d = 0; d < 3; ++d) mean[3 * q + d] = nb[q] ? __ddiv_rn(s1[12 * q + d], c) : 0.0;
}

__global__ void k_prop_final(int64_t nn, const int64_t* __restrict__ node_size,
                             const unsigned long long* __restrict__ nb, const uint8_t* __restrict__ is_halo,
                             const double* __restrict__ s1, const double* __restrict__ s2,
                             const double* __restrict__ mean, const float4* __restrict__ ref,
                             float L, double m, double rho_bar, rs_halo_props_t* __restrict__ out) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nn) return;
  rs_halo_props_t P;
  memset(&P, 0, sizeof(P));
  P.n = node_size[q];
  P.n_bound = int64_t(nb[q]);
  P.is_halo = is_halo[q];
  P.m_bound = __dmul_rn(double(nb[q]), m);
  if (nb[q] > 0) {
    const double c = double(nb[q]);
    const double* S = s1 + 12 * q;
    double varx = 0.0, varv = 0.0;
    const float rp[3] = {ref[q].x, ref[q].y, ref[q].z};
    for (int d = 0; d < 3; ++d) {
      const double mu = mean[3 * q + d];
      const double mv = __ddiv_rn(S[6 + d], c);
      const double tx = __dsub_rn(__ddiv_rn(S[3 + d], c), __dmul_rn(mu, mu));
      const double tv = __dsub_rn(__ddiv_rn(S[9 + d], c), __dmul_rn(mv, mv));
      varx = (d == 0) ? tx : __dadd_rn(varx, tx);
      varv = (d == 0) ? tv : __dadd_rn(varv, tv);
      double cen = __dadd_rn(double(rp[d]), mu);
      if (cen < 0.0) cen = __dadd_rn(cen, double(L));
      else if (cen >= double(L)) cen = __dsub_rn(cen, double(L));
      P.pos[d] = cen;
      P.vel[d] = mv;
    }
    P.sigma_x = __dsqrt_rn(varx > 0.0 ? varx : 0.0);
    P.sigma_v = __dsqrt_rn(varv > 0.0 ? varv : 0.0);
    const double pi = 3.14159265358979323846;
    P.r_vir = cbrt(__ddiv_rn(__dmul_rn(3.0, P.m_bound),
                             __dmul_rn(__dmul_rn(__dmul_rn(4.0, pi), 200.0), rho_bar)));
    for (int k = 0; k < 6; ++k) P.inertia[k] = __ddiv_rn(s2[6 * q + k], c);
  }
  out[q] = P;
}

__global__ void k_halo_decide(int64_t nn, const int64_t* __restrict__ node_size,
                              const unsigned long long* __restrict__ nb, int min_size, int bnum, int bden,
                              uint8_t* __restrict__ is_halo) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nn) return;
  const int64_t c = int64_t(nb[q]);
  is_halo[q] = (c >= min_size && int64_t(bden) * c >= int64_t(bnum) * node_size[q]) ? 1 : 0;
}

// Tiles of the blocked kernel for kBlkR = R (nodes above kBlockedMin members, ordered by size
// class, largest first) and of k_potential (the other selected nodes).
int potential_tiles(rs_ctx* ctx, int64_t sur_min, const int* only, int64_t max_g, int R,
                    int64_t* tile_small, int64_t* tile_perm, uint32_t** perm, cudaStream_t st,
                    unsigned long long* pairs) {
  Hier h = hier_of(ctx);
  const int64_t nn = ctx->n_nodes;
  int64_t* tile_big = scratch_t<int64_t>(ctx, S_U_TILEBIG, size_t(nn) + 1);
  uint64_t* ka = scratch_t<uint64_t>(ctx, S_U_OKEY_A, size_t(nn));
  uint64_t* kb = scratch_t<uint64_t>(ctx, S_U_OKEY_B, size_t(nn));
  uint32_t* va = scratch_t<uint32_t>(ctx, S_U_OVAL_A, size_t(nn));
  uint32_t* vb = scratch_t<uint32_t>(ctx, S_U_OVAL_B, size_t(nn));
  if (!tile_big || !ka || !kb || !va || !vb) return RS_ERR_OOM;
  k_tiles_split<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_size, sur_min, only, max_g, kBlkThreads * R,
                                                 tile_small, tile_big, ka, va, pairs);
  RS_LAUNCHED(ctx, "k_tiles_split");
  uint64_t* ko;
  RS_TRY(radix_sort_u64(ctx, nn, 8, ka, va, kb, vb, &ko, perm, st));
  k_perm_tiles<<<grid_for(nn, kT), kT, 0, st>>>(nn, *perm, tile_big, tile_perm);
  RS_LAUNCHED(ctx, "k_perm_tiles");
  RS_TRY(exclusive_scan_i64(ctx, nn, tile_small, tile_small + nn, st));
  RS_TRY(exclusive_scan_i64(ctx, nn, tile_perm, tile_perm + nn, st));
  return RS_OK;
}

int launch_blocked(rs_ctx* ctx, int R, const int64_t* tile_perm, const uint32_t* perm, float* S,
                   cudaStream_t st) {
  Hier h = hier_of(ctx);
  const int64_t m = ctx->n_members, nn = ctx->n_nodes;
  const float eps2 = ctx->cfg.softening * ctx->cfg.softening;
  const unsigned grid = grid_for(m / (kBlockedMin + 1) + m / (kBlkThreads * R) + 1, 1);
  if (R == 2)
    k_potential_blocked<2><<<grid, kBlkThreads, 0, st>>>(nn, tile_perm, perm, h.node_off, h.node_size, h.U, eps2, S);
  else if (R == 8)
    k_potential_blocked<8><<<grid, kBlkThreads, 0, st>>>(nn, tile_perm, perm, h.node_off, h.node_size, h.U, eps2, S);
  else
    k_potential_blocked<4><<<grid, kBlkThreads, 0, st>>>(nn, tile_perm, perm, h.node_off, h.node_size, h.U, eps2, S);
  RS_LAUNCHED(ctx, "k_potential_blocked");
  return RS_OK;
}

// Float32 direct sums S_i = sum_{j != i} (|u_j - u_i|^2 + eps^2)^(-1/2) of every member of the
// selected nodes (only[k] != 0 if `only` is given, else nodes below sur_min when sur_min > 0,
// else all): nodes up to kBlockedMin members by k_potential, larger ones by the blocked kernel
// with its tiles ordered by node size class, largest first. The blocked kernel's members per
// thread come from the context's autotuner: on the first call with at least kTuneMinMembers
// members, each of 2, 4 and 8 is timed on that call's own nodes (CUDA events; identical sums)
// and the fastest is kept for the context.
int direct_potential(rs_ctx* ctx, int64_t sur_min, const int* only, int64_t max_g, float* S,
                     cudaStream_t st) {
  Hier h = hier_of(ctx);
  const int64_t m = ctx->n_members, nn = ctx->n_nodes;
  const float eps = ctx->cfg.softening;
  int64_t* tile_small = scratch_t<int64_t>(ctx, S_SELECT, size_t(nn) + 1);
  int64_t* tile_perm = scratch_t<int64_t>(ctx, S_U_TILEPERM, size_t(nn) + 1);
  if (!tile_small || !tile_perm) return RS_ERR_OOM;
  uint32_t* perm;
  const bool plain = ctx->cfg.batched == 0;
  if (!plain && ctx->tune_blk_r == 0 && m >= kTuneMinMembers) {
    const int cand[3] = {2, 4, 8};
    float best_ms = 0.f;
    int best = 4;
    cudaEvent_t e0, e1;
    RS_CUDA(ctx, cudaEventCreate(&e0));
    RS_CUDA(ctx, cudaEventCreate(&e1));
    for (int c = 0; c < 3; ++c) {
      RS_TRY(potential_tiles(ctx, sur_min, only, max_g, cand[c], tile_small, tile_perm, &perm, st,
                             nullptr));
      RS_CUDA(ctx, cudaEventRecord(e0, st));
      RS_TRY(launch_blocked(ctx, cand[c], tile_perm, perm, S, st));
      RS_CUDA(ctx, cudaEventRecord(e1, st));
      RS_CUDA(ctx, cudaEventSynchronize(e1));
      float ms = 0.f;
      RS_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
      ctx->tune_blk_ms[c] = ms;
      if (c == 0 || ms < best_ms) {
        best_ms = ms;
        best = cand[c];
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tune_blk_r = best;
  }
  const int R = ctx->tune_blk_r ? ctx->tune_blk_r : 4;
  // pair tallies of this rs_unbind (counters [20], [21], zeroed at its start)
  unsigned long long* pairs = static_cast<unsigned long long*>(ctx->buf[S_SUR_COUNTERS].ptr) + 20;
  RS_TRY(potential_tiles(ctx, sur_min, only, max_g, R, tile_small, tile_perm, &perm, st, pairs));
  {
    ProfScope prof_(ctx, "k_potential", st);
    k_potential<<<grid_for(m, kT), kT, 0, st>>>(m, h.mnode, tile_small, h.node_off, h.node_size, h.U,
                                               eps * eps, S);
  }
  RS_LAUNCHED(ctx, "k_potential");
  if (plain) {  // one member per thread, node order (the plain form has no size-ordered tiles)
    k_tiles_plain<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_size, only, tile_perm);
    RS_LAUNCHED(ctx, "k_tiles_plain");
    RS_TRY(exclusive_scan_i64(ctx, nn, tile_perm, tile_perm + nn, st));
    ProfScope prof_(ctx, "k_potential_tiled", st);
    k_potential_tiled<<<grid_for(m / (kBlockedMin + 1) + m / kTileThreads + 1, 1), kTileThreads, 0, st>>>(
        nn, tile_perm, h.node_off, h.node_size, h.U, eps * eps, S);
    RS_LAUNCHED(ctx, "k_potential_tiled");
    return RS_OK;
  }
  {
    ProfScope prof_(ctx, "k_potential_blocked", st);
    RS_TRY(launch_blocked(ctx, R, tile_perm, perm, S, st));
  }
  return RS_OK;
}

// Passes 2.. of iterative unbinding: each recomputes the bulk velocity and the potential of the
// members still bound over the members still bound (the others moved to +inf in a masked copy
// of U, which the potential kernels read in place of U during the pass) and re-flags them, until
// a pass removes nobody or `passes` passes have run. The float32 sums keep their certified
// bounds and the float64 fallback sees the same masked copy, so every pass's flags are exact.
int unbind_passes(rs_ctx* ctx, int passes, bool tree, int64_t max_g, double* vbulk, uint8_t* bound,
                  float* S, float* potential_out, uint32_t* ambig, unsigned long long* counters,
                  cudaStream_t st) {
  Hier h = hier_of(ctx);
  const int64_t m = ctx->n_members, nn = ctx->n_nodes;
  const double Gm = ctx->cfg.G * ctx->cfg.particle_mass;
  uint8_t* in = scratch_t<uint8_t>(ctx, S_U_PREV, size_t(m));
  float4* Um = scratch_t<float4>(ctx, S_U_UM, size_t(m));
  unsigned long long* cnt = scratch_t<unsigned long long>(ctx, S_U_PCNT, size_t(nn) + 1);
  if (!in || !Um || !cnt) return RS_ERR_OOM;
  unsigned long long* removed = cnt + nn;
  for (int pass = 2; pass <= passes; ++pass) {
    RS_CUDA(ctx, cudaMemcpyAsync(in, bound, size_t(m), cudaMemcpyDeviceToDevice, st));
    RS_CUDA(ctx, cudaMemsetAsync(cnt, 0, 8 * (size_t(nn) + 1), st));
    k_bound_count<<<grid_for(m, kT), kT, 0, st>>>(m, h.mnode, in, cnt);
    RS_LAUNCHED(ctx, "k_bound_count");
    RS_TRY((cro_segmented<3, VelTermMasked>(ctx, nn, h.node_off, h.node_size, m, VelTermMasked{h.V, in},
                                            vbulk, st)));
    k_vbulk_masked<<<grid_for(3 * nn, kT), kT, 0, st>>>(nn, cnt, vbulk);
    RS_LAUNCHED(ctx, "k_vbulk_masked");
    k_mask_u<<<grid_for(m, kT), kT, 0, st>>>(m, h.U, in, Um);
    RS_LAUNCHED(ctx, "k_mask_u");
    std::swap(ctx->buf[S_H_U], ctx->buf[S_U_UM]);  // the pass's kernels read the masked copy
    int rc = direct_potential(ctx, 0, nullptr, max_g, S, st);
    Hier hm = hier_of(ctx);
    if (rc == RS_OK) {
      k_flags<<<grid_for(m, kT), kT, 0, st>>>(m, hm.mnode, hm.node_size, hm.V, vbulk, S, Gm, kCertB, bound,
                                             potential_out, ambig, counters + 7, 0, nullptr, max_g, in);
      rc = after_launch(ctx, "k_flags");
    }
    if (rc == RS_OK) rc = unbind_fallback(ctx, counters + 7, ambig, vbulk, bound, st, potential_out);
    if (rc == RS_OK && tree) rc = tree_build(ctx, st);
    if (rc == RS_OK && tree) rc = tree_decide(ctx, nullptr, in, vbulk, bound, counters, st);
    std::swap(ctx->buf[S_H_U], ctx->buf[S_U_UM]);
    if (rc != RS_OK) return rc;
    RS_CUDA(ctx, cudaMemsetAsync(removed, 0, 8, st));
    k_removed<<<grid_for(m, kT), kT, 0, st>>>(m, in, bound, removed);
    RS_LAUNCHED(ctx, "k_removed");
    RS_TRY(read_back(ctx, removed, 8, st));
    ctx->unbind_passes_run = pass;
    if (ctx->host_box[0] == 0) break;
  }
  return RS_OK;
}

}  // namespace

extern "C" int rs_unbind(rs_ctx* ctx, const float* pos, const float* vel, float* potential_out,
                         uint8_t* bound_out, int64_t* n_fallback_out, void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  ctx->have_unbind = false;
  if (!ctx->have_hier) return set_error(ctx, RS_ERR_STATE, "rs_fof6d has not run on this context");
  const int64_t m = ctx->n_members, nn = ctx->n_nodes;
  if (m > 0 && !bound_out) return set_error(ctx, RS_ERR_INVALID_ARG, "bound_out is NULL");
  if (m > 0 && (!pos || !vel)) return set_error(ctx, RS_ERR_INVALID_ARG, "null pos/vel");
  const bool sur = ctx->cfg.use_surrogate != 0;
  const int passes = std::max(1, int(ctx->cfg.unbind_passes));
  if (sur && passes > 1)
    return set_error(ctx, RS_ERR_INVALID_ARG, "iterative unbinding runs in the plain and batched forms");
  if (sur && potential_out)
    return set_error(ctx, RS_ERR_INVALID_ARG, "potential_out must be NULL with the surrogate");
  if (sur && !ctx->have_mlp)
    return set_error(ctx, RS_ERR_STATE, "the surrogate needs weights (rs_mlp_train or set_params)");
  const int64_t sur_min = sur ? kSurrogateMinMembers : 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  if (pos != ctx->h_pos || vel != ctx->h_vel) {  // other arrays than rs_fof6d's: re-gather
    RS_TRY(gather_members(ctx, 0, m, 0, nn, pos, vel, st));
    ctx->h_pos = pos;
    ctx->h_vel = vel;
  }
  Hier h = hier_of(ctx);
  uint8_t* bound = scratch_t<uint8_t>(ctx, S_U_BOUND, size_t(std::max<int64_t>(m, 1)));
  float* S = scratch_t<float>(ctx, S_U_PHI, size_t(std::max<int64_t>(m, 1)));
  unsigned long long* nb = scratch_t<unsigned long long>(ctx, S_U_NB, size_t(std::max<int64_t>(nn, 1)));
  double* vbulk = scratch_t<double>(ctx, S_U_VBULK, size_t(std::max<int64_t>(nn, 1)) * 3);
  uint32_t* ambig = scratch_t<uint32_t>(ctx, S_U_AMBIG, size_t(std::max<int64_t>(m, 1)));
  uint8_t* halo = scratch_t<uint8_t>(ctx, S_U_FLAGS, size_t(std::max<int64_t>(nn, 1)));
  // counters: [0..6], [8..11], [19] surrogate path (rs_surrogate.cu), [7] float64 fallbacks of
  // the direct sums, [12..18] certified tree bound (rs_tree.cu), [20..21] direct-sum pairs
  unsigned long long* counters = scratch_t<unsigned long long>(ctx, S_SUR_COUNTERS, kCounters);
  if (!bound || !S || !nb || !vbulk || !ambig || !halo || !counters) return RS_ERR_OOM;
  unsigned long long* n_ambig = counters + 7;
  // certified tree bound: batched forms, when no potential is asked for
  const bool tree = ctx->tree_min > 0 && potential_out == nullptr && ctx->cfg.batched != 0;
  const int64_t tree_min = ctx->tree_min;
  const int64_t max_g = (tree && !sur) ? tree_min : 0;
  ctx->tree_recorded = false;
  double* rec = nullptr;
  if (tree && ctx->tree_record && m > 0) {
    rec = scratch_t<double>(ctx, S_T_REC, 2 * size_t(m));
    if (!rec) return RS_ERR_OOM;
    RS_CUDA(ctx, cudaMemsetAsync(rec, 0xff, 16 * size_t(m), st));  // NaN: not bounded
  }
  int64_t nfb = 0;
  for (int i = 0; i < 11; ++i) ctx->sur_stats[i] = 0;
  for (int i = 0; i < 8; ++i) ctx->tree_stats[i] = 0;
  ctx->pot_pairs[0] = ctx->pot_pairs[1] = 0;
  ctx->tree_nt = ctx->tree_T = ctx->tree_C = 0;
  ctx->unbind_passes_run = 1;
  if (m > 0) {
    const double Gm = ctx->cfg.G * ctx->cfg.particle_mass;
    RS_CUDA(ctx, cudaMemsetAsync(counters, 0, kCounters * sizeof(unsigned long long), st));
    RS_TRY((cro_segmented<3, VelTerm>(ctx, nn, h.node_off, h.node_size, m, VelTerm{h.V}, vbulk, st)));
    k_vbulk<<<grid_for(3 * nn, kT), kT, 0, st>>>(nn, h.node_size, vbulk);  // sums -> bulk velocities
    RS_LAUNCHED(ctx, "k_vbulk");
    RS_TRY(direct_potential(ctx, sur_min, nullptr, max_g, S, st));
    k_flags<<<grid_for(m, kT), kT, 0, st>>>(m, h.mnode, h.node_size, h.V, vbulk, S, Gm, kCertB, bound,
                                           potential_out, ambig, n_ambig, sur_min, nullptr, max_g,
                                           nullptr);
    RS_LAUNCHED(ctx, "k_flags");
    RS_TRY(unbind_fallback(ctx, n_ambig, ambig, vbulk, bound, st, potential_out));
    if (tree) RS_TRY(tree_build(ctx, st));
    if (tree && !sur) RS_TRY(tree_decide(ctx, nullptr, nullptr, vbulk, bound, counters, st));
    if (sur) RS_TRY(surrogate_unbind(ctx, vbulk, bound, counters, st));
    if (passes > 1) RS_TRY(unbind_passes(ctx, passes, tree, max_g, vbulk, bound, S, potential_out, ambig,
                                         counters, st));
    RS_CUDA(ctx, cudaMemsetAsync(nb, 0, 8 * nn, st));
    k_bound_count<<<grid_for(m, kT), kT, 0, st>>>(m, h.mnode, bound, nb);
    RS_LAUNCHED(ctx, "k_bound_count");
    k_halo_decide<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_size, nb, ctx->cfg.min_halo_particles,
                                                  ctx->cfg.bound_num, ctx->cfg.bound_den, halo);
    RS_LAUNCHED(ctx, "k_halo_decide");
    k_copy_u8<<<grid_for(m, kT), kT, 0, st>>>(m, bound, bound_out);
    RS_LAUNCHED(ctx, "k_copy_u8");
    RS_TRY(read_back(ctx, counters, kCounters * sizeof(unsigned long long), st));
    // stats: surrogate members, gated, exact (exact-path list + calibration members, outside
    // nodes sent whole), spot-checked, failed nodes, fp64 (surrogate path), fp64 (direct sums),
    // re-run members, members of nodes sent whole to the direct sum, members whose flag the
    // surrogate decided, spot-checked members whose surrogate flag was wrong
    ctx->sur_stats[0] = sur ? ctx->sur_members : 0;
    ctx->sur_stats[1] = ctx->host_box[5];
    ctx->sur_stats[2] = ctx->host_box[0] + ctx->host_box[11];
    ctx->sur_stats[3] = ctx->host_box[1];
    ctx->sur_stats[4] = ctx->host_box[4];
    ctx->sur_stats[5] = ctx->host_box[6];
    ctx->sur_stats[6] = ctx->host_box[7];
    ctx->sur_stats[7] = ctx->host_box[3];
    ctx->sur_stats[8] = ctx->host_box[8];
    ctx->sur_stats[9] = ctx->host_box[10];
    ctx->sur_stats[10] = ctx->host_box[19];
    // tree: nodes, members, decided by the bound, sent to the exact list, expansions, direct
    // pairs, pair terms of the exact list sums (tree and surrogate paths)
    ctx->tree_stats[0] = ctx->tree_nt;
    ctx->tree_stats[1] = ctx->tree_T;
    for (int i = 0; i < 4; ++i) ctx->tree_stats[2 + i] = ctx->host_box[12 + i];
    ctx->tree_stats[6] = ctx->host_box[18];
    ctx->pot_pairs[0] = ctx->host_box[20];
    ctx->pot_pairs[1] = ctx->host_box[21];
    nfb = ctx->host_box[7] + ctx->host_box[6];
    ctx->tree_recorded = rec != nullptr;
  }
  if (n_fallback_out) *n_fallback_out = nfb;
  ctx->have_unbind = true;
  ctx->last_unbind_surrogate = sur;
  return RS_OK;
}

extern "C" int rs_potential_pairs(rs_ctx* ctx, int64_t* pairs_out) {
  if (!ctx || !pairs_out) return RS_ERR_INVALID_ARG;
  pairs_out[0] = ctx->pot_pairs[0];
  pairs_out[1] = ctx->pot_pairs[1];
  return RS_OK;
}

// Exact unbinding of the nodes flagged in `only` (int [n_nodes]): register-blocked float32
// potential of all their members, certified flags, float64 fallback for the ambiguous ones;
// nodes with a built tree (tree_build of this rs_unbind) go through the certified tree bound.
int rs::unbind_nodes(rs_ctx* ctx, const int* only, const double* vbulk, uint8_t* bound,
                     uint32_t* ambig, unsigned long long* n_ambig, cudaStream_t st,
                     unsigned long long* counters) {
  Hier h = hier_of(ctx);
  const int64_t m = ctx->n_members;
  float* S = static_cast<float*>(ctx->buf[S_U_PHI].ptr);
  const double Gm = ctx->cfg.G * ctx->cfg.particle_mass;
  const int64_t max_g = ctx->tree_nt > 0 ? ctx->tree_min : 0;
  RS_TRY(direct_potential(ctx, 0, only, max_g, S, st));
  k_flags<<<grid_for(m, kT), kT, 0, st>>>(m, h.mnode, h.node_size, h.V, vbulk, S, Gm, kCertB, bound, nullptr,
                                         ambig, n_ambig, 0, only, max_g, nullptr);
  RS_LAUNCHED(ctx, "k_flags");
  RS_TRY(unbind_fallback(ctx, n_ambig, ambig, vbulk, bound, st));
  if (ctx->tree_nt > 0) RS_TRY(tree_decide(ctx, only, nullptr, vbulk, bound, counters, st));
  return RS_OK;
}

int rs::unbind_fallback(rs_ctx* ctx, const unsigned long long* n_ambig, const uint32_t* ambig,
                        const double* vbulk, uint8_t* bound, cudaStream_t st, float* phi_out) {
  Hier h = hier_of(ctx);
  const double Gm = ctx->cfg.G * ctx->cfg.particle_mass;
  const double eps = ctx->cfg.softening;
  unsigned long long* mc = scratch_t<unsigned long long>(ctx, S_U_FBMAX, 1);
  if (!mc) return RS_ERR_OOM;
  RS_CUDA(ctx, cudaMemsetAsync(mc, 0, sizeof(unsigned long long), st));
  k_fallback_max_chunks<<<152, kT, 0, st>>>(n_ambig, ambig, h.mnode, h.node_size, mc);
  RS_LAUNCHED(ctx, "k_fallback_max_chunks");
  RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box, n_ambig, 8, cudaMemcpyDeviceToHost, st));
  RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box + 1, mc, 8, cudaMemcpyDeviceToHost, st));
  RS_CUDA(ctx, cudaStreamSynchronize(st));
  const int64_t n = ctx->host_box[0], max_chunks = ctx->host_box[1];
  if (n == 0) return RS_OK;
  double* chunk_tot = scratch_t<double>(ctx, S_U_FBCHUNK, size_t(n) * size_t(max_chunks));
  if (!chunk_tot) return RS_ERR_OOM;
  {
    ProfScope prof_(ctx, "k_fallback", st);
    for (int64_t w0 = 0; w0 < n; w0 += 65535) {
      const dim3 grid(unsigned((max_chunks + kT / 32 - 1) / (kT / 32)), unsigned(std::min<int64_t>(65535, n - w0)));
      k_fallback_chunks<<<grid, kT, 0, st>>>(w0, ambig, h.mnode, h.node_off, h.node_size, h.U, eps * eps,
                                              max_chunks, chunk_tot);
    }
  }
  RS_LAUNCHED(ctx, "k_fallback_chunks");
  k_fallback_finish<<<grid_for(n, kT), kT, 0, st>>>(n, ambig, h.mnode, h.node_size, h.V, vbulk, Gm, max_chunks,
                                                   chunk_tot, bound, phi_out);
  RS_LAUNCHED(ctx, "k_fallback_finish");
  return RS_OK;
}

extern "C" int rs_unbind_passes(rs_ctx* ctx) { return ctx ? ctx->unbind_passes_run : 0; }

extern "C" int rs_halo_props(rs_ctx* ctx, rs_halo_props_t* props_out, void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (!ctx->have_hier || !ctx->have_unbind)
    return set_error(ctx, RS_ERR_STATE, "rs_halo_props needs rs_fof6d and rs_unbind first");
  const int64_t m = ctx->n_members, nn = ctx->n_nodes;
  if (nn == 0) return RS_OK;
  if (!props_out) return set_error(ctx, RS_ERR_INVALID_ARG, "props_out is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  Hier h = hier_of(ctx);
  uint8_t* bound = static_cast<uint8_t*>(ctx->buf[S_U_BOUND].ptr);
  unsigned long long* nb = static_cast<unsigned long long*>(ctx->buf[S_U_NB].ptr);
  uint8_t* halo = static_cast<uint8_t*>(ctx->buf[S_U_FLAGS].ptr);
  double* s1 = scratch_t<double>(ctx, S_NODE_TMP, size_t(nn) * 12);
  double* s2 = scratch_t<double>(ctx, S_GVAL_B, size_t(nn) * 6);
  double* mean = scratch_t<double>(ctx, S_GKEY_B, size_t(nn) * 3);
  if (!s1 || !s2 || !mean) return RS_ERR_OOM;
  RS_TRY((cro_segmented<12, PropTerm1>(ctx, nn, h.node_off, h.node_size, m, PropTerm1{h.U, h.V, bound},
                                       s1, st)));
  k_prop_means<<<grid_for(nn, kT), kT, 0, st>>>(nn, nb, s1, mean);
  RS_LAUNCHED(ctx, "k_prop_means");
  RS_TRY((cro_segmented<6, PropTerm2>(ctx, nn, h.node_off, h.node_size, m, PropTerm2{h.U, bound, mean},
                                      s2, st)));
  const double L = ctx->cfg.box_L;
  const double rho_bar = double(ctx->n_particles) * ctx->cfg.particle_mass / (L * L * L);
  k_prop_final<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_size, nb, halo, s1, s2, mean, h.ref,
                                               ctx->cfg.box_L, ctx->cfg.particle_mass, rho_bar,
                                               props_out);
  RS_LAUNCHED(ctx, "k_prop_final");
  return RS_OK;
}

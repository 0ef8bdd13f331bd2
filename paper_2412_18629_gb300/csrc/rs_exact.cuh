// Exact float32 potential sums of a LIST of members (the members whose flag is still open after
// a gate), with certified flags; shared by the surrogate path and the certified tree bound.
//
// A list entry k indexes a member-position map (mem_of[k] = p, the member's position in the
// hierarchy's member CSR); the list is grouped by node, with per-node ranges [lofs, lend).
#pragma once

#include "rs_cro.cuh"

namespace {

constexpr double kU = 5.9604644775390625e-08;
// per-member warp sum: per term <= 8u, 32-term lane blocks <= 31u, Kahan <= 2u, 5-level warp
// tree <= 5u; 48u with slack.
constexpr double kCertB2 = 48.0 * kU + 1e-12;

// Blocked direct sum over a list: 128 threads x kListR members per block (kListR: a template
// parameter the autotuner picks among 2, 4, 8).
constexpr int kListThreads = 128;

// 0.5 |v - v_bulk|^2 in float64, every operation rounded (the oracle's kinetic energy).
__device__ __forceinline__ double kinetic(float4 v, const double* vb) {
  const double dvx = __dsub_rn(rsd::f2d(v.x), vb[0]);
  const double dvy = __dsub_rn(rsd::f2d(v.y), vb[1]);
  const double dvz = __dsub_rn(rsd::f2d(v.z), vb[2]);
  const double s = __dadd_rn(__dadd_rn(__dmul_rn(dvx, dvx), __dmul_rn(dvy, dvy)), __dmul_rn(dvz, dvz));
  return __dmul_rn(0.5, s);
}

// Float32 sums S_all,i = sum over ALL members j of the node (self included) of
// (|u_j - u_i|^2 + eps^2)^(-1/2) for the members i of the exact-path list: block b covers one
// 512-member tile of one big node's list; j-tiles of 128 members staged duplicated in shared
// memory, packed float32x2 arithmetic, 32-term sequential blocks added with Kahan compensation
// (the same per-member summation as the direct-sum kernels). Including the self term, whose
// computed value is exactly w0 = rsqrt(eps^2), removes every per-pair index test; k_flags_list
// subtracts it and widens the certified bound accordingly.
template <int kListR>
__global__ void __launch_bounds__(kListThreads)
k_potential_list(int64_t nbig, const int64_t* __restrict__ tile_off, const int64_t* __restrict__ nodes,
                 const int64_t* __restrict__ lofs, const int64_t* __restrict__ lend,
                 const uint32_t* __restrict__ list, const uint32_t* __restrict__ mem_of,
                 const int64_t* __restrict__ node_off, const int64_t* __restrict__ node_size,
                 const float4* __restrict__ U, float eps2, float* __restrict__ Sx) {
  __shared__ float4 sxy[kListThreads];
  __shared__ float2 sz[kListThreads];
  const int64_t b = blockIdx.x;
  if (b >= tile_off[nbig]) return;
  const int64_t bi = rsd::upper_bound_i64(tile_off, nbig, b) - 1;
  const int64_t q = nodes[bi], t = b - tile_off[bi];
  const int64_t base = node_off[q], g = node_size[q];
  const int64_t l0 = lofs[bi] + t * (kListThreads * kListR), l1 = lend[bi];
  float2 nx[kListR / 2], ny[kListR / 2], nz[kListR / 2];
  float S[kListR], C[kListR];
#pragma unroll
  for (int pp = 0; pp < kListR / 2; ++pp) {
    const int64_t a0 = l0 + threadIdx.x + kListThreads * (2 * pp), a1 = a0 + kListThreads;
    const float4 u0 = a0 < l1 ? U[mem_of[list[a0]]] : make_float4(0, 0, 0, 0);
    const float4 u1 = a1 < l1 ? U[mem_of[list[a1]]] : make_float4(0, 0, 0, 0);
    nx[pp] = make_float2(-u0.x, -u1.x);
    ny[pp] = make_float2(-u0.y, -u1.y);
    nz[pp] = make_float2(-u0.z, -u1.z);
  }
#pragma unroll
  for (int k = 0; k < kListR; ++k) {
    S[k] = 0.f;
    C[k] = 0.f;
  }
  const float2 e2 = make_float2(eps2, eps2);
  for (int64_t j0 = 0; j0 < g; j0 += kListThreads) {
    const int64_t j = j0 + threadIdx.x;
    if (j < g) {
      const float4 u = U[base + j];
      sxy[threadIdx.x] = make_float4(u.x, u.x, u.y, u.y);
      sz[threadIdx.x] = make_float2(u.z, u.z);
    }
    __syncthreads();
    const int jn = int(rsd::min64(kListThreads, g - j0));
    for (int jb = 0; jb < jn; jb += 32) {
      const int je = min(jb + 32, jn);
      float2 blk[kListR / 2];
#pragma unroll
      for (int pp = 0; pp < kListR / 2; ++pp) blk[pp] = make_float2(0.f, 0.f);
#pragma unroll 8
      for (int jj = jb; jj < je; ++jj) {
        const float4 a = sxy[jj];
        const float2 zz = sz[jj];
#pragma unroll
        for (int pp = 0; pp < kListR / 2; ++pp) {
          const float2 dx = __fadd2_rn(make_float2(a.x, a.y), nx[pp]);
          const float2 dy = __fadd2_rn(make_float2(a.z, a.w), ny[pp]);
          const float2 dz = __fadd2_rn(zz, nz[pp]);
          const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
          blk[pp] = __fadd2_rn(blk[pp], make_float2(rsqrtf(r2.x), rsqrtf(r2.y)));
        }
      }
#pragma unroll
      for (int k = 0; k < kListR; ++k) {
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
  for (int k = 0; k < kListR; ++k) {
    const int64_t a = l0 + threadIdx.x + kListThreads * k;
    if (a < l1) Sx[list[a]] = S[k];
  }
}

// Flags of the exact-path list from S_all: S = fl(S_all - w0). With B = 41u the bound of the
// blocked sum relative to S_all = S + w0, |S - S_true| <= B (S + w0) + u S, so the member's
// relative bound is Bi = B (1 + w0 / S) + u (plus slack); the flag is certain when
// |KE + phi~| > 2 Bi |phi~|, otherwise the member is queued for the float64 potential.
__global__ void k_flags_list(const unsigned long long* __restrict__ count, const uint32_t* __restrict__ list,
                             const uint32_t* __restrict__ mem_of, const uint32_t* __restrict__ mnode,
                             const float4* __restrict__ V, const double* __restrict__ vbulk,
                             float eps2, double Gm, float* __restrict__ Sx, uint8_t* __restrict__ bound,
                             uint32_t* __restrict__ ambig, unsigned long long* __restrict__ n_ambig) {
  const int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= int64_t(*count)) return;
  const uint32_t k = list[w];
  const uint32_t p = mem_of[k], q = mnode[p];
  const float w0 = rsqrtf(eps2);
  const float S = __fsub_rn(Sx[k], w0);
  Sx[k] = S;
  const double ph = -__dmul_rn(Gm, double(S));
  const double e = __dadd_rn(kinetic(V[p], vbulk + 3 * int64_t(q)), ph);
  const double Bi = 41.0 * kU * (1.0 + double(w0) / fmax(double(S), 1e-30)) + 2.0 * kU + 1e-12;
  if (S > 0.f && fabs(e) > 2.0 * Bi * fabs(ph)) {
    bound[p] = e < 0.0 ? 1 : 0;
  } else {
    ambig[atomicAdd(n_ambig, 1ull)] = p;
  }
}

}  // namespace

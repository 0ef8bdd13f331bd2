// Segmented float64 sums in the canonical reduction order (CRO), used for every FP64 sum of the
// path: node moments (sigma_x, sigma_v of the 6D metric), bulk velocities, the exact FP64
// potential and halo properties.
//
// CRO of a[0..m): chunks of 1024 consecutive terms; inside chunk c lane l (0..31) adds
// a[1024c + l + 32k], k = 0..31, in order starting from 0.0; the 32 lane sums combine by the
// halving tree s[l] += s[l + off], off = 16..1 (an xor butterfly gives lane 0 the same value);
// chunk totals combine by the level-by-level pairwise tree with an odd last element carried up.
// That tree equals "merge equal-height subtrees as chunks arrive, then fold the remaining stack
// right to left", which is how the device evaluates it in O(log m) registers.
#pragma once

#include "rs_common.cuh"

namespace rsd {

// Streaming evaluation of the pairwise tree over chunk totals.
struct CroTree {
  double stk[40];
  int hgt[40];
  int sp = 0;
  __device__ __forceinline__ void push(double v) {
    int h = 0;
    while (sp > 0 && hgt[sp - 1] == h) {
      v = __dadd_rn(stk[sp - 1], v);
      --sp;
      ++h;
    }
    stk[sp] = v;
    hgt[sp] = h;
    ++sp;
  }
  __device__ __forceinline__ double result() const {
    if (sp == 0) return 0.0;
    double v = stk[sp - 1];
    for (int k = sp - 2; k >= 0; --k) v = __dadd_rn(stk[k], v);
    return v;
  }
};

__device__ __forceinline__ int64_t upper_bound_i64(const int64_t* a, int64_t n, int64_t v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One warp per chunk of 1024 terms of one segment. Term::add<first>(q, p, idx, acc) adds the NS
// terms of element p (global member position; idx = position inside the segment) of segment q
// (first: the lane's first term, added to 0.0 by rsd::cro_add<true>).
// chunk_off has nseg + 1 entries (the last one is the total number of chunks).
template <int NS, class Term>
__global__ void __launch_bounds__(256)
k_cro_chunks(int64_t nseg, const int64_t* __restrict__ chunk_off,
             const int64_t* __restrict__ seg_off, const int64_t* __restrict__ seg_size, Term term,
             double* __restrict__ out) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= chunk_off[nseg]) return;
  const int64_t q = upper_bound_i64(chunk_off, nseg, w) - 1;
  const int64_t cc = w - chunk_off[q];
  const int64_t base = seg_off[q], g = seg_size[q];
  double acc[NS];
  const int64_t i0 = cc * 1024 + lane;
  if (i0 < g) {
    term.template add<true>(q, base + i0, i0, acc);
  } else {
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  }
  for (int k = 1; k < 32; ++k) {
    const int64_t idx = i0 + 32 * k;
    if (idx < g) term.template add<false>(q, base + idx, idx, acc);
  }
  const int64_t cs = g - cc * 1024;  // terms in this chunk (lanes at or above cs hold 0.0)
  int off0 = 16;
  while (off0 > 1 && cs <= off0) off0 >>= 1;
  if (cs <= 1) off0 = 0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const double v = warp_cro_combine(acc[s], off0);
    if (lane == 0) out[w * NS + s] = v;
  }
}

// Pairwise tree over each segment's chunk totals -> seg_sums[q][NS]. One thread per segment.
template <int NS>
__global__ void __launch_bounds__(128)
k_cro_tree(int64_t nseg, const int64_t* __restrict__ chunk_off,
           const double* __restrict__ chunk_sums, double* __restrict__ seg_sums) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nseg) return;
  const int64_t c0 = chunk_off[q];
  const int64_t c1 = chunk_off[q + 1];
  for (int s = 0; s < NS; ++s) {
    CroTree t;
    for (int64_t c = c0; c < c1; ++c) t.push(chunk_sums[c * NS + s]);
    seg_sums[q * NS + s] = t.result();
  }
}

}  // namespace rsd

namespace rs {

// Segmented CRO driver: segment q covers global positions [seg_off[q], seg_off[q] + seg_size[q]);
// `total` = sum of the sizes (bounds the chunk count without a host round trip).
// Writes seg_sums[q * NS + s]. Uses the S_CHUNK_OFF / S_CHUNK_SUM scratch slots.
// chunk_off[q] = sum over earlier segments of ceil(size / 1024); chunk_off[nseg] = total chunks.
int cro_prepare(rs_ctx* ctx, int64_t nseg, const int64_t* seg_size, int64_t** chunk_off,
                cudaStream_t st);

template <int NS, class Term>
int cro_segmented(rs_ctx* ctx, int64_t nseg, const int64_t* seg_off, const int64_t* seg_size,
                  int64_t total, Term term, double* seg_sums, cudaStream_t st) {
  if (nseg <= 0) return RS_OK;
  int64_t* chunk_off;
  RS_TRY(cro_prepare(ctx, nseg, seg_size, &chunk_off, st));
  const int64_t nchunks_ub = nseg + total / 1024 + 1;
  double* chunk_sums = scratch_t<double>(ctx, S_CHUNK_SUM, size_t(nchunks_ub) * NS);
  if (!chunk_sums) return RS_ERR_OOM;
  rsd::k_cro_chunks<NS, Term><<<grid_for(nchunks_ub * 32, 256), 256, 0, st>>>(
      nseg, chunk_off, seg_off, seg_size, term, chunk_sums);
  RS_LAUNCHED(ctx, "k_cro_chunks");
  rsd::k_cro_tree<NS><<<grid_for(nseg, 128), 128, 0, st>>>(nseg, chunk_off, chunk_sums, seg_sums);
  RS_LAUNCHED(ctx, "k_cro_tree");
  return RS_OK;
}

}  // namespace rs

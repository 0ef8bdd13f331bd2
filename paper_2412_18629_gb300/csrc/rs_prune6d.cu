// Pruned 6D nearest-neighbour and link searches for the batched form of rs_fof6d.
//
// The plain form evaluates d6 for every pair of a node. Here the members of every node of a
// level are ordered by a 3D Morton key of their scaled position offsets (every candidate of a
// 6D search lies within sqrt(bound / inv_sx2) in position) and cut into buckets of 32
// consecutive members; each bucket has a 6D bounding box, four 8-member sub-boxes, and every
// 32 consecutive buckets of a node form a superbucket with its own box. Persistent warps pull
// query buckets from a queue ordered by node size (largest first) and, lane = member, visit
// the node's superbuckets, buckets and sub-buckets, skipping any whose lower bound exceeds the
// lane's current best (nearest neighbour) or l2 (link, upper triangle of bucket pairs).
// Lower bounds are computed with the same round-to-nearest float32 operations as d6 on the
// per-axis gaps to the box: every step is monotone, so the bound never exceeds the computed
// d6 of any member inside the box, and pruning cannot change the minimum or the set of links.
// Results are therefore bit-identical to the brute-force kernels (and to the definition).
#include "rs_cro.cuh"

namespace rs {
int prune6d_prepare(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m,
                    const double* sums, cudaStream_t st);
int prune6d_nn(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, float* nn2,
               cudaStream_t st);
int prune6d_link(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, const float* nn2,
                 uint32_t* uf, cudaStream_t st);
}  // namespace rs

using namespace rs;

namespace {

constexpr int kT = 256;
constexpr int kWarpsPerBlock = 8;

struct Bucket {
  uint32_t start;    // level-local sorted position of the first member
  uint32_t count;    // 1..32
  uint32_t node;     // global node index
  uint32_t first;    // index of the node's first bucket
  uint32_t last;     // index of the node's last bucket
  uint32_t sbfirst;  // index of the node's first superbucket
  uint32_t sbcount;  // superbuckets of the node
  uint32_t pad;
};

struct Box {
  float4 ulo, uhi, vlo, vhi;
};

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
  // place the 10 bits of x at positions 0, 3, 6, ..., 27
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__device__ __forceinline__ uint32_t quant10(float c) {
  // scaled offset (in units of the node's total position sigma) in [-4, 4) -> 0..1023
  float t = (c + 4.0f) * 128.0f;
  t = fminf(fmaxf(t, 0.0f), 1023.0f);
  return uint32_t(t);
}

// 3D Morton key of each member's position offset from the node mean (scaled by the node's
// sigma_x), prefixed by the node index.
__global__ void k_morton3(int64_t mb, int64_t m, int64_t nb, const uint32_t* __restrict__ mnode,
                          const float4* __restrict__ U, const float4* __restrict__ inv,
                          const float4* __restrict__ mean_u, uint64_t* __restrict__ keys,
                          uint32_t* __restrict__ vals) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const uint32_t q = mnode[mb + p];
  const float sx = sqrtf(inv[q].x);
  const float4 u = U[mb + p], mu = mean_u[q];
  const uint32_t code = spread10(quant10((u.x - mu.x) * sx)) |
                        (spread10(quant10((u.y - mu.y) * sx)) << 1) |
                        (spread10(quant10((u.z - mu.z) * sx)) << 2);
  keys[p] = (uint64_t(q - nb) << 30) | uint64_t(code);
  vals[p] = uint32_t(p);
}

// Node mean positions (float) from the canonical-order moment sums, for the quantisation only.
__global__ void k_node_means(int64_t nb, int64_t nn, const int64_t* __restrict__ node_size,
                             const double* __restrict__ sums, float4* __restrict__ mean_u) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const double g = double(node_size[nb + k]);
  const double* S = sums + 12 * k;
  mean_u[nb + k] = make_float4(float(S[0] / g), float(S[1] / g), float(S[2] / g), 0.f);
}

__global__ void k_gather_sorted(int64_t mb, int64_t m, const uint32_t* __restrict__ order,
                                const float4* __restrict__ U, const float4* __restrict__ V,
                                float4* __restrict__ Us, float4* __restrict__ Vs,
                                uint32_t* __restrict__ sp) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= m) return;
  const uint32_t p = order[s];
  Us[s] = U[mb + p];
  Vs[s] = V[mb + p];
  sp[s] = p;
}

__global__ void k_gather_nn2(int64_t m, const uint32_t* __restrict__ sp, const float* __restrict__ nn2,
                             float* __restrict__ nn2s) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s < m) nn2s[s] = nn2[sp[s]];
}

__global__ void k_bucket_counts(int64_t nb, int64_t nn, const int64_t* __restrict__ node_size,
                                int64_t* __restrict__ bcnt, int64_t* __restrict__ sbcnt) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const int64_t c = (node_size[nb + k] + 31) / 32;
  bcnt[k] = c;
  sbcnt[k] = (c + 31) / 32;
}

__device__ __forceinline__ void warp_box(const float (&a)[6], bool valid, int lo_off, int hi_off,
                                         float (&lo)[6], float (&hi)[6]) {
  const float inf = __int_as_float(0x7f800000);
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    if (lo_off == 1) {
      lo[d] = valid ? a[d] : inf;
      hi[d] = valid ? a[d] : -inf;
    }
#pragma unroll
    for (int off = lo_off; off <= hi_off; off <<= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
    }
  }
}

__device__ __forceinline__ Box make_box(const float (&lo)[6], const float (&hi)[6]) {
  return Box{make_float4(lo[0], lo[1], lo[2], 0.f), make_float4(hi[0], hi[1], hi[2], 0.f),
             make_float4(lo[3], lo[4], lo[5], 0.f), make_float4(hi[3], hi[4], hi[5], 0.f)};
}

// Node size class for the work queue: 8 * floor(log2 g) + the next 3 bits of g (monotone in
// g, 0..254 for g < 2^31), so one 8-bit radix pass orders the buckets largest node first.
__device__ __forceinline__ uint32_t size_class(int64_t g) {
  const int L = 63 - __clzll(uint64_t(g));
  const uint32_t f = L >= 3 ? uint32_t((uint64_t(g) >> (L - 3)) & 7u) : uint32_t((uint64_t(g) << (3 - L)) & 7u);
  return uint32_t(min(L, 31)) * 8u + f > 254u ? 254u : uint32_t(min(L, 31)) * 8u + f;
}

// One warp per bucket (padding warps write a queue key that sorts last): bucket table entry,
// box, four 8-member sub-boxes (an empty sub-bucket gets lo = +inf, hi = -inf, so every gap to
// it is +inf), and the work-queue key (largest node first).
__global__ void __launch_bounds__(kT)
k_buckets(int64_t nb, int64_t nn, int64_t mb, int64_t nbk_ub, const int64_t* __restrict__ bucket_off,
          const int64_t* __restrict__ sb_off, const int64_t* __restrict__ node_off,
          const int64_t* __restrict__ node_size, const float4* __restrict__ Us,
          const float4* __restrict__ Vs, Bucket* __restrict__ bk, Box* __restrict__ box,
          Box* __restrict__ sub, uint64_t* __restrict__ qkey, uint32_t* __restrict__ qval) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nbk_ub) return;
  if (w >= bucket_off[nn]) {
    if (lane == 0) {
      qkey[w] = 255u;  // after every real bucket (their keys are < 255: nodes have >= 2 members)
      qval[w] = uint32_t(w);
    }
    return;
  }
  const int64_t k = rsd::upper_bound_i64(bucket_off, nn, w) - 1;
  const int64_t q = nb + k;
  const int64_t kb = w - bucket_off[k];
  const int64_t start = node_off[q] - mb + 32 * kb;
  const int cnt = int(rsd::min64(32, node_size[q] - 32 * kb));
  const bool valid = lane < cnt;
  const float4 u = Us[start + (valid ? lane : 0)], v = Vs[start + (valid ? lane : 0)];
  const float a[6] = {u.x, u.y, u.z, v.x, v.y, v.z};
  float lo[6], hi[6];
  warp_box(a, valid, 1, 4, lo, hi);
  if ((lane & 7) == 0) sub[4 * w + (lane >> 3)] = make_box(lo, hi);
  warp_box(a, valid, 8, 16, lo, hi);
  if (lane == 0) {
    Bucket b;
    b.start = uint32_t(start);
    b.count = uint32_t(cnt);
    b.node = uint32_t(q);
    b.first = uint32_t(bucket_off[k]);
    b.last = uint32_t(bucket_off[k + 1] - 1);
    b.sbfirst = uint32_t(sb_off[k]);
    b.sbcount = uint32_t(sb_off[k + 1] - sb_off[k]);
    b.pad = 0;
    bk[w] = b;
    box[w] = make_box(lo, hi);
    qkey[w] = 255u - size_class(node_size[q]);
    qval[w] = uint32_t(w);
  }
}

// One warp per superbucket: the box of its (up to 32) bucket boxes.
__global__ void __launch_bounds__(kT)
k_superboxes(int64_t nn, const int64_t* __restrict__ bucket_off, const int64_t* __restrict__ sb_off,
             const Box* __restrict__ box, Box* __restrict__ sbox) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= sb_off[nn]) return;
  const int64_t k = rsd::upper_bound_i64(sb_off, nn, w) - 1;
  const int64_t b0 = bucket_off[k] + 32 * (w - sb_off[k]);
  const int64_t b1 = rsd::min64(b0 + 32, bucket_off[k + 1]);
  const bool valid = b0 + lane < b1;
  const Box B = box[valid ? b0 + lane : b0];
  const float inf = __int_as_float(0x7f800000);
  float lo[6] = {B.ulo.x, B.ulo.y, B.ulo.z, B.vlo.x, B.vlo.y, B.vlo.z};
  float hi[6] = {B.uhi.x, B.uhi.y, B.uhi.z, B.vhi.x, B.vhi.y, B.vhi.z};
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    lo[d] = valid ? lo[d] : inf;
    hi[d] = valid ? hi[d] : -inf;
#pragma unroll
    for (int off = 1; off <= 16; off <<= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
    }
  }
  if (lane == 0) sbox[w] = make_box(lo, hi);
}

// Gap from x to [lo, hi] rounded like the d6 differences (monotone: never above |fl(y - x)| for
// any y in the interval).
__device__ __forceinline__ float gap1(float x, float lo, float hi) {
  return x < lo ? __fsub_rn(lo, x) : (x > hi ? __fsub_rn(x, hi) : 0.f);
}

__device__ __forceinline__ float gap2(float alo, float ahi, float blo, float bhi) {
  return blo > ahi ? __fsub_rn(blo, ahi) : (alo > bhi ? __fsub_rn(alo, bhi) : 0.f);
}

__device__ __forceinline__ float lb_point_box(float4 u, float4 v, const Box& b, float isx, float isv) {
  const float rx = rsd::sq3(gap1(u.x, b.ulo.x, b.uhi.x), gap1(u.y, b.ulo.y, b.uhi.y), gap1(u.z, b.ulo.z, b.uhi.z));
  const float rv = rsd::sq3(gap1(v.x, b.vlo.x, b.vhi.x), gap1(v.y, b.vlo.y, b.vhi.y), gap1(v.z, b.vlo.z, b.vhi.z));
  return __fadd_rn(__fmul_rn(rx, isx), __fmul_rn(rv, isv));
}

__device__ __forceinline__ float lb_box_box(const Box& a, const Box& b, float isx, float isv) {
  const float rx = rsd::sq3(gap2(a.ulo.x, a.uhi.x, b.ulo.x, b.uhi.x), gap2(a.ulo.y, a.uhi.y, b.ulo.y, b.uhi.y),
                            gap2(a.ulo.z, a.uhi.z, b.ulo.z, b.uhi.z));
  const float rv = rsd::sq3(gap2(a.vlo.x, a.vhi.x, b.vlo.x, b.vhi.x), gap2(a.vlo.y, a.vhi.y, b.vlo.y, b.vhi.y),
                            gap2(a.vlo.z, a.vhi.z, b.vlo.z, b.vhi.z));
  return __fadd_rn(__fmul_rn(rx, isx), __fmul_rn(rv, isv));
}

__device__ __forceinline__ float d6(float4 ui, float4 vi, float4 uj, float4 vj, float isx, float isv) {
  const float rx = rsd::sq3(__fsub_rn(uj.x, ui.x), __fsub_rn(uj.y, ui.y), __fsub_rn(uj.z, ui.z));
  const float rv = rsd::sq3(__fsub_rn(vj.x, vi.x), __fsub_rn(vj.y, vi.y), __fsub_rn(vj.z, vi.z));
  return __fadd_rn(__fmul_rn(rx, isx), __fmul_rn(rv, isv));
}

// Index visited at step t of the outward walk from a: a, a+1, a-1, a+2, a-2, ...
__device__ __forceinline__ int64_t outward(int64_t a, int64_t t) {
  const int64_t h = (t + 1) >> 1;
  return (t & 1) ? a + h : a - h;
}

// Next query bucket from the size-ordered queue (one atomic per warp).
__device__ __forceinline__ int64_t next_work(unsigned long long* counter, int lane) {
  unsigned long long w = 0;
  if (lane == 0) w = atomicAdd(counter, 1ull);
  return int64_t(__shfl_sync(0xffffffffu, w, 0));
}

struct NNArgs {
  const int64_t* nbuckets;
  const Bucket* bk;
  const Box* box;
  const Box* sub;
  const Box* sbox;
  const uint32_t* order;
  const float4* Us;
  const float4* Vs;
  const uint32_t* sp;
  const float4* inv;
  unsigned long long* counter;
  unsigned long long* work;  // [4]: NN d6, NN box tests, link d6, link box tests (counting variant)
  const float* nn2s;         // nearest-neighbour d6 in sorted member order (link pass)
};

// Per-lane tallies of the counting variant (evaluated d6 and box tests).
struct Tally {
  unsigned long long d6 = 0, box = 0;
};

// Evaluate target bucket b for the warp's query lanes (nearest-neighbour search).
template <bool kCount>
__device__ __forceinline__ void nn_bucket(const NNArgs& A, int64_t a, int64_t b, bool valid, float4 ui,
                                          float4 vi, float isx, float isv, float& best, int lane,
                                          float4 (&su)[32], float4 (&sv)[32], Tally& T) {
  const Box B = A.box[b];
  const bool need = valid && lb_point_box(ui, vi, B, isx, isv) <= best;
  if (kCount) T.box += valid;
  if (!__any_sync(0xffffffffu, need)) return;
  const Bucket Bb = A.bk[b];
  __syncwarp();
  if (lane < int(Bb.count)) {
    su[lane] = A.Us[Bb.start + lane];
    sv[lane] = A.Vs[Bb.start + lane];
  }
  __syncwarp();
  const uint32_t self = (b == a) ? uint32_t(lane) : 0xffffffffu;
  for (uint32_t s0 = 0; s0 < Bb.count; s0 += 8) {
    const Box Sb = A.sub[4 * b + (s0 >> 3)];
    const bool sneed = need && lb_point_box(ui, vi, Sb, isx, isv) <= best;
    if (kCount) T.box += need;
    if (!__any_sync(0xffffffffu, sneed)) continue;
    if (sneed) {
      const uint32_t s1 = min(s0 + 8, Bb.count);
      if (kCount) T.d6 += s1 - s0;
      for (uint32_t j = s0; j < s1; ++j) {
        if (j == self) continue;
        best = fminf(best, d6(ui, vi, su[j], sv[j], isx, isv));
      }
    }
  }
}

template <bool kCount>
__device__ __forceinline__ void flush_tally(const Tally& T, unsigned long long* work, int lane) {
  if (!kCount) return;
  unsigned long long d = T.d6, b = T.box;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    d += __shfl_xor_sync(0xffffffffu, d, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
  }
  if (lane == 0) {
    atomicAdd(work, d);
    atomicAdd(work + 1, b);
  }
}

template <bool kCount>
__global__ void __launch_bounds__(kT) k_nn6d_pruned(NNArgs A, float* __restrict__ nn2) {
  __shared__ float4 su[kWarpsPerBlock][32], sv[kWarpsPerBlock][32];
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int64_t nbk = *A.nbuckets;
  Tally T;
  while (true) {
    const int64_t w = next_work(A.counter, lane);
    if (w >= nbk) break;
    const int64_t a = A.order[w];
    const Bucket Aq = A.bk[a];
    const float4 iv = A.inv[Aq.node];
    const float isx = iv.x, isv = iv.y;
    const bool valid = lane < int(Aq.count);
    const uint32_t si = Aq.start + (valid ? lane : 0);
    const float4 ui = A.Us[si], vi = A.Vs[si];
    float best = __int_as_float(0x7f800000);
    const int64_t own = (a - int64_t(Aq.first)) >> 5, nsb = Aq.sbcount;
    for (int64_t t = 0; t <= 2 * nsb; ++t) {
      const int64_t s = outward(own, t);
      if (s < 0 || s >= nsb) continue;
      const Box SB = A.sbox[Aq.sbfirst + s];
      const bool need = valid && lb_point_box(ui, vi, SB, isx, isv) <= best;
      if (kCount) T.box += valid;
      if (!__any_sync(0xffffffffu, need)) continue;
      const int64_t b_lo = int64_t(Aq.first) + 32 * s;
      const int64_t b_hi = rsd::min64(b_lo + 32, int64_t(Aq.last) + 1);
      if (s == own) {
        for (int64_t t2 = 0; t2 <= 2 * 32; ++t2) {
          const int64_t b = outward(a, t2);
          if (b < b_lo || b >= b_hi) continue;
          nn_bucket<kCount>(A, a, b, valid, ui, vi, isx, isv, best, lane, su[wb], sv[wb], T);
        }
      } else if (s > own) {
        for (int64_t b = b_lo; b < b_hi; ++b)
          nn_bucket<kCount>(A, a, b, valid, ui, vi, isx, isv, best, lane, su[wb], sv[wb], T);
      } else {
        for (int64_t b = b_hi - 1; b >= b_lo; --b)
          nn_bucket<kCount>(A, a, b, valid, ui, vi, isx, isv, best, lane, su[wb], sv[wb], T);
      }
    }
    if (valid) nn2[A.sp[si]] = best;
  }
  flush_tally<kCount>(T, A.work, lane);
}

// Link pairs of query bucket a (box Abox) with target bucket b >= a.
template <bool kCount>
__device__ __forceinline__ void link_bucket(const NNArgs& A, int64_t a, int64_t b, const Box& Abox,
                                            bool active, float4 ui, float4 vi, uint32_t pi,
                                            float isx, float isv, float l2, const float* nn2,
                                            uint32_t* uf, int lane, float4 (&su)[32],
                                            float4 (&sv)[32], uint32_t (&sj)[32], float (&snn)[32],
                                            Tally& T) {
  const Box B = A.box[b];
  if (kCount) T.box += (lane == 0);
  if (lb_box_box(Abox, B, isx, isv) > l2) return;
  const bool need = active && lb_point_box(ui, vi, B, isx, isv) <= l2;
  if (kCount) T.box += active;
  if (!__any_sync(0xffffffffu, need)) return;
  const Bucket Bb = A.bk[b];
  __syncwarp();
  if (lane < int(Bb.count)) {
    su[lane] = A.Us[Bb.start + lane];
    sv[lane] = A.Vs[Bb.start + lane];
    sj[lane] = A.sp[Bb.start + lane];
    snn[lane] = A.nn2s[Bb.start + lane];
  }
  __syncwarp();
  const uint32_t j0 = (b == a) ? uint32_t(lane) + 1 : 0u;
  for (uint32_t s0 = 0; s0 < Bb.count; s0 += 8) {
    const Box Sb = A.sub[4 * b + (s0 >> 3)];
    if (kCount) T.box += (lane == 0);
    if (lb_box_box(Abox, Sb, isx, isv) > l2) continue;
    const bool sneed = need && lb_point_box(ui, vi, Sb, isx, isv) <= l2;
    if (kCount) T.box += need;
    if (!__any_sync(0xffffffffu, sneed)) continue;
    if (sneed) {
      const uint32_t s1 = min(s0 + 8, Bb.count);
      if (kCount) T.d6 += s1 > max(s0, j0) ? s1 - max(s0, j0) : 0u;
      for (uint32_t j = max(s0, j0); j < s1; ++j) {
        if (snn[j] > l2) continue;
        if (d6(ui, vi, su[j], sv[j], isx, isv) <= l2) rsd::uf_unite(uf, pi, sj[j]);
      }
    }
  }
}

template <bool kCount>
__global__ void __launch_bounds__(kT)
k_link6d_pruned(NNArgs A, const float* __restrict__ nn2, uint32_t* __restrict__ uf) {
  Tally T;
  __shared__ float4 su[kWarpsPerBlock][32], sv[kWarpsPerBlock][32];
  __shared__ uint32_t sj[kWarpsPerBlock][32];
  __shared__ float snn[kWarpsPerBlock][32];
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int64_t nbk = *A.nbuckets;
  while (true) {
    const int64_t w = next_work(A.counter, lane);
    if (w >= nbk) break;
    const int64_t a = A.order[w];
    const Bucket Aq = A.bk[a];
    const float4 iv = A.inv[Aq.node];
    const float isx = iv.x, isv = iv.y, l2 = iv.z;
    const bool valid = lane < int(Aq.count);
    const uint32_t si = Aq.start + (valid ? lane : 0);
    const float4 ui = A.Us[si], vi = A.Vs[si];
    const uint32_t pi = A.sp[si];
    const bool active = valid && A.nn2s[si] <= l2;
    if (!__any_sync(0xffffffffu, active)) continue;
    const Box Abox = A.box[a];
    const int64_t own = (a - int64_t(Aq.first)) >> 5, nsb = Aq.sbcount;
    for (int64_t s = own; s < nsb; ++s) {
      const Box SB = A.sbox[Aq.sbfirst + s];
      if (kCount) T.box += (lane == 0);
      if (lb_box_box(Abox, SB, isx, isv) > l2) continue;
      const bool need = active && lb_point_box(ui, vi, SB, isx, isv) <= l2;
      if (kCount) T.box += active;
      if (!__any_sync(0xffffffffu, need)) continue;
      const int64_t b_lo = rsd::min64(int64_t(Aq.first) + 32 * s, int64_t(Aq.last) + 1);
      const int64_t b_hi = rsd::min64(int64_t(Aq.first) + 32 * s + 32, int64_t(Aq.last) + 1);
      for (int64_t b = (s == own ? a : b_lo); b < b_hi; ++b)
        link_bucket<kCount>(A, a, b, Abox, active, ui, vi, pi, isx, isv, l2, nn2, uf, lane, su[wb], sv[wb],
                            sj[wb], snn[wb], T);
    }
  }
  flush_tally<kCount>(T, A.work + 2, lane);
}

int bits_for(uint64_t v) {
  int b = 1;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

NNArgs nn_args(rs_ctx* ctx, int64_t nn) {
  Hier h = hier_of(ctx);
  NNArgs A;
  A.nbuckets = static_cast<const int64_t*>(ctx->buf[S_P_BOFF].ptr) + nn;
  A.bk = static_cast<const Bucket*>(ctx->buf[S_P_BUCKET].ptr);
  A.box = static_cast<const Box*>(ctx->buf[S_P_BOX].ptr);
  A.sub = static_cast<const Box*>(ctx->buf[S_P_SUB].ptr);
  A.sbox = static_cast<const Box*>(ctx->buf[S_P_SBOX].ptr);
  A.order = static_cast<const uint32_t*>(ctx->buf[S_P_ORDER].ptr);
  A.Us = static_cast<const float4*>(ctx->buf[S_P_US].ptr);
  A.Vs = static_cast<const float4*>(ctx->buf[S_P_VS].ptr);
  A.sp = static_cast<const uint32_t*>(ctx->buf[S_P_SP].ptr);
  A.inv = h.inv;
  A.counter = static_cast<unsigned long long*>(ctx->buf[S_P_QCTR].ptr);
  A.work = static_cast<unsigned long long*>(ctx->buf[S_P_WORK].ptr);
  A.nn2s = nullptr;
  return A;
}

}  // namespace

int rs::prune6d_prepare(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m,
                        const double* sums, cudaStream_t st) {
  Hier h = hier_of(ctx);
  float4* mean_u = scratch_t<float4>(ctx, S_P_MEANU, size_t(nb + nn));
  uint64_t* ka = scratch_t<uint64_t>(ctx, S_KEY_A, size_t(m));
  uint64_t* kb = scratch_t<uint64_t>(ctx, S_KEY_B, size_t(m));
  uint32_t* va = scratch_t<uint32_t>(ctx, S_VAL_A, size_t(m));
  uint32_t* vb = scratch_t<uint32_t>(ctx, S_VAL_B, size_t(m));
  float4* Us = scratch_t<float4>(ctx, S_P_US, size_t(m));
  float4* Vs = scratch_t<float4>(ctx, S_P_VS, size_t(m));
  uint32_t* sp = scratch_t<uint32_t>(ctx, S_P_SP, size_t(m));
  int64_t* boff = scratch_t<int64_t>(ctx, S_P_BOFF, size_t(nn) + 1);
  int64_t* sboff = scratch_t<int64_t>(ctx, S_P_SBOFF, size_t(nn) + 1);
  const int64_t nbk_ub = nn + m / 32 + 1;
  const int64_t nsb_ub = nn + nbk_ub / 32 + 1;
  Bucket* bk = scratch_t<Bucket>(ctx, S_P_BUCKET, size_t(nbk_ub));
  Box* box = scratch_t<Box>(ctx, S_P_BOX, size_t(nbk_ub));
  Box* sub = scratch_t<Box>(ctx, S_P_SUB, size_t(nbk_ub) * 4);
  Box* sbox = scratch_t<Box>(ctx, S_P_SBOX, size_t(nsb_ub));
  unsigned long long* qctr = scratch_t<unsigned long long>(ctx, S_P_QCTR, 2);
  if (!scratch_t<unsigned long long>(ctx, S_P_WORK, 4)) return RS_ERR_OOM;
  if (!mean_u || !ka || !kb || !va || !vb || !Us || !Vs || !sp || !boff || !sboff || !bk || !box ||
      !sub || !sbox || !qctr)
    return RS_ERR_OOM;
  k_node_means<<<grid_for(nn, kT), kT, 0, st>>>(nb, nn, h.node_size, sums, mean_u);
  RS_LAUNCHED(ctx, "k_node_means");
  k_morton3<<<grid_for(m, kT), kT, 0, st>>>(mb, m, nb, h.mnode, h.U, h.inv, mean_u, ka, va);
  RS_LAUNCHED(ctx, "k_morton3");
  uint64_t* keys;
  uint32_t* order;
  RS_TRY(radix_sort_u64(ctx, m, 30 + bits_for(uint64_t(nn)), ka, va, kb, vb, &keys, &order, st));
  k_gather_sorted<<<grid_for(m, kT), kT, 0, st>>>(mb, m, order, h.U, h.V, Us, Vs, sp);
  RS_LAUNCHED(ctx, "k_gather_sorted");
  k_bucket_counts<<<grid_for(nn, kT), kT, 0, st>>>(nb, nn, h.node_size, boff, sboff);
  RS_LAUNCHED(ctx, "k_bucket_counts");
  RS_TRY(exclusive_scan_i64(ctx, nn, boff, boff + nn, st));
  RS_TRY(exclusive_scan_i64(ctx, nn, sboff, sboff + nn, st));
  // bucket tables and the work queue (keys/values reuse the sort buffers: m >= buckets)
  uint64_t* qk = scratch_t<uint64_t>(ctx, S_KEY_A, size_t(std::max(m, nbk_ub)));
  uint64_t* qk2 = scratch_t<uint64_t>(ctx, S_KEY_B, size_t(std::max(m, nbk_ub)));
  uint32_t* qv = scratch_t<uint32_t>(ctx, S_VAL_A, size_t(std::max(m, nbk_ub)));
  uint32_t* qv2 = scratch_t<uint32_t>(ctx, S_VAL_B, size_t(std::max(m, nbk_ub)));
  if (!qk || !qk2 || !qv || !qv2) return RS_ERR_OOM;
  k_buckets<<<grid_for(nbk_ub * 32, kT), kT, 0, st>>>(nb, nn, mb, nbk_ub, boff, sboff, h.node_off,
                                                     h.node_size, Us, Vs, bk, box, sub, qk, qv);
  RS_LAUNCHED(ctx, "k_buckets");
  k_superboxes<<<grid_for(nsb_ub * 32, kT), kT, 0, st>>>(nn, boff, sboff, box, sbox);
  RS_LAUNCHED(ctx, "k_superboxes");
  uint64_t* qk_out;
  uint32_t* qv_out;
  RS_TRY(radix_sort_u64(ctx, nbk_ub, 8, qk, qv, qk2, qv2, &qk_out, &qv_out, st));
  uint32_t* qorder = scratch_t<uint32_t>(ctx, S_P_ORDER, size_t(nbk_ub));
  if (!qorder) return RS_ERR_OOM;
  RS_CUDA(ctx, cudaMemcpyAsync(qorder, qv_out, sizeof(uint32_t) * nbk_ub, cudaMemcpyDeviceToDevice, st));
  return RS_OK;
}

int rs::prune6d_nn(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, float* nn2,
                   cudaStream_t st) {
  (void)nb;
  (void)mb;
  NNArgs A = nn_args(ctx, nn);
  const int64_t nbk_ub = nn + m / 32 + 1;
  const unsigned grid = unsigned(std::min<int64_t>((nbk_ub + kWarpsPerBlock - 1) / kWarpsPerBlock, 152 * 8));
  RS_CUDA(ctx, cudaMemsetAsync(A.counter, 0, sizeof(unsigned long long), st));
  if (ctx->count_work) {
    k_nn6d_pruned<true><<<grid, kT, 0, st>>>(A, nn2);
  } else {
    ProfScope prof_(ctx, "k_nn6d_pruned", st);
    k_nn6d_pruned<false><<<grid, kT, 0, st>>>(A, nn2);
  }
  RS_LAUNCHED(ctx, "k_nn6d_pruned");
  return RS_OK;
}

int rs::prune6d_link(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, const float* nn2,
                     uint32_t* uf, cudaStream_t st) {
  (void)nb;
  (void)mb;
  NNArgs A = nn_args(ctx, nn);
  A.counter += 1;
  float* nn2s = scratch_t<float>(ctx, S_P_NN2S, size_t(std::max<int64_t>(m, 1)));
  if (!nn2s) return RS_ERR_OOM;
  k_gather_nn2<<<grid_for(m, kT), kT, 0, st>>>(m, A.sp, nn2, nn2s);
  RS_LAUNCHED(ctx, "k_gather_nn2");
  A.nn2s = nn2s;
  const int64_t nbk_ub = nn + m / 32 + 1;
  const unsigned grid = unsigned(std::min<int64_t>((nbk_ub + kWarpsPerBlock - 1) / kWarpsPerBlock, 152 * 8));
  RS_CUDA(ctx, cudaMemsetAsync(A.counter, 0, sizeof(unsigned long long), st));
  if (ctx->count_work) {
    k_link6d_pruned<true><<<grid, kT, 0, st>>>(A, nn2, uf);
  } else {
    ProfScope prof_(ctx, "k_link6d_pruned", st);
    k_link6d_pruned<false><<<grid, kT, 0, st>>>(A, nn2, uf);
  }
  RS_LAUNCHED(ctx, "k_link6d_pruned");
  return RS_OK;
}

// Pruned 6D nearest-neighbour and link searches for the batched form of rs_fof6d.
//
// The plain form evaluates d6 for every pair of a node. Here the members of every node of a
// level are ordered by a 3D Morton key of their scaled position offsets, cut into buckets of 32
// consecutive members, and each bucket gets its 6D bounding box. A warp takes one query bucket
// (lane = member) and visits the node's buckets outward from its own in key order:
//   nearest neighbour: a bucket is skipped for a lane when the box lower bound exceeds the
//     lane's current best; otherwise all its members are evaluated;
//   link: a bucket pair is skipped when the box-to-box lower bound exceeds l2.
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
  uint32_t start;  // level-local sorted position of the first member
  uint32_t count;  // 1..32
  uint32_t node;   // global node index
  uint32_t first;  // index of the node's first bucket
  uint32_t last;   // index of the node's last bucket
  uint32_t pad[3];
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
// sigma_x), prefixed by the node index. Position-only ordering gives spatially tight buckets:
// every candidate of a 6D search lies within sqrt(bound / inv_sx2) in position.
__global__ void k_morton6(int64_t mb, int64_t m, int64_t nb, int nodebits,
                          const uint32_t* __restrict__ mnode, const float4* __restrict__ U,
                          const float4* __restrict__ V, const float4* __restrict__ inv,
                          const float4* __restrict__ mean_u, const float4* __restrict__ mean_v,
                          uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
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
  (void)nodebits;
  (void)V;
  (void)mean_v;
}

// Node means (float) from the CRO moment sums, for the Morton quantisation only.
__global__ void k_node_means(int64_t nb, int64_t nn, const int64_t* __restrict__ node_size,
                             const double* __restrict__ sums, float4* __restrict__ mean_u,
                             float4* __restrict__ mean_v) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const double g = double(node_size[nb + k]);
  const double* S = sums + 12 * k;
  mean_u[nb + k] = make_float4(float(S[0] / g), float(S[1] / g), float(S[2] / g), 0.f);
  mean_v[nb + k] = make_float4(float(S[6] / g), float(S[7] / g), float(S[8] / g), 0.f);
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

__global__ void k_bucket_counts(int64_t nb, int64_t nn, const int64_t* __restrict__ node_size,
                                int64_t* __restrict__ out) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < nn) out[k] = (node_size[nb + k] + 31) / 32;
}

// One warp per bucket: its table entry and its 6D bounding box.
__global__ void __launch_bounds__(kT)
k_buckets(int64_t nb, int64_t nn, int64_t mb, const int64_t* __restrict__ bucket_off,
          const int64_t* __restrict__ node_off, const int64_t* __restrict__ node_size,
          const float4* __restrict__ Us, const float4* __restrict__ Vs, Bucket* __restrict__ bk,
          Box* __restrict__ box) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= bucket_off[nn]) return;
  const int64_t k = rsd::upper_bound_i64(bucket_off, nn, w) - 1;
  const int64_t q = nb + k;
  const int64_t kb = w - bucket_off[k];
  const int64_t start = node_off[q] - mb + 32 * kb;
  const int cnt = int(rsd::min64(32, node_size[q] - 32 * kb));
  const bool valid = lane < cnt;
  const float4 u = Us[start + (valid ? lane : 0)], v = Vs[start + (valid ? lane : 0)];
  float a[6] = {u.x, u.y, u.z, v.x, v.y, v.z};
  float lo[6], hi[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    lo[d] = a[d];
    hi[d] = a[d];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
    }
  }
  if (lane == 0) {
    Bucket b;
    b.start = uint32_t(start);
    b.count = uint32_t(cnt);
    b.node = uint32_t(q);
    b.first = uint32_t(bucket_off[k]);
    b.last = uint32_t(bucket_off[k + 1] - 1);
    b.pad[0] = b.pad[1] = b.pad[2] = 0;
    bk[w] = b;
    box[w] = Box{make_float4(lo[0], lo[1], lo[2], 0.f), make_float4(hi[0], hi[1], hi[2], 0.f),
                 make_float4(lo[3], lo[4], lo[5], 0.f), make_float4(hi[3], hi[4], hi[5], 0.f)};
  }
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

// Bucket visited at step t of the outward walk from bucket a within [first, last]:
// a, a+1, a-1, a+2, a-2, ... (indices outside the range are skipped by the caller).
__device__ __forceinline__ int64_t outward(int64_t a, int64_t t) {
  const int64_t h = (t + 1) >> 1;
  return (t & 1) ? a + h : a - h;
}

__global__ void __launch_bounds__(kT)
k_nn6d_pruned(const int64_t* __restrict__ nbuckets_dev, const Bucket* __restrict__ bk,
              const Box* __restrict__ box, const float4* __restrict__ Us,
              const float4* __restrict__ Vs, const uint32_t* __restrict__ sp,
              const float4* __restrict__ inv, float* __restrict__ nn2) {
  __shared__ float4 su[kWarpsPerBlock][32], sv[kWarpsPerBlock][32];
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int64_t nbk = *nbuckets_dev;
  const int64_t stride = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t a = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; a < nbk; a += stride) {
    const Bucket A = bk[a];
    const float4 iv = inv[A.node];
    const float isx = iv.x, isv = iv.y;
    const bool valid = lane < int(A.count);
    const uint32_t si = A.start + (valid ? lane : 0);
    const float4 ui = Us[si], vi = Vs[si];
    float best = __int_as_float(0x7f800000);
    const int64_t span = int64_t(A.last) - int64_t(A.first);
    for (int64_t t = 0; t <= 2 * span; ++t) {
      const int64_t b = outward(a, t);
      if (b < int64_t(A.first) || b > int64_t(A.last)) continue;
      const Box B = box[b];
      const bool need = valid && lb_point_box(ui, vi, B, isx, isv) <= best;
      if (!__any_sync(0xffffffffu, need)) continue;
      const Bucket Bb = bk[b];
      __syncwarp();
      if (lane < int(Bb.count)) {
        su[wb][lane] = Us[Bb.start + lane];
        sv[wb][lane] = Vs[Bb.start + lane];
      }
      __syncwarp();
      if (need) {
        const uint32_t self = (b == a) ? uint32_t(lane) : 0xffffffffu;
        for (uint32_t j = 0; j < Bb.count; ++j) {
          if (j == self) continue;
          best = fminf(best, d6(ui, vi, su[wb][j], sv[wb][j], isx, isv));
        }
      }
    }
    if (valid) nn2[sp[si]] = best;
  }
}

__global__ void __launch_bounds__(kT)
k_link6d_pruned(const int64_t* __restrict__ nbuckets_dev, const Bucket* __restrict__ bk,
                const Box* __restrict__ box, const float4* __restrict__ Us,
                const float4* __restrict__ Vs, const uint32_t* __restrict__ sp,
                const float4* __restrict__ inv, const float* __restrict__ nn2,
                uint32_t* __restrict__ uf) {
  __shared__ float4 su[kWarpsPerBlock][32], sv[kWarpsPerBlock][32];
  __shared__ uint32_t sj[kWarpsPerBlock][32];
  __shared__ float snn[kWarpsPerBlock][32];
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int64_t nbk = *nbuckets_dev;
  const int64_t stride = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t a = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; a < nbk; a += stride) {
    const Bucket A = bk[a];
    const float4 iv = inv[A.node];
    const float isx = iv.x, isv = iv.y, l2 = iv.z;
    const bool valid = lane < int(A.count);
    const uint32_t si = A.start + (valid ? lane : 0);
    const float4 ui = Us[si], vi = Vs[si];
    const uint32_t pi = sp[si];
    const bool active = valid && nn2[pi] <= l2;
    if (!__any_sync(0xffffffffu, active)) continue;
    const Box Abox = box[a];
    for (int64_t b = a; b <= int64_t(A.last); ++b) {
      const Box B = box[b];
      if (lb_box_box(Abox, B, isx, isv) > l2) continue;
      const bool need = active && lb_point_box(ui, vi, B, isx, isv) <= l2;
      if (!__any_sync(0xffffffffu, need)) continue;
      const Bucket Bb = bk[b];
      __syncwarp();
      if (lane < int(Bb.count)) {
        su[wb][lane] = Us[Bb.start + lane];
        sv[wb][lane] = Vs[Bb.start + lane];
        sj[wb][lane] = sp[Bb.start + lane];
        snn[wb][lane] = nn2[sp[Bb.start + lane]];
      }
      __syncwarp();
      if (need) {
        const uint32_t j0 = (b == a) ? uint32_t(lane) + 1 : 0u;
        for (uint32_t j = j0; j < Bb.count; ++j) {
          if (snn[wb][j] > l2) continue;
          if (d6(ui, vi, su[wb][j], sv[wb][j], isx, isv) <= l2) rsd::uf_unite(uf, pi, sj[wb][j]);
        }
      }
    }
  }
}

int bits_for(uint64_t v) {
  int b = 1;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

}  // namespace

int rs::prune6d_prepare(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m,
                        const double* sums, cudaStream_t st) {
  Hier h = hier_of(ctx);
  float4* mean_u = scratch_t<float4>(ctx, S_P_MEANU, size_t(nb + nn));
  float4* mean_v = scratch_t<float4>(ctx, S_P_MEANV, size_t(nb + nn));
  uint64_t* ka = scratch_t<uint64_t>(ctx, S_KEY_A, size_t(m));
  uint64_t* kb = scratch_t<uint64_t>(ctx, S_KEY_B, size_t(m));
  uint32_t* va = scratch_t<uint32_t>(ctx, S_VAL_A, size_t(m));
  uint32_t* vb = scratch_t<uint32_t>(ctx, S_VAL_B, size_t(m));
  float4* Us = scratch_t<float4>(ctx, S_P_US, size_t(m));
  float4* Vs = scratch_t<float4>(ctx, S_P_VS, size_t(m));
  uint32_t* sp = scratch_t<uint32_t>(ctx, S_P_SP, size_t(m));
  int64_t* boff = scratch_t<int64_t>(ctx, S_P_BOFF, size_t(nn) + 1);
  const int64_t nbk_ub = nn + m / 32 + 1;
  Bucket* bk = scratch_t<Bucket>(ctx, S_P_BUCKET, size_t(nbk_ub));
  Box* box = scratch_t<Box>(ctx, S_P_BOX, size_t(nbk_ub));
  if (!mean_u || !mean_v || !ka || !kb || !va || !vb || !Us || !Vs || !sp || !boff || !bk || !box)
    return RS_ERR_OOM;
  k_node_means<<<grid_for(nn, kT), kT, 0, st>>>(nb, nn, h.node_size, sums, mean_u, mean_v);
  RS_LAUNCHED(ctx, "k_node_means");
  k_morton6<<<grid_for(m, kT), kT, 0, st>>>(mb, m, nb, 0, h.mnode, h.U, h.V, h.inv, mean_u, mean_v, ka, va);
  RS_LAUNCHED(ctx, "k_morton6");
  uint64_t* keys;
  uint32_t* order;
  RS_TRY(radix_sort_u64(ctx, m, 30 + bits_for(uint64_t(nn)), ka, va, kb, vb, &keys, &order, st));
  k_gather_sorted<<<grid_for(m, kT), kT, 0, st>>>(mb, m, order, h.U, h.V, Us, Vs, sp);
  RS_LAUNCHED(ctx, "k_gather_sorted");
  k_bucket_counts<<<grid_for(nn, kT), kT, 0, st>>>(nb, nn, h.node_size, boff);
  RS_LAUNCHED(ctx, "k_bucket_counts");
  RS_TRY(exclusive_scan_i64(ctx, nn, boff, boff + nn, st));
  k_buckets<<<grid_for(nbk_ub * 32, kT), kT, 0, st>>>(nb, nn, mb, boff, h.node_off, h.node_size, Us, Vs,
                                                     bk, box);
  RS_LAUNCHED(ctx, "k_buckets");
  return RS_OK;
}

int rs::prune6d_nn(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, float* nn2,
                   cudaStream_t st) {
  (void)nb;
  (void)mb;
  Hier h = hier_of(ctx);
  const int64_t* boff = static_cast<const int64_t*>(ctx->buf[S_P_BOFF].ptr);
  const Bucket* bk = static_cast<const Bucket*>(ctx->buf[S_P_BUCKET].ptr);
  const Box* box = static_cast<const Box*>(ctx->buf[S_P_BOX].ptr);
  const float4* Us = static_cast<const float4*>(ctx->buf[S_P_US].ptr);
  const float4* Vs = static_cast<const float4*>(ctx->buf[S_P_VS].ptr);
  const uint32_t* sp = static_cast<const uint32_t*>(ctx->buf[S_P_SP].ptr);
  const int64_t nbk_ub = nn + m / 32 + 1;
  const unsigned grid = unsigned(std::min<int64_t>((nbk_ub + kWarpsPerBlock - 1) / kWarpsPerBlock, 152 * 16));
  {
    ProfScope prof_(ctx, "k_nn6d_pruned", st);
    k_nn6d_pruned<<<grid, kT, 0, st>>>(boff + nn, bk, box, Us, Vs, sp, h.inv, nn2);
  }
  RS_LAUNCHED(ctx, "k_nn6d_pruned");
  return RS_OK;
}

int rs::prune6d_link(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, const float* nn2,
                     uint32_t* uf, cudaStream_t st) {
  (void)nb;
  (void)mb;
  Hier h = hier_of(ctx);
  const int64_t* boff = static_cast<const int64_t*>(ctx->buf[S_P_BOFF].ptr);
  const Bucket* bk = static_cast<const Bucket*>(ctx->buf[S_P_BUCKET].ptr);
  const Box* box = static_cast<const Box*>(ctx->buf[S_P_BOX].ptr);
  const float4* Us = static_cast<const float4*>(ctx->buf[S_P_US].ptr);
  const float4* Vs = static_cast<const float4*>(ctx->buf[S_P_VS].ptr);
  const uint32_t* sp = static_cast<const uint32_t*>(ctx->buf[S_P_SP].ptr);
  const int64_t nbk_ub = nn + m / 32 + 1;
  const unsigned grid = unsigned(std::min<int64_t>((nbk_ub + kWarpsPerBlock - 1) / kWarpsPerBlock, 152 * 16));
  {
    ProfScope prof_(ctx, "k_link6d_pruned", st);
    k_link6d_pruned<<<grid, kT, 0, st>>>(boff + nn, bk, box, Us, Vs, sp, h.inv, nn2, uf);
  }
  RS_LAUNCHED(ctx, "k_link6d_pruned");
  return RS_OK;
}

// Pruned 6D nearest-neighbour and link searches for the batched form of rs_fof6d.
//
// The plain form evaluates d6 for every pair of a node. Here the members of every node of a
// level are ordered by a 3D Hilbert key of their scaled position offsets (every candidate of a
// 6D search lies within sqrt(bound / inv_sx2) in position) and cut into buckets of 32
// consecutive members; each bucket has a 6D bounding box, four 8-member sub-boxes, and every
// 32 consecutive buckets of a node form a superbucket with its own box. Persistent warps pull
// query buckets from a queue ordered by node size (largest first) and, lane = member, visit
// the node's superbuckets, buckets and sub-buckets, skipping any whose lower bound exceeds the
// lane's current best (nearest neighbour) or l2 (link, upper triangle of bucket pairs). The
// link pass runs on the members with a friend only (nn2 <= l2: no other member can be linked),
// compacted in the same order and bucketed again, so its boxes are tighter and no lane idles.
// Nodes of 4096 members or more search their nearest neighbours within bounds of l2 taken
// from an exactly searched sample (see k_sample_bounds; a device check re-searches any node
// whose l2 falls outside them). Distances and bounds use packed float32x2 arithmetic with each
// half rounded like the scalar operation. Lower bounds are computed with the same
// round-to-nearest float32 operations as d6 on the per-axis gaps to the box: every step is
// monotone, so the bound never exceeds the computed d6 of any member inside the box, and
// pruning cannot change the minimum or the set of links. Results are therefore bit-identical
// to the brute-force kernels (and to the definition).
#include "rs_cro.cuh"

namespace rs {
int prune6d_prepare(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m,
                    const double* sums, cudaStream_t st);
int prune6d_nn(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, float* nn2,
               cudaStream_t st);
int prune6d_check(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t m, float* nn2, const int** failed_out,
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

// 6D box, stored for the packed float32x2 bounds: (position, velocity) pairs per axis, the
// lower corner and the NEGATED upper corner (so both gaps are additions).
struct Box {
  float4 lo01;   // (x, vx, y, vy)
  float4 nhi01;  // -(x, vx, y, vy) of the upper corner
  float2 lo2;    // (z, vz)
  float2 nhi2;
};

__device__ __forceinline__ uint32_t quant8(float c) {
  // scaled offset (in units of the node's total position sigma) in [-4, 4) -> 0..255
  float t = (c + 4.0f) * 32.0f;
  t = fminf(fmaxf(t, 0.0f), 255.0f);
  return uint32_t(t);
}

// 3D Hilbert key of each member's position offset from the node mean (scaled by the node's
// sigma_x), prefixed by the node index.
__global__ void k_hilbert3(int64_t mb, int64_t m, int64_t nb, const uint32_t* __restrict__ mnode,
                          const float4* __restrict__ U, const float4* __restrict__ inv,
                          const float4* __restrict__ mean_u, uint64_t* __restrict__ keys,
                          uint32_t* __restrict__ vals) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const uint32_t q = mnode[mb + p];
  const float sx = sqrtf(inv[q].x);
  const float4 u = U[mb + p], mu = mean_u[q];
  const uint32_t code = rsd::hilbert3<8>(quant8((u.x - mu.x) * sx), quant8((u.y - mu.y) * sx),
                                   quant8((u.z - mu.z) * sx));
  keys[p] = (uint64_t(q - nb) << 24) | uint64_t(code);
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

// Members of each node of the level in the bucketed arrays: start (level-local sorted
// position) and count; all members for the NN pass, the members with a friend for the link pass.
__global__ void k_node_ranges(int64_t nb, int64_t nn, int64_t mb, const int64_t* __restrict__ node_off,
                              const int64_t* __restrict__ node_size, int64_t* __restrict__ start,
                              int64_t* __restrict__ cnt) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  start[k] = node_off[nb + k] - mb;
  cnt[k] = node_size[nb + k];
}

__global__ void k_bucket_counts(int64_t nn, const int64_t* __restrict__ cnt, int64_t* __restrict__ bcnt,
                                int64_t* __restrict__ sbcnt) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const int64_t c = (cnt[k] + 31) / 32;
  bcnt[k] = c;
  sbcnt[k] = (c + 31) / 32;
}

// Link pass: the members with a friend (nn2 <= l2 of their node), compacted in sorted order.
__global__ void k_active_flags(int64_t m, int64_t mb, const uint32_t* __restrict__ sp,
                               const uint32_t* __restrict__ mnode, const float4* __restrict__ inv,
                               const float* __restrict__ nn2, int64_t* __restrict__ flag) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= m) return;
  const uint32_t p = sp[s];
  flag[s] = nn2[p] <= inv[mnode[mb + p]].z ? 1 : 0;
}

__global__ void k_compact_active(int64_t m, const int64_t* __restrict__ pos, const float4* __restrict__ Us,
                                 const float4* __restrict__ Vs, const uint32_t* __restrict__ sp,
                                 float4* __restrict__ UsA, float4* __restrict__ VsA,
                                 uint32_t* __restrict__ spA) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= m || pos[s + 1] == pos[s]) return;
  const int64_t a = pos[s];
  UsA[a] = Us[s];
  VsA[a] = Vs[s];
  spA[a] = sp[s];
}

__global__ void k_active_ranges(int64_t nb, int64_t nn, int64_t mb, const int64_t* __restrict__ node_off,
                                const int64_t* __restrict__ node_size, const int64_t* __restrict__ pos,
                                int64_t* __restrict__ start, int64_t* __restrict__ cnt) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const int64_t s0 = node_off[nb + k] - mb;
  start[k] = pos[s0];
  cnt[k] = pos[s0 + node_size[nb + k]] - pos[s0];
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

// lo, hi indexed (x, y, z, vx, vy, vz).
__device__ __forceinline__ Box make_box(const float (&lo)[6], const float (&hi)[6]) {
  return Box{make_float4(lo[0], lo[3], lo[1], lo[4]), make_float4(-hi[0], -hi[3], -hi[1], -hi[4]),
             make_float2(lo[2], lo[5]), make_float2(-hi[2], -hi[5])};
}

// One warp per bucket (padding warps write a queue key that sorts last): bucket table entry,
// box, four 8-member sub-boxes (an empty sub-bucket gets lo = +inf, hi = -inf, so every gap to
// it is +inf), and the work-queue key (largest node first).
__global__ void __launch_bounds__(kT)
k_buckets(int64_t nb, int64_t nn, int64_t nbk_ub, const int64_t* __restrict__ bucket_off,
          const int64_t* __restrict__ sb_off, const int64_t* __restrict__ nstart,
          const int64_t* __restrict__ ncnt, const float4* __restrict__ Us,
          const float4* __restrict__ Vs, Bucket* __restrict__ bk, Box* __restrict__ box,
          Box* __restrict__ sub, uint64_t* __restrict__ qkey, uint32_t* __restrict__ qval) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nbk_ub) return;
  if (w >= bucket_off[nn]) {
    if (lane == 0) {
      qkey[w] = 255u;  // the largest key: after every real bucket (stable sort, higher indices)
      qval[w] = uint32_t(w);
    }
    return;
  }
  const int64_t k = rsd::upper_bound_i64(bucket_off, nn, w) - 1;
  const int64_t q = nb + k;
  const int64_t kb = w - bucket_off[k];
  const int64_t start = nstart[k] + 32 * kb;
  const int cnt = int(rsd::min64(32, ncnt[k] - 32 * kb));
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
    qkey[w] = 255u - rsd::size_class(ncnt[k]);
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
  float lo[6] = {B.lo01.x, B.lo01.z, B.lo2.x, B.lo01.y, B.lo01.w, B.lo2.y};
  float hi[6] = {-B.nhi01.x, -B.nhi01.z, -B.nhi2.x, -B.nhi01.y, -B.nhi01.w, -B.nhi2.y};
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

// Packed float32x2 add and multiply, each half rounded exactly like __fadd_rn / __fmul_rn. The
// float2 intrinsics let the compiler fuse a multiply into a following add (an FMA: one rounding
// instead of two, which changes d6 in the last bit); inline PTX with the product taken as an
// fma with a +0 addend keeps every rounding (fl(a b + 0) = fl(a b) for the non-negative
// products used here).
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rz, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rz, 0;\n\tfma.rn.f32x2 rd, ra, rb, rz;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// A query lane's coordinates, packed for the float32x2 arithmetic: (position, velocity)
// pairs per axis and their negations for the box bounds; each coordinate negated and
// duplicated for the distances to two targets at once; the metric scales.
struct Query {
  float2 qa, qb, qc, na, nb, nc;
  float2 nux, nuy, nuz, nvx, nvy, nvz;
  float2 s;         // (inv_sx2, inv_sv2)
  float2 sx2, sv2;  // (inv_sx2, inv_sx2), (inv_sv2, inv_sv2)
};

__device__ __forceinline__ Query make_query(float4 u, float4 v, float isx, float isv) {
  Query Q;
  Q.qa = make_float2(u.x, v.x);
  Q.qb = make_float2(u.y, v.y);
  Q.qc = make_float2(u.z, v.z);
  Q.na = make_float2(-u.x, -v.x);
  Q.nb = make_float2(-u.y, -v.y);
  Q.nc = make_float2(-u.z, -v.z);
  Q.nux = make_float2(-u.x, -u.x);
  Q.nuy = make_float2(-u.y, -u.y);
  Q.nuz = make_float2(-u.z, -u.z);
  Q.nvx = make_float2(-v.x, -v.x);
  Q.nvy = make_float2(-v.y, -v.y);
  Q.nvz = make_float2(-v.z, -v.z);
  Q.s = make_float2(isx, isv);
  Q.sx2 = make_float2(isx, isx);
  Q.sv2 = make_float2(isv, isv);
  return Q;
}

__device__ __forceinline__ float2 max0(float2 a, float2 b) {
  return make_float2(fmaxf(fmaxf(a.x, b.x), 0.f), fmaxf(fmaxf(a.y, b.y), 0.f));
}

// Per-axis gap from q to [lo, hi]: max(fl(lo - q), fl(q - hi), 0). When q < lo this is
// fl(lo - q) (the other difference is negative), when q > hi it is fl(q - hi), otherwise 0:
// rounded like the d6 differences, hence never above |fl(y - q)| for any y in the interval.
__device__ __forceinline__ float2 gap_pt(float2 lo, float2 nhi, float2 q, float2 nq) {
  return max0(padd(lo, nq), padd(q, nhi));
}

// Gap between two intervals: max(fl(blo - ahi), fl(alo - bhi), 0).
__device__ __forceinline__ float2 gap_bb(float2 alo, float2 anhi, float2 blo, float2 bnhi) {
  return max0(padd(blo, anhi), padd(alo, bnhi));
}

// fl(fl(rx * inv_sx2) + fl(rv * inv_sv2)) with (rx, rv) = ((ga^2 + gb^2) + gc^2) per half:
// the operation order of d6.
__device__ __forceinline__ float metric(float2 ga, float2 gb, float2 gc, float2 s) {
  const float2 r = padd(padd(pmul(ga, ga), pmul(gb, gb)), pmul(gc, gc));
  const float2 t = pmul(r, s);
  return __fadd_rn(t.x, t.y);
}

__device__ __forceinline__ float lb_point_box(const Query& Q, const Box& b) {
  return metric(gap_pt(make_float2(b.lo01.x, b.lo01.y), make_float2(b.nhi01.x, b.nhi01.y), Q.qa, Q.na),
                gap_pt(make_float2(b.lo01.z, b.lo01.w), make_float2(b.nhi01.z, b.nhi01.w), Q.qb, Q.nb),
                gap_pt(b.lo2, b.nhi2, Q.qc, Q.nc), Q.s);
}

__device__ __forceinline__ float lb_box_box(const Box& a, const Box& b, float2 s) {
  return metric(gap_bb(make_float2(a.lo01.x, a.lo01.y), make_float2(a.nhi01.x, a.nhi01.y),
                       make_float2(b.lo01.x, b.lo01.y), make_float2(b.nhi01.x, b.nhi01.y)),
                gap_bb(make_float2(a.lo01.z, a.lo01.w), make_float2(a.nhi01.z, a.nhi01.w),
                       make_float2(b.lo01.z, b.lo01.w), make_float2(b.nhi01.z, b.nhi01.w)),
                gap_bb(a.lo2, a.nhi2, b.lo2, b.nhi2), s);
}

// Staged targets of one warp, structure of arrays (x, y, z, vx, vy, vz); slots past the
// bucket's count hold NaN, whose distance is NaN: it lowers no minimum and passes no test.
struct __align__(16) Stage {  // 16-byte aligned: pairs of slots load as float2
  float c[6][32];
};

// d6 of the query to targets j and j + 1 (j even): fl(fl(rx * isx) + fl(rv * isv)) with
// rx = (dx^2 + dy^2) + dz^2, d = fl(u_j - u_i) formed as u_j + (-u_i), every operation rounded
// separately; each half equals the scalar d6.
__device__ __forceinline__ float2 d6_pair(const Query& Q, const Stage& S, int j) {
  const float2 dx = padd(*reinterpret_cast<const float2*>(&S.c[0][j]), Q.nux);
  const float2 dy = padd(*reinterpret_cast<const float2*>(&S.c[1][j]), Q.nuy);
  const float2 dz = padd(*reinterpret_cast<const float2*>(&S.c[2][j]), Q.nuz);
  const float2 ex = padd(*reinterpret_cast<const float2*>(&S.c[3][j]), Q.nvx);
  const float2 ey = padd(*reinterpret_cast<const float2*>(&S.c[4][j]), Q.nvy);
  const float2 ez = padd(*reinterpret_cast<const float2*>(&S.c[5][j]), Q.nvz);
  const float2 rx = padd(padd(pmul(dx, dx), pmul(dy, dy)), pmul(dz, dz));
  const float2 rv = padd(padd(pmul(ex, ex), pmul(ey, ey)), pmul(ez, ez));
  return padd(pmul(rx, Q.sx2), pmul(rv, Q.sv2));
}

__device__ __forceinline__ void stage(Stage& S, const float4* __restrict__ Us, const float4* __restrict__ Vs,
                                      uint32_t start, int cnt, int lane) {
  const float nan = __int_as_float(0x7fc00000);
  float4 u = make_float4(nan, nan, nan, nan), v = u;
  if (lane < cnt) {
    u = Us[start + lane];
    v = Vs[start + lane];
  }
  S.c[0][lane] = u.x;
  S.c[1][lane] = u.y;
  S.c[2][lane] = u.z;
  S.c[3][lane] = v.x;
  S.c[4][lane] = v.y;
  S.c[5][lane] = v.z;
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
  const float2* bounds;      // NN only: per node of the level (node - nb): (lo, hi), or nullptr
  int64_t nb;
};

// Search limit of a nearest-neighbour lane with current minimum `best` and node bounds
// [lo, hi]: boxes whose lower bound exceeds it are skipped. A lane below lo is done (-1: no
// bound is negative); otherwise min(best, hi): a minimum above hi only needs to be known above
// hi. With (lo, hi) = (-inf, +inf) this is best itself: the exact search.
__device__ __forceinline__ float nn_limit(float best, float lo, float hi) {
  return best < lo ? -1.f : fminf(best, hi);
}

// Per-lane tallies of the counting variant (evaluated d6 and box tests).
struct Tally {
  unsigned long long d6 = 0, box = 0;
};

// Evaluate target bucket b for the warp's query lanes (nearest-neighbour search).
template <bool kCount>
__device__ __forceinline__ void nn_bucket(const NNArgs& A, int64_t a, int64_t b, bool valid, const Query& Q,
                                          float& best, float lo, float hi, int lane, Stage& S, Tally& T) {
  const Box B = A.box[b];
  const bool need = valid && lb_point_box(Q, B) <= nn_limit(best, lo, hi);
  if (kCount) T.box += valid;
  if (!__any_sync(0xffffffffu, need)) return;
  const Bucket Bb = A.bk[b];
  __syncwarp();
  stage(S, A.Us, A.Vs, Bb.start, int(Bb.count), lane);
  __syncwarp();
  for (uint32_t s0 = 0; s0 < Bb.count; s0 += 8) {
    const Box Sb = A.sub[4 * b + (s0 >> 3)];
    const bool sneed = need && lb_point_box(Q, Sb) <= nn_limit(best, lo, hi);
    if (kCount) T.box += need;
    if (!__any_sync(0xffffffffu, sneed)) continue;
    if (sneed) {
      const int s1 = int(min(s0 + 8, Bb.count));
      if (kCount) T.d6 += uint32_t(s1) - s0;
      if (b == a) {
        for (int j = int(s0); j < s1; j += 2) {
          const float2 d = d6_pair(Q, S, j);
          best = fminf(best, j == lane ? best : d.x);
          best = fminf(best, j + 1 == lane ? best : d.y);
        }
      } else {
#pragma unroll
        for (int j = int(s0); j < int(s0) + 8; j += 2) {
          if (j < s1) {
            const float2 d = d6_pair(Q, S, j);
            best = fminf(fminf(best, d.x), d.y);
          }
        }
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
__global__ void __launch_bounds__(kT, 4) k_nn6d_pruned(NNArgs A, float* __restrict__ nn2) {
  __shared__ Stage stg[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int64_t nbk = *A.nbuckets;
  Tally T;
  while (true) {
    const int64_t w = next_work(A.counter, lane);
    if (w >= nbk) break;
    const int64_t a = A.order[w];
    const Bucket Aq = A.bk[a];
    const float4 iv = A.inv[Aq.node];
    const bool valid = lane < int(Aq.count);
    const uint32_t si = Aq.start + (valid ? lane : 0);
    const Query Q = make_query(A.Us[si], A.Vs[si], iv.x, iv.y);
    float best = __int_as_float(0x7f800000);
    float lo = -best, hi = best;
    if (A.bounds) {
      const float2 bd = A.bounds[int64_t(Aq.node) - A.nb];
      lo = bd.x;
      hi = bd.y;
    }
    const int64_t own = (a - int64_t(Aq.first)) >> 5, nsb = Aq.sbcount;
    for (int64_t t = 0; t <= 2 * nsb; ++t) {
      if (__all_sync(0xffffffffu, !valid || best < lo)) break;  // every lane known below lo
      const int64_t s = outward(own, t);
      if (s < 0 || s >= nsb) continue;
      const Box SB = A.sbox[Aq.sbfirst + s];
      const bool need = valid && lb_point_box(Q, SB) <= nn_limit(best, lo, hi);
      if (kCount) T.box += valid;
      if (!__any_sync(0xffffffffu, need)) continue;
      const int64_t b_lo = int64_t(Aq.first) + 32 * s;
      const int64_t b_hi = rsd::min64(b_lo + 32, int64_t(Aq.last) + 1);
      if (s == own) {
        for (int64_t t2 = 0; t2 <= 2 * 32; ++t2) {
          const int64_t b = outward(a, t2);
          if (b < b_lo || b >= b_hi) continue;
          nn_bucket<kCount>(A, a, b, valid, Q, best, lo, hi, lane, stg[wb], T);
        }
      } else if (s > own) {
        for (int64_t b = b_lo; b < b_hi; ++b)
          nn_bucket<kCount>(A, a, b, valid, Q, best, lo, hi, lane, stg[wb], T);
      } else {
        for (int64_t b = b_hi - 1; b >= b_lo; --b)
          nn_bucket<kCount>(A, a, b, valid, Q, best, lo, hi, lane, stg[wb], T);
      }
    }
    if (valid) nn2[A.sp[si]] = best;
  }
  flush_tally<kCount>(T, A.work, lane);
}

// Pending unions of each lane of a warp: member indices of its friends, lane-major columns.
struct LinkQueue {
  uint32_t j[32][32];
};

// Union the warp's pending friends with their lanes' members, the lanes side by side (the
// union order does not change the resulting components).
__device__ __forceinline__ void flush_links(uint32_t* uf, uint32_t pi, const LinkQueue& LQ, int& qn,
                                            int lane) {
  const int mx = int(__reduce_max_sync(0xffffffffu, uint32_t(qn)));
  for (int k = 0; k < mx; ++k)
    if (k < qn) rsd::uf_unite(uf, pi, LQ.j[k][lane]);
  qn = 0;
}

// Link pairs of query bucket a (box Abox) with target bucket b >= a.
template <bool kCount>
__device__ __forceinline__ void link_bucket(const NNArgs& A, int64_t a, int64_t b, const Box& Abox,
                                            bool active, const Query& Q, uint32_t pi, float l2,
                                            uint32_t* uf, int lane, Stage& S, uint32_t (&sj)[32],
                                            LinkQueue& LQ, int& qn, Tally& T) {
  const Box B = A.box[b];
  if (kCount) T.box += (lane == 0);
  if (lb_box_box(Abox, B, Q.s) > l2) return;
  const bool need = active && lb_point_box(Q, B) <= l2;
  if (kCount) T.box += active;
  if (!__any_sync(0xffffffffu, need)) return;
  const Bucket Bb = A.bk[b];
  __syncwarp();
  stage(S, A.Us, A.Vs, Bb.start, int(Bb.count), lane);
  if (lane < int(Bb.count)) sj[lane] = A.sp[Bb.start + lane];
  __syncwarp();
  const int j0 = (b == a) ? lane + 1 : 0;
  uint32_t pending = 0;  // targets of this bucket the lane links to (unions after the scan)
  for (uint32_t s0 = 0; s0 < Bb.count; s0 += 8) {
    const Box Sb = A.sub[4 * b + (s0 >> 3)];
    if (kCount) T.box += (lane == 0);
    if (lb_box_box(Abox, Sb, Q.s) > l2) continue;
    const bool sneed = need && lb_point_box(Q, Sb) <= l2;
    if (kCount) T.box += need;
    if (!__any_sync(0xffffffffu, sneed)) continue;
    if (sneed) {
      const int s1 = int(min(s0 + 8, Bb.count));
      if (kCount) T.d6 += s1 > max(int(s0), j0) ? uint32_t(s1 - max(int(s0), j0)) : 0u;
      for (int j = int(s0); j < s1; j += 2) {
        if (j + 1 < j0) continue;
        const float2 d = d6_pair(Q, S, j);
        if (j >= j0 && d.x <= l2) pending |= 1u << j;
        if (j + 1 >= j0 && j + 1 < s1 && d.y <= l2) pending |= 2u << j;
      }
    }
  }
  // Friends go to the lane's queue; the queues are flushed (union-find calls of all lanes side
  // by side) when one would overflow and at the end of the query bucket, instead of one
  // diverging lane at a time inside the distance loop.
  if (__any_sync(0xffffffffu, qn + __popc(pending) > 32)) flush_links(uf, pi, LQ, qn, lane);
  while (pending) {
    const int j = __ffs(pending) - 1;
    pending &= pending - 1u;
    LQ.j[qn++][lane] = sj[j];
  }
}

// Over the buckets of the members with a friend: every valid lane is active.
template <bool kCount>
__global__ void __launch_bounds__(kT)
k_link6d_pruned(NNArgs A, uint32_t* __restrict__ uf) {
  Tally T;
  __shared__ Stage stg[kWarpsPerBlock];
  __shared__ uint32_t sj[kWarpsPerBlock][32];
  __shared__ LinkQueue lq[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int64_t nbk = *A.nbuckets;
  while (true) {
    const int64_t w = next_work(A.counter, lane);
    if (w >= nbk) break;
    const int64_t a = A.order[w];
    const Bucket Aq = A.bk[a];
    const float4 iv = A.inv[Aq.node];
    const float l2 = iv.z;
    const bool valid = lane < int(Aq.count);
    const uint32_t si = Aq.start + (valid ? lane : 0);
    const Query Q = make_query(A.Us[si], A.Vs[si], iv.x, iv.y);
    const uint32_t pi = A.sp[si];
    const bool active = valid;
    const Box Abox = A.box[a];
    int qn = 0;  // this lane's pending unions in lq[wb]
    const int64_t own = (a - int64_t(Aq.first)) >> 5, nsb = Aq.sbcount;
    for (int64_t s = own; s < nsb; ++s) {
      const Box SB = A.sbox[Aq.sbfirst + s];
      if (kCount) T.box += (lane == 0);
      if (lb_box_box(Abox, SB, Q.s) > l2) continue;
      const bool need = active && lb_point_box(Q, SB) <= l2;
      if (kCount) T.box += active;
      if (!__any_sync(0xffffffffu, need)) continue;
      const int64_t b_lo = rsd::min64(int64_t(Aq.first) + 32 * s, int64_t(Aq.last) + 1);
      const int64_t b_hi = rsd::min64(int64_t(Aq.first) + 32 * s + 32, int64_t(Aq.last) + 1);
      for (int64_t b = (s == own ? a : b_lo); b < b_hi; ++b)
        link_bucket<kCount>(A, a, b, Abox, active, Q, pi, l2, uf, lane, stg[wb], sj[wb], lq[wb], qn, T);
    }
    flush_links(uf, pi, lq[wb], qn, lane);
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
  A.bounds = nullptr;
  A.nb = 0;
  return A;
}

}  // namespace

namespace {

// Bucket tables of the level over the members [start[k], start[k] + cnt[k]) of each node k in
// the arrays Us, Vs (m entries at most): buckets of 32, boxes, sub-boxes, superboxes and the
// work queue ordered by node size class.
int build_buckets(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t m, const int64_t* start, const int64_t* cnt,
                  const float4* Us, const float4* Vs, cudaStream_t st) {
  int64_t* boff = scratch_t<int64_t>(ctx, S_P_BOFF, size_t(nn) + 1);
  int64_t* sboff = scratch_t<int64_t>(ctx, S_P_SBOFF, size_t(nn) + 1);
  const int64_t nbk_ub = nn + m / 32 + 1;
  const int64_t nsb_ub = nn + nbk_ub / 32 + 1;
  Bucket* bk = scratch_t<Bucket>(ctx, S_P_BUCKET, size_t(nbk_ub));
  Box* box = scratch_t<Box>(ctx, S_P_BOX, size_t(nbk_ub));
  Box* sub = scratch_t<Box>(ctx, S_P_SUB, size_t(nbk_ub) * 4);
  Box* sbox = scratch_t<Box>(ctx, S_P_SBOX, size_t(nsb_ub));
  uint64_t* qk = scratch_t<uint64_t>(ctx, S_P_QKEY_A, size_t(nbk_ub));
  uint64_t* qk2 = scratch_t<uint64_t>(ctx, S_P_QKEY_B, size_t(nbk_ub));
  uint32_t* qv = scratch_t<uint32_t>(ctx, S_P_QVAL_A, size_t(nbk_ub));
  uint32_t* qv2 = scratch_t<uint32_t>(ctx, S_P_QVAL_B, size_t(nbk_ub));
  uint32_t* qorder = scratch_t<uint32_t>(ctx, S_P_ORDER, size_t(nbk_ub));
  if (!boff || !sboff || !bk || !box || !sub || !sbox || !qk || !qk2 || !qv || !qv2 || !qorder)
    return RS_ERR_OOM;
  k_bucket_counts<<<grid_for(nn, kT), kT, 0, st>>>(nn, cnt, boff, sboff);
  RS_LAUNCHED(ctx, "k_bucket_counts");
  RS_TRY(exclusive_scan_i64(ctx, nn, boff, boff + nn, st));
  RS_TRY(exclusive_scan_i64(ctx, nn, sboff, sboff + nn, st));
  k_buckets<<<grid_for(nbk_ub * 32, kT), kT, 0, st>>>(nb, nn, nbk_ub, boff, sboff, start, cnt, Us, Vs, bk, box,
                                                     sub, qk, qv);
  RS_LAUNCHED(ctx, "k_buckets");
  k_superboxes<<<grid_for(nsb_ub * 32, kT), kT, 0, st>>>(nn, boff, sboff, box, sbox);
  RS_LAUNCHED(ctx, "k_superboxes");
  uint64_t* qk_out;
  uint32_t* qv_out;
  RS_TRY(radix_sort_u64(ctx, nbk_ub, 8, qk, qv, qk2, qv2, &qk_out, &qv_out, st));
  RS_CUDA(ctx, cudaMemcpyAsync(qorder, qv_out, sizeof(uint32_t) * nbk_ub, cudaMemcpyDeviceToDevice, st));
  return RS_OK;
}

// ---- Bounded nearest-neighbour searches for large nodes ---------------------------------------
// The split needs each member's nn2 exactly only near the k-th smallest value (the adaptive l2)
// and, elsewhere, only whether it lies below or above it (k_select_l2 and the link pass's
// member filter). For nodes of at least min_members (4096 by default) members a sample of
// buckets (every S-th of the node, about kSampleBuckets of them) is searched exactly first;
// the sample's order statistics around rank p s (p = (k + 1/2) / g) give bounds lo <= hi; the
// other members are searched with the limit of nn_limit: a lane stops once its minimum is below lo (its nn2 is
// then some value below lo) and prunes with hi (a minimum above hi is kept as some value above
// hi). Members whose nn2 lies in [lo, hi] are found exactly, so the k-th smallest of the stored
// values equals the exact one whenever it lies in [lo, hi]; k_bounds_check verifies that per
// node after the selection and sends every node that fails through the exact search again.
constexpr int64_t kBoundMinDefault = 4096;
constexpr int64_t kSampleBuckets = 48;

__device__ __forceinline__ int64_t sample_stride(int64_t nbk) {
  return nbk / kSampleBuckets > 1 ? nbk / kSampleBuckets : 1;
}

// Queue entry w (bucket order[w]) goes to the first, exact queue (flag s: the samples of the
// nodes searched with bounds, and every bucket of the smaller nodes, so that the first launch
// fills the GPU) or to the second (flag r: the other buckets of the bounded nodes).
__global__ void k_queue_flags(int64_t nbk_ub, const int64_t* __restrict__ nbk, const uint32_t* __restrict__ order,
                              const Bucket* __restrict__ bk, const int64_t* __restrict__ node_size,
                              int64_t min_members, int64_t* __restrict__ fs, int64_t* __restrict__ fr) {
  const int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= nbk_ub) return;
  int64_t smp = 0, rest = 0;
  if (w < *nbk) {
    const Bucket B = bk[order[w]];
    const int64_t nb_node = int64_t(B.last) - int64_t(B.first) + 1;
    const bool bounded = node_size[B.node] >= min_members;
    smp = !bounded || ((int64_t(order[w]) - int64_t(B.first)) % sample_stride(nb_node)) == 0;
    rest = !smp;
  }
  fs[w] = smp;
  fr[w] = rest;
}

// Stable scatter of the two queues (order preserved: largest nodes first in both); counts at
// qcount[0] (sample) and qcount[1] (others).
__global__ void k_queue_scatter(int64_t nbk_ub, const uint32_t* __restrict__ order, const int64_t* __restrict__ fs,
                                const int64_t* __restrict__ fr, uint32_t* __restrict__ qs,
                                uint32_t* __restrict__ qr, int64_t* __restrict__ qcount) {
  const int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w == 0) {
    qcount[0] = fs[nbk_ub];
    qcount[1] = fr[nbk_ub];
  }
  if (w >= nbk_ub) return;
  if (fs[w + 1] != fs[w]) qs[fs[w]] = order[w];
  if (fr[w + 1] != fr[w]) qr[fr[w]] = order[w];
}

// Radix select (4 passes of 8 bits over non-negative float bit patterns) of rank k among the
// sample values of one node, read through `val(t)` for t < n (invalid entries return false).
template <class Val>
__device__ float block_select(Val val, int64_t n, uint32_t k, uint32_t* hist, uint32_t* s_prefix,
                              uint32_t* s_k) {
  if (threadIdx.x == 0) {
    *s_prefix = 0;
    *s_k = k;
  }
  uint32_t mask = 0;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0;
    __syncthreads();
    const uint32_t prefix = *s_prefix;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
      float v;
      if (!val(t, v)) continue;
      const uint32_t bits = __float_as_uint(v);
      if ((bits & mask) == prefix) atomicAdd(&hist[(bits >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t kk = *s_k, cum = 0;
      int d = 0;
      for (; d < 255; ++d) {
        if (cum + hist[d] > kk) break;
        cum += hist[d];
      }
      *s_k = kk - cum;
      *s_prefix = prefix | (uint32_t(d) << shift);
    }
    mask |= 255u << shift;
    __syncthreads();
  }
  return __uint_as_float(*s_prefix);
}

// One block per node of the level: bounds (lo, hi) from the sample of a node of at least
// min_members members, (-inf, +inf) (exact search) otherwise. The sample of a node is every
// S-th of its buckets; its size s and the target rank r = p s with p = (k + 1/2) / g; the
// bounds are the sample's order statistics at r -+ d, d = 6 sqrt(s p (1 - p)) + 8 (twice
// three binomial standard deviations: the sampled buckets are clusters of neighbours).
__global__ void __launch_bounds__(256)
k_sample_bounds(int64_t nb, int64_t nn, const int64_t* __restrict__ node_size, const int64_t* __restrict__ boff,
                const Bucket* __restrict__ bk, const uint32_t* __restrict__ sp, const float* __restrict__ nn2,
                int f_num, int f_den, float margin, int64_t min_members, float2* __restrict__ bounds) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_prefix, s_k;
  const int64_t k = blockIdx.x;
  if (k >= nn) return;
  const int64_t g = node_size[nb + k];
  const float inf = __int_as_float(0x7f800000);
  if (g < min_members) {
    if (threadIdx.x == 0) bounds[k] = make_float2(-inf, inf);
    return;
  }
  const int64_t b0 = boff[k], nbk = boff[k + 1] - b0;
  const int64_t S = sample_stride(nbk), ns = (nbk + S - 1) / S;
  // sample members: 32 per sampled bucket except possibly the node's last bucket
  const Bucket last = bk[b0 + nbk - 1];
  const bool last_sampled = ((nbk - 1) % S) == 0;
  const int64_t s = ns * 32 - (last_sampled ? 32 - int64_t(last.count) : 0);
  const int64_t kk = (int64_t(f_num) * g + f_den - 1) / f_den - 1;
  const double p = (double(kk) + 0.5) / double(g);
  const double r = p * double(s);
  const double d = double(margin) * (6.0 * sqrt(double(s) * p * (1.0 - p)) + 8.0);
  const int64_t r_lo = int64_t(floor(r - d)), r_hi = int64_t(ceil(r + d));
  if (r_lo > r_hi) {  // empty bounds (margin < 0: the exact fallback under test)
    if (threadIdx.x == 0) bounds[k] = make_float2(inf, -inf);
    return;
  }
  auto val = [&](int64_t t, float& v) -> bool {
    const Bucket B = bk[b0 + (t >> 5) * S];
    const uint32_t l = uint32_t(t & 31);
    if (l >= B.count) return false;
    v = nn2[sp[B.start + l]];
    return true;
  };
  const float lo = r_lo <= 0 ? -inf : block_select(val, ns * 32, uint32_t(r_lo), hist, &s_prefix, &s_k);
  __syncthreads();
  const float hi = r_hi >= s - 1 ? inf : block_select(val, ns * 32, uint32_t(r_hi), hist, &s_prefix, &s_k);
  if (threadIdx.x == 0) bounds[k] = make_float2(lo, hi);
}

// After the selection: a bounded node whose l2 lies outside its [lo, hi] failed (its stored
// values are not exact there): mark it, reset its bounds to the exact search and queue all its
// buckets again (qcount[2]; order of the queue does not matter for exact results).
// tally (counting variant, may be null): [0] nodes searched with bounds, [1] nodes that failed.
__global__ void k_bounds_check(int64_t nb, int64_t nn, const float4* __restrict__ inv, float2* __restrict__ bounds,
                               int* __restrict__ failed, unsigned long long* __restrict__ tally) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const float inf = __int_as_float(0x7f800000);
  const float2 bd = bounds[k];
  const float l2 = inv[nb + k].z;
  const bool bad = !(bd.x <= l2 && l2 <= bd.y);
  failed[k] = bad ? 1 : 0;
  if (bad) bounds[k] = make_float2(-inf, inf);
  if (tally && (bd.x > -inf || bd.y < inf)) {
    atomicAdd(tally, 1ull);
    if (bad) atomicAdd(tally + 1, 1ull);
  }
}

__global__ void k_fail_queue(int64_t nbk_ub, const int64_t* __restrict__ nbk, const uint32_t* __restrict__ order,
                             const Bucket* __restrict__ bk, int64_t nb, const int* __restrict__ failed,
                             uint32_t* __restrict__ qf, unsigned long long* __restrict__ qcount) {
  const int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= nbk_ub || w >= *nbk) return;
  const uint32_t a = order[w];
  if (failed[int64_t(bk[a].node) - nb]) qf[atomicAdd(qcount, 1ull)] = a;
}

unsigned persistent_grid(int64_t nbk_ub) {
  return unsigned(std::min<int64_t>((nbk_ub + kWarpsPerBlock - 1) / kWarpsPerBlock, 152 * 8));
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
  int64_t* nstart = scratch_t<int64_t>(ctx, S_P_NSTART, size_t(nn));
  int64_t* ncnt = scratch_t<int64_t>(ctx, S_P_NCNT, size_t(nn));
  unsigned long long* qctr = scratch_t<unsigned long long>(ctx, S_P_QCTR, 2);
  if (!scratch_t<unsigned long long>(ctx, S_P_WORK, 6)) return RS_ERR_OOM;
  if (!mean_u || !ka || !kb || !va || !vb || !Us || !Vs || !sp || !nstart || !ncnt || !qctr) return RS_ERR_OOM;
  k_node_means<<<grid_for(nn, kT), kT, 0, st>>>(nb, nn, h.node_size, sums, mean_u);
  RS_LAUNCHED(ctx, "k_node_means");
  k_hilbert3<<<grid_for(m, kT), kT, 0, st>>>(mb, m, nb, h.mnode, h.U, h.inv, mean_u, ka, va);
  RS_LAUNCHED(ctx, "k_hilbert3");
  uint64_t* keys;
  uint32_t* order;
  RS_TRY(radix_sort_u64(ctx, m, 24 + bits_for(uint64_t(nn)), ka, va, kb, vb, &keys, &order, st));
  k_gather_sorted<<<grid_for(m, kT), kT, 0, st>>>(mb, m, order, h.U, h.V, Us, Vs, sp);
  RS_LAUNCHED(ctx, "k_gather_sorted");
  k_node_ranges<<<grid_for(nn, kT), kT, 0, st>>>(nb, nn, mb, h.node_off, h.node_size, nstart, ncnt);
  RS_LAUNCHED(ctx, "k_node_ranges");
  return build_buckets(ctx, nb, nn, m, nstart, ncnt, Us, Vs, st);
}

// One persistent launch of the nearest-neighbour kernel over the queue (order, count).
static int run_nn(rs_ctx* ctx, NNArgs A, const uint32_t* order, const int64_t* count, int64_t nbk_ub,
                  float* nn2, cudaStream_t st) {
  A.order = order;
  A.nbuckets = count;
  const unsigned grid = persistent_grid(nbk_ub);
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

// Nearest neighbours of the level: the smaller nodes and the sample of every large node
// exactly, the large nodes' bounds, then their other buckets with those bounds. No host round
// trip: the queues and their counts stay on the device.
int rs::prune6d_nn(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, float* nn2,
                   cudaStream_t st) {
  (void)mb;
  Hier h = hier_of(ctx);
  NNArgs A = nn_args(ctx, nn);
  const int64_t nbk_ub = nn + m / 32 + 1;
  const int64_t bmin = ctx->nn_bound_min > 0 ? ctx->nn_bound_min : kBoundMinDefault;
  ctx->nn_bounded_level = m >= bmin;  // a node of bmin members needs that many at the level
  if (!ctx->nn_bounded_level) return run_nn(ctx, A, A.order, A.nbuckets, nbk_ub, nn2, st);
  int64_t* fs = scratch_t<int64_t>(ctx, S_P_QFS, size_t(nbk_ub) + 1);
  int64_t* fr = scratch_t<int64_t>(ctx, S_P_QFR, size_t(nbk_ub) + 1);
  uint32_t* qs = scratch_t<uint32_t>(ctx, S_P_QS, size_t(nbk_ub));
  uint32_t* qr = scratch_t<uint32_t>(ctx, S_P_QR, size_t(nbk_ub));
  int64_t* qcount = scratch_t<int64_t>(ctx, S_P_QCOUNT, 4);
  float2* bounds = scratch_t<float2>(ctx, S_P_BOUNDS, size_t(std::max<int64_t>(nn, 1)));
  if (!fs || !fr || !qs || !qr || !qcount || !bounds) return RS_ERR_OOM;
  k_queue_flags<<<grid_for(nbk_ub, kT), kT, 0, st>>>(nbk_ub, A.nbuckets, A.order, A.bk, h.node_size, bmin, fs,
                                                     fr);
  RS_LAUNCHED(ctx, "k_queue_flags");
  RS_TRY(exclusive_scan_i64(ctx, nbk_ub, fs, fs + nbk_ub, st));
  RS_TRY(exclusive_scan_i64(ctx, nbk_ub, fr, fr + nbk_ub, st));
  k_queue_scatter<<<grid_for(nbk_ub, kT), kT, 0, st>>>(nbk_ub, A.order, fs, fr, qs, qr, qcount);
  RS_LAUNCHED(ctx, "k_queue_scatter");
  RS_TRY(run_nn(ctx, A, qs, qcount + 0, nbk_ub, nn2, st));  // exactly
  const int64_t* boff = static_cast<const int64_t*>(ctx->buf[S_P_BOFF].ptr);
  k_sample_bounds<<<unsigned(std::max<int64_t>(nn, 1)), 256, 0, st>>>(nb, nn, h.node_size, boff, A.bk, A.sp, nn2,
                                                                   ctx->cfg.f_num, ctx->cfg.f_den,
                                                                   ctx->nn_bound_margin, bmin, bounds);
  RS_LAUNCHED(ctx, "k_sample_bounds");
  A.bounds = bounds;
  A.nb = nb;
  return run_nn(ctx, A, qr, qcount + 1, nbk_ub, nn2, st);
}

// After the selection of l2: nodes whose l2 fell outside their bounds are searched again
// exactly (*failed_out: int [nn], 1 for those nodes, for the selection to be repeated there).
int rs::prune6d_check(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t m, float* nn2, const int** failed_out,
                      cudaStream_t st) {
  *failed_out = nullptr;
  if (!ctx->nn_bounded_level) return RS_OK;  // every search of the level was exact
  Hier h = hier_of(ctx);
  NNArgs A = nn_args(ctx, nn);
  const int64_t nbk_ub = nn + m / 32 + 1;
  float2* bounds = static_cast<float2*>(ctx->buf[S_P_BOUNDS].ptr);
  int* failed = scratch_t<int>(ctx, S_P_FAILED, size_t(std::max<int64_t>(nn, 1)));
  uint32_t* qf = scratch_t<uint32_t>(ctx, S_P_QS, size_t(nbk_ub));  // the sample queue is done
  unsigned long long* fcount = reinterpret_cast<unsigned long long*>(
      static_cast<int64_t*>(ctx->buf[S_P_QCOUNT].ptr) + 2);
  if (!failed || !qf) return RS_ERR_OOM;
  k_bounds_check<<<grid_for(nn, kT), kT, 0, st>>>(nb, nn, h.inv, bounds, failed,
                                                  ctx->count_work ? A.work + 4 : nullptr);
  RS_LAUNCHED(ctx, "k_bounds_check");
  RS_CUDA(ctx, cudaMemsetAsync(fcount, 0, sizeof(unsigned long long), st));
  k_fail_queue<<<grid_for(nbk_ub, kT), kT, 0, st>>>(nbk_ub, A.nbuckets, A.order, A.bk, nb, failed, qf, fcount);
  RS_LAUNCHED(ctx, "k_fail_queue");
  A.bounds = bounds;
  A.nb = nb;
  RS_TRY(run_nn(ctx, A, qf, reinterpret_cast<const int64_t*>(fcount), nbk_ub, nn2, st));
  *failed_out = failed;
  return RS_OK;
}

// The link pass runs over the members with a friend only (the others can join no link): they
// are compacted in the sorted order and get their own, tighter buckets.
int rs::prune6d_link(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, const float* nn2,
                     uint32_t* uf, cudaStream_t st) {
  Hier h = hier_of(ctx);
  const float4* Us = static_cast<const float4*>(ctx->buf[S_P_US].ptr);
  const float4* Vs = static_cast<const float4*>(ctx->buf[S_P_VS].ptr);
  const uint32_t* sp = static_cast<const uint32_t*>(ctx->buf[S_P_SP].ptr);
  int64_t* pos = scratch_t<int64_t>(ctx, S_P_APOS, size_t(m) + 1);
  float4* UsA = scratch_t<float4>(ctx, S_P_USA, size_t(std::max<int64_t>(m, 1)));
  float4* VsA = scratch_t<float4>(ctx, S_P_VSA, size_t(std::max<int64_t>(m, 1)));
  uint32_t* spA = scratch_t<uint32_t>(ctx, S_P_SPA, size_t(std::max<int64_t>(m, 1)));
  int64_t* nstart = scratch_t<int64_t>(ctx, S_P_NSTART, size_t(nn));
  int64_t* ncnt = scratch_t<int64_t>(ctx, S_P_NCNT, size_t(nn));
  if (!pos || !UsA || !VsA || !spA || !nstart || !ncnt) return RS_ERR_OOM;
  k_active_flags<<<grid_for(m, kT), kT, 0, st>>>(m, mb, sp, h.mnode, h.inv, nn2, pos);
  RS_LAUNCHED(ctx, "k_active_flags");
  RS_TRY(exclusive_scan_i64(ctx, m, pos, pos + m, st));
  k_compact_active<<<grid_for(m, kT), kT, 0, st>>>(m, pos, Us, Vs, sp, UsA, VsA, spA);
  RS_LAUNCHED(ctx, "k_compact_active");
  k_active_ranges<<<grid_for(nn, kT), kT, 0, st>>>(nb, nn, mb, h.node_off, h.node_size, pos, nstart, ncnt);
  RS_LAUNCHED(ctx, "k_active_ranges");
  RS_TRY(build_buckets(ctx, nb, nn, m, nstart, ncnt, UsA, VsA, st));
  NNArgs A = nn_args(ctx, nn);
  A.Us = UsA;
  A.Vs = VsA;
  A.sp = spA;
  A.counter += 1;
  const unsigned grid = persistent_grid(nn + m / 32 + 1);
  RS_CUDA(ctx, cudaMemsetAsync(A.counter, 0, sizeof(unsigned long long), st));
  if (ctx->count_work) {
    k_link6d_pruned<true><<<grid, kT, 0, st>>>(A, uf);
  } else {
    ProfScope prof_(ctx, "k_link6d_pruned", st);
    k_link6d_pruned<false><<<grid, kT, 0, st>>>(A, uf);
  }
  RS_LAUNCHED(ctx, "k_link6d_pruned");
  return RS_OK;
}

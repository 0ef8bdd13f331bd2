// Learned surrogate of the binding energy inside rs_unbind (batched + surrogate form).
//
// For every node with at least kSurMin members ("big" nodes), instead of the O(g^2) potential:
//   1. features per member (k_sur_features): r / r_vir, the enclosed-member fractions within
//      0.5, 1 and 2 times the member's radius (binary searches in the node's radially sorted
//      members), the potential of the spherically averaged node (enclosed count over r plus the
//      suffix sum of 1 / r_j over the members outside), |v - v_bulk| / sigma_v,1D, log10 g and
//      the relative size of the deepest hierarchy node holding the member; r is measured from
//      the node's mean position, r_vir = (3 g m / (4 pi 200 rho_bar))^(1/3);
//   2. the MLP predicts psi = phi r_vir / (G g m); E_pred = KE + psi_hat G g m / r_vir;
//   3. gate (k_sur_gate): a member is classified by the surrogate iff
//      |E_pred| > margin_factor * err_max * G g m / r_vir, err_max being the MLP's held-out
//      maximum error; every other member takes the exact path;
//   4. spot check: per node, the spot_check gated members with the smallest margin are also
//      evaluated exactly; if any has |psi_hat - psi| > err_max or a different flag, the whole
//      node falls back to the exact path;
//   5. exact path per member (k_pot_member): float32 direct sum over the node (one warp per
//      member, certified bound kCertB2) and the float64 canonical-order potential when the
//      energy is within the bound of zero -- the same flag as the plain form.
#include <cmath>

#include "rs_cro.cuh"

namespace rs {
int mlp_forward(rs_ctx* ctx, int64_t n, const float* x, float* y, cudaStream_t st);
int surrogate_unbind(rs_ctx* ctx, const double* vbulk, uint8_t* bound, unsigned long long* counters,
                     cudaStream_t st);
}  // namespace rs

using namespace rs;

namespace {

constexpr int kT = 256;
constexpr int64_t kSurMin = kSurrogateMinMembers;
constexpr double kU = 5.9604644775390625e-08;
// per-member warp sum: per term <= 8u, 32-term lane blocks <= 31u, Kahan <= 2u, 5-level warp
// tree <= 5u; 48u with slack.
constexpr double kCertB2 = 48.0 * kU + 1e-12;

struct NodeStat {
  float cx, cy, cz, r_vir;
  float sig_v1d, log_g, pad0, pad1;
  double gm_over_rvir;
  double pad2;
};

struct StatTerm {  // u (3), v (3), v^2 (3)
  const float4* U;
  const float4* V;
  __device__ __forceinline__ void add(int64_t, int64_t p, int64_t, double* acc) const {
    const float4 u = U[p], v = V[p];
    const double a[3] = {double(u.x), double(u.y), double(u.z)};
    const double b[3] = {double(v.x), double(v.y), double(v.z)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      acc[d] = __dadd_rn(acc[d], a[d]);
      acc[3 + d] = __dadd_rn(acc[3 + d], b[d]);
      acc[6 + d] = __dadd_rn(acc[6 + d], __dmul_rn(b[d], b[d]));
    }
  }
};

__global__ void k_sur_node_flags(int64_t nn, const int64_t* __restrict__ node_size,
                                 int64_t* __restrict__ szm, int64_t* __restrict__ bigf) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nn) return;
  const bool big = node_size[q] >= kSurMin;
  szm[q] = big ? node_size[q] : 0;
  bigf[q] = big ? 1 : 0;
}

__global__ void k_sur_stats(int64_t nn, const int64_t* __restrict__ node_size,
                            const double* __restrict__ sums, double m, double G, double rho_bar,
                            NodeStat* __restrict__ st) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nn) return;
  const double g = double(node_size[q]);
  const double* S = sums + 9 * q;
  NodeStat s;
  s.cx = float(S[0] / g);
  s.cy = float(S[1] / g);
  s.cz = float(S[2] / g);
  double var = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double mv = S[3 + d] / g;
    var += S[6 + d] / g - mv * mv;
  }
  s.sig_v1d = float(sqrt(fmax(var, 0.0) / 3.0));
  const double rv = cbrt(3.0 * g * m / (4.0 * 3.14159265358979323846 * 200.0 * rho_bar));
  s.r_vir = float(rv);
  s.log_g = float(log10(g));
  s.gm_over_rvir = G * g * m / rv;
  s.pad0 = s.pad1 = 0.f;
  s.pad2 = 0.0;
  st[q] = s;
}

__global__ void k_sur_members(int64_t m, const uint32_t* __restrict__ mnode,
                              const int64_t* __restrict__ node_off, const int64_t* __restrict__ node_size,
                              const int64_t* __restrict__ sur_off, uint32_t* __restrict__ sur_mem) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const uint32_t q = mnode[p];
  if (node_size[q] < kSurMin) return;
  sur_mem[sur_off[q] + (p - node_off[q])] = uint32_t(p);
}

__device__ __forceinline__ float member_radius(float4 u, const NodeStat& s) {
  const float dx = u.x - s.cx, dy = u.y - s.cy, dz = u.z - s.cz;
  return sqrtf(dx * dx + dy * dy + dz * dz);
}

// Radial sort key of every (node, member): node index above the radius bits, so each node's
// members stay in the node's own member range [node_off, node_off + g) after sorting.
__global__ void k_all_radius(int64_t m, const uint32_t* __restrict__ mnode, const float4* __restrict__ U,
                             const NodeStat* __restrict__ st, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const uint32_t q = mnode[p];
  const float r = member_radius(U[p], st[q]);
  keys[p] = (uint64_t(q) << 32) | uint64_t(__float_as_uint(r));
  vals[p] = uint32_t(p);
}

__device__ __forceinline__ int64_t count_below(const uint64_t* __restrict__ rkeys, int64_t lo, int64_t hi,
                                               float v) {
  // members of the segment whose radius is < v (radius bits are the low 32 bits of the keys)
  const int64_t base = lo;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (__uint_as_float(uint32_t(rkeys[mid] & 0xffffffffull)) < v) lo = mid + 1; else hi = mid;
  }
  return lo - base;
}

constexpr double kFix = 16777216.0;  // 2^24: fixed-point scale of the 1/r suffix sums

// Per radially sorted position s: fixed-point 1 / max(r, eps) (to be prefix-summed) and the
// sorted position of each surrogate member.
__global__ void k_sur_inv_r(int64_t ns, const uint64_t* __restrict__ rkeys, const uint32_t* __restrict__ rvals,
                            float eps, int64_t* __restrict__ fix, uint32_t* __restrict__ spos) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const float r = __uint_as_float(uint32_t(rkeys[s] & 0xffffffffull));
  fix[s] = llrint(kFix / double(fmaxf(r, eps)));
  spos[rvals[s]] = uint32_t(s);
}

// psi_sph of every (node, member): the potential of the spherically averaged node at the
// member, in units of G g m / r_vir: -(r_vir / g) (#inside / max(r, eps) + sum over members
// outside of 1 / max(r_j, eps)), from the radially sorted member ranges.
__global__ void k_psi_sph(int64_t m, const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_off,
                          const int64_t* __restrict__ node_size, const NodeStat* __restrict__ st,
                          const float4* __restrict__ U, const int64_t* __restrict__ fix,
                          const uint32_t* __restrict__ spos, float eps, float* __restrict__ psi_sph) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const uint32_t q = mnode[p];
  const NodeStat s = st[q];
  const int64_t g = node_size[q], lo = node_off[q], hi = lo + g;
  const int64_t si = spos[p];
  const double outer = double(fix[hi] - fix[si + 1]) / kFix;
  const double inner = double(si - lo) / double(fmaxf(member_radius(U[p], s), eps));
  psi_sph[p] = float(-(double(s.r_vir) / double(g)) * (inner + outer));
}

// Features of surrogate member k, in this order: r / r_vir; fractions of the node's members
// with radius below 0.5 r, r and 2 r; psi_sph of the node; |v - v_bulk| / sigma_v,1D;
// log10 g; psi_sph of the deepest node holding the member, converted to this node's units
// (g_d / g) (r_vir / r_vir,d) -- the well of the member's own substructure.
__global__ void k_sur_features(int64_t ns, const uint32_t* __restrict__ sur_mem,
                               const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_off,
                               const int64_t* __restrict__ node_size, const float4* __restrict__ U,
                               const float4* __restrict__ V, const NodeStat* __restrict__ st,
                               const double* __restrict__ vbulk, const uint64_t* __restrict__ rkeys,
                               const float* __restrict__ psi_sph, const uint32_t* __restrict__ mem,
                               const int64_t* __restrict__ deepest,
                               const uint32_t* __restrict__ deepest_pos, float* __restrict__ feat) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t p = sur_mem[k], q = mnode[p];
  const NodeStat s = st[q];
  const int64_t g = node_size[q], lo = node_off[q], hi = lo + g;
  const float r = member_radius(U[p], s);
  const float inv_g = 1.0f / float(g);
  const float f05 = float(count_below(rkeys, lo, hi, 0.5f * r)) * inv_g;
  const float f1 = float(count_below(rkeys, lo, hi, r)) * inv_g;
  const float f2 = float(count_below(rkeys, lo, hi, 2.0f * r)) * inv_g;
  const float4 v = V[p];
  const float dvx = v.x - float(vbulk[3 * q]), dvy = v.y - float(vbulk[3 * q + 1]),
              dvz = v.z - float(vbulk[3 * q + 2]);
  const uint32_t part = mem[p];
  const int64_t d = deepest[part];
  const float sub = psi_sph[deepest_pos[part]] * (float(node_size[d]) / float(g)) *
                    (s.r_vir / st[d].r_vir);
  float* F = feat + 8 * k;
  F[0] = r / s.r_vir;
  F[1] = f05;
  F[2] = f1;
  F[3] = f2;
  F[4] = psi_sph[p];
  F[5] = sqrtf(dvx * dvx + dvy * dvy + dvz * dvz) / fmaxf(s.sig_v1d, 1e-30f);
  F[6] = s.log_g;
  F[7] = sub;
}

__global__ void k_sur_targets(int64_t ns, const uint32_t* __restrict__ sur_mem,
                              const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_size,
                              const NodeStat* __restrict__ st, const float* __restrict__ S,
                              float* __restrict__ psi) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t p = sur_mem[k], q = mnode[p];
  psi[k] = float(-double(S[p]) * double(st[q].r_vir) / double(node_size[q]));
}

__device__ __forceinline__ double kinetic(float4 v, const double* vb) {
  const double dvx = __dsub_rn(double(v.x), vb[0]);
  const double dvy = __dsub_rn(double(v.y), vb[1]);
  const double dvz = __dsub_rn(double(v.z), vb[2]);
  const double s = __dadd_rn(__dadd_rn(__dmul_rn(dvx, dvx), __dmul_rn(dvy, dvy)), __dmul_rn(dvz, dvz));
  return __dmul_rn(0.5, s);
}

// counters: [0] exact per-member list, [1] check list, [2] fp64 list (current pass), [3] rerun
// list, [4] failed nodes, [5] gated, [6] fp64 total (surrogate path), [7] fp64 of the direct
// sums, [8] members of nodes sent whole to the direct sum
__global__ void k_sur_gate(int64_t ns, const uint32_t* __restrict__ sur_mem, const uint32_t* __restrict__ mnode,
                           const int64_t* __restrict__ node_size, const float4* __restrict__ V,
                           const double* __restrict__ vbulk, const NodeStat* __restrict__ st,
                           const float* __restrict__ psi_hat, float thr_psi, uint8_t* __restrict__ bound,
                           uint8_t* __restrict__ sflag, float* __restrict__ margin,
                           unsigned int* __restrict__ gcount, unsigned int* __restrict__ ecount,
                           unsigned long long* __restrict__ counters) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t p = sur_mem[k], q = mnode[p];
  const double gmr = st[q].gm_over_rvir;
  const double e = kinetic(V[p], vbulk + 3 * int64_t(q)) + double(psi_hat[k]) * gmr;
  const double thr = double(thr_psi) * gmr;
  if (fabs(e) > thr) {
    const uint8_t f = e < 0.0 ? 1 : 0;
    bound[p] = f;
    sflag[k] = f;
    margin[k] = float((fabs(e) - thr) / gmr);
    atomicAdd(gcount + q, 1u);
    atomicAdd(counters + 5, 1ull);
  } else {
    sflag[k] = 2;
    margin[k] = __int_as_float(0x7f800000);
    atomicAdd(ecount + q, 1u);
  }
}

// A node whose ungated share exceeds 1/4 is cheaper as a whole through the blocked direct sum.
__global__ void k_sur_full(int64_t nbig, const int64_t* __restrict__ big_nodes,
                           const int64_t* __restrict__ node_size, const unsigned int* __restrict__ ecount,
                           int* __restrict__ full, unsigned long long* __restrict__ counters) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nbig) return;
  const int64_t q = big_nodes[b];
  const bool f = 4 * int64_t(ecount[q]) > node_size[q];
  full[q] = f ? 1 : 0;
  if (f) atomicAdd(counters + 8, (unsigned long long)node_size[q]);
}

__global__ void k_sur_exact_list(int64_t ns, const uint32_t* __restrict__ sur_mem,
                                 const uint32_t* __restrict__ mnode, const uint8_t* __restrict__ sflag,
                                 const int* __restrict__ full, uint32_t* __restrict__ list,
                                 unsigned long long* __restrict__ counters) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  if (sflag[k] == 2 && !full[mnode[sur_mem[k]]]) list[atomicAdd(counters + 0, 1ull)] = uint32_t(k);
}

// Per big node (one block each): the k-th smallest margin (k = min(spot, gated) - 1) by radix
// select on the non-negative float bit patterns; threshold +inf marks "no gated member".
__global__ void __launch_bounds__(kT)
k_sur_select(const int64_t* __restrict__ big_nodes, const int64_t* __restrict__ sur_off,
             const int64_t* __restrict__ node_size, const unsigned int* __restrict__ gcount,
             const float* __restrict__ margin, int spot, const int* __restrict__ full,
             float* __restrict__ tau) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_prefix, s_k;
  const int64_t q = big_nodes[blockIdx.x];
  const int64_t lo = sur_off[q], g = node_size[q];
  const uint32_t ng = gcount[q];
  if (ng == 0 || spot <= 0 || full[q]) {
    if (threadIdx.x == 0) tau[q] = -1.0f;
    return;
  }
  if (threadIdx.x == 0) {
    s_prefix = 0;
    s_k = min(uint32_t(spot), ng) - 1;
  }
  uint32_t mask = 0;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0;
    __syncthreads();
    const uint32_t prefix = s_prefix;
    for (int64_t a = threadIdx.x; a < g; a += blockDim.x) {
      const uint32_t bits = __float_as_uint(margin[lo + a]);
      if ((bits & mask) == prefix) atomicAdd(&hist[(bits >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t kk = s_k, cum = 0;
      int d = 0;
      for (; d < 255; ++d) {
        if (cum + hist[d] > kk) break;
        cum += hist[d];
      }
      s_k = kk - cum;
      s_prefix = prefix | (uint32_t(d) << shift);
    }
    mask |= 255u << shift;
    __syncthreads();
  }
  if (threadIdx.x == 0) tau[q] = __uint_as_float(s_prefix);
}

__global__ void k_sur_spot_mark(int64_t ns, const uint32_t* __restrict__ sur_mem,
                                const uint32_t* __restrict__ mnode, const float* __restrict__ margin,
                                const uint8_t* __restrict__ sflag, const float* __restrict__ tau,
                                uint8_t* __restrict__ checked, uint32_t* __restrict__ check_list,
                                unsigned long long* __restrict__ counters) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t q = mnode[sur_mem[k]];
  const bool c = sflag[k] != 2 && margin[k] <= tau[q];
  checked[k] = c ? 1 : 0;
  if (c) check_list[atomicAdd(counters + 1, 1ull)] = uint32_t(k);
}

// Exact float32 potential of listed members (one warp each) and the certified flag; members
// whose energy is within the bound of zero are queued for the float64 potential.
__global__ void __launch_bounds__(kT)
k_pot_member(const unsigned long long* __restrict__ count, const uint32_t* __restrict__ list,
             const uint32_t* __restrict__ sur_mem, const uint32_t* __restrict__ mnode,
             const int64_t* __restrict__ node_off, const int64_t* __restrict__ node_size,
             const float4* __restrict__ U, const float4* __restrict__ V, const double* __restrict__ vbulk,
             float eps2, double Gm, float* __restrict__ Sx, uint8_t* __restrict__ bound,
             uint32_t* __restrict__ ambig, unsigned long long* __restrict__ n_ambig) {
  const int lane = threadIdx.x & 31;
  const unsigned long long total = *count;
  for (unsigned long long w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < total;
       w += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    const uint32_t k = list[w];
    const uint32_t p = sur_mem[k], q = mnode[p];
    const int64_t base = node_off[q], g = node_size[q], i = int64_t(p) - base;
    const float4 ui = U[p];
    float S = 0.f, C = 0.f;
    for (int64_t j0 = lane; j0 < g; j0 += 32 * 32) {
      float blk = 0.f;
#pragma unroll 4
      for (int t = 0; t < 32; ++t) {
        const int64_t j = j0 + 32 * t;
        if (j < g) {
          const float4 uj = U[base + j];
          const float dx = __fsub_rn(uj.x, ui.x);
          const float dy = __fsub_rn(uj.y, ui.y);
          const float dz = __fsub_rn(uj.z, ui.z);
          const float wv = rsqrtf(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmaf_rn(dz, dz, eps2))));
          blk = __fadd_rn(blk, j == i ? 0.f : wv);
        }
      }
      const float y = __fsub_rn(blk, C);
      const float tt = __fadd_rn(S, y);
      C = __fsub_rn(__fsub_rn(tt, S), y);
      S = tt;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) S = __fadd_rn(S, __shfl_xor_sync(0xffffffffu, S, off));
    if (lane == 0) {
      Sx[k] = S;
      const double ph = -__dmul_rn(Gm, double(S));
      const double e = __dadd_rn(kinetic(V[p], vbulk + 3 * int64_t(q)), ph);
      if (fabs(e) > __dmul_rn(2.0 * kCertB2, fabs(ph))) {
        bound[p] = e < 0.0 ? 1 : 0;
      } else {
        ambig[atomicAdd(n_ambig, 1ull)] = p;
      }
    }
  }
}

__global__ void k_sur_verdict(const unsigned long long* __restrict__ counters,
                              const uint32_t* __restrict__ check_list, const uint32_t* __restrict__ sur_mem,
                              const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_size,
                              const NodeStat* __restrict__ st, const float* __restrict__ Sx,
                              const float* __restrict__ psi_hat, const uint8_t* __restrict__ sflag,
                              const uint8_t* __restrict__ bound, float err_max, int* __restrict__ fail) {
  const unsigned long long total = counters[1];
  for (unsigned long long w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < total;
       w += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t k = check_list[w];
    const uint32_t p = sur_mem[k], q = mnode[p];
    const double psi = -double(Sx[k]) * double(st[q].r_vir) / double(node_size[q]);
    if (fabs(double(psi_hat[k]) - psi) > double(err_max) || sflag[k] != bound[p]) fail[q] = 1;
  }
}

__global__ void k_sur_rerun(int64_t ns, const uint32_t* __restrict__ sur_mem, const uint32_t* __restrict__ mnode,
                            const int* __restrict__ fail, const uint8_t* __restrict__ sflag,
                            const uint8_t* __restrict__ checked, uint32_t* __restrict__ list,
                            unsigned long long* __restrict__ counters) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t q = mnode[sur_mem[k]];
  if (fail[q] && sflag[k] != 2 && !checked[k]) list[atomicAdd(counters + 3, 1ull)] = uint32_t(k);
}

__global__ void k_count_fail(int64_t nn, const int* __restrict__ fail, unsigned long long* __restrict__ counters) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < nn && fail[q]) atomicAdd(counters + 4, 1ull);
}

__global__ void k_acc_counter(unsigned long long* __restrict__ counters, int from, int to) {
  counters[to] += counters[from];
  counters[from] = 0;
}

__global__ void k_big_list(int64_t nn, const int64_t* __restrict__ node_size,
                           const int64_t* __restrict__ rank, int64_t* __restrict__ big_nodes) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < nn && node_size[q] >= kSurMin) big_nodes[rank[q]] = q;
}

int bits_for(uint64_t v) {
  int b = 1;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

// k_fallback of rs_unbind.cu (float64 canonical-order potential of queued members)
}  // namespace

namespace rs {
int unbind_fallback(rs_ctx* ctx, const unsigned long long* n_ambig, const uint32_t* ambig,
                    const double* vbulk, uint8_t* bound, cudaStream_t st);
int unbind_nodes(rs_ctx* ctx, const int* only, const double* vbulk, uint8_t* bound,
                 uint32_t* ambig, unsigned long long* n_ambig, cudaStream_t st);

// Shared set-up: big-node member list, node statistics, radial sort, features.
// Returns the number of surrogate members through *ns_out (host).
static int sur_prepare(rs_ctx* ctx, const double* vbulk, int64_t* ns_out, cudaStream_t st) {
  Hier h = hier_of(ctx);
  const int64_t nn = ctx->n_nodes, m = ctx->n_members;
  int64_t* sur_off = scratch_t<int64_t>(ctx, S_SUR_OFF, size_t(nn) + 1);
  int64_t* rank = scratch_t<int64_t>(ctx, S_SUR_RANK, size_t(nn) + 1);
  NodeStat* stt = scratch_t<NodeStat>(ctx, S_SUR_STAT, size_t(nn));
  double* sums = scratch_t<double>(ctx, S_NODE_TMP, size_t(nn) * 9);
  if (!sur_off || !rank || !stt || !sums) return RS_ERR_OOM;
  k_sur_node_flags<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_size, sur_off, rank);
  RS_LAUNCHED(ctx, "k_sur_node_flags");
  RS_TRY(exclusive_scan_i64(ctx, nn, sur_off, sur_off + nn, st));
  RS_TRY(exclusive_scan_i64(ctx, nn, rank, rank + nn, st));
  RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box, sur_off + nn, 8, cudaMemcpyDeviceToHost, st));
  RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box + 1, rank + nn, 8, cudaMemcpyDeviceToHost, st));
  RS_CUDA(ctx, cudaStreamSynchronize(st));
  const int64_t ns = ctx->host_box[0], nbig = ctx->host_box[1];
  *ns_out = ns;
  ctx->sur_nbig = nbig;
  if (ns == 0) return RS_OK;
  RS_TRY((cro_segmented<9, StatTerm>(ctx, nn, h.node_off, h.node_size, m, StatTerm{h.U, h.V}, sums, st)));
  const double L = ctx->cfg.box_L;
  const double rho_bar = double(ctx->n_particles) * ctx->cfg.particle_mass / (L * L * L);
  k_sur_stats<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_size, sums, ctx->cfg.particle_mass, ctx->cfg.G,
                                              rho_bar, stt);
  RS_LAUNCHED(ctx, "k_sur_stats");
  uint32_t* sur_mem = scratch_t<uint32_t>(ctx, S_SUR_MEM, size_t(ns));
  int64_t* big_nodes = scratch_t<int64_t>(ctx, S_SUR_BIG, size_t(nbig) + 1);
  uint64_t* ka = scratch_t<uint64_t>(ctx, S_KEY_A, size_t(m));
  uint64_t* kb = scratch_t<uint64_t>(ctx, S_KEY_B, size_t(m));
  uint32_t* va = scratch_t<uint32_t>(ctx, S_VAL_A, size_t(m));
  uint32_t* vb = scratch_t<uint32_t>(ctx, S_VAL_B, size_t(m));
  float* feat = scratch_t<float>(ctx, S_SUR_FEAT, size_t(ns) * 8);
  float* psi_sph = scratch_t<float>(ctx, S_SUR_PSISPH, size_t(m));
  if (!sur_mem || !big_nodes || !ka || !kb || !va || !vb || !feat || !psi_sph) return RS_ERR_OOM;
  k_sur_members<<<grid_for(m, kT), kT, 0, st>>>(m, h.mnode, h.node_off, h.node_size, sur_off, sur_mem);
  RS_LAUNCHED(ctx, "k_sur_members");
  // rank holds the exclusive scan of big flags: rank of each big node
  k_big_list<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_size, rank, big_nodes);
  RS_LAUNCHED(ctx, "k_big_list");
  // radial order of every node's members (all levels)
  k_all_radius<<<grid_for(m, kT), kT, 0, st>>>(m, h.mnode, h.U, stt, ka, va);
  RS_LAUNCHED(ctx, "k_all_radius");
  uint64_t* rkeys;
  uint32_t* rvals;
  RS_TRY(radix_sort_u64(ctx, m, 32 + bits_for(uint64_t(nn)), ka, va, kb, vb, &rkeys, &rvals, st));
  ctx->sur_rkeys = rkeys;
  int64_t* fix = scratch_t<int64_t>(ctx, S_SUR_FIX, size_t(m) + 1);
  uint32_t* spos = scratch_t<uint32_t>(ctx, S_SUR_SPOS, size_t(m));
  if (!fix || !spos) return RS_ERR_OOM;
  const float eps = std::max(ctx->cfg.softening, 1e-6f);
  k_sur_inv_r<<<grid_for(m, kT), kT, 0, st>>>(m, rkeys, rvals, eps, fix, spos);
  RS_LAUNCHED(ctx, "k_sur_inv_r");
  RS_TRY(exclusive_scan_i64(ctx, m, fix, fix + m, st));
  k_psi_sph<<<grid_for(m, kT), kT, 0, st>>>(m, h.mnode, h.node_off, h.node_size, stt, h.U, fix, spos, eps,
                                           psi_sph);
  RS_LAUNCHED(ctx, "k_psi_sph");
  {
    ProfScope prof_(ctx, "k_sur_features", st);
    k_sur_features<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, h.node_off, h.node_size, h.U,
                                                   h.V, stt, vbulk, rkeys, psi_sph, h.mem, h.deepest,
                                                   h.deepest_pos, feat);
  }
  RS_LAUNCHED(ctx, "k_sur_features");
  return RS_OK;
}

int surrogate_unbind(rs_ctx* ctx, const double* vbulk, uint8_t* bound, unsigned long long* counters,
                     cudaStream_t st) {
  Hier h = hier_of(ctx);
  const int64_t nn = ctx->n_nodes;
  int64_t ns = 0;
  RS_TRY(sur_prepare(ctx, vbulk, &ns, st));
  ctx->sur_members = ns;
  if (ns == 0) return RS_OK;
  const NodeStat* stt = static_cast<const NodeStat*>(ctx->buf[S_SUR_STAT].ptr);
  const int64_t* sur_off = static_cast<const int64_t*>(ctx->buf[S_SUR_OFF].ptr);
  const uint32_t* sur_mem = static_cast<const uint32_t*>(ctx->buf[S_SUR_MEM].ptr);
  const int64_t* big_nodes = static_cast<const int64_t*>(ctx->buf[S_SUR_BIG].ptr);
  const float* feat = static_cast<const float*>(ctx->buf[S_SUR_FEAT].ptr);
  float* psi_hat = scratch_t<float>(ctx, S_SUR_PSI, size_t(ns));
  float* margin = scratch_t<float>(ctx, S_SUR_MARGIN, size_t(ns));
  uint8_t* sflag = scratch_t<uint8_t>(ctx, S_SUR_SFLAG, size_t(ns));
  uint8_t* checked = scratch_t<uint8_t>(ctx, S_SUR_CHECKED, size_t(ns));
  float* Sx = scratch_t<float>(ctx, S_SUR_SX, size_t(ns));
  uint32_t* exact_list = scratch_t<uint32_t>(ctx, S_SUR_LIST_A, size_t(ns));
  uint32_t* check_list = scratch_t<uint32_t>(ctx, S_SUR_LIST_B, size_t(ns));
  uint32_t* ambig = scratch_t<uint32_t>(ctx, S_U_AMBIG, size_t(ctx->n_members) + 1);
  unsigned int* gcount = scratch_t<unsigned int>(ctx, S_SUR_GCOUNT, size_t(nn));
  float* tau = scratch_t<float>(ctx, S_SUR_TAU, size_t(nn));
  int* fail = scratch_t<int>(ctx, S_SUR_FAIL, size_t(nn));
  unsigned int* ecount = scratch_t<unsigned int>(ctx, S_SUR_ECOUNT, size_t(nn));
  int* full = scratch_t<int>(ctx, S_SUR_FULL, size_t(nn));
  if (!psi_hat || !margin || !sflag || !checked || !Sx || !exact_list || !check_list || !ambig ||
      !gcount || !tau || !fail || !ecount || !full)
    return RS_ERR_OOM;
  RS_TRY(mlp_forward(ctx, ns, feat, psi_hat, st));
  RS_CUDA(ctx, cudaMemsetAsync(gcount, 0, 4 * nn, st));
  RS_CUDA(ctx, cudaMemsetAsync(ecount, 0, 4 * nn, st));
  RS_CUDA(ctx, cudaMemsetAsync(fail, 0, 4 * nn, st));
  RS_CUDA(ctx, cudaMemsetAsync(full, 0, 4 * nn, st));
  const float thr_psi = ctx->cfg.margin_factor * ctx->mlp_err_max;
  k_sur_gate<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, h.node_size, h.V, vbulk, stt, psi_hat,
                                             thr_psi, bound, sflag, margin, gcount, ecount, counters);
  RS_LAUNCHED(ctx, "k_sur_gate");
  if (ctx->sur_nbig > 0) {
    k_sur_full<<<grid_for(ctx->sur_nbig, kT), kT, 0, st>>>(ctx->sur_nbig, big_nodes, h.node_size, ecount,
                                                           full, counters);
    RS_LAUNCHED(ctx, "k_sur_full");
  }
  k_sur_exact_list<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, sflag, full, exact_list, counters);
  RS_LAUNCHED(ctx, "k_sur_exact_list");
  // nodes mostly outside the gate: whole-node blocked direct sum
  RS_TRY(unbind_nodes(ctx, full, vbulk, bound, ambig, counters + 2, st));
  k_acc_counter<<<1, 1, 0, st>>>(counters, 2, 7);
  RS_LAUNCHED(ctx, "k_acc_counter");
  if (ctx->sur_nbig > 0) {
    k_sur_select<<<unsigned(ctx->sur_nbig), kT, 0, st>>>(big_nodes, sur_off, h.node_size, gcount, margin,
                                                         ctx->cfg.spot_check, full, tau);
    RS_LAUNCHED(ctx, "k_sur_select");
  }
  k_sur_spot_mark<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, margin, sflag, tau, checked,
                                                  check_list, counters);
  RS_LAUNCHED(ctx, "k_sur_spot_mark");
  const double Gm = ctx->cfg.G * ctx->cfg.particle_mass;
  const float eps = ctx->cfg.softening;
  const unsigned grid = 152 * 8;
  // exact members, then the spot checks (counters 0 and 1), fp64 fallback after each pass
  for (int pass = 0; pass < 2; ++pass) {
    const uint32_t* list = pass == 0 ? exact_list : check_list;
    {
      ProfScope prof_(ctx, "k_pot_member", st);
      k_pot_member<<<grid, kT, 0, st>>>(counters + pass, list, sur_mem, h.mnode, h.node_off, h.node_size,
                                        h.U, h.V, vbulk, eps * eps, Gm, Sx, bound, ambig, counters + 2);
    }
    RS_LAUNCHED(ctx, "k_pot_member");
    RS_TRY(unbind_fallback(ctx, counters + 2, ambig, vbulk, bound, st));
    k_acc_counter<<<1, 1, 0, st>>>(counters, 2, 6);
    RS_LAUNCHED(ctx, "k_acc_counter");
  }
  k_sur_verdict<<<grid, kT, 0, st>>>(counters, check_list, sur_mem, h.mnode, h.node_size, stt, Sx, psi_hat,
                                     sflag, bound, ctx->mlp_err_max, fail);
  RS_LAUNCHED(ctx, "k_sur_verdict");
  k_sur_rerun<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, fail, sflag, checked, exact_list,
                                              counters);
  RS_LAUNCHED(ctx, "k_sur_rerun");
  {
    ProfScope prof_(ctx, "k_pot_member", st);
    k_pot_member<<<grid, kT, 0, st>>>(counters + 3, exact_list, sur_mem, h.mnode, h.node_off, h.node_size,
                                      h.U, h.V, vbulk, eps * eps, Gm, Sx, bound, ambig, counters + 2);
  }
  RS_LAUNCHED(ctx, "k_pot_member");
  RS_TRY(unbind_fallback(ctx, counters + 2, ambig, vbulk, bound, st));
  k_acc_counter<<<1, 1, 0, st>>>(counters, 2, 6);
  RS_LAUNCHED(ctx, "k_acc_counter");
  k_count_fail<<<grid_for(nn, kT), kT, 0, st>>>(nn, fail, counters);
  RS_LAUNCHED(ctx, "k_count_fail");
  return RS_OK;
}

}  // namespace rs

extern "C" int rs_surrogate_features(rs_ctx* ctx, float* feat_out, float* psi_out, int64_t* n_out,
                                     void* stream) {
  if (!ctx || !n_out) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (!ctx->have_hier || !ctx->have_unbind)
    return set_error(ctx, RS_ERR_STATE, "needs rs_fof6d and rs_unbind first");
  if (psi_out && ctx->last_unbind_surrogate)
    return set_error(ctx, RS_ERR_STATE, "targets need an rs_unbind without the surrogate");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  const double* vbulk = static_cast<const double*>(ctx->buf[S_U_VBULK].ptr);
  int64_t ns = 0;
  RS_TRY(sur_prepare(ctx, vbulk, &ns, st));
  *n_out = ns;
  if (ns == 0) return RS_OK;
  if (feat_out)
    RS_CUDA(ctx, cudaMemcpyAsync(feat_out, ctx->buf[S_SUR_FEAT].ptr, sizeof(float) * 8 * ns,
                                 cudaMemcpyDeviceToDevice, st));
  if (psi_out) {
    Hier h = hier_of(ctx);
    k_sur_targets<<<grid_for(ns, kT), kT, 0, st>>>(
        ns, static_cast<const uint32_t*>(ctx->buf[S_SUR_MEM].ptr), h.mnode, h.node_size,
        static_cast<const NodeStat*>(ctx->buf[S_SUR_STAT].ptr),
        static_cast<const float*>(ctx->buf[S_U_PHI].ptr), psi_out);
    RS_LAUNCHED(ctx, "k_sur_targets");
  }
  return RS_OK;
}

extern "C" int rs_surrogate_stats(rs_ctx* ctx, int64_t* stats_out) {
  if (!ctx || !stats_out) return RS_ERR_INVALID_ARG;
  for (int i = 0; i < 10; ++i) stats_out[i] = ctx->sur_stats[i];
  return RS_OK;
}

// Learned surrogate of the binding energy inside rs_unbind (batched + surrogate form).
//
// For every node with at least kSurMin members ("big" nodes), instead of the O(g^2) potential:
//   1. features per member (k_sur_features): r / r_vir, the enclosed-member fractions within
//      0.5, 1, 2 and 4 times the member's radius (binary searches in the node's radially sorted
//      members), |v - v_bulk| / sigma_v,1D, log10 g, and in the eighth input the node's
//      potential at the member from the radially split multipole expansion to quadrupole order
//      (psi_mp: monopole = spherically averaged node, plus the dipole and quadrupole moments of
//      the members inside and outside the member's radius, from fixed-point prefix sums over
//      the radial order); r is measured from the node's mean position,
//      r_vir = (3 g m / (4 pi 200 rho_bar))^(1/3);
//   2. the MLP predicts psi = phi r_vir / (G g m); E_pred = KE + psi_hat G g m / r_vir;
//   3. gate (k_sur_gate): a member is classified by the surrogate iff
//      |E_pred| > margin_factor * err * G g m / r_vir, with err the MLP's held-out maximum error
//      from training (err_max: the default gate), or, opted in (surrogate_gate = 1), a per-node
//      calibrated error: kCalib members of the node evenly spaced in member order are evaluated
//      exactly and err = max(their max |psi_hat - psi|, err_max / 8);
//   4. every other member takes the exact path: the certified tree bound for nodes with a tree,
//      a register-blocked float32 sum over the node for the list of such members (with the self
//      term included and subtracted, and a per-member certified bound), the float64
//      canonical-order potential when the energy is within that bound of zero; a node with at
//      most 1/20 of its members gated goes whole to the exact path;
//   5. spot check: per node, the spot_check gated members with the smallest margin and about
//      spot_check more drawn at every margin (a seeded hash of the member position) are also
//      evaluated exactly; if any has a different flag (counted), or |psi_hat - psi| above half
//      the gate's margin, the whole node is recomputed exactly.
// Zero flag mismatches against the exact path is a measured result (the tests compare every
// member's flag on held-out snapshots), not a guarantee: a member the network mispredicts by
// more than the margin and that no spot check samples keeps a wrong flag.
#include <cmath>

#include "rs_exact.cuh"

namespace rs {
int mlp_forward(rs_ctx* ctx, int64_t n, const float* x, float* y, cudaStream_t st);
int surrogate_unbind(rs_ctx* ctx, const double* vbulk, uint8_t* bound, unsigned long long* counters,
                     cudaStream_t st);
}  // namespace rs

using namespace rs;

namespace {

constexpr int kT = 256;
constexpr int64_t kSurMin = kSurrogateMinMembers;
constexpr int64_t kTuneMinSurMembers = 1 << 20;  // the autotuner times candidates on lists this large

struct NodeStat {
  float cx, cy, cz, r_vir;
  float sig_v1d, log_g, pad0, pad1;
  double gm_over_rvir;
  double pad2;
};

__global__ void k_sur_node_flags(int64_t nn, const int64_t* __restrict__ node_size,
                                 int64_t* __restrict__ szm, int64_t* __restrict__ bigf) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nn) return;
  const bool big = node_size[q] >= kSurMin;
  szm[q] = big ? node_size[q] : 0;
  bigf[q] = big ? 1 : 0;
}

// Node statistics of the features: centre and sigma_v,1D from the moments of the node's 6D
// split (canonical-order float64 sums of u and v), r_vir from g.
__global__ void k_sur_stats(int64_t nn, const int64_t* __restrict__ node_size, const float4* __restrict__ mom,
                            double m, double G, double rho_bar, NodeStat* __restrict__ st) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nn) return;
  const double g = double(node_size[q]);
  const float4 M = mom[q];
  NodeStat s;
  s.cx = M.x;
  s.cy = M.y;
  s.cz = M.z;
  s.sig_v1d = M.w;
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

// Radial sort key of every surrogate member k (surrogate order is node-grouped): the big
// node's rank above the radius bits (31: a radius is never negative), so each node's members stay in their range
// [sur_off[q], sur_off[q] + g) after sorting.
__global__ void k_big_radius(int64_t ns, const uint32_t* __restrict__ sur_mem, const uint32_t* __restrict__ mnode,
                             const int64_t* __restrict__ big_rank, const float4* __restrict__ U,
                             const NodeStat* __restrict__ st, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t p = sur_mem[k], q = mnode[p];
  const float r = member_radius(U[p], st[q]);
  keys[k] = (uint64_t(big_rank[q]) << 31) | uint64_t(__float_as_uint(r));  // r >= 0: 31 bits
  vals[k] = uint32_t(k);
}

__device__ __forceinline__ int64_t count_below(const uint64_t* __restrict__ rkeys, int64_t lo, int64_t hi,
                                               float v) {
  // members of the segment whose radius is < v (radius bits are the low 31 bits of the keys)
  const int64_t base = lo;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (__uint_as_float(uint32_t(rkeys[mid] & 0x7fffffffull)) < v) lo = mid + 1; else hi = mid;
  }
  return lo - base;
}

constexpr double kFix = 16777216.0;  // 2^24: fixed-point scale of the 1/r suffix sums

// Per radially sorted position s: fixed-point 1 / max(r, eps) (to be prefix-summed) and the
// sorted position of each surrogate member (spos[k]).
__global__ void k_sur_inv_r(int64_t ns, const uint64_t* __restrict__ rkeys, const uint32_t* __restrict__ rvals,
                            float eps, int64_t* __restrict__ fix, uint32_t* __restrict__ spos) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const float r = __uint_as_float(uint32_t(rkeys[s] & 0x7fffffffull));
  fix[s] = llrint(kFix / double(fmaxf(r, eps)));
  spos[rvals[s]] = uint32_t(s);
}

// psi_sph of every surrogate member k: the potential of the spherically averaged node at the
// member, in units of G g m / r_vir: -(r_vir / g) (#inside / max(r, eps) + sum over members
// outside of 1 / max(r_j, eps)), from the radially sorted member ranges.
__global__ void k_psi_sph(int64_t ns, const uint32_t* __restrict__ sur_mem, const uint32_t* __restrict__ mnode,
                          const int64_t* __restrict__ sur_off, const int64_t* __restrict__ node_size,
                          const NodeStat* __restrict__ st, const float4* __restrict__ U,
                          const int64_t* __restrict__ fix, const uint32_t* __restrict__ spos, float eps,
                          float* __restrict__ psi_sph) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t p = sur_mem[k], q = mnode[p];
  const NodeStat s = st[q];
  const int64_t g = node_size[q], lo = sur_off[q], hi = lo + g;
  const int64_t si = spos[k];
  const float outer = float(fix[hi] - fix[si + 1]) * (1.0f / float(kFix));
  const float inner = float(si - lo) / fmaxf(member_radius(U[p], s), eps);
  psi_sph[k] = -(s.r_vir / float(g)) * (inner + outer);
}

constexpr float kFixIn = 16777216.0f;  // 2^24: scale of the inner moment sums
constexpr float kFixOut = 65536.0f;    // 2^16: scale of the outer moment sums
constexpr int kMpTerms = 18;

// Multipole terms of every surrogate member at its radially sorted position c (the node's
// range is [sur_off[q], sur_off[q] + g)), with x = u - centre, r = |x|, rr = max(r, eps):
// inner (scale 2^24): x (3), T = 3 x x^T - r^2 I (xx, yy, zz, xy, xz, yz);
// outer (scale 2^16): x / rr^3 (3), T / rr^5 (6). Float32 terms rounded to int64 fixed point,
// so the prefix sums are exact and independent of the scan's order. Row t of `terms` has
// ns + 1 entries (the last one 0); the rows are prefix-summed as one array, since only
// differences inside a row are used.
__global__ void k_mp_terms(const uint32_t* __restrict__ rvals, const uint32_t* __restrict__ sur_mem,
                           const uint32_t* __restrict__ mnode, const NodeStat* __restrict__ st,
                           const float4* __restrict__ U, float eps, int64_t ns, int64_t* __restrict__ terms) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c < kMpTerms) terms[c * (ns + 1) + ns] = 0;  // the slot after each row
  if (c >= ns) return;
  const uint32_t p = sur_mem[rvals[c]], q = mnode[p];
  const NodeStat S = st[q];
  const float4 u = U[p];
  const float x = u.x - S.cx, y = u.y - S.cy, z = u.z - S.cz;
  const float r2 = x * x + y * y + z * z;
  const float rr = fmaxf(sqrtf(r2), eps);
  const float i3 = 1.0f / (rr * rr * rr), i5 = i3 / (rr * rr);
  const float T[6] = {3 * x * x - r2, 3 * y * y - r2, 3 * z * z - r2, 3 * x * y, 3 * x * z, 3 * y * z};
  const float v[kMpTerms] = {x * kFixIn, y * kFixIn, z * kFixIn,
                             T[0] * kFixIn, T[1] * kFixIn, T[2] * kFixIn,
                             T[3] * kFixIn, T[4] * kFixIn, T[5] * kFixIn,
                             x * i3 * kFixOut, y * i3 * kFixOut, z * i3 * kFixOut,
                             T[0] * i5 * kFixOut, T[1] * i5 * kFixOut, T[2] * i5 * kFixOut,
                             T[3] * i5 * kFixOut, T[4] * i5 * kFixOut, T[5] * i5 * kFixOut};
#pragma unroll
  for (int t = 0; t < kMpTerms; ++t) terms[int64_t(t) * (ns + 1) + c] = llrintf(v[t]);
}

// psi_mp of surrogate member k: psi_sph plus the dipole and quadrupole terms of the radially
// split expansion, -(r_vir / g) [x.D_in / rr^3 + x.D_out + (x^T Q_in x / rr^5 + x^T Q_out x) / 2],
// D_in, Q_in over the members before it in the radial order, D_out, Q_out over those after it.
__device__ __forceinline__ float psi_multipole(const int64_t* __restrict__ terms, int64_t ns, int64_t lo,
                                               int64_t hi, int64_t c, float4 u, const NodeStat& S,
                                               float eps, int64_t g, float psi_sph) {
  const float x = u.x - S.cx, y = u.y - S.cy, z = u.z - S.cz;
  const float rr = fmaxf(sqrtf(x * x + y * y + z * z), eps);
  float a[kMpTerms];
#pragma unroll
  for (int t = 0; t < kMpTerms; ++t) {
    const int64_t* row = terms + int64_t(t) * (ns + 1);
    a[t] = t < 9 ? float(row[c] - row[lo]) * (1.0f / kFixIn) : float(row[hi] - row[c + 1]) * (1.0f / kFixOut);
  }
  const float quad_in = a[3] * x * x + a[4] * y * y + a[5] * z * z + 2 * (a[6] * x * y + a[7] * x * z + a[8] * y * z);
  const float quad_out = a[12] * x * x + a[13] * y * y + a[14] * z * z +
                         2 * (a[15] * x * y + a[16] * x * z + a[17] * y * z);
  const float r3 = rr * rr * rr;
  const float dip = (a[0] * x + a[1] * y + a[2] * z) / r3 + (a[9] * x + a[10] * y + a[11] * z);
  const float quad = 0.5f * (quad_in / (r3 * rr * rr) + quad_out);
  return psi_sph - (S.r_vir / float(g)) * (dip + quad);
}

// Features of surrogate member k, in this order: r / r_vir; fractions of the node's members
// with radius below 0.5 r, r, 2 r and 4 r; |v - v_bulk| / sigma_v,1D; log10 g; and psi_mp, the
// node's potential at the member from the radially split multipole expansion.
__global__ void k_sur_features(int64_t ns, const uint32_t* __restrict__ sur_mem,
                               const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_size,
                               const float4* __restrict__ U, const float4* __restrict__ V,
                               const NodeStat* __restrict__ st, const double* __restrict__ vbulk,
                               const uint64_t* __restrict__ rkeys, const float* __restrict__ psi_sph,
                               const int64_t* __restrict__ sur_off, const uint32_t* __restrict__ spos,
                               const int64_t* __restrict__ terms, float eps, float* __restrict__ feat) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t p = sur_mem[k], q = mnode[p];
  const NodeStat s = st[q];
  const int64_t g = node_size[q], lo = sur_off[q], hi = lo + g;
  const float r = member_radius(U[p], s);
  const float inv_g = 1.0f / float(g);
  const float4 v = V[p];
  const float dvx = v.x - float(vbulk[3 * q]), dvy = v.y - float(vbulk[3 * q + 1]),
              dvz = v.z - float(vbulk[3 * q + 2]);
  float* F = feat + 8 * k;
  F[0] = r / s.r_vir;
  F[1] = float(count_below(rkeys, lo, hi, 0.5f * r)) * inv_g;
  F[2] = float(count_below(rkeys, lo, hi, r)) * inv_g;
  F[3] = float(count_below(rkeys, lo, hi, 2.0f * r)) * inv_g;
  F[4] = float(count_below(rkeys, lo, hi, 4.0f * r)) * inv_g;
  F[5] = sqrtf(dvx * dvx + dvy * dvy + dvz * dvz) / fmaxf(s.sig_v1d, 1e-30f);
  F[6] = s.log_g;
  F[7] = psi_multipole(terms, ns, lo, hi, int64_t(spos[k]), U[p], s, eps, g, psi_sph[k]);
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

// counters: [0] exact per-member list, [1] check list, [2] fp64 list (current pass), [3] rerun
// list, [4] failed nodes, [5] gated, [6] fp64 total (surrogate path), [7] fp64 of the direct
// sums, [8] members of nodes sent whole to the direct sum
__global__ void k_sur_gate(int64_t ns, const uint32_t* __restrict__ sur_mem, const uint32_t* __restrict__ mnode,
                           const int64_t* __restrict__ node_size, const float4* __restrict__ V,
                           const double* __restrict__ vbulk, const NodeStat* __restrict__ st,
                           const float* __restrict__ psi_hat, const float* __restrict__ errn, float err_floor,
                           float margin_factor, uint8_t* __restrict__ bound, uint8_t* __restrict__ sflag,
                           float* __restrict__ margin, unsigned int* __restrict__ gcount,
                           unsigned int* __restrict__ ecount, unsigned long long* __restrict__ counters) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  // every lane stays to the end for the warp-aggregated counters
  const bool in = k < ns;
  const bool calib = in && sflag[k] == 3;  // calibration member: exact already
  const uint32_t p = in ? sur_mem[k] : 0u, q = in ? mnode[p] : 0u;
  bool gated = false;
  if (in && !calib) {
    // predicted energy in units of G g m / r_vir, float32 (the gate's margin dwarfs its rounding)
    const float inv_gmr = float(1.0 / st[q].gm_over_rvir);
    const float4 v = V[p];
    const float dvx = v.x - float(vbulk[3 * q]), dvy = v.y - float(vbulk[3 * q + 1]),
                dvz = v.z - float(vbulk[3 * q + 2]);
    const float e = 0.5f * (dvx * dvx + dvy * dvy + dvz * dvz) * inv_gmr + psi_hat[k];
    const float thr = margin_factor * (errn ? fmaxf(errn[q], err_floor) : err_floor);
    if (fabsf(e) > thr) {
      const uint8_t f = e < 0.f ? 1 : 0;
      bound[p] = f;
      sflag[k] = f;
      margin[k] = fabsf(e) - thr;
      gated = true;
    } else {
      sflag[k] = 2;
      margin[k] = __int_as_float(0x7f800000);
    }
  }
  if (calib) margin[k] = __int_as_float(0x7f800000);
  rsd::warp_run_add(gcount, q, gated, 1u);
  rsd::warp_run_add(ecount, q, in && !calib && !gated, 1u);
  rsd::warp_count(counters + 5, gated);
}

// Calibration members: kCalib per big node, evenly spaced in member order (sflag = 3).
constexpr int kCalib = 64;
static_assert(kCalib % 4 == 0, "k_pot_member4 groups the calibration list by 4 members of one node");

__global__ void k_sur_calib_list(int64_t nbig, const int64_t* __restrict__ big_nodes,
                                 const int64_t* __restrict__ sur_off, const int64_t* __restrict__ node_size,
                                 uint32_t* __restrict__ list, uint8_t* __restrict__ sflag,
                                 unsigned long long* __restrict__ counters) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t == 0) counters[9] = (unsigned long long)(nbig * kCalib);
  if (t >= nbig * kCalib) return;
  const int64_t b = t / kCalib, i = t % kCalib, q = big_nodes[b], g = node_size[q];
  const int64_t k = sur_off[q] + (i * (g - 1)) / (kCalib - 1);
  list[t] = uint32_t(k);
  sflag[k] = 3;
}

// err_node[q] = max over the node's calibration members of |psi_hat - psi| (float bits of a
// non-negative value, so the integer maximum is the float maximum and order-independent).
__global__ void k_sur_err(const unsigned long long* __restrict__ count, const uint32_t* __restrict__ list,
                          const uint32_t* __restrict__ sur_mem, const uint32_t* __restrict__ mnode,
                          const int64_t* __restrict__ node_size, const NodeStat* __restrict__ st,
                          const float* __restrict__ Sx, const float* __restrict__ psi_hat,
                          unsigned int* __restrict__ errn) {
  const int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= int64_t(*count)) return;
  const uint32_t k = list[w];
  const uint32_t q = mnode[sur_mem[k]];
  const double psi = -double(Sx[k]) * double(st[q].r_vir) / double(node_size[q]);
  const float e = float(fabs(double(psi_hat[k]) - psi));
  atomicMax(errn + q, __float_as_uint(e));
}

// A node with at most 1/20 of its members gated goes whole through the blocked direct sum.
__global__ void k_sur_full(int64_t nbig, const int64_t* __restrict__ big_nodes,
                           const int64_t* __restrict__ node_size, const unsigned int* __restrict__ ecount,
                           int ncalib, int* __restrict__ full, unsigned long long* __restrict__ counters) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nbig) return;
  const int64_t q = big_nodes[b], g = node_size[q];
  const bool f = 20 * (int64_t(ecount[q]) + ncalib) >= 19 * g;
  full[q] = f ? 1 : 0;
  if (f) atomicAdd(counters + 8, (unsigned long long)g);
}

// Ungated members of nodes not sent whole: the exact-path list (lf), except in nodes with a
// certified tree (tmin > 0, at least tmin members), whose members are marked in `want` for it.
__global__ void k_sur_exact_flags(int64_t ns, const uint32_t* __restrict__ sur_mem,
                                  const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_size,
                                  const uint8_t* __restrict__ sflag, const int* __restrict__ full,
                                  int64_t tmin, int64_t* __restrict__ lf, uint8_t* __restrict__ want) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t p = sur_mem[k], q = mnode[p];
  const bool open = sflag[k] == 2 && !full[q];
  const bool tree = tmin > 0 && node_size[q] >= tmin;
  lf[k] = (open && !tree) ? 1 : 0;
  if (want) want[p] = (open && tree) ? 1 : 0;
}

// Exact-path list in surrogate-member order (so grouped by node), per-node list offsets and
// the blocked kernel's tile counts per big node.
__global__ void k_sur_exact_list(int64_t ns, const int64_t* __restrict__ lf, uint32_t* __restrict__ list,
                                 unsigned long long* __restrict__ counters) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k == 0) counters[0] = (unsigned long long)lf[ns];
  if (k >= ns) return;
  if (lf[k + 1] != lf[k]) list[lf[k]] = uint32_t(k);
}

__global__ void k_sur_list_tiles(int64_t nbig, const int64_t* __restrict__ big_nodes,
                                 const int64_t* __restrict__ sur_off, const int64_t* __restrict__ node_size,
                                 const int64_t* __restrict__ lf, int list_tile, int64_t* __restrict__ lofs,
                                 int64_t* __restrict__ tiles, unsigned long long* __restrict__ list_pairs) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nbig) return;
  const int64_t q = big_nodes[b];
  const int64_t a = lf[sur_off[q]], e = lf[sur_off[q] + node_size[q]];
  lofs[b] = a;
  tiles[b] = (e - a + list_tile - 1) / list_tile;
  if (list_pairs && e > a) atomicAdd(list_pairs, (unsigned long long)((e - a) * node_size[q]));
}

__global__ void k_sur_list_end(int64_t nbig, const int64_t* __restrict__ big_nodes,
                               const int64_t* __restrict__ sur_off, const int64_t* __restrict__ node_size,
                               const int64_t* __restrict__ lf, int64_t* __restrict__ lend) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nbig) return;
  const int64_t q = big_nodes[b];
  lend[b] = lf[sur_off[q] + node_size[q]];
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

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", 2014)
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// Spot-checked gated members: the `spot` of smallest margin (margin <= tau) and, at every
// margin, a seeded pseudo-random sample of about `spot` more (hash of the member position).
__global__ void k_sur_spot_mark(int64_t ns, const uint32_t* __restrict__ sur_mem,
                                const uint32_t* __restrict__ mnode, const float* __restrict__ margin,
                                const uint8_t* __restrict__ sflag, const float* __restrict__ tau,
                                const unsigned int* __restrict__ gcount, int spot, const int* __restrict__ full,
                                uint8_t* __restrict__ checked, uint32_t* __restrict__ check_list,
                                unsigned long long* __restrict__ counters) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t p = sur_mem[k], q = mnode[p];
  const uint64_t period = spot > 0 ? uint64_t(max(1u, gcount[q] / uint32_t(spot))) : 0;
  const bool sampled = period > 0 && !full[q] && splitmix64(uint64_t(p) ^ 0x5eedull) % period == 0;
  const bool c = sflag[k] < 2 && (margin[k] <= tau[q] || sampled);
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

// k_pot_member for groups of 4 consecutive list entries of the same node (the calibration
// list: 64 per node): one warp per group shares every target load among the 4 members; each
// member's sum has the same per-lane order as k_pot_member (bit-identical result).
__global__ void __launch_bounds__(kT)
k_pot_member4(const unsigned long long* __restrict__ count, const uint32_t* __restrict__ list,
              const uint32_t* __restrict__ sur_mem, const uint32_t* __restrict__ mnode,
              const int64_t* __restrict__ node_off, const int64_t* __restrict__ node_size,
              const float4* __restrict__ U, const float4* __restrict__ V, const double* __restrict__ vbulk,
              float eps2, double Gm, float* __restrict__ Sx, uint8_t* __restrict__ bound,
              uint32_t* __restrict__ ambig, unsigned long long* __restrict__ n_ambig) {
  const int lane = threadIdx.x & 31;
  const unsigned long long total = *count / 4;
  for (unsigned long long w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < total;
       w += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    uint32_t k[4], p[4];
    int64_t i[4];
    float4 ui[4];
    float S[4], C[4];
    const uint32_t q = mnode[sur_mem[list[4 * w]]];
    const int64_t base = node_off[q], g = node_size[q];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      k[r] = list[4 * w + r];
      p[r] = sur_mem[k[r]];
      i[r] = int64_t(p[r]) - base;
      ui[r] = U[p[r]];
      S[r] = 0.f;
      C[r] = 0.f;
    }
    for (int64_t j0 = lane; j0 < g; j0 += 32 * 32) {
      float blk[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
      for (int t = 0; t < 32; ++t) {
        const int64_t j = j0 + 32 * t;
        if (j < g) {
          const float4 uj = U[base + j];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float dx = __fsub_rn(uj.x, ui[r].x);
            const float dy = __fsub_rn(uj.y, ui[r].y);
            const float dz = __fsub_rn(uj.z, ui[r].z);
            const float wv = rsqrtf(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmaf_rn(dz, dz, eps2))));
            blk[r] = __fadd_rn(blk[r], j == i[r] ? 0.f : wv);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float y = __fsub_rn(blk[r], C[r]);
        const float tt = __fadd_rn(S[r], y);
        C[r] = __fsub_rn(__fsub_rn(tt, S[r]), y);
        S[r] = tt;
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) S[r] = __fadd_rn(S[r], __shfl_xor_sync(0xffffffffu, S[r], off));
    }
    if (lane < 4) {
      const float Sr = lane == 0 ? S[0] : lane == 1 ? S[1] : lane == 2 ? S[2] : S[3];
      const uint32_t kr = k[lane], pr = p[lane];
      Sx[kr] = Sr;
      const double ph = -__dmul_rn(Gm, double(Sr));
      const double e = __dadd_rn(kinetic(V[pr], vbulk + 3 * int64_t(q)), ph);
      if (fabs(e) > __dmul_rn(2.0 * kCertB2, fabs(ph))) {
        bound[pr] = e < 0.0 ? 1 : 0;
      } else {
        ambig[atomicAdd(n_ambig, 1ull)] = pr;
      }
    }
  }
}

__global__ void k_sur_verdict(unsigned long long* __restrict__ counters,
                              const uint32_t* __restrict__ check_list, const uint32_t* __restrict__ sur_mem,
                              const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_size,
                              const NodeStat* __restrict__ st, const float* __restrict__ Sx,
                              const float* __restrict__ psi_hat, const uint8_t* __restrict__ sflag,
                              const uint8_t* __restrict__ bound, const float* __restrict__ errn,
                              float err_floor, float margin_factor, int* __restrict__ fail) {
  const unsigned long long total = counters[1];
  for (unsigned long long w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < total;
       w += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t k = check_list[w];
    const uint32_t p = sur_mem[k], q = mnode[p];
    const double psi = -double(Sx[k]) * double(st[q].r_vir) / double(node_size[q]);
    const double err = 0.5 * double(margin_factor) * double(errn ? fmaxf(errn[q], err_floor) : err_floor);
    const bool flag_differs = sflag[k] != bound[p];
    if (flag_differs) atomicAdd(counters + 19, 1ull);
    if (fabs(double(psi_hat[k]) - psi) > err || flag_differs) fail[q] = 1;
  }
}

// Gated, unchecked members of nodes that failed the spot check (recomputed with their node).
__global__ void k_sur_rerun(int64_t ns, const uint32_t* __restrict__ sur_mem, const uint32_t* __restrict__ mnode,
                            const int* __restrict__ fail, const uint8_t* __restrict__ sflag,
                            const uint8_t* __restrict__ checked, unsigned long long* __restrict__ counters) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const uint32_t q = mnode[sur_mem[k]];
  if (fail[q] && sflag[k] < 2 && !checked[k]) atomicAdd(counters + 3, 1ull);
}

// Members whose flag the surrogate decided (gated, in a node neither sent whole to the direct
// sum nor failed, and not spot-checked) -> counters[10]; calibration members of nodes not sent
// whole -> counters[11].
__global__ void k_sur_decided(int64_t ns, const uint32_t* __restrict__ sur_mem, const uint32_t* __restrict__ mnode,
                              const uint8_t* __restrict__ sflag, const uint8_t* __restrict__ checked,
                              const int* __restrict__ full, const int* __restrict__ fail,
                              unsigned long long* __restrict__ counters) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool in = k < ns;
  const uint32_t q = in ? mnode[sur_mem[k]] : 0u;
  const bool keep = in && !full[q];
  rsd::warp_count(counters + 10, keep && sflag[k] < 2 && !checked[k] && !fail[q]);
  rsd::warp_count(counters + 11, keep && sflag[k] == 3);
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

// Sort keys of the big nodes: largest size class first (stable: node order within a class).
__global__ void k_big_keys(int64_t nbig, const int64_t* __restrict__ big_nodes,
                           const int64_t* __restrict__ node_size, uint64_t* __restrict__ keys,
                           uint32_t* __restrict__ vals) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nbig) return;
  keys[b] = 255u - rsd::size_class(node_size[big_nodes[b]]);
  vals[b] = uint32_t(big_nodes[b]);
}

__global__ void k_big_store(int64_t nbig, const uint32_t* __restrict__ vals, int64_t* __restrict__ big_nodes) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b < nbig) big_nodes[b] = int64_t(vals[b]);
}

int bits_for(uint64_t v) {
  int b = 1;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

// The float64 canonical-order potential of queued members (rs_unbind.cu)
}  // namespace

namespace rs {
int unbind_fallback(rs_ctx* ctx, const unsigned long long* n_ambig, const uint32_t* ambig,
                    const double* vbulk, uint8_t* bound, cudaStream_t st, float* phi_out = nullptr);
int unbind_nodes(rs_ctx* ctx, const int* only, const double* vbulk, uint8_t* bound,
                 uint32_t* ambig, unsigned long long* n_ambig, cudaStream_t st,
                 unsigned long long* counters);
int tree_decide(rs_ctx* ctx, const int* only, const uint8_t* want, const double* vbulk,
                uint8_t* bound, unsigned long long* counters, cudaStream_t st);

// Shared set-up: big-node member list, node statistics, radial sort, features.
// Returns the number of surrogate members through *ns_out (host).
static int sur_prepare(rs_ctx* ctx, const double* vbulk, int64_t* ns_out, cudaStream_t st) {
  Hier h = hier_of(ctx);
  const int64_t nn = ctx->n_nodes, m = ctx->n_members;
  int64_t* sur_off = scratch_t<int64_t>(ctx, S_SUR_OFF, size_t(nn) + 1);
  int64_t* rank = scratch_t<int64_t>(ctx, S_SUR_RANK, size_t(nn) + 1);
  NodeStat* stt = scratch_t<NodeStat>(ctx, S_SUR_STAT, size_t(nn));
  if (!sur_off || !rank || !stt) return RS_ERR_OOM;
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
  const double L = ctx->cfg.box_L;
  const double rho_bar = double(ctx->n_particles) * ctx->cfg.particle_mass / (L * L * L);
  k_sur_stats<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_size, h.mom, ctx->cfg.particle_mass, ctx->cfg.G,
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
  {  // big nodes largest first, so the per-node work of the surrogate path starts with them
    uint64_t* bka = scratch_t<uint64_t>(ctx, S_U_OKEY_A, size_t(nbig));
    uint64_t* bkb = scratch_t<uint64_t>(ctx, S_U_OKEY_B, size_t(nbig));
    uint32_t* bva = scratch_t<uint32_t>(ctx, S_U_OVAL_A, size_t(nbig));
    uint32_t* bvb = scratch_t<uint32_t>(ctx, S_U_OVAL_B, size_t(nbig));
    if (!bka || !bkb || !bva || !bvb) return RS_ERR_OOM;
    k_big_keys<<<grid_for(nbig, kT), kT, 0, st>>>(nbig, big_nodes, h.node_size, bka, bva);
    RS_LAUNCHED(ctx, "k_big_keys");
    uint64_t* bko;
    uint32_t* bvo;
    RS_TRY(radix_sort_u64(ctx, nbig, 8, bka, bva, bkb, bvb, &bko, &bvo, st));
    k_big_store<<<grid_for(nbig, kT), kT, 0, st>>>(nbig, bvo, big_nodes);
    RS_LAUNCHED(ctx, "k_big_store");
  }
  // radial order of the surrogate members inside their node
  k_big_radius<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, rank, h.U, stt, ka, va);
  RS_LAUNCHED(ctx, "k_big_radius");
  uint64_t* rkeys;
  uint32_t* rvals;
  RS_TRY(radix_sort_u64(ctx, ns, 31 + bits_for(uint64_t(nbig)), ka, va, kb, vb, &rkeys, &rvals, st));
  ctx->sur_rkeys = rkeys;
  int64_t* fix = scratch_t<int64_t>(ctx, S_SUR_FIX, size_t(ns) + 1);
  uint32_t* spos = scratch_t<uint32_t>(ctx, S_SUR_SPOS, size_t(ns));
  if (!fix || !spos) return RS_ERR_OOM;
  const float eps = std::max(ctx->cfg.softening, 1e-6f);
  k_sur_inv_r<<<grid_for(ns, kT), kT, 0, st>>>(ns, rkeys, rvals, eps, fix, spos);
  RS_LAUNCHED(ctx, "k_sur_inv_r");
  RS_TRY(exclusive_scan_i64(ctx, ns, fix, fix + ns, st));
  k_psi_sph<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, sur_off, h.node_size, stt, h.U, fix, spos,
                                            eps, psi_sph);
  RS_LAUNCHED(ctx, "k_psi_sph");
  const int64_t nterms = int64_t(kMpTerms) * (ns + 1);
  int64_t* terms = scratch_t<int64_t>(ctx, S_SUR_MP, size_t(nterms) + 1);
  if (!terms) return RS_ERR_OOM;
  k_mp_terms<<<grid_for(std::max<int64_t>(ns, kMpTerms), kT), kT, 0, st>>>(rvals, sur_mem, h.mnode, stt, h.U,
                                                                         eps, ns, terms);
  RS_LAUNCHED(ctx, "k_mp_terms");
  RS_TRY(exclusive_scan_i64(ctx, nterms, terms, terms + nterms, st));
  {
    ProfScope prof_(ctx, "k_sur_features", st);
    k_sur_features<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, h.node_size, h.U, h.V, stt,
                                                   vbulk, rkeys, psi_sph, sur_off, spos, terms, eps,
                                                   feat);
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
  const int64_t nbig = ctx->sur_nbig;
  unsigned int* errn = scratch_t<unsigned int>(ctx, S_SUR_ERRN, size_t(nn));
  uint32_t* calib_list = scratch_t<uint32_t>(ctx, S_SUR_LIST_C, size_t(nbig) * kCalib + 1);
  int64_t* lf = scratch_t<int64_t>(ctx, S_SUR_LSCAN, size_t(ns) + 1);
  int64_t* lofs = scratch_t<int64_t>(ctx, S_SUR_LOFS, size_t(nbig) * 2 + 2);
  int64_t* ltiles = scratch_t<int64_t>(ctx, S_SUR_TILES, size_t(nbig) + 1);
  if (!errn || !calib_list || !lf || !lofs || !ltiles) return RS_ERR_OOM;
  int64_t* lend = lofs + nbig + 1;
  const double Gm = ctx->cfg.G * ctx->cfg.particle_mass;
  const float eps = ctx->cfg.softening;
  const unsigned grid = 152 * 8;
  // gate: the benchmark spec's held-out maximum error of the training (err_max), or, opted in, the
  // per-node calibrated error with err_max / 8 as its floor
  const bool calibrated = ctx->cfg.surrogate_gate == 1;
  const float err_floor = calibrated ? ctx->mlp_err_max / 8.0f : ctx->mlp_err_max;
  RS_TRY(mlp_forward(ctx, ns, feat, psi_hat, st));
  RS_CUDA(ctx, cudaMemsetAsync(gcount, 0, 4 * nn, st));
  RS_CUDA(ctx, cudaMemsetAsync(ecount, 0, 4 * nn, st));
  RS_CUDA(ctx, cudaMemsetAsync(fail, 0, 4 * nn, st));
  RS_CUDA(ctx, cudaMemsetAsync(full, 0, 4 * nn, st));
  RS_CUDA(ctx, cudaMemsetAsync(errn, 0, 4 * nn, st));
  RS_CUDA(ctx, cudaMemsetAsync(sflag, 0, size_t(ns), st));
  if (calibrated) {
    // 1. calibration members: exact potential and flag, then the per-node error of the surrogate
    k_sur_calib_list<<<grid_for(nbig * kCalib, kT), kT, 0, st>>>(nbig, big_nodes, sur_off, h.node_size,
                                                                 calib_list, sflag, counters);
    RS_LAUNCHED(ctx, "k_sur_calib_list");
    {
      ProfScope prof_(ctx, "k_pot_member", st);
      k_pot_member4<<<grid, kT, 0, st>>>(counters + 9, calib_list, sur_mem, h.mnode, h.node_off,
                                         h.node_size, h.U, h.V, vbulk, eps * eps, Gm, Sx, bound, ambig,
                                         counters + 2);
    }
    RS_LAUNCHED(ctx, "k_pot_member4");
    RS_TRY(unbind_fallback(ctx, counters + 2, ambig, vbulk, bound, st));
    k_acc_counter<<<1, 1, 0, st>>>(counters, 2, 6);
    RS_LAUNCHED(ctx, "k_acc_counter");
    k_sur_err<<<grid_for(nbig * kCalib, kT), kT, 0, st>>>(counters + 9, calib_list, sur_mem, h.mnode,
                                                          h.node_size, stt, Sx, psi_hat, errn);
    RS_LAUNCHED(ctx, "k_sur_err");
  }
  const float* errn_f = calibrated ? reinterpret_cast<const float*>(errn) : nullptr;
  // 2. gate
  k_sur_gate<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, h.node_size, h.V, vbulk, stt, psi_hat,
                                             errn_f, err_floor, ctx->cfg.margin_factor, bound, sflag,
                                             margin, gcount, ecount, counters);
  RS_LAUNCHED(ctx, "k_sur_gate");
  if (nbig > 0) {
    k_sur_full<<<grid_for(nbig, kT), kT, 0, st>>>(nbig, big_nodes, h.node_size, ecount,
                                                  calibrated ? kCalib : 0, full, counters);
    RS_LAUNCHED(ctx, "k_sur_full");
  }
  // 3. nodes nearly all outside the gate: whole-node blocked direct sum
  RS_TRY(unbind_nodes(ctx, full, vbulk, bound, ambig, counters + 2, st, counters));
  k_acc_counter<<<1, 1, 0, st>>>(counters, 2, 7);
  RS_LAUNCHED(ctx, "k_acc_counter");
  // 4. the other ungated members: blocked sums over their node, certified flags, float64 fallback
  // (members of nodes with a certified tree: its bound first, the same exact path after it)
  const int64_t tmin = ctx->tree_nt > 0 ? ctx->tree_min : 0;
  uint8_t* want = tmin > 0 ? scratch_t<uint8_t>(ctx, S_SUR_WANT, size_t(ctx->n_members)) : nullptr;
  if (tmin > 0 && !want) return RS_ERR_OOM;
  k_sur_exact_flags<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, h.node_size, sflag, full, tmin, lf,
                                                    want);
  RS_LAUNCHED(ctx, "k_sur_exact_flags");
  if (tmin > 0) RS_TRY(tree_decide(ctx, nullptr, want, vbulk, bound, counters, st));
  RS_TRY(exclusive_scan_i64(ctx, ns, lf, lf + ns, st));
  k_sur_exact_list<<<grid_for(ns, kT), kT, 0, st>>>(ns, lf, exact_list, counters);
  RS_LAUNCHED(ctx, "k_sur_exact_list");
  if (nbig > 0) {
    k_sur_list_end<<<grid_for(nbig, kT), kT, 0, st>>>(nbig, big_nodes, sur_off, h.node_size, lf, lend);
    RS_LAUNCHED(ctx, "k_sur_list_end");
    // members per thread: autotuned on the first call with enough surrogate members (each of
    // 2, 4, 8 timed on this call's list; identical sums), then kept for the context
    const bool tune = ctx->tune_list_r == 0 && ns >= kTuneMinSurMembers;
    const int cand[3] = {2, 4, 8};
    float best_ms = 0.f;
    int best = 4;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (tune) {
      RS_CUDA(ctx, cudaEventCreate(&e0));
      RS_CUDA(ctx, cudaEventCreate(&e1));
    }
    for (int c = tune ? 0 : 3; c <= 3; ++c) {
      const int R = c < 3 ? cand[c] : (ctx->tune_list_r ? ctx->tune_list_r : 4);
      k_sur_list_tiles<<<grid_for(nbig, kT), kT, 0, st>>>(nbig, big_nodes, sur_off, h.node_size, lf,
                                                          kListThreads * R, lofs, ltiles,
                                                          c == 3 ? counters + 18 : nullptr);
      RS_LAUNCHED(ctx, "k_sur_list_tiles");
      RS_TRY(exclusive_scan_i64(ctx, nbig, ltiles, ltiles + nbig, st));
      const unsigned grid = grid_for(ns / (kListThreads * R) + nbig + 1, 1);
      if (c < 3) RS_CUDA(ctx, cudaEventRecord(e0, st));
      {
        ProfScope prof_(ctx, c < 3 ? "k_potential_list_tune" : "k_potential_list", st);
        if (R == 2)
          k_potential_list<2><<<grid, kListThreads, 0, st>>>(nbig, ltiles, big_nodes, lofs, lend, exact_list,
                                                             sur_mem, h.node_off, h.node_size, h.U, eps * eps, Sx);
        else if (R == 8)
          k_potential_list<8><<<grid, kListThreads, 0, st>>>(nbig, ltiles, big_nodes, lofs, lend, exact_list,
                                                             sur_mem, h.node_off, h.node_size, h.U, eps * eps, Sx);
        else
          k_potential_list<4><<<grid, kListThreads, 0, st>>>(nbig, ltiles, big_nodes, lofs, lend, exact_list,
                                                             sur_mem, h.node_off, h.node_size, h.U, eps * eps, Sx);
      }
      RS_LAUNCHED(ctx, "k_potential_list");
      if (c < 3) {
        RS_CUDA(ctx, cudaEventRecord(e1, st));
        RS_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        RS_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        ctx->tune_list_ms[c] = ms;
        if (c == 0 || ms < best_ms) {
          best_ms = ms;
          best = cand[c];
        }
        if (c == 2) ctx->tune_list_r = best;
      }
    }
    if (tune) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
  }
  k_flags_list<<<grid_for(ns, kT), kT, 0, st>>>(counters + 0, exact_list, sur_mem, h.mnode, h.V, vbulk,
                                               eps * eps, Gm, Sx, bound, ambig, counters + 2);
  RS_LAUNCHED(ctx, "k_flags_list");
  RS_TRY(unbind_fallback(ctx, counters + 2, ambig, vbulk, bound, st));
  k_acc_counter<<<1, 1, 0, st>>>(counters, 2, 6);
  RS_LAUNCHED(ctx, "k_acc_counter");
  // 5. spot checks: the smallest-margin gated members of each node, exactly
  if (nbig > 0) {
    k_sur_select<<<unsigned(nbig), kT, 0, st>>>(big_nodes, sur_off, h.node_size, gcount, margin,
                                                ctx->cfg.spot_check, full, tau);
    RS_LAUNCHED(ctx, "k_sur_select");
  }
  k_sur_spot_mark<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, margin, sflag, tau, gcount,
                                                  ctx->cfg.spot_check, full, checked, check_list, counters);
  RS_LAUNCHED(ctx, "k_sur_spot_mark");
  {
    ProfScope prof_(ctx, "k_pot_member", st);
    k_pot_member<<<grid, kT, 0, st>>>(counters + 1, check_list, sur_mem, h.mnode, h.node_off, h.node_size,
                                      h.U, h.V, vbulk, eps * eps, Gm, Sx, bound, ambig, counters + 2);
  }
  RS_LAUNCHED(ctx, "k_pot_member");
  RS_TRY(unbind_fallback(ctx, counters + 2, ambig, vbulk, bound, st));
  k_acc_counter<<<1, 1, 0, st>>>(counters, 2, 6);
  RS_LAUNCHED(ctx, "k_acc_counter");
  k_sur_verdict<<<grid, kT, 0, st>>>(counters, check_list, sur_mem, h.mnode, h.node_size, stt, Sx, psi_hat,
                                     sflag, bound, errn_f, err_floor, ctx->cfg.margin_factor, fail);
  RS_LAUNCHED(ctx, "k_sur_verdict");
  // 6. nodes that failed a spot check: the whole node through the blocked direct sum
  k_sur_rerun<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, fail, sflag, checked, counters);
  RS_LAUNCHED(ctx, "k_sur_rerun");
  RS_TRY(unbind_nodes(ctx, fail, vbulk, bound, ambig, counters + 2, st, counters));
  k_acc_counter<<<1, 1, 0, st>>>(counters, 2, 6);
  RS_LAUNCHED(ctx, "k_acc_counter");
  k_sur_decided<<<grid_for(ns, kT), kT, 0, st>>>(ns, sur_mem, h.mnode, sflag, checked, full, fail, counters);
  RS_LAUNCHED(ctx, "k_sur_decided");
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
  if (psi_out && (ctx->last_unbind_surrogate || ctx->tree_nt > 0))
    return set_error(ctx, RS_ERR_STATE,
                     "targets need an rs_unbind that computed every potential (no surrogate, "
                     "no tree bound: ask it for the potential)");
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
  for (int i = 0; i < 11; ++i) stats_out[i] = ctx->sur_stats[i];
  return RS_OK;
}

// Recursive 6D phase-space friends-of-friends inside every 3D FoF group (Section
// "Parallelization": subhalo finding for each FoF halo from 6D phase-space information;
// metric |dx|^2/sigma_x^2 + |dv|^2/sigma_v^2, linked fraction f and recursion from Rockstar).
//
// Level-synchronous: level 0 = FoF groups with >= min members (sorted by (label, id)); each
// level runs, over all of its nodes at once,
//   k_member_node   owning node of every member position
//   k_gather_uv     u = wrapped offset from the node's smallest-id member, v, as float4
//   CRO moments     12 float64 sums per node -> inv_sx2, inv_sv2 (k_node_inv)
//   k_nn6d          brute-force nearest-neighbour d6 per member, j-tiles in shared memory
//   k_select_l2     exact k-th smallest nn2 per node (radix select on the float bit patterns)
//   k_link6d        union-find over pairs with d6 <= l2 (upper triangle of each node)
//   k_comp_count    roots and component sizes; k_child_flags marks children
//   compaction + stable radix sort by child index -> next level's member list (ascending id
//   inside each child because member positions ascend with id)
// Every float32 operation of d6 is rounded separately (no FMA), so the result equals the
// oracle's plain definition bit for bit.
#include "rs_cro.cuh"

namespace {

constexpr int kT = 256;
constexpr int kTile6 = 128;

// ---------------------------------------------------------------------------------------------
// Level 0 from FoF labels.

// out[0] = max id, out[1] = max label (~0 in both when any id or label is negative).
__global__ void __launch_bounds__(256)
k_max_id(int64_t n, const int64_t* __restrict__ ids, const int64_t* __restrict__ lab,
         unsigned long long* __restrict__ out) {
  __shared__ unsigned long long wmax[2][8];
  unsigned long long mi = 0, ml = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t a = ids[i], b = lab[i];
    if (a < 0 || b < 0) {
      mi = ml = ~0ull;
    } else {
      mi = (unsigned long long)a > mi ? (unsigned long long)a : mi;
      ml = (unsigned long long)b > ml ? (unsigned long long)b : ml;
    }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const unsigned long long oi = __shfl_xor_sync(0xffffffffu, mi, off);
    const unsigned long long ol = __shfl_xor_sync(0xffffffffu, ml, off);
    mi = oi > mi ? oi : mi;
    ml = ol > ml ? ol : ml;
  }
  if ((threadIdx.x & 31) == 0) {
    wmax[0][threadIdx.x >> 5] = mi;
    wmax[1][threadIdx.x >> 5] = ml;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // one atomic per block and value
    for (int w = 1; w < int(blockDim.x >> 5); ++w) {
      mi = wmax[0][w] > mi ? wmax[0][w] : mi;
      ml = wmax[1][w] > ml ? wmax[1][w] : ml;
    }
    atomicMax(out, mi);
    atomicMax(out + 1, ml);
  }
}

// ---- level 0 over a dense label range (max label < 2 n + 4096): per-label member counts, the
// kept labels' node indices and member offsets from two scans over the label range, then one
// sort of the kept particles only, by (node, id).
__global__ void k_label_count(int64_t n, const int64_t* __restrict__ lab, uint32_t* __restrict__ cnt) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool valid = i < n;  // every lane stays for the warp-aggregated atomics
  rsd::warp_run_add<uint32_t>(cnt, valid ? uint32_t(lab[i]) : 0u, valid, 1u);
}

__global__ void k_label_keep(int64_t nl, const uint32_t* __restrict__ cnt, int min_size,
                             int64_t* __restrict__ knode, int64_t* __restrict__ ksize) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  const bool keep = cnt[l] >= uint32_t(min_size);
  knode[l] = keep ? 1 : 0;
  ksize[l] = keep ? int64_t(cnt[l]) : 0;
}

__global__ void k_label_nodes(int64_t nl, const uint32_t* __restrict__ cnt, int min_size,
                              const int64_t* __restrict__ knode, const int64_t* __restrict__ koff,
                              int64_t* __restrict__ node_off, int64_t* __restrict__ node_size,
                              int64_t* __restrict__ node_parent, int32_t* __restrict__ node_level) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= nl || cnt[l] < uint32_t(min_size)) return;
  const int64_t q = knode[l];
  node_off[q] = koff[l];
  node_size[q] = cnt[l];
  node_parent[q] = -1;
  node_level[q] = 0;
}

// Keys (node << bid | id) of the particles of kept groups, appended with one atomic per warp.
__global__ void k_label_keys(int64_t n, const int64_t* __restrict__ ids, const int64_t* __restrict__ lab,
                             const uint32_t* __restrict__ cnt, int min_size,
                             const int64_t* __restrict__ knode, int bid,
                             unsigned long long* __restrict__ ctr, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t l = i < n ? lab[i] : 0;
  const bool keep = i < n && cnt[l] >= uint32_t(min_size);
  const unsigned b = __ballot_sync(0xffffffffu, keep);
  unsigned long long base = 0;
  if (lane == 0 && b) base = atomicAdd(ctr, (unsigned long long)__popc(b));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (!keep) return;
  const unsigned long long pos = base + __popc(b & ((1u << lane) - 1u));
  keys[pos] = (uint64_t(knode[l]) << bid) | uint64_t(ids[i]);
  vals[pos] = uint32_t(i);
}

__global__ void k_level0_minid(int64_t nodes, const int64_t* __restrict__ node_off,
                               const uint32_t* __restrict__ mem, const int64_t* __restrict__ ids,
                               int64_t* __restrict__ node_minid) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < nodes) node_minid[q] = ids[mem[node_off[q]]];  // members ascend by id
}

// Sparse labels: all particles ordered by (label, id) with two stable radix sorts, first by id
// (k_id_keys), then by label (k_label_of: the labels of the id-sorted particles).
__global__ void k_id_keys(int64_t n, const int64_t* __restrict__ ids, uint64_t* __restrict__ keys,
                          uint32_t* __restrict__ vals) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = uint64_t(ids[i]);
  vals[i] = uint32_t(i);
}

__global__ void k_label_of(int64_t n, const uint32_t* __restrict__ vals, const int64_t* __restrict__ lab,
                           uint64_t* __restrict__ keys) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < n) keys[k] = uint64_t(lab[vals[k]]);
}

// head flag per sorted position (1 where a new label starts); run index comes from a scan.
__global__ void k_run_heads(int64_t n, const uint64_t* __restrict__ keys, int b, int64_t* __restrict__ head) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  head[i] = (i == 0 || (keys[i] >> b) != (keys[i - 1] >> b)) ? 1 : 0;
}

// After the scan: run start positions and, at the end, run sizes; runs with >= min members
// become level-0 nodes.
__global__ void k_run_starts(int64_t n, const uint64_t* __restrict__ keys, int b,
                             const int64_t* __restrict__ run_idx, int64_t* __restrict__ run_start) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i == 0 || (keys[i] >> b) != (keys[i - 1] >> b)) run_start[run_idx[i]] = i;
}

__global__ void k_run_keep(int64_t nruns, int64_t n, const int64_t* __restrict__ run_start,
                           int min_size, int64_t* __restrict__ keep, int64_t* __restrict__ size) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= nruns) return;
  const int64_t e = (r + 1 < nruns) ? run_start[r + 1] : n;
  const int64_t s = e - run_start[r];
  size[r] = s;
  keep[r] = s >= min_size ? 1 : 0;
}

// Level-0 node table and member list (particle indices), from kept runs.
__global__ void k_level0_nodes(int64_t nruns, const int64_t* __restrict__ run_start,
                               const int64_t* __restrict__ size, const int64_t* __restrict__ keep,
                               const int64_t* __restrict__ node_of_run /*scan of keep*/,
                               const int64_t* __restrict__ mem_off /*scan of kept sizes*/,
                               const uint32_t* __restrict__ vals, const int64_t* __restrict__ ids,
                               int64_t* __restrict__ node_off, int64_t* __restrict__ node_size,
                               int64_t* __restrict__ node_parent, int32_t* __restrict__ node_level,
                               int64_t* __restrict__ node_minid) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= nruns || !keep[r]) return;
  const int64_t q = node_of_run[r];
  node_off[q] = mem_off[r];
  node_size[q] = size[r];
  node_parent[q] = -1;
  node_level[q] = 0;
  node_minid[q] = ids[vals[run_start[r]]];
}

// run_heads holds the exclusive scan of the head flags: a run start sees its own run index,
// any later element of run r sees r + 1.
__device__ __forceinline__ int64_t run_of(const uint64_t* keys, int b, const int64_t* run_heads,
                                          int64_t i) {
  const bool head = (i == 0 || (keys[i] >> b) != (keys[i - 1] >> b));
  return run_heads[i] - (head ? 0 : 1);
}

__global__ void k_level0_members(int64_t n, const uint64_t* __restrict__ keys, int b,
                                 const int64_t* __restrict__ run_heads,
                                 const int64_t* __restrict__ run_start, const int64_t* __restrict__ keep,
                                 const int64_t* __restrict__ mem_off, const uint32_t* __restrict__ vals,
                                 uint32_t* __restrict__ mem) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t r = run_of(keys, b, run_heads, i);
  if (!keep[r]) return;
  mem[mem_off[r] + (i - run_start[r])] = vals[i];
}

__global__ void k_fill_i64(int64_t n, int64_t* __restrict__ a, int64_t v) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

__global__ void k_size_mask(int64_t n, const int64_t* __restrict__ keep, const int64_t* __restrict__ size,
                            int64_t* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = keep[i] ? size[i] : 0;
}

// ---------------------------------------------------------------------------------------------
// Per-level kernels. Member positions p are global (into the hierarchy's member list);
// level-local position = p - mb.

__global__ void k_member_node(int64_t mb, int64_t me, int64_t nb, int64_t nn,
                              const int64_t* __restrict__ node_off, uint32_t* __restrict__ mnode) {
  const int64_t p = mb + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= me) return;
  mnode[p] = uint32_t(nb + rsd::upper_bound_i64(node_off + nb, nn, p) - 1);
}

__global__ void k_gather_uv(int64_t mb, int64_t me, const uint32_t* __restrict__ mem,
                            const uint32_t* __restrict__ mnode, const int64_t* __restrict__ node_off,
                            const float* __restrict__ pos, const float* __restrict__ vel, float L,
                            float4* __restrict__ U, float4* __restrict__ V) {
  const int64_t p = mb + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= me) return;
  const int64_t i = mem[p];
  const int64_t r = mem[node_off[mnode[p]]];
  const float hL = 0.5f * L;
  U[p] = make_float4(rsd::wrap_diff(pos[3 * r], pos[3 * i], L, hL),
                     rsd::wrap_diff(pos[3 * r + 1], pos[3 * i + 1], L, hL),
                     rsd::wrap_diff(pos[3 * r + 2], pos[3 * i + 2], L, hL), 0.f);
  V[p] = make_float4(vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], 0.f);
}

__global__ void k_node_ref(int64_t nb, int64_t ne, const uint32_t* __restrict__ mem,
                           const int64_t* __restrict__ node_off, const float* __restrict__ pos,
                           float4* __restrict__ ref) {
  const int64_t q = nb + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= ne) return;
  const int64_t r = mem[node_off[q]];
  ref[q] = make_float4(pos[3 * r], pos[3 * r + 1], pos[3 * r + 2], 0.f);
}

struct MomentTerm {
  const float4* U;
  const float4* V;
  template <bool kFirst>
  __device__ __forceinline__ void add(int64_t, int64_t p, int64_t, double* acc) const {
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

// Total variance ((Q0/g - m0^2) + (Q1/g - m1^2)) + (Q2/g - m2^2), m_d = S_d / g.
__device__ __forceinline__ double total_var(const double* S, const double* Q, double g) {
  double var = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double m = __ddiv_rn(S[d], g);
    const double t = __dsub_rn(__ddiv_rn(Q[d], g), __dmul_rn(m, m));
    var = (d == 0) ? t : __dadd_rn(var, t);
  }
  return var;
}

// Metric scales of the node's split, and (mean u, sigma_v,1D) in float32 for the surrogate's
// features.
__global__ void k_node_inv(int64_t nb, int64_t nn, const int64_t* __restrict__ node_size,
                           const double* __restrict__ sums, float4* __restrict__ inv,
                           float4* __restrict__ mom) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const double g = double(node_size[nb + k]);
  const double* S = sums + 12 * k;
  const double vx = total_var(S, S + 3, g);
  const double vv = total_var(S + 6, S + 9, g);
  const float ix = vx > 0.0 ? __double2float_rn(__ddiv_rn(1.0, vx)) : 0.f;
  const float iv = vv > 0.0 ? __double2float_rn(__ddiv_rn(1.0, vv)) : 0.f;
  inv[nb + k] = make_float4(ix, iv, 0.f, 0.f);
  mom[nb + k] = make_float4(float(__ddiv_rn(S[0], g)), float(__ddiv_rn(S[1], g)), float(__ddiv_rn(S[2], g)),
                            float(sqrt(fmax(vv, 0.0) / 3.0)));
}

__device__ __forceinline__ float d6(float4 ui, float4 vi, float4 uj, float4 vj, float isx, float isv) {
  const float rx = rsd::sq3(__fsub_rn(uj.x, ui.x), __fsub_rn(uj.y, ui.y), __fsub_rn(uj.z, ui.z));
  const float rv = rsd::sq3(__fsub_rn(vj.x, vi.x), __fsub_rn(vj.y, vi.y), __fsub_rn(vj.z, vi.z));
  return __fadd_rn(__fmul_rn(rx, isx), __fmul_rn(rv, isv));
}

__global__ void k_tile_counts(int64_t nb, int64_t nn, const int64_t* __restrict__ node_size, int tile,
                              int64_t* __restrict__ out) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < nn) out[k] = (node_size[nb + k] + tile - 1) / tile;
}

// Nearest-neighbour d6 per member: block = (node, i-tile of 128), j-tiles staged in shared memory.
__global__ void __launch_bounds__(kTile6)
k_nn6d(int64_t nb, int64_t nn, const int64_t* __restrict__ tile_off, const int64_t* __restrict__ node_off,
       const int64_t* __restrict__ node_size, const float4* __restrict__ inv,
       const float4* __restrict__ U, const float4* __restrict__ V, float* __restrict__ nn2, int64_t mb) {
  __shared__ float4 su[kTile6], sv[kTile6];
  const int64_t b = blockIdx.x;
  if (b >= tile_off[nn]) return;
  const int64_t k = rsd::upper_bound_i64(tile_off, nn, b) - 1;
  const int64_t t = b - tile_off[k];
  const int64_t q = nb + k;
  const int64_t base = node_off[q], g = node_size[q];
  const float isx = inv[q].x, isv = inv[q].y;
  const int64_t i = t * kTile6 + threadIdx.x;
  const bool valid = i < g;
  const float4 ui = valid ? U[base + i] : make_float4(0, 0, 0, 0);
  const float4 vi = valid ? V[base + i] : make_float4(0, 0, 0, 0);
  float best = __int_as_float(0x7f800000);
  for (int64_t j0 = 0; j0 < g; j0 += kTile6) {
    const int64_t j = j0 + threadIdx.x;
    if (j < g) {
      su[threadIdx.x] = U[base + j];
      sv[threadIdx.x] = V[base + j];
    }
    __syncthreads();
    const int jn = int(rsd::min64(kTile6, g - j0));
    for (int jj = 0; jj < jn; ++jj) {
      if (j0 + jj == i) continue;
      best = fminf(best, d6(ui, vi, su[jj], sv[jj], isx, isv));
    }
    __syncthreads();
  }
  if (valid) nn2[base + i - mb] = best;
}

// Exact k-th smallest nn2 of each node, k = ceil(f_num g / f_den) - 1: 4 passes of 8-bit radix
// select on the (non-negative) float bit patterns. Nodes up to kSelectWarpMax members take one
// warp each (k_select_l2_warp), larger ones a block (k_select_l2).
constexpr int64_t kSelectWarpMax = 4096;
constexpr int64_t kPrunedMinMembers = 4096;

// only (if given): int [nn], the nodes to select for (the others keep their l2).
__global__ void __launch_bounds__(kT)
k_select_l2_warp(int64_t nb, int64_t nn, const int64_t* __restrict__ node_off,
                 const int64_t* __restrict__ node_size, const float* __restrict__ nn2, int64_t mb,
                 int f_num, int f_den, float4* __restrict__ inv, const int* __restrict__ only) {
  __shared__ uint32_t hist[kT / 32][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t k = int64_t(blockIdx.x) * (kT / 32) + w;
  if (k >= nn) return;
  const int64_t q = nb + k;
  const int64_t base = node_off[q] - mb, g = node_size[q];
  if (g > kSelectWarpMax || (only && !only[k])) return;
  uint32_t kk = uint32_t((int64_t(f_num) * g + f_den - 1) / f_den - 1);
  uint32_t prefix = 0, mask = 0;
  uint32_t* h = hist[w];
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int d = lane; d < 256; d += 32) h[d] = 0;
    __syncwarp();
    for (int64_t a = lane; a < g; a += 32) {
      const uint32_t bits = __float_as_uint(nn2[base + a]);
      if ((bits & mask) == prefix) atomicAdd(&h[(bits >> shift) & 255u], 1u);
    }
    __syncwarp();
    // digit d with cum(d) <= kk < cum(d) + h[d]: lane l owns bins 8l .. 8l + 7
    uint32_t c[8], sum = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      c[t] = h[8 * lane + t];
      sum += c[t];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    const uint32_t excl = incl - sum;
    const unsigned owner = __ballot_sync(0xffffffffu, excl <= kk && kk < incl);
    const int L = __ffs(owner) - 1;
    uint32_t d = 0, cum = excl;
    if (lane == L) {
      for (int t = 0; t < 8; ++t) {
        if (cum + c[t] > kk) {
          d = 8 * lane + t;
          break;
        }
        cum += c[t];
      }
    }
    d = __shfl_sync(0xffffffffu, d, L);
    cum = __shfl_sync(0xffffffffu, cum, L);
    kk -= cum;
    prefix |= d << shift;
    mask |= 255u << shift;
    __syncwarp();
  }
  if (lane == 0) inv[q].z = __uint_as_float(prefix);
}

// only (if given): int [nn], the nodes to select for (the others keep their l2).
__global__ void __launch_bounds__(kT)
k_select_l2(int64_t nb, const int64_t* __restrict__ node_off, const int64_t* __restrict__ node_size,
            const float* __restrict__ nn2, int64_t mb, int f_num, int f_den, float4* __restrict__ inv,
            const int* __restrict__ only) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_prefix, s_k;
  const int64_t q = nb + blockIdx.x;
  const int64_t base = node_off[q] - mb, g = node_size[q];
  if (g <= kSelectWarpMax || (only && !only[blockIdx.x])) return;
  if (threadIdx.x == 0) {
    s_prefix = 0;
    s_k = uint32_t((int64_t(f_num) * g + f_den - 1) / f_den - 1);
  }
  uint32_t mask = 0;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0;
    __syncthreads();
    const uint32_t prefix = s_prefix;
    for (int64_t a = threadIdx.x; a < g; a += blockDim.x) {
      const uint32_t bits = __float_as_uint(nn2[base + a]);
      if ((bits & mask) == prefix) atomicAdd(&hist[(bits >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t kk = s_k, cum = 0;
      int d = 0;
      for (; d < 256; ++d) {
        if (cum + hist[d] > kk) break;
        cum += hist[d];
      }
      s_k = kk - cum;
      s_prefix = prefix | (uint32_t(d) << shift);
    }
    mask |= 255u << shift;
    __syncthreads();
  }
  if (threadIdx.x == 0) inv[q].z = __uint_as_float(s_prefix);
}

__global__ void k_iota_u32(int64_t n, uint32_t* __restrict__ a) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) a[i] = uint32_t(i);
}

// Union-find over pairs with d6 <= l2: block = (node, i-tile); j-tiles from the i-tile on.
__global__ void __launch_bounds__(kTile6)
k_link6d(int64_t nb, int64_t nn, const int64_t* __restrict__ tile_off, const int64_t* __restrict__ node_off,
         const int64_t* __restrict__ node_size, const float4* __restrict__ inv,
         const float4* __restrict__ U, const float4* __restrict__ V, const float* __restrict__ nn2,
         uint32_t* __restrict__ uf, int64_t mb) {
  __shared__ float4 su[kTile6], sv[kTile6];
  __shared__ float snn[kTile6];
  const int64_t b = blockIdx.x;
  if (b >= tile_off[nn]) return;
  const int64_t k = rsd::upper_bound_i64(tile_off, nn, b) - 1;
  const int64_t t = b - tile_off[k];
  const int64_t q = nb + k;
  const int64_t base = node_off[q], g = node_size[q];
  const float4 iv = inv[q];
  const float isx = iv.x, isv = iv.y, l2 = iv.z;
  const int64_t i = t * kTile6 + threadIdx.x;
  const bool valid = i < g;
  const float4 ui = valid ? U[base + i] : make_float4(0, 0, 0, 0);
  const float4 vi = valid ? V[base + i] : make_float4(0, 0, 0, 0);
  const bool active = valid && nn2[base + i - mb] <= l2;  // others have no friend at all
  const uint32_t li = uint32_t(base + i - mb);
  for (int64_t j0 = t * kTile6; j0 < g; j0 += kTile6) {
    const int64_t j = j0 + threadIdx.x;
    if (j < g) {
      su[threadIdx.x] = U[base + j];
      sv[threadIdx.x] = V[base + j];
      snn[threadIdx.x] = nn2[base + j - mb];
    }
    __syncthreads();
    const int jn = int(rsd::min64(kTile6, g - j0));
    if (active) {
      for (int jj = 0; jj < jn; ++jj) {
        if (j0 + jj <= i || snn[jj] > l2) continue;
        if (d6(ui, vi, su[jj], sv[jj], isx, isv) <= l2)
          rsd::uf_unite(uf, li, uint32_t(base + j0 + jj - mb));
      }
    }
    __syncthreads();
  }
}

// Roots (full compression) and component sizes.
__global__ void k_comp_count(int64_t m, uint32_t* __restrict__ uf, uint32_t* __restrict__ cnt) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool valid = p < m;  // every lane stays: lanes with the same root add once
  const uint32_t r = valid ? rsd::uf_find_ro(uf, uint32_t(p)) : 0xffffffffu;
  if (valid) uf[p] = r;
  const unsigned peers = __match_any_sync(0xffffffffu, r);
  if (valid && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cnt + r, uint32_t(__popc(peers)));
}

// child flag at each root that forms a child (>= min and < its node's size).
__global__ void k_child_flags(int64_t m, int64_t mb, const uint32_t* __restrict__ uf,
                              const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ mnode,
                              const int64_t* __restrict__ node_size, int min_size,
                              int64_t* __restrict__ flag) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  int64_t f = 0;
  if (uf[p] == uint32_t(p)) {
    const int64_t c = cnt[p];
    f = (c >= min_size && c < node_size[mnode[mb + p]]) ? 1 : 0;
  }
  flag[p] = f;
}

// member flag: 1 if the member's root is a child root.
__global__ void k_member_flags(int64_t m, const uint32_t* __restrict__ uf, const int64_t* __restrict__ cflag,
                               int64_t* __restrict__ mflag) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  mflag[p] = cflag[uf[p]];
}

// Scatter (child index, particle index) of child members into compacted order.
__global__ void k_child_members(int64_t m, int64_t mb, const uint32_t* __restrict__ uf,
                                const int64_t* __restrict__ cidx, const int64_t* __restrict__ cflag,
                                const int64_t* __restrict__ mpos, const uint32_t* __restrict__ mem,
                                uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const uint32_t r = uf[p];
  if (!cflag[r]) return;
  keys[mpos[p]] = uint64_t(cidx[r]);
  vals[mpos[p]] = mem[mb + p];
}

// Child node table entries (global node index ne + child index).
__global__ void k_child_nodes(int64_t m, int64_t mb, int64_t ne, const uint32_t* __restrict__ uf,
                              const uint32_t* __restrict__ cnt, const int64_t* __restrict__ cflag,
                              const int64_t* __restrict__ cidx, const uint32_t* __restrict__ mnode,
                              const uint32_t* __restrict__ mem, const int64_t* __restrict__ ids,
                              int64_t* __restrict__ node_size, int64_t* __restrict__ node_parent,
                              int32_t* node_level, int64_t* __restrict__ node_minid) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= m || uf[p] != uint32_t(p) || !cflag[p]) return;
  const int64_t q = ne + cidx[p];
  const uint32_t par = mnode[mb + p];
  node_size[q] = cnt[p];
  node_parent[q] = par;
  node_level[q] = node_level[par] + 1;
  node_minid[q] = ids[mem[mb + p]];
}

__global__ void k_copy_u32(int64_t n, const uint32_t* __restrict__ src, uint32_t* __restrict__ dst) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

__global__ void k_offsets_add(int64_t n, const int64_t* __restrict__ src, int64_t add,
                              int64_t* __restrict__ dst) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] + add;
}

// Deepest node per particle and the particle's member position in that node.
// Deepest node per particle and the particle's member position in that node, written once:
// at the level where the member does not go on into a child (its root is not a child root).
__global__ void k_deepest(int64_t mb, int64_t me, const uint32_t* __restrict__ mem,
                          const uint32_t* __restrict__ mnode, const uint32_t* __restrict__ uf,
                          const int64_t* __restrict__ cflag, int64_t* __restrict__ deepest,
                          uint32_t* __restrict__ deepest_pos) {
  const int64_t p = mb + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p < me && !cflag[uf[p - mb]]) {
    deepest[mem[p]] = mnode[p];
    deepest_pos[mem[p]] = uint32_t(p);
  }
}

// Grow a persistent hierarchy buffer, keeping its first `used` bytes.
int grow_keep(rs_ctx* ctx, int slot, size_t used, size_t need, cudaStream_t st) {
  rs::Buffer& b = ctx->buf[slot];
  if (b.bytes >= need) return RS_OK;
  size_t want = std::max(need, b.bytes * 3 / 2);
  want = (want + 255) & ~size_t(255);
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    return rs::set_error(ctx, RS_ERR_OOM, "cudaMalloc of %zu bytes failed (slot %d)", want, slot);
  }
  if (used && b.ptr) RS_CUDA(ctx, cudaMemcpyAsync(p, b.ptr, used, cudaMemcpyDeviceToDevice, st));
  RS_CUDA(ctx, cudaStreamSynchronize(st));
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = p;
  b.bytes = want;
  return RS_OK;
}

int bits_for(uint64_t v) {
  int b = 1;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

}  // namespace

namespace rs {

Hier hier_of(rs_ctx* ctx) {
  Hier h;
  h.mem = static_cast<uint32_t*>(ctx->buf[S_H_MEM].ptr);
  h.mnode = static_cast<uint32_t*>(ctx->buf[S_H_MNODE].ptr);
  h.U = static_cast<float4*>(ctx->buf[S_H_U].ptr);
  h.V = static_cast<float4*>(ctx->buf[S_H_V].ptr);
  h.node_off = static_cast<int64_t*>(ctx->buf[S_H_NODE_OFF].ptr);
  h.node_size = static_cast<int64_t*>(ctx->buf[S_H_NODE_SIZE].ptr);
  h.node_parent = static_cast<int64_t*>(ctx->buf[S_H_NODE_PARENT].ptr);
  h.node_level = static_cast<int32_t*>(ctx->buf[S_H_NODE_LEVEL].ptr);
  h.node_minid = static_cast<int64_t*>(ctx->buf[S_H_NODE_MINID].ptr);
  h.inv = static_cast<float4*>(ctx->buf[S_H_NODE_INV].ptr);
  h.mom = static_cast<float4*>(ctx->buf[S_H_NODE_MOM].ptr);
  h.ref = static_cast<float4*>(ctx->buf[S_H_NODE_REF].ptr);
  h.deepest = static_cast<int64_t*>(ctx->buf[S_H_DEEPEST].ptr);
  h.deepest_pos = static_cast<uint32_t*>(ctx->buf[S_H_DEEPPOS].ptr);
  return h;
}

// Batched form: exactly pruned nearest-neighbour and link searches (rs_prune6d.cu).
int prune6d_prepare(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m,
                    const double* sums, cudaStream_t st);
int prune6d_nn(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, float* nn2,
               cudaStream_t st);
int prune6d_check(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t m, float* nn2, const int** failed_out,
                  cudaStream_t st);
int prune6d_link(rs_ctx* ctx, int64_t nb, int64_t nn, int64_t mb, int64_t m, const float* nn2,
                 uint32_t* uf, cudaStream_t st);

// Gather U, V (and node reference positions) for member positions [mb, me) and nodes [nb, ne).
int gather_members(rs_ctx* ctx, int64_t mb, int64_t me, int64_t nb, int64_t ne, const float* pos,
                   const float* vel, cudaStream_t st);

}  // namespace rs

using namespace rs;

int rs::gather_members(rs_ctx* ctx, int64_t mb, int64_t me, int64_t nb, int64_t ne,
                       const float* pos, const float* vel, cudaStream_t st) {
  Hier h = hier_of(ctx);
  if (me > mb) {
    k_gather_uv<<<grid_for(me - mb, kT), kT, 0, st>>>(mb, me, h.mem, h.mnode, h.node_off, pos, vel,
                                                     ctx->cfg.box_L, h.U, h.V);
    RS_LAUNCHED(ctx, "k_gather_uv");
  }
  if (ne > nb) {
    k_node_ref<<<grid_for(ne - nb, kT), kT, 0, st>>>(nb, ne, h.mem, h.node_off, pos, h.ref);
    RS_LAUNCHED(ctx, "k_node_ref");
  }
  return RS_OK;
}

static int ensure_nodes(rs_ctx* ctx, int64_t used, int64_t need, cudaStream_t st) {
  RS_TRY(grow_keep(ctx, S_H_NODE_OFF, size_t(used + 1) * 8, size_t(need + 1) * 8, st));
  RS_TRY(grow_keep(ctx, S_H_NODE_SIZE, size_t(used) * 8, size_t(need) * 8, st));
  RS_TRY(grow_keep(ctx, S_H_NODE_PARENT, size_t(used) * 8, size_t(need) * 8, st));
  RS_TRY(grow_keep(ctx, S_H_NODE_LEVEL, size_t(used) * 4, size_t(need) * 4, st));
  RS_TRY(grow_keep(ctx, S_H_NODE_MINID, size_t(used) * 8, size_t(need) * 8, st));
  RS_TRY(grow_keep(ctx, S_H_NODE_INV, size_t(used) * 16, size_t(need) * 16, st));
  RS_TRY(grow_keep(ctx, S_H_NODE_MOM, size_t(used) * 16, size_t(need) * 16, st));
  RS_TRY(grow_keep(ctx, S_H_NODE_REF, size_t(used) * 16, size_t(need) * 16, st));
  return RS_OK;
}

static int ensure_members(rs_ctx* ctx, int64_t used, int64_t need, cudaStream_t st) {
  RS_TRY(grow_keep(ctx, S_H_MEM, size_t(used) * 4, size_t(need) * 4, st));
  RS_TRY(grow_keep(ctx, S_H_MNODE, size_t(used) * 4, size_t(need) * 4, st));
  RS_TRY(grow_keep(ctx, S_H_U, size_t(used) * 16, size_t(need) * 16, st));
  RS_TRY(grow_keep(ctx, S_H_V, size_t(used) * 16, size_t(need) * 16, st));
  return RS_OK;
}

extern "C" int rs_fof6d(rs_ctx* ctx, int64_t n, const float* pos, const float* vel,
                        const int64_t* ids, const int64_t* fof_label, int64_t* n_nodes_out,
                        int64_t* n_members_out, void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  ctx->have_hier = false;
  ctx->have_unbind = false;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n < 0 || n >= (int64_t(1) << 32) - 1)
    return set_error(ctx, RS_ERR_INVALID_ARG, "n = %lld out of range", (long long)n);
  if (n > 0 && (!pos || !vel || !ids || !fof_label))
    return set_error(ctx, RS_ERR_INVALID_ARG, "null device pointer");
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  const int min_size = ctx->cfg.min_halo_particles;
  const float L = ctx->cfg.box_L;
  // ---------------- level 0 from the FoF labels
  int64_t* deep = scratch_t<int64_t>(ctx, S_H_DEEPEST, size_t(std::max<int64_t>(n, 1)));
  uint32_t* deep_pos = scratch_t<uint32_t>(ctx, S_H_DEEPPOS, size_t(std::max<int64_t>(n, 1)));
  if (!deep) return RS_ERR_OOM;
  int64_t nodes = 0, members = 0;
  if (n == 0) {
    RS_TRY(ensure_nodes(ctx, 0, 1, st));
    RS_TRY(ensure_members(ctx, 0, 1, st));
    k_fill_i64<<<1, 1, 0, st>>>(1, hier_of(ctx).node_off, 0);
    RS_LAUNCHED(ctx, "k_fill_i64");
  } else {
    k_fill_i64<<<grid_for(n, kT), kT, 0, st>>>(n, deep, -1);
    RS_LAUNCHED(ctx, "k_fill_i64");
    if (!deep_pos) return RS_ERR_OOM;
    unsigned long long* mx = scratch_t<unsigned long long>(ctx, S_COUNTER, 16);
    if (!mx) return RS_ERR_OOM;
    RS_CUDA(ctx, cudaMemsetAsync(mx, 0, 16, st));
    k_max_id<<<std::min(grid_for(n, kT), 152u * 8u), kT, 0, st>>>(n, ids, fof_label, mx);
    RS_LAUNCHED(ctx, "k_max_id");
    RS_TRY(read_back(ctx, mx, 16, st));
    const uint64_t max_id = uint64_t(ctx->host_box[0]), max_lab = uint64_t(ctx->host_box[1]);
    if (max_id == ~0ull) return set_error(ctx, RS_ERR_INVALID_ARG, "negative id or label");
    // dense label range: (node << bid | id) keys of the kept particles; otherwise two sorts
    const int bid = bits_for(max_id);
    if (max_lab < std::min<uint64_t>(uint64_t(2 * n + 4096), uint64_t(1) << 31) &&
        bits_for(max_lab + 1) + bid <= 64) {
      // dense label range: count per label, keep, scan, sort the kept particles only
      const int64_t nl = int64_t(max_lab) + 1;
      uint32_t* cntl = scratch_t<uint32_t>(ctx, S_ROOT_CNT, size_t(nl));
      int64_t* knode = scratch_t<int64_t>(ctx, S_GKEY_A, size_t(nl) + 1);
      int64_t* koff = scratch_t<int64_t>(ctx, S_GKEY_B, size_t(nl) + 1);
      if (!cntl || !knode || !koff) return RS_ERR_OOM;
      RS_CUDA(ctx, cudaMemsetAsync(cntl, 0, sizeof(uint32_t) * nl, st));
      k_label_count<<<grid_for(n, kT), kT, 0, st>>>(n, fof_label, cntl);
      RS_LAUNCHED(ctx, "k_label_count");
      k_label_keep<<<grid_for(nl, kT), kT, 0, st>>>(nl, cntl, min_size, knode, koff);
      RS_LAUNCHED(ctx, "k_label_keep");
      RS_TRY(exclusive_scan_i64(ctx, nl, knode, knode + nl, st));
      RS_TRY(exclusive_scan_i64(ctx, nl, koff, koff + nl, st));
      RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box, knode + nl, 8, cudaMemcpyDeviceToHost, st));
      RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box + 1, koff + nl, 8, cudaMemcpyDeviceToHost, st));
      RS_CUDA(ctx, cudaStreamSynchronize(st));
      nodes = ctx->host_box[0];
      members = ctx->host_box[1];
      RS_TRY(ensure_nodes(ctx, 0, std::max<int64_t>(nodes, 1) * 2, st));
      RS_TRY(ensure_members(ctx, 0, std::max<int64_t>(members, 1) * 2, st));
      Hier h = hier_of(ctx);
      if (members > 0) {
        uint64_t* ka = scratch_t<uint64_t>(ctx, S_KEY_A, size_t(members));
        uint64_t* kb = scratch_t<uint64_t>(ctx, S_KEY_B, size_t(members));
        uint32_t* va = scratch_t<uint32_t>(ctx, S_VAL_A, size_t(members));
        uint32_t* vb = scratch_t<uint32_t>(ctx, S_VAL_B, size_t(members));
        if (!ka || !kb || !va || !vb) return RS_ERR_OOM;
        k_label_nodes<<<grid_for(nl, kT), kT, 0, st>>>(nl, cntl, min_size, knode, koff, h.node_off,
                                                      h.node_size, h.node_parent, h.node_level);
        RS_LAUNCHED(ctx, "k_label_nodes");
        RS_CUDA(ctx, cudaMemsetAsync(mx, 0, 8, st));
        k_label_keys<<<grid_for(n, kT), kT, 0, st>>>(n, ids, fof_label, cntl, min_size, knode, bid,
                                                    mx, ka, va);
        RS_LAUNCHED(ctx, "k_label_keys");
        uint64_t* keys;
        uint32_t* vals;
        RS_TRY(radix_sort_u64(ctx, members, bits_for(uint64_t(std::max<int64_t>(nodes - 1, 1))) + bid,
                              ka, va, kb, vb, &keys, &vals, st));
        k_copy_u32<<<grid_for(members, kT), kT, 0, st>>>(members, vals, h.mem);
        RS_LAUNCHED(ctx, "k_copy_u32");
        k_level0_minid<<<grid_for(nodes, kT), kT, 0, st>>>(nodes, h.node_off, h.mem, ids, h.node_minid);
        RS_LAUNCHED(ctx, "k_level0_minid");
      }
    } else {
      uint64_t* ka = scratch_t<uint64_t>(ctx, S_KEY_A, n);
      uint64_t* kb = scratch_t<uint64_t>(ctx, S_KEY_B, n);
      uint32_t* va = scratch_t<uint32_t>(ctx, S_VAL_A, n);
      uint32_t* vb = scratch_t<uint32_t>(ctx, S_VAL_B, n);
      int64_t* head = scratch_t<int64_t>(ctx, S_GKEY_A, size_t(n) + 1);
      int64_t* run_start = scratch_t<int64_t>(ctx, S_GKEY_B, size_t(n) + 1);
      int64_t* rsize = scratch_t<int64_t>(ctx, S_GVAL_A, size_t(n) * 2 + 2);
      int64_t* keep = scratch_t<int64_t>(ctx, S_GVAL_B, size_t(n) * 2 + 2);
      if (!ka || !kb || !va || !vb || !head || !run_start || !rsize || !keep) return RS_ERR_OOM;
      int64_t* node_of_run = rsize + n + 1;
      int64_t* mem_off = keep + n + 1;
      k_id_keys<<<grid_for(n, kT), kT, 0, st>>>(n, ids, ka, va);
      RS_LAUNCHED(ctx, "k_id_keys");
      uint64_t* keys;
      uint32_t* vals;
      RS_TRY(radix_sort_u64(ctx, n, bid, ka, va, kb, vb, &keys, &vals, st));
      {
        uint64_t* lk = keys == ka ? kb : ka;  // labels of the id-sorted particles
        uint32_t* lv = vals == va ? vb : va;
        k_label_of<<<grid_for(n, kT), kT, 0, st>>>(n, vals, fof_label, lk);
        RS_LAUNCHED(ctx, "k_label_of");
        RS_TRY(radix_sort_u64(ctx, n, bits_for(max_lab), lk, vals, keys, lv, &keys, &vals, st));
      }
      const int b = 0;  // keys are the labels themselves
      k_run_heads<<<grid_for(n, kT), kT, 0, st>>>(n, keys, b, head);
      RS_LAUNCHED(ctx, "k_run_heads");
      RS_TRY(exclusive_scan_i64(ctx, n, head, head + n, st));
      RS_TRY(read_back(ctx, head + n, 8, st));
      const int64_t nruns = ctx->host_box[0];
      k_run_starts<<<grid_for(n, kT), kT, 0, st>>>(n, keys, b, head, run_start);
      RS_LAUNCHED(ctx, "k_run_starts");
      k_run_keep<<<grid_for(nruns, kT), kT, 0, st>>>(nruns, n, run_start, min_size, keep, rsize);
      RS_LAUNCHED(ctx, "k_run_keep");
      RS_CUDA(ctx, cudaMemcpyAsync(node_of_run, keep, sizeof(int64_t) * nruns,
                                   cudaMemcpyDeviceToDevice, st));
      RS_TRY(exclusive_scan_i64(ctx, nruns, node_of_run, node_of_run + nruns, st));
      k_size_mask<<<grid_for(nruns, kT), kT, 0, st>>>(nruns, keep, rsize, mem_off);
      RS_LAUNCHED(ctx, "k_size_mask");
      RS_TRY(exclusive_scan_i64(ctx, nruns, mem_off, mem_off + nruns, st));
      RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box, node_of_run + nruns, 8, cudaMemcpyDeviceToHost, st));
      RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box + 1, mem_off + nruns, 8, cudaMemcpyDeviceToHost, st));
      RS_CUDA(ctx, cudaStreamSynchronize(st));
      nodes = ctx->host_box[0];
      members = ctx->host_box[1];
      RS_TRY(ensure_nodes(ctx, 0, std::max<int64_t>(nodes, 1) * 2, st));
      RS_TRY(ensure_members(ctx, 0, std::max<int64_t>(members, 1) * 2, st));
      Hier h = hier_of(ctx);
      if (nruns > 0) {
        k_level0_nodes<<<grid_for(nruns, kT), kT, 0, st>>>(nruns, run_start, rsize, keep, node_of_run,
                                                         mem_off, vals, ids, h.node_off, h.node_size,
                                                         h.node_parent, h.node_level, h.node_minid);
        RS_LAUNCHED(ctx, "k_level0_nodes");
        k_level0_members<<<grid_for(n, kT), kT, 0, st>>>(n, keys, b, head, run_start, keep, mem_off,
                                                         vals, h.mem);
        RS_LAUNCHED(ctx, "k_level0_members");
      }
    }
    Hier h = hier_of(ctx);
    k_fill_i64<<<1, 1, 0, st>>>(1, h.node_off + nodes, members);
    RS_LAUNCHED(ctx, "k_fill_i64");
  }
  // ---------------- levels
  int64_t nb = 0, ne = nodes, mb = 0, me = members;
  int32_t levels = 0;
  const int f_num = ctx->cfg.f_num, f_den = ctx->cfg.f_den;
  while (ne > nb) {
    const int64_t nn = ne - nb, m = me - mb;
    Hier h = hier_of(ctx);
    k_member_node<<<grid_for(m, kT), kT, 0, st>>>(mb, me, nb, nn, h.node_off, h.mnode);
    RS_LAUNCHED(ctx, "k_member_node");
    RS_TRY(gather_members(ctx, mb, me, nb, ne, pos, vel, st));
    double* sums = scratch_t<double>(ctx, S_NODE_TMP, size_t(nn) * 12);
    if (!sums) return RS_ERR_OOM;
    RS_TRY((cro_segmented<12, MomentTerm>(ctx, nn, h.node_off + nb, h.node_size + nb, m,
                                          MomentTerm{h.U, h.V}, sums, st)));
    k_node_inv<<<grid_for(nn, kT), kT, 0, st>>>(nb, nn, h.node_size, sums, h.inv, h.mom);
    RS_LAUNCHED(ctx, "k_node_inv");
    // tiles of 128 members
    int64_t* tile_off = scratch_t<int64_t>(ctx, S_SELECT, size_t(nn) + 1);
    float* nn2 = scratch_t<float>(ctx, S_NN2, size_t(m));
    uint32_t* uf = scratch_t<uint32_t>(ctx, S_UF, size_t(m));
    uint32_t* cnt = scratch_t<uint32_t>(ctx, S_ROOT_CNT, size_t(m));
    int64_t* cflag = scratch_t<int64_t>(ctx, S_FLAGS, size_t(m) + 1);
    int64_t* cidx = scratch_t<int64_t>(ctx, S_CHILD_IDX, size_t(m) + 1);
    int64_t* mpos = scratch_t<int64_t>(ctx, S_GKEY_A, size_t(m) + 1);
    if (!tile_off || !nn2 || !uf || !cnt || !cflag || !cidx || !mpos) return RS_ERR_OOM;
    // batched form: pruned searches, except on levels of at most kPrunedMinMembers members,
    // where the brute-force pair kernels (identical results) cost less than the bucket set-up
    const bool batched = ctx->cfg.batched != 0 && m > kPrunedMinMembers;
    const int64_t tiles_ub = nn + m / kTile6 + 1;
    if (batched) {
      RS_TRY(prune6d_prepare(ctx, nb, nn, mb, m, sums, st));
      RS_TRY(prune6d_nn(ctx, nb, nn, mb, m, nn2, st));
      h = hier_of(ctx);
    } else {
      k_tile_counts<<<grid_for(nn, kT), kT, 0, st>>>(nb, nn, h.node_size, kTile6, tile_off);
      RS_LAUNCHED(ctx, "k_tile_counts");
      RS_TRY(exclusive_scan_i64(ctx, nn, tile_off, tile_off + nn, st));
      {
        ProfScope prof_(ctx, "k_nn6d", st);
        k_nn6d<<<grid_for(tiles_ub, 1), kTile6, 0, st>>>(nb, nn, tile_off, h.node_off, h.node_size, h.inv,
                                                        h.U, h.V, nn2, mb);
      }
      RS_LAUNCHED(ctx, "k_nn6d");
    }
    {
      ProfScope prof_(ctx, "k_select_l2", st);
      k_select_l2_warp<<<grid_for(nn, kT / 32), kT, 0, st>>>(nb, nn, h.node_off, h.node_size, nn2, mb, f_num,
                                                            f_den, h.inv, nullptr);
      k_select_l2<<<unsigned(nn), kT, 0, st>>>(nb, h.node_off, h.node_size, nn2, mb, f_num, f_den, h.inv,
                                               nullptr);
    }
    RS_LAUNCHED(ctx, "k_select_l2");
    if (batched) {  // bounded searches: nodes whose l2 fell outside their bounds, exactly again
      const int* failed = nullptr;
      RS_TRY(prune6d_check(ctx, nb, nn, m, nn2, &failed, st));
      if (failed) {  // bounded nodes can be small enough for the warp selection too
        h = hier_of(ctx);
        ProfScope prof_(ctx, "k_select_l2", st);
        k_select_l2_warp<<<grid_for(nn, kT / 32), kT, 0, st>>>(nb, nn, h.node_off, h.node_size, nn2, mb, f_num,
                                                              f_den, h.inv, failed);
        k_select_l2<<<unsigned(nn), kT, 0, st>>>(nb, h.node_off, h.node_size, nn2, mb, f_num, f_den, h.inv,
                                                 failed);
        RS_LAUNCHED(ctx, "k_select_l2");
      }
    }
    k_iota_u32<<<grid_for(m, kT), kT, 0, st>>>(m, uf);
    RS_LAUNCHED(ctx, "k_iota_u32");
    if (batched) {
      RS_TRY(prune6d_link(ctx, nb, nn, mb, m, nn2, uf, st));
    } else {
      {
        ProfScope prof_(ctx, "k_link6d", st);
        k_link6d<<<grid_for(tiles_ub, 1), kTile6, 0, st>>>(nb, nn, tile_off, h.node_off, h.node_size,
                                                          h.inv, h.U, h.V, nn2, uf, mb);
      }
      RS_LAUNCHED(ctx, "k_link6d");
    }
    RS_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * m, st));
    k_comp_count<<<grid_for(m, kT), kT, 0, st>>>(m, uf, cnt);
    RS_LAUNCHED(ctx, "k_comp_count");
    k_child_flags<<<grid_for(m, kT), kT, 0, st>>>(m, mb, uf, cnt, h.mnode, h.node_size, min_size, cflag);
    RS_LAUNCHED(ctx, "k_child_flags");
    RS_CUDA(ctx, cudaMemcpyAsync(cidx, cflag, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, st));
    RS_TRY(exclusive_scan_i64(ctx, m, cidx, cidx + m, st));
    k_member_flags<<<grid_for(m, kT), kT, 0, st>>>(m, uf, cflag, mpos);
    RS_LAUNCHED(ctx, "k_member_flags");
    RS_TRY(exclusive_scan_i64(ctx, m, mpos, mpos + m, st));
    k_deepest<<<grid_for(m, kT), kT, 0, st>>>(mb, me, h.mem, h.mnode, uf, cflag, deep, deep_pos);
    RS_LAUNCHED(ctx, "k_deepest");
    RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box, cidx + m, 8, cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box + 1, mpos + m, 8, cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    const int64_t nchild = ctx->host_box[0], mchild = ctx->host_box[1];
    ++levels;
    if (nchild == 0) {
      nb = ne;
      break;
    }
    RS_TRY(ensure_nodes(ctx, ne, ne + nchild, st));
    RS_TRY(ensure_members(ctx, me, me + mchild, st));
    h = hier_of(ctx);
    uint64_t* ka = scratch_t<uint64_t>(ctx, S_KEY_A, size_t(mchild));
    uint64_t* kb = scratch_t<uint64_t>(ctx, S_KEY_B, size_t(mchild));
    uint32_t* va = scratch_t<uint32_t>(ctx, S_VAL_A, size_t(mchild));
    uint32_t* vb = scratch_t<uint32_t>(ctx, S_VAL_B, size_t(mchild));
    int64_t* csize = scratch_t<int64_t>(ctx, S_GVAL_A, size_t(nchild) + 1);
    if (!ka || !kb || !va || !vb || !csize) return RS_ERR_OOM;
    k_child_members<<<grid_for(m, kT), kT, 0, st>>>(m, mb, uf, cidx, cflag, mpos, h.mem, ka, va);
    RS_LAUNCHED(ctx, "k_child_members");
    uint64_t* skeys;
    uint32_t* svals;
    RS_TRY(radix_sort_u64(ctx, mchild, bits_for(uint64_t(nchild)), ka, va, kb, vb, &skeys, &svals, st));
    k_copy_u32<<<grid_for(mchild, kT), kT, 0, st>>>(mchild, svals, h.mem + me);
    RS_LAUNCHED(ctx, "k_copy_u32");
    k_child_nodes<<<grid_for(m, kT), kT, 0, st>>>(m, mb, ne, uf, cnt, cflag, cidx, h.mnode, h.mem, ids,
                                                 h.node_size, h.node_parent, h.node_level,
                                                 h.node_minid);
    RS_LAUNCHED(ctx, "k_child_nodes");
    RS_CUDA(ctx, cudaMemcpyAsync(csize, h.node_size + ne, sizeof(int64_t) * nchild,
                                 cudaMemcpyDeviceToDevice, st));
    RS_TRY(exclusive_scan_i64(ctx, nchild, csize, csize + nchild, st));
    k_offsets_add<<<grid_for(nchild + 1, kT), kT, 0, st>>>(nchild + 1, csize, me, h.node_off + ne);
    RS_LAUNCHED(ctx, "k_offsets_add");
    nb = ne;
    ne += nchild;
    mb = me;
    me += mchild;
  }
  ctx->have_hier = true;
  ctx->h_pos = pos;
  ctx->h_vel = vel;
  ctx->n_particles = n;
  ctx->n_nodes = ne;
  ctx->n_members = me;
  ctx->n_levels = levels;
  if (n_nodes_out) *n_nodes_out = ne;
  if (n_members_out) *n_members_out = me;
  return RS_OK;
}

namespace {
__global__ void k_u32_to_i64(int64_t n, const uint32_t* __restrict__ a, int64_t* __restrict__ b) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}
}  // namespace

extern "C" int rs_fof6d_copy(rs_ctx* ctx, int64_t* node_parent, int32_t* node_level,
                             int64_t* node_min_id, int64_t* node_size, int64_t* member_offsets,
                             int64_t* member_idx, int64_t* particle_deepest_node, void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (!ctx->have_hier) return set_error(ctx, RS_ERR_STATE, "rs_fof6d has not run on this context");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  Hier h = hier_of(ctx);
  const int64_t nn = ctx->n_nodes, nm = ctx->n_members;
  auto cp = [&](void* dst, const void* src, size_t bytes) -> int {
    if (dst && bytes) RS_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
    return RS_OK;
  };
  RS_TRY(cp(node_parent, h.node_parent, 8 * nn));
  RS_TRY(cp(node_level, h.node_level, 4 * nn));
  RS_TRY(cp(node_min_id, h.node_minid, 8 * nn));
  RS_TRY(cp(node_size, h.node_size, 8 * nn));
  RS_TRY(cp(member_offsets, h.node_off, 8 * (nn + 1)));
  RS_TRY(cp(particle_deepest_node, h.deepest, 8 * ctx->n_particles));
  if (member_idx && nm) {
    k_u32_to_i64<<<grid_for(nm, kT), kT, 0, st>>>(nm, h.mem, member_idx);
    RS_LAUNCHED(ctx, "k_u32_to_i64");
  }
  return RS_OK;
}

extern "C" int rs_fof6d_node_params(rs_ctx* ctx, float* params_out, void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (!ctx->have_hier) return set_error(ctx, RS_ERR_STATE, "rs_fof6d has not run on this context");
  if (!params_out && ctx->n_nodes) return set_error(ctx, RS_ERR_INVALID_ARG, "params_out is NULL");
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  if (ctx->n_nodes)
    RS_CUDA(ctx, cudaMemcpyAsync(params_out, hier_of(ctx).inv, 16 * ctx->n_nodes,
                                 cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
  return RS_OK;
}

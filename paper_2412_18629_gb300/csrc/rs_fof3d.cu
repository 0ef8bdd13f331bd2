// 3D friends-of-friends over a periodic snapshot (Section "Parallelization": every process runs
// 3D FoF on its particles before subhalo finding).
//
// Pipeline (one stream, no host round trip except the optional group count):
//   k_cell_keys   cell key per particle on a grid of sub-cells of side sc <= 0.99 ll / sqrt(3)
//                 (so two particles in one sub-cell are always linked) -> mixed-radix key
//                 (z ns + y) ns + x; value = particle index
//   radix sort    (key, index), ceil(log2 ns^3) key bits (32 for ns = 1600, not 3*11)
//   k_gather_pos  sorted positions as float4; keys re-packed (z, y, x) with XB bits per axis
//   k_row_start   dense table of the first sorted position of every (z, y) row
//   k_cell_bounds cell start (union-find parent = the cell's first particle: every sub-cell is a
//                 clique) and cell end per sorted position
//   k_fof_link    per particle (particles alone in their sub-cell, then the others, in two
//                 launches), the half stencil of rows within R sub-cells; a neighbour cell is
//                 skipped when its root already equals the particle's root, otherwise scanned
//                 until the first linked member (one link joins the whole clique)
//   k_fof_roots   after full path compression: each root stores its id and counts as a group;
//                 k_fof_member_min lowers it to the smallest member id (atomicMin)
//   k_fof_labels  label of every particle in input order
#include <cmath>

#include "rs_common.cuh"

namespace {

constexpr int kThreads = 256;

struct Grid3 {
  int ns;        // sub-cells per axis
  int xb;        // key bits per axis
  int R;         // stencil radius in sub-cells
  bool full;     // 2R+1 > ns: visit every cell once instead of the half stencil
  float inv_sc;  // ns / L
  int64_t nrows; // 2^(2 xb)
};

int make_grid(rs_ctx* ctx, float L, float ll, Grid3* g) {
  if (!(L > 0.f) || !(ll > 0.f) || !std::isfinite(L) || !std::isfinite(ll))
    return rs::set_error(ctx, RS_ERR_INVALID_ARG, "box_L and link_len must be positive");
  const double sc_target = 0.99 * double(ll) / std::sqrt(3.0);
  double nsd = std::ceil(double(L) / sc_target);
  if (nsd < 1) nsd = 1;
  if (nsd > 4096)
    return rs::set_error(ctx, RS_ERR_INVALID_ARG,
                         "box_L / link_len = %g needs more than 4096 sub-cells per axis",
                         double(L) / double(ll));
  g->ns = int(nsd);
  const double sc = double(L) / g->ns;
  int R = 1;
  while (R * sc <= double(ll) * (1.0 + 1e-3)) ++R;
  g->R = R;
  g->full = (2 * R + 1) > g->ns;
  int xb = 1;
  while ((1 << xb) < g->ns) ++xb;
  g->xb = xb;
  g->nrows = int64_t(1) << (2 * xb);
  g->inv_sc = float(double(g->ns) / double(L));
  return RS_OK;
}

__global__ void __launch_bounds__(kThreads)
k_cell_keys(int64_t n, const float* __restrict__ pos, float inv_sc, int ns, int xb,
            uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float x = pos[3 * i + d];
    int k = int(__fmul_rn(x, inv_sc));
    k = k < 0 ? 0 : (k >= ns ? ns - 1 : k);
    c[d] = uint32_t(k);
  }
  keys[i] = (uint64_t(c[2]) * uint64_t(ns) + c[1]) * uint64_t(ns) + c[0];  // mixed radix
  vals[i] = uint32_t(i);
}

// Sorted positions as float4, and the sorted mixed-radix keys (z ns + y) ns + x (the fewest key
// bits for the sort, same order) re-packed with XB bits per axis for the row and cell lookups.
__global__ void __launch_bounds__(kThreads)
k_gather_pos(int64_t n, const uint32_t* __restrict__ idx, const float* __restrict__ pos,
             const uint64_t* __restrict__ mkeys, int ns, int xb, float4* __restrict__ posS,
             uint64_t* __restrict__ keys) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t s = idx[i];
  posS[i] = make_float4(pos[3 * s], pos[3 * s + 1], pos[3 * s + 2], 0.f);
  const uint64_t k = mkeys[i];
  uint64_t x, y, z;
  if (k < (uint64_t(1) << 32)) {  // 32-bit division whenever ns^3 fits (ns <= 1625)
    const uint32_t k32 = uint32_t(k), n32 = uint32_t(ns);
    const uint32_t yz = k32 / n32;
    x = k32 - yz * n32;
    z = yz / n32;
    y = yz - uint32_t(z) * n32;
  } else {
    const uint64_t yz = k / uint64_t(ns);
    x = k - yz * uint64_t(ns);
    z = yz / uint64_t(ns);
    y = yz - z * uint64_t(ns);
  }
  keys[i] = (((z << xb) | y) << xb) | x;
}

__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t* __restrict__ a, uint32_t lo,
                                                    uint32_t hi, uint64_t v) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// row_start[r] = first sorted position whose row (key >> xb) is >= r, for r in [0, nrows]: one
// thread per row, binary search over the sorted keys (neighbouring rows share search paths).
__global__ void __launch_bounds__(kThreads)
k_row_start(int64_t n, const uint64_t* __restrict__ keys, int xb, int64_t nrows,
            uint32_t* __restrict__ row_start) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r > nrows) return;
  row_start[r] = lower_bound_u64(keys, 0u, uint32_t(n), uint64_t(r) << xb);
}

__device__ __forceinline__ uint32_t upper_bound_u64(const uint64_t* __restrict__ a, uint32_t lo,
                                                    uint32_t hi, uint64_t v) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads)
k_cell_bounds(int64_t n, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ row_start,
              int xb, uint32_t* __restrict__ cell_end, uint32_t* __restrict__ parent) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = keys[i];
  const uint64_t r = k >> xb;
  const uint32_t a = row_start[r], b = row_start[r + 1];
  parent[i] = lower_bound_u64(keys, a, uint32_t(i), k);
  cell_end[i] = upper_bound_u64(keys, uint32_t(i) + 1, b, k);
}

struct LinkArgs {
  const uint64_t* keys;
  const float4* posS;
  const uint32_t* row_start;
  const uint32_t* cell_end;
  uint32_t* parent;
  int ns, xb, R;
  bool full;
  float L, hL, ll2;
};

// Scan cells with x sub-cell in [x0, x1] of row (zz, yy) against particle i.
__device__ __forceinline__ void scan_cells(const LinkArgs& A, uint32_t i, uint64_t key_i,
                                           float4 pi, uint32_t& root_i, int zz, int yy, int x0,
                                           int x1) {
  const uint64_t row = (uint64_t(zz) << A.xb) | uint64_t(yy);
  const uint32_t a = A.row_start[row], b = A.row_start[row + 1];
  if (a == b) return;
  const uint64_t kmin = (row << A.xb) | uint64_t(x0);
  const uint64_t kmax = (row << A.xb) | uint64_t(x1);
  uint32_t j = lower_bound_u64(A.keys, a, b, kmin);
  while (j < b) {
    const uint64_t kj = A.keys[j];
    if (kj > kmax) break;
    const uint32_t e = A.cell_end[j];
    if (kj != key_i) {
      root_i = rsd::uf_find(A.parent, root_i);
      const uint32_t rj = rsd::uf_find(A.parent, j);
      if (rj != root_i) {
        for (uint32_t jj = j; jj < e; ++jj) {
          const float4 pj = A.posS[jj];
          const float dx = rsd::wrap_diff(pi.x, pj.x, A.L, A.hL);
          const float dy = rsd::wrap_diff(pi.y, pj.y, A.L, A.hL);
          const float dz = rsd::wrap_diff(pi.z, pj.z, A.L, A.hL);
          if (rsd::sq3(dx, dy, dz) <= A.ll2) {
            rsd::uf_unite(A.parent, i, jj);
            root_i = rsd::uf_find(A.parent, i);
            break;
          }
        }
      }
    }
    j = e;
  }
}

__device__ __forceinline__ void scan_row(const LinkArgs& A, uint32_t i, uint64_t key_i, float4 pi,
                                         uint32_t& root_i, int zz, int yy, int xa, int xb_) {
  const int ns = A.ns;
  // periodic wrap of offsets within one box length (|offset| <= R < ns): a compare and an add
  // instead of an integer division
  zz += zz < 0 ? ns : (zz >= ns ? -ns : 0);
  yy += yy < 0 ? ns : (yy >= ns ? -ns : 0);
  if (xa < 0) {
    scan_cells(A, i, key_i, pi, root_i, zz, yy, xa + ns, ns - 1);
    scan_cells(A, i, key_i, pi, root_i, zz, yy, 0, xb_);
  } else if (xb_ >= ns) {
    scan_cells(A, i, key_i, pi, root_i, zz, yy, xa, ns - 1);
    scan_cells(A, i, key_i, pi, root_i, zz, yy, 0, xb_ - ns);
  } else {
    scan_cells(A, i, key_i, pi, root_i, zz, yy, xa, xb_);
  }
}

// Two launches: particles alone in their sub-cell (sparse regions: short scans, few links),
// then particles of shared sub-cells (dense regions: many occupied neighbour cells). Keeping the
// two kinds in different launches keeps a warp's lanes on similar amounts of work, and each
// launch reads the particles in sorted order. Measured on 2^27 particles in L = 512 Mpc/h, two
// alternatives were slower: occupancy bits per row segment to skip empty stencil rows (their
// random reads into a 0.5 GB bit array cost more than the row searches they save) and one
// launch over a partition of the two kinds (its warps gather scattered particles).
__global__ void __launch_bounds__(kThreads) k_fof_link(int64_t n, LinkArgs A, bool alone) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t i = uint32_t(t);
  const uint64_t key_i = A.keys[i];
  const bool single = (i == 0 || A.keys[i - 1] != key_i) && (t + 1 == n || A.keys[i + 1] != key_i);
  if (single != alone) return;
  const uint32_t mask = (1u << A.xb) - 1u;
  const int kx = int(key_i & mask), ky = int((key_i >> A.xb) & mask), kz = int(key_i >> (2 * A.xb));
  const float4 pi = A.posS[i];
  uint32_t root_i = rsd::uf_find(A.parent, i);
  const int R = A.R;
  if (!A.full) {
    for (int dz = 0; dz <= R; ++dz)
      for (int dy = (dz == 0 ? 0 : -R); dy <= R; ++dy) {
        const int xlo = (dz == 0 && dy == 0) ? 1 : -R;
        scan_row(A, i, key_i, pi, root_i, kz + dz, ky + dy, kx + xlo, kx + R);
      }
  } else {
    for (int zz = 0; zz < A.ns; ++zz)
      for (int yy = 0; yy < A.ns; ++yy) scan_cells(A, i, key_i, pi, root_i, zz, yy, 0, A.ns - 1);
  }
}

// After full compression parent[i] is i's root. Each root stores its own id (a plain store:
// most roots are single particles) and counts as a group; then every other particle lowers its
// root's entry to its id (warp-aggregated atomicMin over runs of equal roots).
__global__ void __launch_bounds__(kThreads)
k_fof_roots(int64_t n, const uint32_t* __restrict__ parent, const uint32_t* __restrict__ idx,
            const int64_t* __restrict__ ids, unsigned long long* __restrict__ minid,
            unsigned long long* __restrict__ counter) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool root = i < n && parent[i] == uint32_t(i);  // every lane stays for the count
  if (root) minid[i] = (unsigned long long)ids[idx[i]];
  rsd::warp_count(counter, root);
}

__global__ void __launch_bounds__(kThreads)
k_fof_member_min(int64_t n, const uint32_t* __restrict__ parent, const uint32_t* __restrict__ idx,
                 const int64_t* __restrict__ ids, unsigned long long* __restrict__ minid) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint32_t r = i < n ? parent[i] : 0u;
  const bool member = i < n && r != uint32_t(i);  // every lane stays for the run reduction
  rsd::warp_run_min(minid, r, member, member ? (unsigned long long)ids[idx[i]] : ~0ull);
}

__global__ void __launch_bounds__(kThreads)
k_fof_compress(int64_t n, uint32_t* __restrict__ parent) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  parent[i] = rsd::uf_find_ro(parent, uint32_t(i));
}

__global__ void __launch_bounds__(kThreads)
k_fof_labels(int64_t n, const uint32_t* __restrict__ parent, const uint32_t* __restrict__ idx,
             const unsigned long long* __restrict__ minid, int64_t* __restrict__ label_out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  label_out[idx[i]] = int64_t(minid[parent[i]]);
}

}  // namespace

namespace {
__global__ void k_ids_as_keys(int64_t n, const int64_t* __restrict__ ids, uint64_t* __restrict__ keys,
                              uint32_t* __restrict__ vals) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = uint64_t(ids[i]);
  vals[i] = uint32_t(i);
}

// Invalid ids among the sorted ids: a repeated value, or a negative one (sorted last as uint64).
__global__ void k_bad_ids(int64_t n, const uint64_t* __restrict__ keys, unsigned long long* __restrict__ bad) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool b = (i > 0 && keys[i] == keys[i - 1]) || (keys[i] >> 63) != 0;
  rsd::warp_count(bad, b);
}
}  // namespace

// The optional check that ids are unique and non-negative (rs_config.check_ids): a 64-bit radix
// sort of the ids and a comparison of neighbours.
static int check_ids(rs_ctx* ctx, int64_t n, const int64_t* ids, cudaStream_t st) {
  using namespace rs;
  uint64_t* ka = scratch_t<uint64_t>(ctx, S_KEY_A, n);
  uint64_t* kb = scratch_t<uint64_t>(ctx, S_KEY_B, n);
  uint32_t* va = scratch_t<uint32_t>(ctx, S_VAL_A, n);
  uint32_t* vb = scratch_t<uint32_t>(ctx, S_VAL_B, n);
  unsigned long long* bad = scratch_t<unsigned long long>(ctx, S_COUNTER, 8);
  if (!ka || !kb || !va || !vb || !bad) return RS_ERR_OOM;
  k_ids_as_keys<<<grid_for(n, 256), 256, 0, st>>>(n, ids, ka, va);
  RS_LAUNCHED(ctx, "k_ids_as_keys");
  uint64_t* ks;
  uint32_t* vs;
  RS_TRY(radix_sort_u64(ctx, n, 64, ka, va, kb, vb, &ks, &vs, st));
  RS_CUDA(ctx, cudaMemsetAsync(bad, 0, 8, st));
  k_bad_ids<<<grid_for(n, 256), 256, 0, st>>>(n, ks, bad);
  RS_LAUNCHED(ctx, "k_bad_ids");
  RS_TRY(read_back(ctx, bad, 8, st));
  if (ctx->host_box[0] != 0)
    return set_error(ctx, RS_ERR_INVALID_ARG, "%lld repeated or negative ids",
                     (long long)ctx->host_box[0]);
  return RS_OK;
}

extern "C" int rs_fof3d(rs_ctx* ctx, int64_t n, const float* pos, const int64_t* ids,
                        int64_t* label_out, int64_t* n_groups_out, void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n < 0 || n >= (int64_t(1) << 32) - 1)
    return rs::set_error(ctx, RS_ERR_INVALID_ARG, "n = %lld out of range", (long long)n);
  if (n > 0 && (!pos || !ids || !label_out))
    return rs::set_error(ctx, RS_ERR_INVALID_ARG, "null device pointer");
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  if (n == 0) {
    if (n_groups_out) *n_groups_out = 0;
    return RS_OK;
  }
  if (ctx->cfg.check_ids) RS_TRY(check_ids(ctx, n, ids, st));
  Grid3 g;
  RS_TRY(make_grid(ctx, ctx->cfg.box_L, ctx->cfg.link_len, &g));
  using namespace rs;
  uint64_t* ka = scratch_t<uint64_t>(ctx, S_KEY_A, n);
  uint64_t* kb = scratch_t<uint64_t>(ctx, S_KEY_B, n);
  uint32_t* va = scratch_t<uint32_t>(ctx, S_VAL_A, n);
  uint32_t* vb = scratch_t<uint32_t>(ctx, S_VAL_B, n);
  float4* posS = scratch_t<float4>(ctx, S_POS_SORTED, n);
  uint32_t* row_start = scratch_t<uint32_t>(ctx, S_ROW_START, size_t(g.nrows) + 1);
  uint32_t* cend = scratch_t<uint32_t>(ctx, S_CELL_END, n);
  uint32_t* parent = scratch_t<uint32_t>(ctx, S_PARENT, n);
  unsigned long long* minid = scratch_t<unsigned long long>(ctx, S_MINID, n);
  unsigned long long* counter = scratch_t<unsigned long long>(ctx, S_COUNTER, 8);
  if (!ka || !kb || !va || !vb || !posS || !row_start || !cend || !parent || !minid || !counter)
    return RS_ERR_OOM;
  const unsigned grid = grid_for(n, kThreads);
  k_cell_keys<<<grid, kThreads, 0, st>>>(n, pos, g.inv_sc, g.ns, g.xb, ka, va);
  RS_LAUNCHED(ctx, "k_cell_keys");
  uint64_t* mkeys;
  uint32_t* idx;
  const uint64_t ns3 = uint64_t(g.ns) * uint64_t(g.ns) * uint64_t(g.ns);
  int kbits = 1;
  while (kbits < 64 && ((ns3 - 1) >> kbits) != 0) ++kbits;
  RS_TRY(radix_sort_u64(ctx, n, kbits, ka, va, kb, vb, &mkeys, &idx, st));
  uint64_t* keys = (mkeys == ka) ? kb : ka;  // the other key buffer receives the packed keys
  k_gather_pos<<<grid, kThreads, 0, st>>>(n, idx, pos, mkeys, g.ns, g.xb, posS, keys);
  RS_LAUNCHED(ctx, "k_gather_pos");
  k_row_start<<<grid_for(g.nrows + 1, kThreads), kThreads, 0, st>>>(n, keys, g.xb, g.nrows, row_start);
  RS_LAUNCHED(ctx, "k_row_start");
  {
    ProfScope prof_(ctx, "k_cell_bounds", st);
    k_cell_bounds<<<grid, kThreads, 0, st>>>(n, keys, row_start, g.xb, cend, parent);
  }
  RS_LAUNCHED(ctx, "k_cell_bounds");
  LinkArgs A{keys, posS, row_start, cend, parent, g.ns, g.xb, g.R, g.full,
             ctx->cfg.box_L, 0.5f * ctx->cfg.box_L, ctx->cfg.link_len * ctx->cfg.link_len};
  for (const bool alone : {true, false}) {
    {
      ProfScope prof_(ctx, "k_fof_link", st);
      k_fof_link<<<grid, kThreads, 0, st>>>(n, A, alone);
    }
    RS_LAUNCHED(ctx, "k_fof_link");
  }
  RS_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
  k_fof_compress<<<grid, kThreads, 0, st>>>(n, parent);
  RS_LAUNCHED(ctx, "k_fof_compress");
  k_fof_roots<<<grid, kThreads, 0, st>>>(n, parent, idx, ids, minid, counter);
  RS_LAUNCHED(ctx, "k_fof_roots");
  k_fof_member_min<<<grid, kThreads, 0, st>>>(n, parent, idx, ids, minid);
  RS_LAUNCHED(ctx, "k_fof_member_min");
  k_fof_labels<<<grid, kThreads, 0, st>>>(n, parent, idx, minid, label_out);
  RS_LAUNCHED(ctx, "k_fof_labels");
  if (n_groups_out) {
    RS_TRY(read_back(ctx, counter, sizeof(int64_t), st));
    *n_groups_out = ctx->host_box[0];
  }
  return RS_OK;
}

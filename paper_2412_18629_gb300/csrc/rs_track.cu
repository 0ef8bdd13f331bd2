// Temporal tracking of seed halos between two snapshots of the same particles (the paper's
// Summary names temporal tracking among Rockstar's features; the reading implemented here, the
// CPU oracle's bit for bit): particles are matched by id; the progenitor of a seed h2 of the
// later snapshot is the seed h1 of the earlier one holding the most of h2's particles (ties: the
// smaller index; -1 when none of them is in a seed earlier), and the descendant of h1 is the
// seed h2 receiving the most of h1's particles (ties: the smaller index).
//   k_trk_keys   earlier snapshot's ids as sort keys -> stable radix sort by id
//   k_trk_match  per particle of the later snapshot: the earlier seed of its id (binary search)
//   k_trk_pairs  (h2, h1) and (h1, h2) keys of the matched particles -> two radix sorts
//   k_trk_heads, k_trk_runs   run-length counts of equal keys
//   k_trk_best   per group (same first index): the run with the largest count, first = smallest
#include "rs_common.cuh"

using namespace rs;

namespace {

constexpr int kT = 256;

__global__ void k_trk_keys(int64_t n, const int64_t* __restrict__ ids, uint64_t* __restrict__ keys,
                           uint32_t* __restrict__ vals) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = uint64_t(ids[i]);
  vals[i] = uint32_t(i);
}

__global__ void k_trk_match(int64_t n2, const int64_t* __restrict__ ids2, const int64_t* __restrict__ seed2,
                            int64_t n1, const uint64_t* __restrict__ sid1, const uint32_t* __restrict__ sidx1,
                            const int64_t* __restrict__ seed1, int64_t* __restrict__ h1_of,
                            int64_t* __restrict__ flag) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n2) return;
  int64_t h1 = -1;
  if (seed2[j] >= 0) {
    const uint64_t id = uint64_t(ids2[j]);
    int64_t lo = 0, hi = n1;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (sid1[mid] < id) lo = mid + 1; else hi = mid;
    }
    if (lo < n1 && sid1[lo] == id) h1 = seed1[sidx1[lo]];
  }
  h1_of[j] = h1;
  flag[j] = h1 >= 0 ? 1 : 0;
}

__global__ void k_trk_pairs(int64_t n2, const int64_t* __restrict__ flag, const int64_t* __restrict__ seed2,
                            const int64_t* __restrict__ h1_of, uint64_t* __restrict__ k21,
                            uint64_t* __restrict__ k12, uint32_t* __restrict__ v21, uint32_t* __restrict__ v12) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n2 || flag[j + 1] == flag[j]) return;
  const int64_t k = flag[j];
  const uint64_t h2 = uint64_t(seed2[j]), h1 = uint64_t(h1_of[j]);
  k21[k] = (h2 << 32) | h1;
  k12[k] = (h1 << 32) | h2;
  v21[k] = uint32_t(k);
  v12[k] = uint32_t(k);
}

__global__ void k_trk_heads(int64_t np, const uint64_t* __restrict__ keys, int64_t* __restrict__ head) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < np) head[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1 : 0;
}

// After the scan of the heads: run r starts at run_start[r]; run_start[nruns] = np.
__global__ void k_trk_runs(int64_t np, const uint64_t* __restrict__ keys, const int64_t* __restrict__ hs,
                           int64_t* __restrict__ run_start, uint64_t* __restrict__ run_key) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k == 0) run_start[hs[np]] = np;
  if (k >= np) return;
  if (k == 0 || keys[k] != keys[k - 1]) {
    run_start[hs[k]] = k;
    run_key[hs[k]] = keys[k];
  }
}

// One thread per group (runs with the same upper 32 bits, consecutive, lower bits ascending):
// the run of largest count; the first one found is the smallest partner index.
__global__ void k_trk_best(int64_t nruns, const uint64_t* __restrict__ run_key,
                           const int64_t* __restrict__ run_start, int64_t* __restrict__ best,
                           int64_t* __restrict__ best_count) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= nruns) return;
  const uint64_t g = run_key[r] >> 32;
  if (r > 0 && (run_key[r - 1] >> 32) == g) return;  // not the group's first run
  int64_t arg = -1, cnt = 0;
  for (int64_t s = r; s < nruns && (run_key[s] >> 32) == g; ++s) {
    const int64_t c = run_start[s + 1] - run_start[s];
    if (c > cnt) {
      cnt = c;
      arg = int64_t(run_key[s] & 0xffffffffull);
    }
  }
  best[g] = arg;
  best_count[g] = cnt;
}

__global__ void k_trk_fill(int64_t n, int64_t* __restrict__ a, int64_t va, int64_t* __restrict__ b, int64_t vb) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  a[i] = va;
  b[i] = vb;
}

int bits_for(uint64_t v) {
  int b = 1;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

// Sorted (key) pairs -> per group the best partner and its count.
int best_of(rs_ctx* ctx, int64_t np, uint64_t* ka, uint32_t* va, uint64_t* kb, uint32_t* vb, int nbits,
            int64_t* best, int64_t* best_count, cudaStream_t st) {
  uint64_t* keys;
  uint32_t* vals;
  RS_TRY(radix_sort_u64(ctx, np, nbits, ka, va, kb, vb, &keys, &vals, st));
  int64_t* hs = scratch_t<int64_t>(ctx, S_TRK_HEAD, size_t(np) + 1);
  int64_t* rstart = scratch_t<int64_t>(ctx, S_TRK_RSTART, size_t(np) + 1);
  uint64_t* rkey = scratch_t<uint64_t>(ctx, S_TRK_RKEY, size_t(np) + 1);
  if (!hs || !rstart || !rkey) return RS_ERR_OOM;
  k_trk_heads<<<grid_for(np, kT), kT, 0, st>>>(np, keys, hs);
  RS_LAUNCHED(ctx, "k_trk_heads");
  RS_TRY(exclusive_scan_i64(ctx, np, hs, hs + np, st));
  k_trk_runs<<<grid_for(np, kT), kT, 0, st>>>(np, keys, hs, rstart, rkey);
  RS_LAUNCHED(ctx, "k_trk_runs");
  RS_TRY(read_back(ctx, hs + np, 8, st));
  const int64_t nruns = ctx->host_box[0];
  k_trk_best<<<grid_for(nruns, kT), kT, 0, st>>>(nruns, rkey, rstart, best, best_count);
  RS_LAUNCHED(ctx, "k_trk_best");
  return RS_OK;
}

}  // namespace

extern "C" int rs_track(rs_ctx* ctx, int64_t n1, const int64_t* ids1, const int64_t* seed1,
                        int64_t n_nodes1, int64_t n2, const int64_t* ids2, const int64_t* seed2,
                        int64_t n_nodes2, int64_t* progenitor, int64_t* prog_shared,
                        int64_t* descendant, int64_t* desc_shared, void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  const int64_t lim = (int64_t(1) << 32) - 1;
  if (n1 < 0 || n2 < 0 || n1 >= lim || n2 >= lim || n_nodes1 < 0 || n_nodes2 < 0 ||
      n_nodes1 >= lim || n_nodes2 >= lim)
    return set_error(ctx, RS_ERR_INVALID_ARG, "sizes out of range");
  if ((n1 > 0 && (!ids1 || !seed1)) || (n2 > 0 && (!ids2 || !seed2)) ||
      (n_nodes2 > 0 && (!progenitor || !prog_shared)) || (n_nodes1 > 0 && (!descendant || !desc_shared)))
    return set_error(ctx, RS_ERR_INVALID_ARG, "null device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  if (n_nodes2 > 0) {
    k_trk_fill<<<grid_for(n_nodes2, kT), kT, 0, st>>>(n_nodes2, progenitor, -1, prog_shared, 0);
    RS_LAUNCHED(ctx, "k_trk_fill");
  }
  if (n_nodes1 > 0) {
    k_trk_fill<<<grid_for(n_nodes1, kT), kT, 0, st>>>(n_nodes1, descendant, -1, desc_shared, 0);
    RS_LAUNCHED(ctx, "k_trk_fill");
  }
  if (n1 == 0 || n2 == 0) return RS_OK;
  const int64_t nmax = std::max(n1, n2);
  uint64_t* ka = scratch_t<uint64_t>(ctx, S_KEY_A, size_t(nmax));
  uint64_t* kb = scratch_t<uint64_t>(ctx, S_KEY_B, size_t(nmax));
  uint32_t* va = scratch_t<uint32_t>(ctx, S_VAL_A, size_t(nmax));
  uint32_t* vb = scratch_t<uint32_t>(ctx, S_VAL_B, size_t(nmax));
  uint64_t* k2a = scratch_t<uint64_t>(ctx, S_TRK_KA, size_t(n2));
  uint64_t* k2b = scratch_t<uint64_t>(ctx, S_TRK_KB, size_t(n2));
  uint32_t* v2a = scratch_t<uint32_t>(ctx, S_TRK_VA, size_t(n2));
  uint32_t* v2b = scratch_t<uint32_t>(ctx, S_TRK_VB, size_t(n2));
  int64_t* h1_of = scratch_t<int64_t>(ctx, S_TRK_H1, size_t(n2));
  int64_t* flag = scratch_t<int64_t>(ctx, S_TRK_FLAG, size_t(n2) + 1);
  if (!ka || !kb || !va || !vb || !k2a || !k2b || !v2a || !v2b || !h1_of || !flag) return RS_ERR_OOM;
  // earlier snapshot by id
  k_trk_keys<<<grid_for(n1, kT), kT, 0, st>>>(n1, ids1, ka, va);
  RS_LAUNCHED(ctx, "k_trk_keys");
  uint64_t* sid1;
  uint32_t* sidx1;
  RS_TRY(radix_sort_u64(ctx, n1, 63, ka, va, kb, vb, &sid1, &sidx1, st));
  k_trk_match<<<grid_for(n2, kT), kT, 0, st>>>(n2, ids2, seed2, n1, sid1, sidx1, seed1, h1_of, flag);
  RS_LAUNCHED(ctx, "k_trk_match");
  RS_TRY(exclusive_scan_i64(ctx, n2, flag, flag + n2, st));
  RS_TRY(read_back(ctx, flag + n2, 8, st));
  const int64_t np = ctx->host_box[0];
  if (np == 0) return RS_OK;
  // (h2, h1) pairs into the free key buffers, (h1, h2) pairs into the tracker's own
  uint64_t* k21 = (sid1 == ka) ? kb : ka;
  uint32_t* v21 = (sidx1 == va) ? vb : va;
  k_trk_pairs<<<grid_for(n2, kT), kT, 0, st>>>(n2, flag, seed2, h1_of, k21, k2a, v21, v2a);
  RS_LAUNCHED(ctx, "k_trk_pairs");
  uint64_t* k21b = (k21 == ka) ? kb : ka;  // the earlier snapshot's sorted ids are no longer needed
  uint32_t* v21b = (v21 == va) ? vb : va;
  const int bits = 32 + bits_for(uint64_t(std::max<int64_t>(std::max(n_nodes1, n_nodes2), 1)));
  RS_TRY(best_of(ctx, np, k21, v21, k21b, v21b, bits, progenitor, prog_shared, st));
  RS_TRY(best_of(ctx, np, k2a, v2a, k2b, v2b, bits, descendant, desc_shared, st));
  return RS_OK;
}

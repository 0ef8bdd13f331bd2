// Seed halos, the assignment of every FoF-group particle to a seed, and the seeds' host
// relations: the step after the 6D hierarchy (Section "Parallelization": subhalo finding inside
// every FoF halo from 6D phase-space information). The paper gives no formulas for it; the
// reading implemented here:
//   seeds   the nodes without children (each level-0 node has at least one under it);
//   frame   u = wrapped offset from the level-0 node's reference member r0 (smallest id);
//   seed s  centre c_s = float(double(wrap(x_{r_s} - x_{r0})) + CRO(u^s) / g_s), u^s the
//           offsets from s's own reference member r_s (the hierarchy's U), bulk velocity
//           w_s = float(CRO(v) / g_s), and the metric scales (inv_sx2, inv_sv2) of s's split;
//   metric  fl(|u - c_s|^2 inv_sx2_s) + fl(|v - w_s|^2 inv_sv2_s), float32 in d6's order;
//   particle  the seed holding it when its deepest node is a seed, otherwise the nearest seed
//           under its deepest node (ties: the smaller node index);
//   host    of a seed s: among the other seeds of the same level-0 node ranking above it (more
//           assigned particles; equal counts: the smaller node index), the nearest by the
//           candidate's metric at (c_s, w_s); -1 if none.
// Every comparison uses the same float32 operations as the CPU oracle, so the results are
// identical to it.
#include "rs_cro.cuh"

namespace rs {
int gather_members(rs_ctx* ctx, int64_t mb, int64_t me, int64_t nb, int64_t ne, const float* pos,
                   const float* vel, cudaStream_t st);
}  // namespace rs

using namespace rs;

namespace {

constexpr int kT = 256;

__global__ void k_seed_kids(int64_t nn, const int64_t* __restrict__ parent, int* __restrict__ nkids) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < nn && parent[q] >= 0) atomicAdd(nkids + parent[q], 1);
}

__global__ void k_seed_total(int64_t nn, const int* __restrict__ nkids, unsigned long long* __restrict__ n_seeds) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  rsd::warp_count(n_seeds, q < nn && nkids[q] == 0);
}

// Pointer jumping towards the level-0 ancestor: out[q] = in[in[q]] (level-0 nodes point at
// themselves).
__global__ void k_seed_jump(int64_t nn, const int64_t* __restrict__ in, int64_t* __restrict__ out) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < nn) out[q] = in[in[q]];
}

__global__ void k_seed_root_init(int64_t nn, const int64_t* __restrict__ parent, int64_t* __restrict__ r) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < nn) r[q] = parent[q] < 0 ? q : parent[q];
}

// Per seed: add 1 to every ancestor's (and its own) count of seeds under it.
__global__ void k_seed_under_count(int64_t nn, const int64_t* __restrict__ parent, const int* __restrict__ nkids,
                                   unsigned long long* __restrict__ cnt) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= nn || nkids[s] != 0) return;
  for (int64_t q = s; q >= 0; q = parent[q]) atomicAdd(cnt + q, 1ull);
}

__global__ void k_seed_under_fill(int64_t nn, const int64_t* __restrict__ parent, const int* __restrict__ nkids,
                                  const int64_t* __restrict__ off, unsigned long long* __restrict__ fill,
                                  int64_t* __restrict__ list) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= nn || nkids[s] != 0) return;
  for (int64_t q = s; q >= 0; q = parent[q]) list[off[q] + int64_t(atomicAdd(fill + q, 1ull))] = s;
}

// Segments of the seeds for the canonical-order sums (node offset and size; size 0 otherwise).
__global__ void k_seed_segments(int64_t nn, const int* __restrict__ nkids, const int64_t* __restrict__ node_size,
                                int64_t* __restrict__ seg_size) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < nn) seg_size[q] = nkids[q] == 0 ? node_size[q] : 0;
}

struct SeedTerm {  // u^s and v of a member of seed s
  const float4* U;
  const float4* V;
  template <bool kFirst>
  __device__ __forceinline__ void add(int64_t, int64_t p, int64_t, double* acc) const {
    const float4 u = U[p], v = V[p];
    rsd::cro_add<kFirst>(acc[0], rsd::f2d(u.x));
    rsd::cro_add<kFirst>(acc[1], rsd::f2d(u.y));
    rsd::cro_add<kFirst>(acc[2], rsd::f2d(u.z));
    rsd::cro_add<kFirst>(acc[3], rsd::f2d(v.x));
    rsd::cro_add<kFirst>(acc[4], rsd::f2d(v.y));
    rsd::cro_add<kFirst>(acc[5], rsd::f2d(v.z));
  }
};

// Seed centres (level-0 frame) and bulk velocities from the canonical-order sums.
__global__ void k_seed_stats(int64_t nn, const int* __restrict__ nkids, const int64_t* __restrict__ root,
                             const int64_t* __restrict__ node_off, const int64_t* __restrict__ node_size,
                             const uint32_t* __restrict__ mem, const float* __restrict__ pos, float L,
                             const double* __restrict__ sums, float4* __restrict__ cen,
                             float4* __restrict__ bulk) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= nn || nkids[s] != 0) return;
  const int64_t rs_ = mem[node_off[s]], r0 = mem[node_off[root[s]]];
  const double g = double(node_size[s]);
  const double* S = sums + 6 * s;
  const float hL = 0.5f * L;
  float c[3], w[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float o = rsd::wrap_diff(pos[3 * r0 + d], pos[3 * rs_ + d], L, hL);
    c[d] = __double2float_rn(__dadd_rn(double(o), __ddiv_rn(S[d], g)));
    w[d] = __double2float_rn(__ddiv_rn(S[3 + d], g));
  }
  cen[s] = make_float4(c[0], c[1], c[2], 0.f);
  bulk[s] = make_float4(w[0], w[1], w[2], 0.f);
}

__device__ __forceinline__ float seed_metric(float ax, float ay, float az, float4 c, float vx, float vy,
                                             float vz, float4 w, float isx, float isv) {
  const float rx = rsd::sq3(__fsub_rn(ax, c.x), __fsub_rn(ay, c.y), __fsub_rn(az, c.z));
  const float rv = rsd::sq3(__fsub_rn(vx, w.x), __fsub_rn(vy, w.y), __fsub_rn(vz, w.z));
  return __fadd_rn(__fmul_rn(rx, isx), __fmul_rn(rv, isv));
}

// One thread per particle: its seed (argmin over the seeds under its deepest node).
__global__ void k_seed_assign(int64_t n, const int64_t* __restrict__ deepest, const int* __restrict__ nkids,
                              const int64_t* __restrict__ root, const int64_t* __restrict__ node_off,
                              const uint32_t* __restrict__ mem, const float* __restrict__ pos,
                              const float* __restrict__ vel, float L, const int64_t* __restrict__ uoff,
                              const int64_t* __restrict__ ulist, const float4* __restrict__ cen,
                              const float4* __restrict__ bulk, const float4* __restrict__ inv,
                              int64_t* __restrict__ seed, unsigned long long* __restrict__ count) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t dq = deepest[i];
  if (dq < 0) {
    seed[i] = -1;
    return;
  }
  int64_t arg = dq;
  if (nkids[dq] != 0) {
    const int64_t r0 = mem[node_off[root[dq]]];
    const float hL = 0.5f * L;
    const float ux = rsd::wrap_diff(pos[3 * r0], pos[3 * i], L, hL);
    const float uy = rsd::wrap_diff(pos[3 * r0 + 1], pos[3 * i + 1], L, hL);
    const float uz = rsd::wrap_diff(pos[3 * r0 + 2], pos[3 * i + 2], L, hL);
    const float vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
    float best = 0.f;
    arg = -1;
    for (int64_t k = uoff[dq]; k < uoff[dq + 1]; ++k) {
      const int64_t s = ulist[k];
      const float4 sc = inv[s];
      const float d = seed_metric(ux, uy, uz, cen[s], vx, vy, vz, bulk[s], sc.x, sc.y);
      if (arg < 0 || d < best || (d == best && s < arg)) {
        best = d;
        arg = s;
      }
    }
  }
  seed[i] = arg;
  atomicAdd(count + arg, 1ull);
}

// One thread per seed: its host among the seeds of its level-0 node ranking above it.
__global__ void k_seed_host(int64_t nn, const int* __restrict__ nkids, const int64_t* __restrict__ root,
                            const int64_t* __restrict__ uoff, const int64_t* __restrict__ ulist,
                            const float4* __restrict__ cen, const float4* __restrict__ bulk,
                            const float4* __restrict__ inv, const unsigned long long* __restrict__ count,
                            int64_t* __restrict__ host, int64_t* __restrict__ count_out) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= nn) return;
  if (nkids[s] != 0) {
    if (host) host[s] = -2;
    if (count_out) count_out[s] = 0;
    return;
  }
  const unsigned long long ns = count[s];
  const float4 c = cen[s], w = bulk[s];
  const int64_t r = root[s];
  float best = 0.f;
  int64_t arg = -1;
  for (int64_t k = uoff[r]; k < uoff[r + 1]; ++k) {
    const int64_t h = ulist[k];
    if (h == s) continue;
    const unsigned long long nh = count[h];
    if (!(nh > ns || (nh == ns && h < s))) continue;
    const float4 sc = inv[h];
    const float d = seed_metric(c.x, c.y, c.z, cen[h], w.x, w.y, w.z, bulk[h], sc.x, sc.y);
    if (arg < 0 || d < best || (d == best && h < arg)) {
      best = d;
      arg = h;
    }
  }
  if (host) host[s] = arg;
  if (count_out) count_out[s] = int64_t(ns);
}

}  // namespace

extern "C" int rs_assign_seeds(rs_ctx* ctx, const float* pos, const float* vel, int64_t* particle_seed,
                               int64_t* node_host, int64_t* node_count, int64_t* n_seeds_out,
                               void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (!ctx->have_hier) return set_error(ctx, RS_ERR_STATE, "rs_fof6d has not run on this context");
  const int64_t n = ctx->n_particles, nn = ctx->n_nodes, m = ctx->n_members;
  if (n > 0 && (!pos || !vel || !particle_seed))
    return set_error(ctx, RS_ERR_INVALID_ARG, "null device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  if (n_seeds_out) *n_seeds_out = 0;
  if (nn == 0) {
    if (n > 0) RS_CUDA(ctx, cudaMemsetAsync(particle_seed, 0xff, 8 * size_t(n), st));  // -1
    return RS_OK;
  }
  if (pos != ctx->h_pos || vel != ctx->h_vel) {  // other arrays than rs_fof6d's: re-gather
    RS_TRY(gather_members(ctx, 0, m, 0, nn, pos, vel, st));
    ctx->h_pos = pos;
    ctx->h_vel = vel;
  }
  Hier h = hier_of(ctx);
  int* nkids = scratch_t<int>(ctx, S_SEED_KIDS, size_t(nn));
  int64_t* ra = scratch_t<int64_t>(ctx, S_SEED_ROOT, 2 * size_t(nn));
  unsigned long long* ucnt = scratch_t<unsigned long long>(ctx, S_SEED_UCNT, 2 * size_t(nn) + 2);
  int64_t* uoff = scratch_t<int64_t>(ctx, S_SEED_UOFF, size_t(nn) + 1);
  float4* cen = scratch_t<float4>(ctx, S_SEED_CEN, 2 * size_t(nn));
  double* sums = scratch_t<double>(ctx, S_SEED_SUMS, 6 * size_t(nn));
  int64_t* segsz = scratch_t<int64_t>(ctx, S_SEED_SEG, size_t(nn));
  unsigned long long* count = scratch_t<unsigned long long>(ctx, S_SEED_COUNT, size_t(nn));
  if (!nkids || !ra || !ucnt || !uoff || !cen || !sums || !segsz || !count) return RS_ERR_OOM;
  float4* bulk = cen + nn;
  unsigned long long* fill = ucnt + nn + 1;
  RS_CUDA(ctx, cudaMemsetAsync(nkids, 0, 4 * size_t(nn), st));
  k_seed_kids<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_parent, nkids);
  RS_LAUNCHED(ctx, "k_seed_kids");
  // level-0 ancestor of every node: pointer jumping (2^7 > any depth of the hierarchy)
  int64_t* rin = ra;
  int64_t* rout = ra + nn;
  k_seed_root_init<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_parent, rin);
  RS_LAUNCHED(ctx, "k_seed_root_init");
  for (int it = 0; it < 7; ++it) {
    k_seed_jump<<<grid_for(nn, kT), kT, 0, st>>>(nn, rin, rout);
    RS_LAUNCHED(ctx, "k_seed_jump");
    std::swap(rin, rout);
  }
  const int64_t* root = rin;
  // the seeds under every node: counts, offsets, lists
  RS_CUDA(ctx, cudaMemsetAsync(ucnt, 0, 8 * (2 * size_t(nn) + 2), st));
  k_seed_under_count<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_parent, nkids, ucnt);
  RS_LAUNCHED(ctx, "k_seed_under_count");
  static_assert(sizeof(unsigned long long) == sizeof(int64_t), "counts scanned as int64");
  RS_CUDA(ctx, cudaMemcpyAsync(uoff, ucnt, 8 * size_t(nn), cudaMemcpyDeviceToDevice, st));
  RS_TRY(exclusive_scan_i64(ctx, nn, uoff, uoff + nn, st));
  RS_TRY(read_back(ctx, uoff + nn, 8, st));
  const int64_t total = ctx->host_box[0];
  int64_t* ulist = scratch_t<int64_t>(ctx, S_SEED_LIST, size_t(std::max<int64_t>(total, 1)));
  if (!ulist) return RS_ERR_OOM;
  k_seed_under_fill<<<grid_for(nn, kT), kT, 0, st>>>(nn, h.node_parent, nkids, uoff, fill, ulist);
  RS_LAUNCHED(ctx, "k_seed_under_fill");
  // seed centres and bulk velocities (canonical-order sums over the seeds' members)
  k_seed_segments<<<grid_for(nn, kT), kT, 0, st>>>(nn, nkids, h.node_size, segsz);
  RS_LAUNCHED(ctx, "k_seed_segments");
  RS_TRY((cro_segmented<6, SeedTerm>(ctx, nn, h.node_off, segsz, m, SeedTerm{h.U, h.V}, sums, st)));
  k_seed_stats<<<grid_for(nn, kT), kT, 0, st>>>(nn, nkids, root, h.node_off, h.node_size, h.mem, pos,
                                               ctx->cfg.box_L, sums, cen, bulk);
  RS_LAUNCHED(ctx, "k_seed_stats");
  RS_CUDA(ctx, cudaMemsetAsync(count, 0, 8 * size_t(nn), st));
  {
    ProfScope prof_(ctx, "k_seed_assign", st);
    k_seed_assign<<<grid_for(n, kT), kT, 0, st>>>(n, h.deepest, nkids, root, h.node_off, h.mem, pos, vel,
                                                 ctx->cfg.box_L, uoff, ulist, cen, bulk, h.inv,
                                                 particle_seed, count);
  }
  RS_LAUNCHED(ctx, "k_seed_assign");
  k_seed_host<<<grid_for(nn, kT), kT, 0, st>>>(nn, nkids, root, uoff, ulist, cen, bulk, h.inv, count,
                                              node_host, node_count);
  RS_LAUNCHED(ctx, "k_seed_host");
  if (n_seeds_out) {
    unsigned long long* ns = fill + nn;  // the spare last counter slot
    RS_CUDA(ctx, cudaMemsetAsync(ns, 0, 8, st));
    k_seed_total<<<grid_for(nn, kT), kT, 0, st>>>(nn, nkids, ns);
    RS_LAUNCHED(ctx, "k_seed_total");
    RS_TRY(read_back(ctx, ns, 8, st));
    *n_seeds_out = ctx->host_box[0];
  }
  return RS_OK;
}

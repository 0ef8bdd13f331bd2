// Context management and the small utility entry points of the C ABI.
#include "rs_cro.cuh"

using namespace rs;

extern "C" int rs_ctx_create(rs_ctx** out, const rs_config* cfg, int device) {
  if (!out || !cfg) return RS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(cfg->box_L > 0.f) || !(cfg->link_len > 0.f) || !(cfg->softening >= 0.f) ||
      !(cfg->particle_mass > 0.0) || !(cfg->G > 0.0) || cfg->f_num <= 0 || cfg->f_den <= 0 ||
      cfg->f_num > cfg->f_den || cfg->min_halo_particles < 2 || cfg->bound_num < 0 ||
      cfg->bound_den <= 0 || !(cfg->tree_theta >= 0.f && cfg->tree_theta <= 0.9f) ||
      cfg->surrogate_gate < 0 || cfg->surrogate_gate > 1 || cfg->spot_check < 0 ||
      cfg->unbind_passes < 0)
    return RS_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return RS_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return RS_ERR_CUDA;
  rs_ctx* ctx = new rs_ctx();
  ctx->cfg = *cfg;
  ctx->device = device;
  // certified tree bound: batched forms only
  ctx->tree_min = cfg->batched == 0 || cfg->tree_min_members < 0
                      ? 0
                      : (cfg->tree_min_members == 0 ? rs::kTreeMinDefault : int64_t(cfg->tree_min_members));
  ctx->tree_theta = cfg->tree_theta > 0.f ? cfg->tree_theta : rs::kTreeThetaDefault;
  if (cudaMallocHost(&ctx->host_box, 64 * sizeof(int64_t)) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return RS_ERR_OOM;
  }
  *out = ctx;
  return RS_OK;
}

static void prof_resolve(rs_ctx* ctx) {
  for (auto& r : ctx->prof_pending) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    bool found = false;
    for (auto& t : ctx->prof_tot)
      if (t.name == r.name) {
        t.ms += ms;
        t.launches += 1;
        found = true;
      }
    if (!found) ctx->prof_tot.push_back({r.name, double(ms), 1});
    ctx->prof_free.push_back(r.a);
    ctx->prof_free.push_back(r.b);
  }
  ctx->prof_pending.clear();
  cudaGetLastError();
}

extern "C" int rs_profile(rs_ctx* ctx, int enable) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  prof_resolve(ctx);
  ctx->prof_tot.clear();
  ctx->profile = enable != 0;
  return RS_OK;
}

extern "C" int rs_profile_get(rs_ctx* ctx, int index, char* name, int name_cap, double* total_ms,
                              int64_t* launches) {
  if (!ctx || index < 0) return RS_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  prof_resolve(ctx);
  if (index >= int(ctx->prof_tot.size())) return RS_ERR_CAPACITY;
  const auto& t = ctx->prof_tot[index];
  if (name && name_cap > 0) {
    strncpy(name, t.name.c_str(), size_t(name_cap) - 1);
    name[name_cap - 1] = 0;
  }
  if (total_ms) *total_ms = t.ms;
  if (launches) *launches = t.launches;
  return RS_OK;
}

extern "C" int rs_count_work(rs_ctx* ctx, int enable, int64_t* counts_out) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  unsigned long long* w = scratch_t<unsigned long long>(ctx, rs::S_P_WORK, 6);
  if (!w) return RS_ERR_OOM;
  if (counts_out) {
    RS_CUDA(ctx, cudaDeviceSynchronize());
    unsigned long long h[6];
    RS_CUDA(ctx, cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 6; ++i) counts_out[i] = int64_t(h[i]);
  }
  if (enable) RS_CUDA(ctx, cudaMemset(w, 0, 6 * sizeof(unsigned long long)));
  ctx->count_work = enable != 0;
  return RS_OK;
}

extern "C" int rs_tuning(rs_ctx* ctx, int32_t* choice_out, float* ms_out) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  if (choice_out) {
    choice_out[0] = ctx->tune_blk_r;
    choice_out[1] = ctx->tune_list_r;
  }
  if (ms_out)
    for (int c = 0; c < 3; ++c) {
      ms_out[c] = ctx->tune_blk_ms[c];
      ms_out[3 + c] = ctx->tune_list_ms[c];
    }
  return RS_OK;
}

extern "C" int rs_ctx_destroy(rs_ctx* ctx) {
  if (!ctx) return RS_OK;
  cudaSetDevice(ctx->device);
  for (rs_ctx* lane : ctx->lanes) rs_ctx_destroy(lane);
  for (void* s : ctx->lane_streams) cudaStreamDestroy(static_cast<cudaStream_t>(s));
  if (ctx->lane_event) cudaEventDestroy(static_cast<cudaEvent_t>(ctx->lane_event));
  if (ctx->graph_stream) cudaStreamDestroy(static_cast<cudaStream_t>(ctx->graph_stream));
  prof_resolve(ctx);
  for (auto e : ctx->prof_free) cudaEventDestroy(e);
  for (auto& b : ctx->buf)
    if (b.ptr) cudaFree(b.ptr);
  if (ctx->host_box) cudaFreeHost(ctx->host_box);
  delete ctx;
  return RS_OK;
}

extern "C" const char* rs_last_error(rs_ctx* ctx) { return ctx ? ctx->err : "null context"; }

extern "C" int64_t rs_kernel_launches(rs_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" int64_t rs_sort_keypasses(rs_ctx* ctx) { return ctx ? ctx->sort_keypasses : 0; }

extern "C" int rs_nn_bounds(rs_ctx* ctx, float margin_scale, int64_t min_members) {
  if (!ctx || !(margin_scale == margin_scale) || min_members < 0) return RS_ERR_INVALID_ARG;
  ctx->nn_bound_margin = margin_scale;
  ctx->nn_bound_min = min_members;
  return RS_OK;
}

extern "C" int rs_use_graphs(rs_ctx* ctx, int enable) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->use_graphs = enable != 0;
  for (rs_ctx* lane : ctx->lanes) lane->use_graphs = ctx->use_graphs;
  return RS_OK;
}

namespace {
struct ArrayTerm {
  const double* a;
  template <bool kFirst>
  __device__ __forceinline__ void add(int64_t, int64_t p, int64_t, double* acc) const {
    rsd::cro_add<kFirst>(acc[0], a[p]);
  }
};

__global__ void k_seg_init(int64_t m, int64_t* off_size) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    off_size[0] = 0;
    off_size[1] = m;
  }
}
}  // namespace

extern "C" int rs_cro_sum(rs_ctx* ctx, int64_t m, const double* a, double* out, void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (m < 0 || !out || (m > 0 && !a)) return set_error(ctx, RS_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  int64_t* seg = scratch_t<int64_t>(ctx, S_GVAL_B, 2);
  if (!seg) return RS_ERR_OOM;
  k_seg_init<<<1, 32, 0, st>>>(m, seg);
  RS_LAUNCHED(ctx, "k_seg_init");
  return cro_segmented<1, ArrayTerm>(ctx, 1, seg, seg + 1, m, ArrayTerm{a}, out, st);
}

extern "C" int rs_sort_pairs(rs_ctx* ctx, int64_t n, int nbits, uint64_t* keys, uint32_t* vals,
                             void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (n < 0 || nbits < 0 || nbits > 64 || (n > 0 && (!keys || !vals)))
    return set_error(ctx, RS_ERR_INVALID_ARG, "bad arguments");
  if (n <= 1 || nbits == 0) return RS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  uint64_t* kb = scratch_t<uint64_t>(ctx, S_KEY_B, size_t(n));
  uint32_t* vb = scratch_t<uint32_t>(ctx, S_VAL_B, size_t(n));
  if (!kb || !vb) return RS_ERR_OOM;
  uint64_t* ko;
  uint32_t* vo;
  RS_TRY(radix_sort_u64(ctx, n, nbits, keys, vals, kb, vb, &ko, &vo, st));
  if (ko != keys) {
    RS_CUDA(ctx, cudaMemcpyAsync(keys, ko, 8 * size_t(n), cudaMemcpyDeviceToDevice, st));
    RS_CUDA(ctx, cudaMemcpyAsync(vals, vo, 4 * size_t(n), cudaMemcpyDeviceToDevice, st));
  }
  return RS_OK;
}

// rs_run_batched: the pipeline over a stream of independent snapshots.
//
// The paper spreads independent units of work (FoF halos) over OpenMP threads so that no core
// idles (Section "Parallelization"). On one GPU the unit that must not idle is the device: the
// level-synchronous pipeline reads counts back between its kernels (next level's node and
// member counts, the exact paths' list lengths), and while one snapshot's host thread waits on
// such a count the GPU has nothing of that snapshot to run. Several lanes - each a context
// with its own CUDA stream and host thread - take snapshots largest first from one shared
// counter, so the kernels of one lane fill the gaps of another. A lane runs exactly the calls
// a caller would run on one snapshot, so outputs are identical to the single-snapshot path.

#include <atomic>
#include <numeric>
#include <thread>

#include "rs_common.cuh"

using namespace rs;

namespace {

constexpr int kMaxLanes = 16;

struct LaneResult {
  int rc = RS_OK;
  std::string msg;
};

// The four calls on one snapshot; counts = {groups, nodes, members, levels}.
int run_snapshot(rs_ctx* L, const rs_snapshot& s, cudaStream_t st, int64_t* counts,
                 std::atomic<bool>* short_capacity) {
  L->cfg.box_L = s.box_L;
  L->cfg.link_len = s.link_len;
  L->cfg.softening = s.softening;
  int64_t ng = 0, nn = 0, nm = 0;
  RS_TRY(rs_fof3d(L, s.n, s.pos, s.ids, s.label_out, &ng, st));
  RS_TRY(rs_fof6d(L, s.n, s.pos, s.vel, s.ids, s.label_out, &nn, &nm, st));
  uint8_t* bound = scratch_t<uint8_t>(L, S_BATCH_BOUND, size_t(std::max<int64_t>(nm, 1)));
  if (!bound) return set_error(L, RS_ERR_OOM, "bound flags of %lld members", (long long)nm);
  RS_TRY(rs_unbind(L, s.pos, s.vel, nullptr, bound, nullptr, st));
  const bool fits = nn <= s.node_capacity;
  if ((s.props_out || s.node_parent_out) && !fits) short_capacity->store(true);
  if (s.props_out && fits) RS_TRY(rs_halo_props(L, s.props_out, st));
  int64_t* parent = fits ? s.node_parent_out : nullptr;
  if (s.deepest_out || parent)
    RS_TRY(rs_fof6d_copy(L, parent, nullptr, nullptr, nullptr, nullptr, nullptr, s.deepest_out, st));
  counts[0] = ng;
  counts[1] = nn;
  counts[2] = nm;
  counts[3] = L->n_levels;
  return RS_OK;
}

int check_snapshot(rs_ctx* ctx, int i, const rs_snapshot& s) {
  if (s.n < 0 || s.n >= (int64_t(1) << 32) - 1)
    return set_error(ctx, RS_ERR_INVALID_ARG, "snapshot %d: n = %lld out of range", i, (long long)s.n);
  if (!(s.box_L > 0.f) || !(s.link_len > 0.f) || !(s.softening >= 0.f))
    return set_error(ctx, RS_ERR_INVALID_ARG, "snapshot %d: box_L, link_len must be > 0, softening >= 0", i);
  if (s.n > 0 && (!s.pos || !s.vel || !s.ids || !s.label_out))
    return set_error(ctx, RS_ERR_INVALID_ARG, "snapshot %d: null device pointer", i);
  if (s.node_capacity < 0)
    return set_error(ctx, RS_ERR_INVALID_ARG, "snapshot %d: negative node_capacity", i);
  return RS_OK;
}

// Creates lanes up to `lanes` (kept on ctx until rs_ctx_destroy).
int ensure_lanes(rs_ctx* ctx, int lanes) {
  if (!ctx->lane_event) {
    cudaEvent_t e;
    RS_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->lane_event = e;
  }
  while (int(ctx->lanes.size()) < lanes) {
    rs_ctx* L = nullptr;
    const int rc = rs_ctx_create(&L, &ctx->cfg, ctx->device);
    if (rc != RS_OK) return set_error(ctx, rc, "creating lane %d failed", int(ctx->lanes.size()));
    cudaStream_t s;
    const cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      rs_ctx_destroy(L);
      return set_error(ctx, RS_ERR_CUDA, "cudaStreamCreateWithFlags: %s", cudaGetErrorString(e));
    }
    ctx->lanes.push_back(L);
    ctx->lane_streams.push_back(s);
  }
  return RS_OK;
}

}  // namespace

extern "C" int rs_run_batched(rs_ctx* ctx, int32_t n_snap, const rs_snapshot* snaps, int32_t lanes,
                              int64_t* counts_out, void* stream) {
  if (!ctx) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (n_snap < 0 || (n_snap > 0 && !snaps))
    return set_error(ctx, RS_ERR_INVALID_ARG, "n_snap = %d with snaps %p", n_snap, (const void*)snaps);
  if (lanes < 1 || lanes > kMaxLanes)
    return set_error(ctx, RS_ERR_INVALID_ARG, "lanes = %d outside 1..%d", lanes, kMaxLanes);
  for (int i = 0; i < n_snap; ++i) RS_TRY(check_snapshot(ctx, i, snaps[i]));
  if (ctx->cfg.use_surrogate && !ctx->have_mlp)
    return set_error(ctx, RS_ERR_STATE, "use_surrogate needs a trained surrogate on the context");
  if (n_snap == 0) return RS_OK;
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  lanes = std::min(lanes, n_snap);
  RS_TRY(ensure_lanes(ctx, lanes));
  cudaEvent_t start = static_cast<cudaEvent_t>(ctx->lane_event);
  RS_CUDA(ctx, cudaEventRecord(start, static_cast<cudaStream_t>(stream)));
  int64_t launches0 = 0, keypasses0 = 0;
  for (int l = 0; l < lanes; ++l) {
    rs_ctx* L = ctx->lanes[l];
    cudaStream_t st = static_cast<cudaStream_t>(ctx->lane_streams[l]);
    // the lanes share ctx's configuration of this call (the snapshot fields are set per run)
    L->cfg = ctx->cfg;
    L->tree_min = ctx->tree_min;
    L->tree_theta = ctx->tree_theta;
    L->use_graphs = ctx->use_graphs;
    RS_CUDA(ctx, cudaStreamWaitEvent(st, start, 0));
    if (ctx->cfg.use_surrogate) {
      const int rc = mlp_copy(L, ctx, st);
      if (rc != RS_OK) return set_error(ctx, rc, "lane %d: %s", l, L->err);
    }
    launches0 += L->launches;
    keypasses0 += L->sort_keypasses;
  }
  // largest snapshots first, taken from one counter
  std::vector<int> order(n_snap);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return snaps[a].n > snaps[b].n; });
  std::vector<int64_t> counts(size_t(n_snap) * 4, 0);
  std::atomic<int> next{0};
  std::atomic<bool> failed{false}, short_capacity{false};
  std::vector<LaneResult> res(lanes);
  auto body = [&](int l) {
    rs_ctx* L = ctx->lanes[l];
    cudaStream_t st = static_cast<cudaStream_t>(ctx->lane_streams[l]);
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
      res[l] = {RS_ERR_CUDA, "cudaSetDevice failed in a lane"};
      failed.store(true);
      return;
    }
    for (;;) {
      if (failed.load()) break;
      const int k = next.fetch_add(1);
      if (k >= n_snap) break;
      const int i = order[k];
      const int rc = run_snapshot(L, snaps[i], st, &counts[size_t(i) * 4], &short_capacity);
      if (rc != RS_OK) {
        res[l] = {rc, "snapshot " + std::to_string(i) + ": " + L->err};
        failed.store(true);
        break;
      }
    }
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && res[l].rc == RS_OK) {
      res[l] = {RS_ERR_CUDA, std::string("lane stream: ") + cudaGetErrorString(e)};
      failed.store(true);
    }
  };
  std::vector<std::thread> threads;
  threads.reserve(lanes - 1);
  for (int l = 1; l < lanes; ++l) threads.emplace_back(body, l);
  body(0);
  for (auto& t : threads) t.join();
  for (int l = 0; l < lanes; ++l) {
    ctx->launches += ctx->lanes[l]->launches;
    ctx->sort_keypasses += ctx->lanes[l]->sort_keypasses;
  }
  ctx->launches -= launches0;
  ctx->sort_keypasses -= keypasses0;
  if (counts_out) std::copy(counts.begin(), counts.end(), counts_out);
  for (int l = 0; l < lanes; ++l)
    if (res[l].rc != RS_OK) return set_error(ctx, res[l].rc, "lane %d, %s", l, res[l].msg.c_str());
  if (short_capacity.load())
    return set_error(ctx, RS_ERR_CAPACITY, "a snapshot has more nodes than its node_capacity");
  return RS_OK;
}

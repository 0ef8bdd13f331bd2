// Device-wide primitives used by every stage: LSD radix sort of (uint64 key, uint32 value)
// pairs, exclusive scans, plus the context's scratch allocator, error reporting and
// read-back helpers.
#include "rs_common.cuh"

namespace rs {

int set_error(rs_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

void* scratch(rs_ctx* ctx, int slot, size_t bytes) {
  Buffer& b = ctx->buf[slot];
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return b.ptr;
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
  size_t want = bytes + bytes / 8;  // headroom so small growth does not reallocate
  want = (want + 255) & ~size_t(255);
  if (cudaMalloc(&b.ptr, want) != cudaSuccess) {
    cudaGetLastError();
    b.ptr = nullptr;
    set_error(ctx, RS_ERR_OOM, "cudaMalloc of %zu bytes failed (slot %d)", want, slot);
    return nullptr;
  }
  b.bytes = want;
  return b.ptr;
}

int after_launch(rs_ctx* ctx, const char* name) {
  ctx->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_error(ctx, RS_ERR_CUDA, "launch of %s failed: %s", name, cudaGetErrorString(e));
  return RS_OK;
}

int begin_capture(rs_ctx* ctx, cudaStream_t* cs) {
  if (!ctx->graph_stream) {
    cudaStream_t s;
    RS_CUDA(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    ctx->graph_stream = s;
  }
  *cs = static_cast<cudaStream_t>(ctx->graph_stream);
  RS_CUDA(ctx, cudaStreamBeginCapture(*cs, cudaStreamCaptureModeThreadLocal));
  return RS_OK;
}

int end_capture(rs_ctx* ctx, cudaStream_t cs, int body_rc, int64_t launches0, bool profile,
                cudaGraphExec_t* exec, int64_t* launches) {
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &g);
  ctx->profile = profile;
  *launches = ctx->launches - launches0;
  ctx->launches = launches0;
  *exec = nullptr;
  if (body_rc != RS_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (body_rc != RS_OK) return body_rc;
    return set_error(ctx, RS_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ce));
  }
  const cudaError_t ie = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    *exec = nullptr;
    return set_error(ctx, RS_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
  }
  return RS_OK;
}

int launch_graph(rs_ctx* ctx, cudaGraphExec_t exec, int64_t launches, cudaStream_t st) {
  RS_CUDA(ctx, cudaGraphLaunch(exec, st));
  ctx->launches += launches;
  return RS_OK;
}

static cudaEvent_t prof_event(rs_ctx* ctx) {
  if (!ctx->prof_free.empty()) {
    cudaEvent_t e = ctx->prof_free.back();
    ctx->prof_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

ProfScope::ProfScope(rs_ctx* c, const char* name, cudaStream_t s) : ctx(c), st(s) {
  if (!ctx->profile) return;
  rs_ctx::ProfRec r{name, prof_event(ctx), prof_event(ctx)};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, st);
  idx = int(ctx->prof_pending.size());
  ctx->prof_pending.push_back(r);
}

ProfScope::~ProfScope() {
  if (idx >= 0) cudaEventRecord(ctx->prof_pending[idx].b, st);
}

int read_back(rs_ctx* ctx, const void* dev, size_t bytes, cudaStream_t st) {
  if (bytes > 64 * sizeof(int64_t)) return set_error(ctx, RS_ERR_INVALID_ARG, "read_back too big");
  RS_CUDA(ctx, cudaMemcpyAsync(ctx->host_box, dev, bytes, cudaMemcpyDeviceToHost, st));
  RS_CUDA(ctx, cudaStreamSynchronize(st));
  return RS_OK;
}

// ------------------------------------------------------------------------------------------
// Radix sort. One pass per 8-bit digit: per-block digit histograms (k_sort_hist), a scan of
// each digit's row of the digit-major histogram table (k_sort_scan_rows), then a stable scatter
// (k_sort_scatter) in which each block ranks its tiles with warp vote masks, reorders a tile
// in shared memory and writes each digit's run contiguously.
namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kKeysPerThread = 8;
constexpr int kTile = kSortThreads * kKeysPerThread;  // 2048
constexpr int kMaxSortBlocks = 4096;                   // bound on the histogram table's rows

__global__ void __launch_bounds__(kSortThreads)
k_sort_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, uint32_t dmask,
            int64_t tiles_per_block, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kSortWarps][kRadix];
  const int warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < kSortWarps * kRadix; t += blockDim.x) (&h[0][0])[t] = 0;
  __syncthreads();
  const int64_t begin = int64_t(blockIdx.x) * tiles_per_block * kTile;
  const int64_t end = min(n, begin + tiles_per_block * kTile);
  for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x)
    atomicAdd(&h[warp][(keys[i] >> shift) & dmask], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
    uint32_t s = 0;
    for (int w = 0; w < kSortWarps; ++w) s += h[w][d];
    hist[int64_t(d) * gridDim.x + blockIdx.x] = s;
  }
}

// Scan of the digit-major histogram table, one block per digit: each row (the digit's count in
// every sort block, in block order) becomes its exclusive prefix, and the row total goes to
// totals[d]. The scatter adds the exclusive prefix of the totals over the digits.
constexpr int kScanRowThreads = 256;

__global__ void __launch_bounds__(kScanRowThreads)
k_sort_scan_rows(uint32_t* __restrict__ hist, int64_t nblocks, uint32_t* __restrict__ totals) {
  __shared__ uint32_t wsum[kScanRowThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* row = hist + int64_t(blockIdx.x) * nblocks;
  const int64_t per = (nblocks + kScanRowThreads - 1) / kScanRowThreads;
  const int64_t b0 = rsd::min64(nblocks, int64_t(threadIdx.x) * per);
  const int64_t b1 = rsd::min64(nblocks, b0 + per);
  uint32_t s = 0;
  for (int64_t b = b0; b < b1; ++b) s += row[b];
  uint32_t incl = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kScanRowThreads / 32; ++w) {
    if (w < warp) before += wsum[w];
    all += wsum[w];
  }
  uint32_t run = before + incl - s;
  for (int64_t b = b0; b < b1; ++b) {
    const uint32_t c = row[b];
    row[b] = run;
    run += c;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = all;
}

__global__ void __launch_bounds__(kSortThreads)
k_sort_scatter(const uint64_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
               uint64_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int64_t n,
               int shift, uint32_t dmask, int64_t tiles_per_block,
               const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ totals) {
  __shared__ uint64_t skey[kTile];
  __shared__ uint32_t sval[kTile];
  __shared__ uint32_t wcount[kSortWarps][kRadix];
  __shared__ uint32_t run[kRadix];
  __shared__ uint32_t tile_start[kRadix];
  __shared__ uint32_t tot[kRadix];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  if (threadIdx.x < 32) {  // run[d] = (digits < d over all blocks) + (digit d in blocks before)
    uint32_t v[kRadix / 32];
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kRadix / 32; ++q) {
      v[q] = totals[lane * (kRadix / 32) + q];
      s += v[q];
    }
    uint32_t incl = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += t;
    }
    uint32_t ex = incl - s;
#pragma unroll
    for (int q = 0; q < kRadix / 32; ++q) {
      const int d = lane * (kRadix / 32) + q;
      run[d] = ex + offsets[int64_t(d) * gridDim.x + blockIdx.x];
      ex += v[q];
    }
  }
  __syncthreads();
  const int64_t tile0 = int64_t(blockIdx.x) * tiles_per_block;
  const int64_t ntiles_total = (n + kTile - 1) / kTile;
  const int64_t tile1 = min(ntiles_total, tile0 + tiles_per_block);
  for (int64_t tile = tile0; tile < tile1; ++tile) {
    const int64_t tbase = tile * kTile;
    const int cnt = int(rsd::min64(kTile, n - tbase));
    uint64_t key[kKeysPerThread];
    uint32_t val[kKeysPerThread];
    uint32_t dig[kKeysPerThread];
    uint32_t rank[kKeysPerThread];
    for (int t = threadIdx.x; t < kSortWarps * kRadix; t += blockDim.x) (&wcount[0][0])[t] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kKeysPerThread; ++k) {
      const int e = warp * (32 * kKeysPerThread) + k * 32 + lane;
      const bool valid = e < cnt;
      key[k] = valid ? keys_in[tbase + e] : 0ull;
      val[k] = valid ? vals_in[tbase + e] : 0u;
      dig[k] = valid ? uint32_t((key[k] >> shift) & dmask) : uint32_t(kRadix);
    }
#pragma unroll
    for (int k = 0; k < kKeysPerThread; ++k) {
      // lanes with the same digit: one vote per digit bit (ALU votes instead of a match, whose
      // shared-pipe latency dominated the scatter)
      const bool valid = dig[k] < kRadix;
      uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
      for (int bit = 0; bit < kRadixBits; ++bit) {
        const bool set = (dig[k] >> bit) & 1u;
        const uint32_t vb = __ballot_sync(0xffffffffu, set);
        peers &= set ? vb : ~vb;
      }
      uint32_t base = valid ? wcount[warp][dig[k]] : 0u;
      rank[k] = base + __popc(peers & lt_mask);
      __syncwarp();
      const int leader = __ffs(peers) - 1;
      if (valid && lane == leader) wcount[warp][dig[k]] = base + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
      uint32_t s = 0;
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = wcount[w][d];
        wcount[w][d] = s;
        s += c;
      }
      tot[d] = s;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of tot[] over the 256 digits by one warp
      uint32_t v[kRadix / 32];
      uint32_t s = 0;
#pragma unroll
      for (int q = 0; q < kRadix / 32; ++q) {
        v[q] = tot[lane * (kRadix / 32) + q];
        s += v[q];
      }
      uint32_t incl = s;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
      }
      uint32_t ex = incl - s;
#pragma unroll
      for (int q = 0; q < kRadix / 32; ++q) {
        tile_start[lane * (kRadix / 32) + q] = ex;
        ex += v[q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kKeysPerThread; ++k) {
      if (dig[k] < kRadix) {
        const uint32_t pos = tile_start[dig[k]] + wcount[warp][dig[k]] + rank[k];
        skey[pos] = key[k];
        sval[pos] = val[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kKeysPerThread; ++k) {
      const int pos = k * kSortThreads + threadIdx.x;
      if (pos < cnt) {
        const uint64_t kk = skey[pos];
        const uint32_t d = uint32_t((kk >> shift) & dmask);
        const uint32_t dest = run[d] + (uint32_t(pos) - tile_start[d]);
        keys_out[dest] = kk;
        vals_out[dest] = sval[pos];
      }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) run[d] += tot[d];
    __syncthreads();
  }
}

}  // namespace

int radix_sort_u64(rs_ctx* ctx, int64_t n, int nbits, uint64_t* keys_a, uint32_t* vals_a,
                   uint64_t* keys_b, uint32_t* vals_b, uint64_t** keys_out,
                   uint32_t** vals_out, cudaStream_t st) {
  *keys_out = keys_a;
  *vals_out = vals_a;
  if (n <= 1 || nbits <= 0) return RS_OK;
  if (n >= (int64_t(1) << 32) - 1) return set_error(ctx, RS_ERR_INVALID_ARG, "sort size %lld", (long long)n);
  if (ctx->sort_blocks == 0) {  // one wave of scatter blocks: every block holds its share of tiles
    int dev_sms = 0, per_sm = 0;
    RS_CUDA(ctx, cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    RS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_scatter, kSortThreads, 0));
    ctx->sort_blocks = std::max(1, std::min(dev_sms * std::max(per_sm, 1), kMaxSortBlocks));
  }
  const int64_t ntiles = (n + kTile - 1) / kTile;
  int64_t blocks = rsd::min64(ntiles, ctx->sort_blocks);
  const int64_t tpb = (ntiles + blocks - 1) / blocks;
  blocks = (ntiles + tpb - 1) / tpb;
  uint32_t* hist = scratch_t<uint32_t>(ctx, S_SORT_HIST, size_t(kRadix) * (blocks + 1));
  if (!hist) return RS_ERR_OOM;
  uint32_t* totals = hist + size_t(kRadix) * blocks;
  uint64_t* kin = keys_a;
  uint32_t* vin = vals_a;
  uint64_t* kout = keys_b;
  uint32_t* vout = vals_b;
  for (int shift = 0; shift < nbits; shift += kRadixBits) {
    ctx->sort_keypasses += n;  // 24 B of key + value traffic per key and pass
    const int dbits = std::min(kRadixBits, nbits - shift);
    const uint32_t dmask = (1u << dbits) - 1u;
    {
      ProfScope prof_(ctx, "k_sort_hist", st);
      k_sort_hist<<<unsigned(blocks), kSortThreads, 0, st>>>(kin, n, shift, dmask, tpb, hist);
    }
    RS_LAUNCHED(ctx, "k_sort_hist");
    k_sort_scan_rows<<<kRadix, kScanRowThreads, 0, st>>>(hist, blocks, totals);
    RS_LAUNCHED(ctx, "k_sort_scan_rows");
    {
      ProfScope prof_(ctx, "k_sort_scatter", st);
      k_sort_scatter<<<unsigned(blocks), kSortThreads, 0, st>>>(kin, vin, kout, vout, n, shift, dmask,
                                                               tpb, hist, totals);
    }
    RS_LAUNCHED(ctx, "k_sort_scatter");
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  *keys_out = kin;
  *vals_out = vin;
  return RS_OK;
}

// ------------------------------------------------------------------------------------------
// Exclusive scan of int64 values: per-block sums, a looping single-block scan of those, then a
// block-local scan that adds each block's offset.
namespace {
constexpr int kScanThreads = 512;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int64_t block_exclusive_i64(int64_t v, int64_t* sh, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x / 32;
    int64_t w = lane < nw ? sh[lane] : 0;
    int64_t wi = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += t;
    }
    if (lane < nw) sh[lane] = wi - w;
    if (lane == nw - 1) sh[32] = wi;
  }
  __syncthreads();
  const int64_t r = sh[warp] + incl - v;
  *total = sh[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int64_t* d, int64_t n, int64_t* bsum) {
  __shared__ int64_t sh[33];
  const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanPer;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k)
    if (base + k < n) s += d[base + k];
  int64_t tot;
  block_exclusive_i64(s, sh, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_single_i64(int64_t* d, int64_t m, int64_t* total) {
  __shared__ int64_t sh[33];
  int64_t carry = 0;
  for (int64_t base0 = 0; base0 < m; base0 += kScanTile) {
    const int64_t base = base0 + int64_t(threadIdx.x) * kScanPer;
    int64_t v[kScanPer];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      v[k] = base + k < m ? d[base + k] : 0;
      s += v[k];
    }
    int64_t tot;
    int64_t run = carry + block_exclusive_i64(s, sh, &tot);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      if (base + k < m) d[base + k] = run;
      run += v[k];
    }
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int64_t* d, int64_t n, const int64_t* boff) {
  __shared__ int64_t sh[33];
  const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanPer;
  int64_t v[kScanPer];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = base + k < n ? d[base + k] : 0;
    s += v[k];
  }
  int64_t tot;
  int64_t run = boff[blockIdx.x] + block_exclusive_i64(s, sh, &tot);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) d[base + k] = run;
    run += v[k];
  }
}
}  // namespace

int exclusive_scan_i64(rs_ctx* ctx, int64_t n, int64_t* data, int64_t* total_dev,
                       cudaStream_t st) {
  if (n <= kScanTile) {
    k_scan_single_i64<<<1, kScanThreads, 0, st>>>(data, n, total_dev);
    RS_LAUNCHED(ctx, "k_scan_single_i64");
    return RS_OK;
  }
  const int64_t blocks = (n + kScanTile - 1) / kScanTile;
  int64_t* bsum = scratch_t<int64_t>(ctx, S_SCAN_TMP, size_t(blocks));
  if (!bsum) return RS_ERR_OOM;
  k_scan_reduce<<<unsigned(blocks), kScanThreads, 0, st>>>(data, n, bsum);
  RS_LAUNCHED(ctx, "k_scan_reduce");
  k_scan_single_i64<<<1, kScanThreads, 0, st>>>(bsum, blocks, total_dev);
  RS_LAUNCHED(ctx, "k_scan_single_i64");
  k_scan_apply<<<unsigned(blocks), kScanThreads, 0, st>>>(data, n, bsum);
  RS_LAUNCHED(ctx, "k_scan_apply");
  return RS_OK;
}

// ------------------------------------------------------------------------------------------
// Chunk offsets for segmented canonical-order sums.
namespace {
__global__ void k_chunk_counts(int64_t nseg, const int64_t* __restrict__ seg_size,
                               int64_t* __restrict__ counts) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < nseg) counts[q] = (seg_size[q] + 1023) / 1024;
}
}  // namespace

int cro_prepare(rs_ctx* ctx, int64_t nseg, const int64_t* seg_size, int64_t** chunk_off,
                cudaStream_t st) {
  int64_t* off = scratch_t<int64_t>(ctx, S_CHUNK_OFF, size_t(nseg) + 1);
  if (!off) return RS_ERR_OOM;
  k_chunk_counts<<<grid_for(nseg, 256), 256, 0, st>>>(nseg, seg_size, off);
  RS_LAUNCHED(ctx, "k_chunk_counts");
  RS_TRY(exclusive_scan_i64(ctx, nseg, off, off + nseg, st));
  *chunk_off = off;
  return RS_OK;
}

}  // namespace rs

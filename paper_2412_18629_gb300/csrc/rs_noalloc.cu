// rs_cro_sum_noalloc: the canonical-order float64 sum of rs_cro_sum for callers that cannot
// allocate device memory -- code running while a CUDA stream is being captured into a graph,
// code inside an allocator or memory-pool callback, or embedders that forbid the library from
// touching the device heap. It needs no context (creating one allocates pinned host memory)
// and calls no cudaMalloc / cudaFree or allocating library routine.
//
// Its only scratch is the file-scope array below: one float64 chunk total per 1024 terms, for
// at most kMaxTerms terms (512 KiB). Every GPU that loads this library holds the array until the
// process exits. Host code cannot use the array's name as a device address, so the first call
// on each device (with that device current) looks the address up with cudaGetSymbolAddress and
// caches it; that first call should therefore happen before any stream capture begins. The
// cache is keyed by device ordinal only: cudaDeviceReset (or any other teardown of the primary
// context) invalidates the address, and the library cannot notice that. All
// calls share the array and it keeps the last call's contents: calls whose kernels overlap on
// the GPU (different streams, or different host threads on one device) race on it and must be
// serialised by the caller. Nothing needs clearing: a call writes every chunk slot it later
// reads.
#include <mutex>

#include "rs_cro.cuh"

namespace {

constexpr int64_t kMaxTerms = int64_t(1) << 26;
constexpr int64_t kMaxChunks = kMaxTerms / 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_chunk_totals[kMaxChunks];

std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {nullptr};

// One warp per chunk of 1024 terms: lane sums in order, halving-tree combine (rs_cro.cuh).
__global__ void __launch_bounds__(256)
k_noalloc_chunks(int64_t m, const double* __restrict__ a, double* __restrict__ chunk_totals) {
  const int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c * 1024 >= m) return;
  double acc = 0.0;
  for (int k = 0; k < 32; ++k) {
    const int64_t idx = c * 1024 + lane + 32 * k;
    if (idx < m) acc = __dadd_rn(acc, a[idx]);
  }
  acc = rsd::warp_cro_combine(acc);
  if (lane == 0) chunk_totals[c] = acc;
}

// Pairwise tree over the chunk totals (0.0 when there are none).
__global__ void k_noalloc_tree(int64_t nchunks, const double* __restrict__ chunk_totals,
                               double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  rsd::CroTree t;
  for (int64_t c = 0; c < nchunks; ++c) t.push(chunk_totals[c]);
  out[0] = t.result();
}

int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return RS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[dev]) {
    double* p = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_chunk_totals) != cudaSuccess || !p) {
      cudaGetLastError();
      return RS_ERR_CUDA;
    }
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return RS_OK;
}

}  // namespace

extern "C" int rs_cro_sum_noalloc(int64_t m, const double* a, double* out, void* stream) {
  if (m < 0 || !out || (m > 0 && !a)) return RS_ERR_INVALID_ARG;
  if (m > kMaxTerms) return RS_ERR_CAPACITY;
  double* scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != RS_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nchunks = (m + 1023) / 1024;
  if (nchunks > 0) {
    k_noalloc_chunks<<<unsigned((nchunks * 32 + 255) / 256), 256, 0, st>>>(m, a, scratch);
    if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
  }
  k_noalloc_tree<<<1, 32, 0, st>>>(nchunks, scratch, out);
  if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
  return RS_OK;
}

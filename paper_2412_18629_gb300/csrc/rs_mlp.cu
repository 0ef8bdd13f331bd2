// BF16 tensor-core MLP (8 -> 64 -> 64 -> 1, ReLU) for the binding-energy surrogate: inference,
// one-batch gradients, and Adam training on float32 master weights.
//
// Definition (what every kernel here computes):
//   x~ = bf16(x) (8 features, padded with zeros to 16);  W1 [16x64], W2 [64x64], W3 [64] are
//   bf16(master); b1, b2, b3 float32.
//   z1 = b1 + W1^T x~   (float32 accumulation)      h1 = bf16(max(z1, 0))
//   z2 = b2 + W2^T h1                                h2 = bf16(max(z2, 0))
//   y  = b3 + sum_k W3[k] h2[k]  (float32: four partial sums over the columns 16 s + 2q +
//        {0, 1, 8, 9}, s = 0..3, for q = 0..3, combined as (p0 + p1) + (p2 + p3))
// Loss over a batch of B samples: L = (1/B) sum (y - t)^2. Backward: dy = 2 (y - t) / B;
//   dW3 = sum_b dy h2; db3 = sum_b dy; dz2 = bf16(dy W3 [h2 > 0]); db2 = sum_b dz2;
//   dW2 = sum_b h1 dz2^T; dz1 = bf16((W2 dz2) [h1 > 0]); db1 = sum_b dz1; dW1 = sum_b x~ dz1^T.
// Products of bf16 operands run on mma.sync.m16n8k16 (bf16 in, float32 accumulate); batch
// reductions are deterministic (per-block partials summed in a fixed order).
//
// Parameter vector layout (float32, kParams entries): W1 [8][64] at 0, b1 [64] at 512,
// W2 [64][64] at 576 (row = input unit), b2 [64] at 4672, W3 [64] at 4736, b3 at 4800.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>

#include "rs_cro.cuh"

namespace rs {
constexpr int kParams = 4801;
constexpr int kOffW1 = 0, kOffB1 = 512, kOffW2 = 576, kOffB2 = 4672, kOffW3 = 4736, kOffB3 = 4800;
int mlp_forward(rs_ctx* ctx, int64_t n, const float* x, float* y, cudaStream_t st);
}  // namespace rs

using namespace rs;

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kRowsPerBlock = kWarps * 16;  // 128 samples per block in the training kernel

// Device copy of the weights used by the kernels: the B fragments of W1 and W2 for
// mma.m16n8k16 already packed per (k-slice, n-tile, lane), and the row-major bf16 matrices the
// backward pass reads.
struct MlpDev {
  uint2 f1[8][32];            // W1 fragments: [n-tile][lane]
  uint2 f2[4][8][32];         // W2 fragments: [k-slice][n-tile][lane]
  __nv_bfloat16 w1[16 * 64];  // [in 16][out 64], rows 8..15 zero
  __nv_bfloat16 w2[64 * 64];  // [in 64][out 64]
  __nv_bfloat16 w3[64];
  float b1[64], b2[64], b3;
};

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Forward of 16 samples held by one warp. xa: A fragment of x~ (one k-slice). Produces the
// post-activation h1, h2 as A fragments (4 k-slices each) and y for rows g and g + 8 (valid in
// lanes with q == 0 after the reduction).
struct Fwd {
  uint32_t h1[4][4];  // A fragments of h1 (k-slices 0..3)
  uint32_t h2[4][4];
  float y_lo, y_hi;   // outputs of rows g and g + 8 (all lanes hold them after the reduction)
};

__device__ __forceinline__ void fwd16(const MlpDev& W, const uint32_t (&xa)[4], int lane, Fwd& f) {
  const int q = lane & 3;
  // layer 1: 8 n-tiles of 8 outputs; d fragment of tile nt covers columns 8 nt + 2q, +1
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float c0 = W.b1[nt * 8 + 2 * q], c1 = W.b1[nt * 8 + 2 * q + 1];
    acc[nt][0] = c0;
    acc[nt][1] = c1;
    acc[nt][2] = c0;
    acc[nt][3] = c1;
    const uint2 b = W.f1[nt][lane];
    mma_bf16(acc[nt], xa[0], xa[1], xa[2], xa[3], b.x, b.y);
  }
  // h1 = bf16(relu(z1)) as A fragments: k-slice s = n-tiles 2s, 2s+1
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const float* lo = acc[2 * s];
    const float* hi = acc[2 * s + 1];
    f.h1[s][0] = pack2(__float2bfloat16_rn(fmaxf(lo[0], 0.f)), __float2bfloat16_rn(fmaxf(lo[1], 0.f)));
    f.h1[s][1] = pack2(__float2bfloat16_rn(fmaxf(lo[2], 0.f)), __float2bfloat16_rn(fmaxf(lo[3], 0.f)));
    f.h1[s][2] = pack2(__float2bfloat16_rn(fmaxf(hi[0], 0.f)), __float2bfloat16_rn(fmaxf(hi[1], 0.f)));
    f.h1[s][3] = pack2(__float2bfloat16_rn(fmaxf(hi[2], 0.f)), __float2bfloat16_rn(fmaxf(hi[3], 0.f)));
  }
  // layer 2
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float c0 = W.b2[nt * 8 + 2 * q], c1 = W.b2[nt * 8 + 2 * q + 1];
    acc[nt][0] = c0;
    acc[nt][1] = c1;
    acc[nt][2] = c0;
    acc[nt][3] = c1;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const uint2 b = W.f2[s][nt][lane];
      mma_bf16(acc[nt], f.h1[s][0], f.h1[s][1], f.h1[s][2], f.h1[s][3], b.x, b.y);
    }
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const float* lo = acc[2 * s];
    const float* hi = acc[2 * s + 1];
    f.h2[s][0] = pack2(__float2bfloat16_rn(fmaxf(lo[0], 0.f)), __float2bfloat16_rn(fmaxf(lo[1], 0.f)));
    f.h2[s][1] = pack2(__float2bfloat16_rn(fmaxf(lo[2], 0.f)), __float2bfloat16_rn(fmaxf(lo[3], 0.f)));
    f.h2[s][2] = pack2(__float2bfloat16_rn(fmaxf(hi[0], 0.f)), __float2bfloat16_rn(fmaxf(hi[1], 0.f)));
    f.h2[s][3] = pack2(__float2bfloat16_rn(fmaxf(hi[2], 0.f)), __float2bfloat16_rn(fmaxf(hi[3], 0.f)));
  }
  // layer 3 in float32: each lane's partial sum over the 16 h2 columns it holds (16 s + 2q +
  // {0, 1, 8, 9}, s = 0..3, in that order), then the quad's four partials by an xor tree,
  // then the bias.
  float plo = 0.f, phi = 0.f;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int c = 16 * s + 2 * q;
    const float w0 = __bfloat162float(W.w3[c]), w1 = __bfloat162float(W.w3[c + 1]);
    const float w8 = __bfloat162float(W.w3[c + 8]), w9 = __bfloat162float(W.w3[c + 9]);
    plo = __fmaf_rn(w0, __uint_as_float(f.h2[s][0] << 16), plo);
    plo = __fmaf_rn(w1, __uint_as_float(f.h2[s][0] & 0xffff0000u), plo);
    plo = __fmaf_rn(w8, __uint_as_float(f.h2[s][2] << 16), plo);
    plo = __fmaf_rn(w9, __uint_as_float(f.h2[s][2] & 0xffff0000u), plo);
    phi = __fmaf_rn(w0, __uint_as_float(f.h2[s][1] << 16), phi);
    phi = __fmaf_rn(w1, __uint_as_float(f.h2[s][1] & 0xffff0000u), phi);
    phi = __fmaf_rn(w8, __uint_as_float(f.h2[s][3] << 16), phi);
    phi = __fmaf_rn(w9, __uint_as_float(f.h2[s][3] & 0xffff0000u), phi);
  }
#pragma unroll
  for (int off = 1; off <= 2; off <<= 1) {
    plo = __fadd_rn(plo, __shfl_xor_sync(0xffffffffu, plo, off));
    phi = __fadd_rn(phi, __shfl_xor_sync(0xffffffffu, phi, off));
  }
  f.y_lo = __fadd_rn(W.b3, plo);
  f.y_hi = __fadd_rn(W.b3, phi);
}

// A fragment of x~ for the warp's 16 rows (row0 = first sample), from float [n][8] features.
__device__ __forceinline__ void load_x(const float* __restrict__ x, int64_t n, int64_t row0, int lane,
                                       uint32_t (&xa)[4]) {
  const int g = lane >> 2, q = lane & 3;
  const int64_t r0 = row0 + g, r1 = row0 + g + 8;
  const int c = 2 * q;  // columns c, c+1 (c+8, c+9 are padding: zero)
  const float x00 = r0 < n ? x[r0 * 8 + c] : 0.f, x01 = r0 < n ? x[r0 * 8 + c + 1] : 0.f;
  const float x10 = r1 < n ? x[r1 * 8 + c] : 0.f, x11 = r1 < n ? x[r1 * 8 + c + 1] : 0.f;
  xa[0] = pack2(__float2bfloat16_rn(x00), __float2bfloat16_rn(x01));
  xa[1] = pack2(__float2bfloat16_rn(x10), __float2bfloat16_rn(x11));
  xa[2] = 0u;
  xa[3] = 0u;
}

__global__ void __launch_bounds__(kThreads)
k_mlp_fwd(int64_t n, const float* __restrict__ x, const MlpDev* __restrict__ Wg, float* __restrict__ y) {
  __shared__ MlpDev W;
  for (int i = threadIdx.x; i < int(sizeof(MlpDev) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t*>(&W)[i] = reinterpret_cast<const uint32_t*>(Wg)[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w * 16 < n; w += warps) {
    uint32_t xa[4];
    load_x(x, n, w * 16, lane, xa);
    Fwd f;
    fwd16(W, xa, lane, f);
    const int g = lane >> 2;
    if ((lane & 3) == 0) {
      if (w * 16 + g < n) y[w * 16 + g] = f.y_lo;
      if (w * 16 + g + 8 < n) y[w * 16 + g + 8] = f.y_hi;
    }
  }
}

// Training forward + backward for a batch: one block per 128 samples, writing its partial
// gradient (kParams floats) to part[blockIdx.x]; also the block's sum of squared errors.
__global__ void __launch_bounds__(kThreads)
k_mlp_grad_block(int64_t n, const float* __restrict__ x, const float* __restrict__ t,
                 const int64_t* __restrict__ idx, float inv_b, const MlpDev* __restrict__ Wg,
                 float* __restrict__ part, double* __restrict__ sse_part) {
  extern __shared__ __align__(16) unsigned char smem[];
  MlpDev& W = *reinterpret_cast<MlpDev*>(smem);
  __nv_bfloat16* sX = reinterpret_cast<__nv_bfloat16*>(smem + sizeof(MlpDev));  // [128][16]
  __nv_bfloat16* sH1 = sX + kRowsPerBlock * 16;                                   // [128][64]
  __nv_bfloat16* sH2 = sH1 + kRowsPerBlock * 64;
  __nv_bfloat16* sD2 = sH2 + kRowsPerBlock * 64;                                  // dz2
  __nv_bfloat16* sD1 = sD2 + kRowsPerBlock * 64;                                  // dz1
  float* sDy = reinterpret_cast<float*>(sD1 + kRowsPerBlock * 64);                // [128]
  for (int i = threadIdx.x; i < int(sizeof(MlpDev) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t*>(&W)[i] = reinterpret_cast<const uint32_t*>(Wg)[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int64_t row0 = int64_t(blockIdx.x) * kRowsPerBlock + warp * 16;
  // gather this warp's 16 samples (through idx) into the A fragment of x~
  uint32_t xa[4];
  {
    const int64_t r0 = row0 + g, r1 = row0 + g + 8;
    const int c = 2 * q;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (r0 < n) {
      const int64_t s = idx ? idx[r0] : r0;
      v[0] = x[s * 8 + c];
      v[1] = x[s * 8 + c + 1];
    }
    if (r1 < n) {
      const int64_t s = idx ? idx[r1] : r1;
      v[2] = x[s * 8 + c];
      v[3] = x[s * 8 + c + 1];
    }
    xa[0] = pack2(__float2bfloat16_rn(v[0]), __float2bfloat16_rn(v[1]));
    xa[1] = pack2(__float2bfloat16_rn(v[2]), __float2bfloat16_rn(v[3]));
    xa[2] = 0u;
    xa[3] = 0u;
  }
  Fwd f;
  fwd16(W, xa, lane, f);
  // dy, squared error
  const int lr0 = warp * 16 + g, lr1 = lr0 + 8;
  float dy0 = 0.f, dy1 = 0.f;
  double se = 0.0;
  if (row0 + g < n) {
    const int64_t s = idx ? idx[row0 + g] : row0 + g;
    const float e = f.y_lo - t[s];
    dy0 = 2.0f * e * inv_b;
    se += double(e) * double(e);
  }
  if (row0 + g + 8 < n) {
    const int64_t s = idx ? idx[row0 + g + 8] : row0 + g + 8;
    const float e = f.y_hi - t[s];
    dy1 = 2.0f * e * inv_b;
    se += double(e) * double(e);
  }
  if (q == 0) {
    sDy[lr0] = dy0;
    sDy[lr1] = dy1;
  }
  // store x~, h1, h2 rows to shared memory (row-major, bf16)
  {
    const uint32_t* xr = xa;
    reinterpret_cast<uint32_t*>(sX + lr0 * 16)[q] = xr[0];
    reinterpret_cast<uint32_t*>(sX + lr1 * 16)[q] = xr[1];
    reinterpret_cast<uint32_t*>(sX + lr0 * 16 + 8)[q] = 0u;
    reinterpret_cast<uint32_t*>(sX + lr1 * 16 + 8)[q] = 0u;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      reinterpret_cast<uint32_t*>(sH1 + lr0 * 64 + 16 * s)[q] = f.h1[s][0];
      reinterpret_cast<uint32_t*>(sH1 + lr1 * 64 + 16 * s)[q] = f.h1[s][1];
      reinterpret_cast<uint32_t*>(sH1 + lr0 * 64 + 16 * s + 8)[q] = f.h1[s][2];
      reinterpret_cast<uint32_t*>(sH1 + lr1 * 64 + 16 * s + 8)[q] = f.h1[s][3];
      reinterpret_cast<uint32_t*>(sH2 + lr0 * 64 + 16 * s)[q] = f.h2[s][0];
      reinterpret_cast<uint32_t*>(sH2 + lr1 * 64 + 16 * s)[q] = f.h2[s][1];
      reinterpret_cast<uint32_t*>(sH2 + lr0 * 64 + 16 * s + 8)[q] = f.h2[s][2];
      reinterpret_cast<uint32_t*>(sH2 + lr1 * 64 + 16 * s + 8)[q] = f.h2[s][3];
    }
  }
  __syncwarp();
  // dz2 = bf16(dy W3 [h2 > 0]) for the warp's rows, columns 2q, 2q+1 (+8) of each k-slice
  uint32_t d2[4][4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int row = (r & 1) ? lr1 : lr0;
      const int col = 16 * s + 2 * q + ((r & 2) ? 8 : 0);
      const float dyr = sDy[row];
      __nv_bfloat16 v[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float h = __bfloat162float(sH2[row * 64 + col + e]);
        v[e] = __float2bfloat16_rn(h > 0.f ? dyr * __bfloat162float(W.w3[col + e]) : 0.f);
      }
      d2[s][r] = pack2(v[0], v[1]);
      reinterpret_cast<uint32_t*>(sD2 + row * 64 + col)[0] = d2[s][r];
    }
  }
  // dh1 = W2 dz2 : [16 x 64 (dz2 dims)] x [64 x 64]^T -> B operand is W2^T, i.e. B[k = out][n = in]
  // = W2[in][out]; dz1 = bf16(dh1 [h1 > 0])
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int n = nt * 8 + g, k = s * 16 + 2 * q;
      const uint32_t b0 = pack2(W.w2[n * 64 + k], W.w2[n * 64 + k + 1]);
      const uint32_t b1 = pack2(W.w2[n * 64 + k + 8], W.w2[n * 64 + k + 9]);
      mma_bf16(acc, d2[s][0], d2[s][1], d2[s][2], d2[s][3], b0, b1);
    }
    const int col = nt * 8 + 2 * q;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int row = r ? lr1 : lr0;
      __nv_bfloat16 v[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float h = __bfloat162float(sH1[row * 64 + col + e]);
        v[e] = __float2bfloat16_rn(h > 0.f ? acc[2 * r + e] : 0.f);
      }
      reinterpret_cast<uint32_t*>(sD1 + row * 64 + col)[0] = pack2(v[0], v[1]);
    }
  }
  __syncthreads();
  float* P = part + int64_t(blockIdx.x) * kParams;
  // weight gradients over the block's 128 samples (K = 128 in 8 slices), warp w owns n-tile w:
  // dW2[in][out]: M = 64 inputs (4 m-tiles), N = 64 outputs; A[m = in][k = sample] = h1[sample][in],
  // B[k = sample][n = out] = dz2[sample][out].
  {
    const int nt = warp;
    float acc2[4][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc2[mt][e] = 0.f;
    float acc1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int ks = 0; ks < kRowsPerBlock / 16; ++ks) {
      const int k = ks * 16 + 2 * q;
      const int n = nt * 8 + g;
      const uint32_t b0 = pack2(sD2[(k + 0) * 64 + n], sD2[(k + 1) * 64 + n]);
      const uint32_t b1 = pack2(sD2[(k + 8) * 64 + n], sD2[(k + 9) * 64 + n]);
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int m0 = mt * 16 + g;
        const uint32_t a0 = pack2(sH1[(k + 0) * 64 + m0], sH1[(k + 1) * 64 + m0]);
        const uint32_t a1 = pack2(sH1[(k + 0) * 64 + m0 + 8], sH1[(k + 1) * 64 + m0 + 8]);
        const uint32_t a2 = pack2(sH1[(k + 8) * 64 + m0], sH1[(k + 9) * 64 + m0]);
        const uint32_t a3 = pack2(sH1[(k + 8) * 64 + m0 + 8], sH1[(k + 9) * 64 + m0 + 8]);
        mma_bf16(acc2[mt], a0, a1, a2, a3, b0, b1);
      }
      // dW1[in][out]: M = 16 inputs, A[m = in][k = sample] = x~[sample][in], B = dz1
      const uint32_t c0 = pack2(sD1[(k + 0) * 64 + n], sD1[(k + 1) * 64 + n]);
      const uint32_t c1 = pack2(sD1[(k + 8) * 64 + n], sD1[(k + 9) * 64 + n]);
      const int m0 = g;
      const uint32_t a0 = pack2(sX[(k + 0) * 16 + m0], sX[(k + 1) * 16 + m0]);
      const uint32_t a1 = pack2(sX[(k + 0) * 16 + m0 + 8], sX[(k + 1) * 16 + m0 + 8]);
      const uint32_t a2 = pack2(sX[(k + 8) * 16 + m0], sX[(k + 9) * 16 + m0]);
      const uint32_t a3 = pack2(sX[(k + 8) * 16 + m0 + 8], sX[(k + 9) * 16 + m0 + 8]);
      mma_bf16(acc1, a0, a1, a2, a3, c0, c1);
    }
    // d fragment: rows m = g (+8), cols n = nt*8 + 2q, +1
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      const int m0 = mt * 16 + g, ncol = nt * 8 + 2 * q;
      P[kOffW2 + m0 * 64 + ncol] = acc2[mt][0];
      P[kOffW2 + m0 * 64 + ncol + 1] = acc2[mt][1];
      P[kOffW2 + (m0 + 8) * 64 + ncol] = acc2[mt][2];
      P[kOffW2 + (m0 + 8) * 64 + ncol + 1] = acc2[mt][3];
    }
    {
      const int ncol = nt * 8 + 2 * q;
      if (g < 8) {  // rows 8..15 of x~ are padding
        P[kOffW1 + g * 64 + ncol] = acc1[0];
        P[kOffW1 + g * 64 + ncol + 1] = acc1[1];
      }
    }
  }
  // bias and W3 gradients: column sums over the block's 128 rows, in row order
  for (int c = threadIdx.x; c < 64 * 4 + 1; c += blockDim.x) {
    float s = 0.f;
    if (c < 64) {
      for (int r = 0; r < kRowsPerBlock; ++r) s += __bfloat162float(sD1[r * 64 + c]);
      P[kOffB1 + c] = s;
    } else if (c < 128) {
      for (int r = 0; r < kRowsPerBlock; ++r) s += __bfloat162float(sD2[r * 64 + c - 64]);
      P[kOffB2 + c - 64] = s;
    } else if (c < 192) {
      for (int r = 0; r < kRowsPerBlock; ++r) s = __fmaf_rn(sDy[r], __bfloat162float(sH2[r * 64 + c - 128]), s);
      P[kOffW3 + c - 128] = s;
    } else if (c == 256) {
      for (int r = 0; r < kRowsPerBlock; ++r) s += sDy[r];
      P[kOffB3] = s;
    }
  }
  // sum of squared errors of the block (deterministic: warp sums in lane order, then warps)
  __shared__ double sse_w[kWarps];
  double v = (q == 0) ? se : 0.0;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
  if (lane == 0) sse_w[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < kWarps; ++w) tot = __dadd_rn(tot, sse_w[w]);
    sse_part[blockIdx.x] = tot;
  }
}

// grad[p] = sum over blocks of part[b][p], blocks in order.
__global__ void k_mlp_reduce(int nblk, const float* __restrict__ part, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[int64_t(b) * kParams + p];
  grad[p] = s;
}

// Adam step on the float32 masters (k_pack_weights then refreshes the bf16 device weights).
// Step number k = *step (0-based); corr[2k], corr[2k + 1] = 1 - b1^(k+1), 1 - b2^(k+1) (the
// bias corrections, rounded on the host). The step counter lives on the device so that one
// captured epoch replays with the right corrections.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, float lr, float b1, float b2, float eps,
                       const float* __restrict__ corr, const int64_t* __restrict__ step) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  const int64_t k = *step;
  const float c1 = corr[2 * k], c2 = corr[2 * k + 1];
  const float gr = grad[p];
  const float mm = b1 * m[p] + (1.f - b1) * gr;
  const float vv = b2 * v[p] + (1.f - b2) * gr * gr;
  m[p] = mm;
  v[p] = vv;
  const float wn = w[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  w[p] = wn;
}

__device__ __forceinline__ __nv_bfloat16 w1_at(const float* __restrict__ w, int in, int out) {
  return __float2bfloat16_rn(in < 8 ? w[kOffW1 + in * 64 + out] : 0.f);
}

__device__ __forceinline__ __nv_bfloat16 w2_at(const float* __restrict__ w, int in, int out) {
  return __float2bfloat16_rn(w[kOffW2 + in * 64 + out]);
}

// bf16 copies and mma fragments of the float32 weights; advances the Adam step counter (if
// given) once the step's update has been packed.
__global__ void k_pack_weights(const float* __restrict__ w, MlpDev* __restrict__ dev,
                               int64_t* __restrict__ step) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (step && p == 0) *step += 1;
  if (p < 8 * 32) {  // W1 fragments (one k-slice)
    const int nt = p / 32, lane = p % 32, g = lane >> 2, q = lane & 3;
    const int n = nt * 8 + g, k = 2 * q;
    dev->f1[nt][lane] = make_uint2(pack2(w1_at(w, k, n), w1_at(w, k + 1, n)),
                                   pack2(w1_at(w, k + 8, n), w1_at(w, k + 9, n)));
  }
  if (p < 4 * 8 * 32) {  // W2 fragments
    const int ks = p / 256, nt = (p / 32) % 8, lane = p % 32, g = lane >> 2, q = lane & 3;
    const int n = nt * 8 + g, k = ks * 16 + 2 * q;
    dev->f2[ks][nt][lane] = make_uint2(pack2(w2_at(w, k, n), w2_at(w, k + 1, n)),
                                       pack2(w2_at(w, k + 8, n), w2_at(w, k + 9, n)));
  }
  if (p < 16 * 64) {
    const int in = p / 64, out = p % 64;
    dev->w1[p] = __float2bfloat16_rn(in < 8 ? w[kOffW1 + in * 64 + out] : 0.f);
  }
  if (p < 64 * 64) dev->w2[p] = __float2bfloat16_rn(w[kOffW2 + p]);
  if (p < 64) {
    dev->w3[p] = __float2bfloat16_rn(w[kOffW3 + p]);
    dev->b1[p] = w[kOffB1 + p];
    dev->b2[p] = w[kOffB2 + p];
  }
  if (p == 0) dev->b3 = w[kOffB3];
}

// Max |y - t| over samples (non-negative floats compare as their bit patterns).
__global__ void k_abs_err_max(int64_t n, const float* __restrict__ y, const float* __restrict__ t,
                              unsigned int* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  float e = 0.f;
  if (i < n) e = fabsf(y[i] - t[i]);
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(e));
}

__global__ void k_gather_f32(int64_t n, const int64_t* __restrict__ idx, const float* __restrict__ src,
                             int width, float* __restrict__ dst) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n * width) return;
  const int64_t r = i / width, c = i % width;
  dst[i] = src[idx[r] * width + c];
}

size_t grad_smem() {
  return sizeof(MlpDev) + size_t(kRowsPerBlock) * (16 + 4 * 64) * 2 + kRowsPerBlock * 4;
}

// Host-side splitmix64 for the initial weights and the shuffles (reproducible on any host).
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

double uniform01(uint64_t& s) { return double(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

namespace rs {

static int ensure_mlp(rs_ctx* ctx) {
  if (!scratch(ctx, S_MLP_DEV, sizeof(MlpDev))) return RS_ERR_OOM;
  if (!scratch(ctx, S_MLP_W, sizeof(float) * kParams)) return RS_ERR_OOM;
  return RS_OK;
}

int mlp_forward(rs_ctx* ctx, int64_t n, const float* x, float* y, cudaStream_t st) {
  if (!ctx->have_mlp) return set_error(ctx, RS_ERR_STATE, "no surrogate weights on this context");
  if (n <= 0) return RS_OK;
  const MlpDev* dev = static_cast<const MlpDev*>(ctx->buf[S_MLP_DEV].ptr);
  const int64_t warps = (n + 15) / 16;
  const unsigned grid = unsigned(std::min<int64_t>((warps + kWarps - 1) / kWarps, 152 * 8));
  {
    ProfScope prof_(ctx, "k_mlp_fwd", st);
    k_mlp_fwd<<<grid, kThreads, 0, st>>>(n, x, dev, y);
  }
  RS_LAUNCHED(ctx, "k_mlp_fwd");
  return RS_OK;
}

static int set_params_dev(rs_ctx* ctx, const float* w_dev_or_host, bool host, cudaStream_t st) {
  RS_TRY(ensure_mlp(ctx));
  float* w = static_cast<float*>(ctx->buf[S_MLP_W].ptr);
  RS_CUDA(ctx, cudaMemcpyAsync(w, w_dev_or_host, sizeof(float) * kParams,
                               host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  k_pack_weights<<<(64 * 64 + 255) / 256, 256, 0, st>>>(w, static_cast<MlpDev*>(ctx->buf[S_MLP_DEV].ptr),
                                                        nullptr);
  RS_LAUNCHED(ctx, "k_pack_weights");
  ctx->have_mlp = true;
  return RS_OK;
}

int mlp_copy(rs_ctx* dst, rs_ctx* src, cudaStream_t st) {
  if (!src->have_mlp) return set_error(dst, RS_ERR_STATE, "no surrogate weights to copy");
  RS_TRY(set_params_dev(dst, static_cast<const float*>(src->buf[S_MLP_W].ptr), false, st));
  dst->mlp_err_max = src->mlp_err_max;
  return RS_OK;
}

// Full-batch gradient of L = (1/B) sum (y - t)^2 over rows idx[0..n) (or 0..n).
// (capturing: enqueue only - scratch is already sized and the attribute set, so nothing but
// stream work happens while a graph is being captured.)
static int mlp_gradient(rs_ctx* ctx, int64_t n, const float* x, const float* t, const int64_t* idx,
                        float* grad, double* sse_out, cudaStream_t st, bool capturing = false) {
  const int nblk = int((n + kRowsPerBlock - 1) / kRowsPerBlock);
  float* part = scratch_t<float>(ctx, S_MLP_PART, size_t(nblk) * kParams);
  double* sse = scratch_t<double>(ctx, S_MLP_SSE, size_t(nblk) + 1);
  if (!part || !sse) return RS_ERR_OOM;
  const size_t smem = grad_smem();
  if (!capturing)
    RS_CUDA(ctx, cudaFuncSetAttribute(k_mlp_grad_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(smem)));
  {
    ProfScope prof_(ctx, "k_mlp_grad_block", st);
    k_mlp_grad_block<<<nblk, kThreads, smem, st>>>(n, x, t, idx, 1.0f / float(n),
                                                   static_cast<const MlpDev*>(ctx->buf[S_MLP_DEV].ptr),
                                                   part, sse);
  }
  RS_LAUNCHED(ctx, "k_mlp_grad_block");
  k_mlp_reduce<<<(kParams + 255) / 256, 256, 0, st>>>(nblk, part, grad);
  RS_LAUNCHED(ctx, "k_mlp_reduce");
  if (sse_out) {
    std::vector<double> h(nblk);
    RS_CUDA(ctx, cudaMemcpyAsync(h.data(), sse, sizeof(double) * nblk, cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : h) s += v;
    *sse_out = s;
  }
  return RS_OK;
}

}  // namespace rs

extern "C" int rs_mlp_set_params(rs_ctx* ctx, const float* params_host) {
  if (!ctx || !params_host) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  RS_TRY(set_params_dev(ctx, params_host, true, nullptr));
  RS_CUDA(ctx, cudaDeviceSynchronize());
  return RS_OK;
}

extern "C" int rs_mlp_get_params(rs_ctx* ctx, float* params_host) {
  if (!ctx || !params_host) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (!ctx->have_mlp) return set_error(ctx, RS_ERR_STATE, "no surrogate weights on this context");
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  RS_CUDA(ctx, cudaMemcpy(params_host, ctx->buf[S_MLP_W].ptr, sizeof(float) * kParams,
                          cudaMemcpyDeviceToHost));
  return RS_OK;
}

extern "C" int rs_mlp_forward(rs_ctx* ctx, int64_t n, const float* x, float* y, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!x || !y))) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  return mlp_forward(ctx, n, x, y, static_cast<cudaStream_t>(stream));
}

extern "C" int rs_mlp_gradient(rs_ctx* ctx, int64_t n, const float* x, const float* t, float* grad,
                               double* sse_out, void* stream) {
  if (!ctx || n <= 0 || !x || !t || !grad) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (!ctx->have_mlp) return set_error(ctx, RS_ERR_STATE, "no surrogate weights on this context");
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  return mlp_gradient(ctx, n, x, t, nullptr, grad, sse_out, static_cast<cudaStream_t>(stream));
}

extern "C" int rs_mlp_train(rs_ctx* ctx, int64_t n, const float* x, const float* t, int32_t epochs,
                            int32_t batch, float lr, uint64_t seed, int32_t holdout_num,
                            int32_t holdout_den, float* err_max_out, double* train_mse_out,
                            void* stream) {
  if (!ctx || n < 16 || !x || !t || epochs < 0 || batch < 16 || !(lr > 0.f) || holdout_num < 0 ||
      holdout_den <= 0 || holdout_num >= holdout_den)
    return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_CUDA(ctx, cudaSetDevice(ctx->device));
  // He-uniform initial weights and zero biases from the seed (host, reproducible).
  std::vector<float> w0(kParams, 0.f);
  uint64_t s = seed;
  const double a1 = std::sqrt(6.0 / 8.0), a2 = std::sqrt(6.0 / 64.0);
  for (int i = 0; i < 512; ++i) w0[kOffW1 + i] = float((2.0 * uniform01(s) - 1.0) * a1);
  for (int i = 0; i < 4096; ++i) w0[kOffW2 + i] = float((2.0 * uniform01(s) - 1.0) * a2);
  for (int i = 0; i < 64; ++i) w0[kOffW3 + i] = float((2.0 * uniform01(s) - 1.0) * a2);
  RS_TRY(set_params_dev(ctx, w0.data(), true, st));
  float* mom = scratch_t<float>(ctx, S_MLP_M, 2 * kParams);
  float* grad = scratch_t<float>(ctx, S_MLP_G, kParams);
  if (!mom || !grad) return RS_ERR_OOM;
  RS_CUDA(ctx, cudaMemsetAsync(mom, 0, sizeof(float) * 2 * kParams, st));
  // Split: the last holdout_num/holdout_den of a seeded permutation is held out.
  std::vector<int64_t> perm(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  for (int64_t i = n - 1; i > 0; --i) std::swap(perm[i], perm[int64_t(splitmix(s) % uint64_t(i + 1))]);
  const int64_t n_hold = n * holdout_num / holdout_den;
  const int64_t n_train = n - n_hold;
  int64_t* idx = scratch_t<int64_t>(ctx, S_MLP_IDX, size_t(n));
  if (!idx) return RS_ERR_OOM;
  RS_CUDA(ctx, cudaMemcpyAsync(idx, perm.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  RS_CUDA(ctx, cudaStreamSynchronize(st));
  float* w = static_cast<float*>(ctx->buf[S_MLP_W].ptr);
  MlpDev* dev = static_cast<MlpDev*>(ctx->buf[S_MLP_DEV].ptr);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int64_t per_epoch = n_train / batch;  // full batches; the remainder is left out
  const int64_t total = int64_t(epochs) * per_epoch;
  // bias corrections of every step, host-rounded: 1 - b^(k+1)
  std::vector<float> corr(size_t(2 * std::max<int64_t>(total, 1)), 1.f);
  for (int64_t k = 0; k < total; ++k) {
    corr[2 * k] = 1.f - std::pow(b1, float(k + 1));
    corr[2 * k + 1] = 1.f - std::pow(b2, float(k + 1));
  }
  float* d_corr = scratch_t<float>(ctx, S_MLP_CORR, corr.size());
  int64_t* d_step = scratch_t<int64_t>(ctx, S_MLP_STEP, 1);
  int64_t* bidx = scratch_t<int64_t>(ctx, S_MLP_BIDX, size_t(std::max<int64_t>(n_train, 1)));
  const int nblk = int((batch + kRowsPerBlock - 1) / kRowsPerBlock);
  double* sse = scratch_t<double>(ctx, S_MLP_SSE, size_t(nblk) + 1);
  if (!d_corr || !d_step || !bidx || !sse || !scratch_t<float>(ctx, S_MLP_PART, size_t(nblk) * kParams))
    return RS_ERR_OOM;
  RS_CUDA(ctx, cudaMemcpyAsync(d_corr, corr.data(), sizeof(float) * corr.size(),
                               cudaMemcpyHostToDevice, st));
  RS_CUDA(ctx, cudaMemsetAsync(d_step, 0, sizeof(int64_t), st));
  RS_CUDA(ctx, cudaFuncSetAttribute(k_mlp_grad_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(grad_smem())));
  RS_CUDA(ctx, cudaStreamSynchronize(st));
  // One epoch's launches: gradient of each batch, Adam update, weight packing. Static (the
  // batch order lives in bidx, the step in d_step), so with graphs on the epoch is captured
  // once and replayed; off, the same launches are issued one by one.
  auto epoch_body = [&](cudaStream_t s, bool capturing) -> int {
    for (int64_t b = 0; b < per_epoch; ++b) {
      RS_TRY(mlp_gradient(ctx, batch, x, t, bidx + b * batch, grad, nullptr, s, capturing));
      k_adam<<<(kParams + 255) / 256, 256, 0, s>>>(w, mom, mom + kParams, grad, lr, b1, b2, eps,
                                                   d_corr, d_step);
      RS_LAUNCHED(ctx, "k_adam");
      k_pack_weights<<<(64 * 64 + 255) / 256, 256, 0, s>>>(w, dev, d_step);
      RS_LAUNCHED(ctx, "k_pack_weights");
    }
    return RS_OK;
  };
  cudaGraphExec_t exec = nullptr;
  int64_t graph_launches = 0;
  std::vector<int64_t> order(n_train);
  int rc = RS_OK;
  for (int e = 0; e < epochs && rc == RS_OK; ++e) {
    for (int64_t i = 0; i < n_train; ++i) order[i] = perm[i];
    for (int64_t i = n_train - 1; i > 0; --i)
      std::swap(order[i], order[int64_t(splitmix(s) % uint64_t(i + 1))]);
    if (n_train > 0) {
      const cudaError_t ce = cudaMemcpyAsync(bidx, order.data(), sizeof(int64_t) * n_train,
                                             cudaMemcpyHostToDevice, st);
      if (ce != cudaSuccess) {
        rc = set_error(ctx, RS_ERR_CUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(ce));
        break;
      }
    }
    if (per_epoch == 0) continue;
    if (!ctx->use_graphs) {
      rc = epoch_body(st, false);
      continue;
    }
    if (!exec) {
      rc = capture_graph(ctx, [&](cudaStream_t cs) { return epoch_body(cs, true); }, &exec,
                         &graph_launches);
      if (rc != RS_OK) break;
    }
    rc = launch_graph(ctx, exec, graph_launches, st);
  }
  if (exec) cudaGraphExecDestroy(exec);
  RS_TRY(rc);
  // squared-error sum of the last batch trained (its per-block partials), host order
  double last_sse = 0.0;
  if (total > 0) {
    std::vector<double> h(nblk);
    RS_CUDA(ctx, cudaMemcpyAsync(h.data(), sse, sizeof(double) * nblk, cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    for (double v : h) last_sse += v;
    last_sse /= double(batch);
  }
  if (train_mse_out) *train_mse_out = last_sse;
  // held-out max |y - t|
  float em = 0.f;
  if (n_hold > 0) {
    float* xh = scratch_t<float>(ctx, S_MLP_XH, size_t(n_hold) * 9 + 2);
    unsigned int* mx = scratch_t<unsigned int>(ctx, S_COUNTER, 2);
    if (!xh || !mx) return RS_ERR_OOM;
    float* th = xh + n_hold * 8;
    float* yh = scratch_t<float>(ctx, S_MLP_YH, size_t(n_hold));
    if (!yh) return RS_ERR_OOM;
    k_gather_f32<<<grid_for(n_hold * 8, 256), 256, 0, st>>>(n_hold, idx + n_train, x, 8, xh);
    RS_LAUNCHED(ctx, "k_gather_f32");
    k_gather_f32<<<grid_for(n_hold, 256), 256, 0, st>>>(n_hold, idx + n_train, t, 1, th);
    RS_LAUNCHED(ctx, "k_gather_f32");
    RS_TRY(mlp_forward(ctx, n_hold, xh, yh, st));
    RS_CUDA(ctx, cudaMemsetAsync(mx, 0, 4, st));
    k_abs_err_max<<<grid_for(n_hold, 256), 256, 0, st>>>(n_hold, yh, th, mx);
    RS_LAUNCHED(ctx, "k_abs_err_max");
    unsigned int bits = 0;
    RS_CUDA(ctx, cudaMemcpyAsync(&bits, mx, 4, cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    std::memcpy(&em, &bits, 4);
  }
  ctx->mlp_err_max = em;
  if (err_max_out) *err_max_out = em;
  return RS_OK;
}

extern "C" int rs_mlp_set_err_max(rs_ctx* ctx, float err_max) {
  if (!ctx || !(err_max >= 0.f)) return RS_ERR_INVALID_ARG;
  ctx->mlp_err_max = err_max;
  return RS_OK;
}

extern "C" int rs_mlp_get_err_max(rs_ctx* ctx, float* err_max_out) {
  if (!ctx || !err_max_out) return RS_ERR_INVALID_ARG;
  *err_max_out = ctx->mlp_err_max;
  return RS_OK;
}

// ---- Surrogate checkpoint: the float32 master parameters and the held-out maximum error in a
// little-endian file: magic "RSMLPv01" (8 bytes), uint32 parameter count (4801), uint32 0,
// float32 err_max, float32 params[4801], uint64 FNV-1a hash of the params' bytes.
namespace {
constexpr char kMagic[8] = {'R', 'S', 'M', 'L', 'P', 'v', '0', '1'};

uint64_t fnv1a(const void* data, size_t bytes) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < bytes; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}
}  // namespace

extern "C" int rs_surrogate_save(rs_ctx* ctx, const char* path) {
  if (!ctx || !path) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  std::vector<float> p(kParams);
  RS_TRY(rs_mlp_get_params(ctx, p.data()));
  FILE* f = std::fopen(path, "wb");
  if (!f) return set_error(ctx, RS_ERR_INVALID_ARG, "cannot open %s for writing", path);
  const uint32_t hdr[2] = {uint32_t(kParams), 0u};
  const float em = ctx->mlp_err_max;
  const uint64_t h = fnv1a(p.data(), sizeof(float) * kParams);
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, 4, 2, f) == 2 &&
            std::fwrite(&em, 4, 1, f) == 1 && std::fwrite(p.data(), 4, kParams, f) == size_t(kParams) &&
            std::fwrite(&h, 8, 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return set_error(ctx, RS_ERR_INVALID_ARG, "short write to %s", path);
  return RS_OK;
}

extern "C" int rs_surrogate_load(rs_ctx* ctx, const char* path) {
  if (!ctx || !path) return RS_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_error(ctx, RS_ERR_INVALID_ARG, "cannot open %s", path);
  char magic[8];
  uint32_t hdr[2];
  float em = 0.f;
  std::vector<float> p(kParams);
  uint64_t h = 0;
  const bool ok = std::fread(magic, 1, 8, f) == 8 && std::fread(hdr, 4, 2, f) == 2 &&
                  std::fread(&em, 4, 1, f) == 1 && std::fread(p.data(), 4, kParams, f) == size_t(kParams) &&
                  std::fread(&h, 8, 1, f) == 1;
  std::fclose(f);
  if (!ok || std::memcmp(magic, kMagic, 8) != 0 || hdr[0] != uint32_t(kParams))
    return set_error(ctx, RS_ERR_INVALID_ARG, "%s is not a surrogate checkpoint", path);
  if (h != fnv1a(p.data(), sizeof(float) * kParams) || !(em >= 0.f))
    return set_error(ctx, RS_ERR_INVALID_ARG, "%s is corrupt (hash or err_max)", path);
  RS_TRY(rs_mlp_set_params(ctx, p.data()));
  ctx->mlp_err_max = em;
  return RS_OK;
}

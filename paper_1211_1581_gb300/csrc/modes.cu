// modes.cu -- the FP32 comparison mode: A and B rounded to FP32 (nearest),
// C = A.B summed in FP32 on the CUDA cores (FFMA), written back as FP64.
// It is reported beside the FP64-accurate modes to show what single
// precision gives on the same inputs; it is not FP64-accurate.
//
// Tiling: 128 x 128 C tile per block, k in steps of 8, 256 threads with an
// 8 x 8 register tile each (rows ty*4 + {0..3, 64..67}, columns tx*4 +
// {0..3, 64..67}); operands staged through double-buffered shared memory,
// converted from FP64 while loading.
#include <cuda_runtime.h>

#include <cstdint>

#include "mxm_internal.h"

namespace mxm {
namespace {

constexpr int BM = 128, BN = 128, BK = 8;

__global__ void __launch_bounds__(256) f32_gemm_kernel(const double* __restrict__ A,
                                                       const double* __restrict__ B,
                                                       double* __restrict__ C, int64_t m,
                                                       int64_t k, int64_t n) {
  __shared__ float As[2][BK][BM];
  __shared__ float Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = static_cast<int64_t>(blockIdx.y) * BM;
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * BN;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  // loader mapping: A tile 128 x 8 (4 values per thread), B tile 8 x 128
  auto load = [&](int buf, int64_t k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = tid + q * 256;      // 0..1023
      const int ar = p >> 3, ac = p & 7;  // A: row, k
      const int64_t gr = m0 + ar, gk = k0 + ac;
      As[buf][ac][ar] = (gr < m && gk < k) ? __double2float_rn(__ldg(A + gr * k + gk)) : 0.f;
      const int br = p >> 7, bc = p & 127;  // B: k, column
      const int64_t hk = k0 + br, hc = n0 + bc;
      Bs[buf][br][bc] = (hk < k && hc < n) ? __double2float_rn(__ldg(B + hk * n + hc)) : 0.f;
    }
  };

  const int64_t nk = (k + BK - 1) / BK;
  load(0, 0);
  __syncthreads();
  for (int64_t kb = 0; kb < nk; ++kb) {
    const int cur = kb & 1;
    if (kb + 1 < nk) load(cur ^ 1, (kb + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[8], b[8];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4 + 64]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4 + 64]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t row = m0 + ty * 4 + (i & 3) + (i >> 2) * 64;
    if (row >= m) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t col = n0 + tx * 4 + (j & 3) + (j >> 2) * 64;
      if (col < n) C[row * n + col] = static_cast<double>(acc[i][j]);
    }
  }
}

}  // namespace

cudaError_t launch_f32_gemm(const double* A, const double* B, double* C, int64_t m, int64_t k,
                            int64_t n, cudaStream_t s) {
  dim3 grid(static_cast<unsigned>((n + BN - 1) / BN), static_cast<unsigned>((m + BM - 1) / BM));
  f32_gemm_kernel<<<grid, 256, 0, s>>>(A, B, C, m, k, n);
  return cudaGetLastError();
}

}  // namespace mxm

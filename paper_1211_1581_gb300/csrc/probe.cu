// probe.cu -- peak-rate probes of single execution units (the roofline
// denominators the driver does not measure: FP64 DFMA, FP64 DMMA, legacy
// IMMA) plus tcgen05 BF16 for comparison with the driver's cuBLAS figure.
// Each probe keeps its operands in registers (or zeroed shared memory), runs
// a fixed number of independent operations per warp (tens of milliseconds of
// work, so that launch overhead and the clock's ramp do not count) and is
// timed with CUDA events; the rate is operations / time over the whole GPU.
#include <cuda_runtime.h>

#include <cstdint>

#include "mxm.h"
#include "mxm_internal.h"
#include "ptx.cuh"

namespace mxm {
namespace {

__global__ void probe_dfma_kernel(int iters, double seed, double* sink) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = seed + i + threadIdx.x;
  const double y = 1.0000001, z = 1e-9;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], y, z);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 12345.678) sink[0] = s;
}

__global__ void probe_dmma_kernel(int iters, double seed, double* sink) {
  double acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0.0;
  double a0 = seed + threadIdx.x, a1 = seed * 2.0, b0 = seed - 1.0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
          "{%0,%1,%2,%3};"
          : "+d"(acc[i][0]), "+d"(acc[i][1]), "+d"(acc[i][2]), "+d"(acc[i][3])
          : "d"(a0), "d"(a1), "d"(b0));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i][0] + acc[i][3];
  if (s == 12345.678) sink[0] = s;
}

__global__ void probe_imma_kernel(int iters, int seed, int* sink) {
  int acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0;
  const uint32_t a0 = seed, a1 = seed + 1, a2 = seed + 2, a3 = seed + 3, b0 = seed * 3,
                 b1 = seed * 5;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};"
          : "+r"(acc[i][0]), "+r"(acc[i][1]), "+r"(acc[i][2]), "+r"(acc[i][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  int s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i][0] + acc[i][3];
  if (s == 12345) sink[0] = s;
}

// tcgen05 BF16: one CTA per SM, one thread issues `iters` MMAs of 128 x N x 16
// from zeroed shared memory into two alternating TMEM accumulators.
template <int N>
__global__ void __launch_bounds__(128, 1) probe_umma_kernel(int iters, int* status) {
  extern __shared__ uint8_t raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  uint8_t* a = base;                       // 128 x 64 bf16
  uint8_t* b = base + 16384;               // N x 64 bf16
  __shared__ uint64_t done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  for (int i = threadIdx.x; i < (16384 + N * 128) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(base)[i] = make_uint4(0, 0, 0, 0);
  fence_async_shared();
  if (threadIdx.x == 0) {
    mbar_init(&done, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if ((threadIdx.x >> 5) == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  if (threadIdx.x == 32) {
    const uint32_t idesc = idesc_bf16_f32(128, N);
    const uint32_t aa = smem_u32(a), bb = smem_u32(b);
    for (int it = 0; it < iters; ++it) {
      const int kk = it & 3;
      mma_bf16_ss(tmem + static_cast<uint32_t>((it & 1) * N), sw128_kmajor_desc(aa + kk * 32),
                  sw128_kmajor_desc(bb + kk * 32), idesc, it > 1 ? 1u : 0u);
    }
    mma_commit(&done);
    (void)mbar_wait_bounded(&done, 0u, &abort_flag, status);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, 512);
}

}  // namespace
}  // namespace mxm

using namespace mxm;

extern "C" mxm_status mxm_peak_probe(int kind, double* tflops) {
  NvtxRange nvtx_range("mxm_peak_probe");
  if (tflops == nullptr || kind < 0 || kind > 4) return MXM_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MXM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MXM_ERR_CUDA;
  void* sink = nullptr;
  int* status = nullptr;
  if (cudaMalloc(&sink, 64) != cudaSuccess) return MXM_ERR_CUDA;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
    cudaFree(sink);
    return MXM_ERR_CUDA;
  }
  cudaMemset(status, 0, sizeof(int));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double ops = 0;
  auto launch = [&](bool timed) -> cudaError_t {
    const int blocks = sms * 4, threads = 256;
    switch (kind) {
      case 0: {
        const int iters = timed ? 16384 : 8;
        probe_dfma_kernel<<<blocks, threads>>>(iters, 1.0, static_cast<double*>(sink));
        ops = 2.0 * 8 * iters * double(blocks) * threads;
        break;
      }
      case 1: {
        const int iters = timed ? 1024 : 2;
        probe_dmma_kernel<<<blocks, threads>>>(iters, 1.0, static_cast<double*>(sink));
        ops = 2.0 * 16 * 8 * 4 * 8.0 * iters * blocks * (threads / 32);
        break;
      }
      case 4: {
        const int iters = timed ? 4096 : 8;
        probe_imma_kernel<<<blocks, threads>>>(iters, 1, static_cast<int*>(sink));
        ops = 2.0 * 16 * 8 * 32 * 8.0 * iters * blocks * (threads / 32);
        break;
      }
      case 2:
      case 3: {
        const int N = kind == 2 ? 128 : 256;
        const int iters = timed ? 65536 : 256;
        // at least 120 KiB so that one CTA (and its 512 TMEM columns) owns each SM
        const size_t smem = 120 * 1024;
        if (N == 128) {
          cudaFuncSetAttribute(probe_umma_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
          probe_umma_kernel<128><<<sms, 128, smem>>>(iters, status);
        } else {
          cudaFuncSetAttribute(probe_umma_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
          probe_umma_kernel<256><<<sms, 128, smem>>>(iters, status);
        }
        ops = 2.0 * 128 * N * 16 * double(iters) * sms;
        break;
      }
    }
    return cudaGetLastError();
  };
  mxm_status st = MXM_OK;
  if (launch(false) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) st = MXM_ERR_CUDA;
  float ms = 0.f;
  if (st == MXM_OK) {
    cudaEventRecord(e0);
    if (launch(true) != cudaSuccess) st = MXM_ERR_CUDA;
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = MXM_ERR_CUDA;
    cudaEventElapsedTime(&ms, e0, e1);
  }
  int sv = 0;
  cudaMemcpy(&sv, status, sizeof(int), cudaMemcpyDeviceToHost);
  if (sv & kStatusTimeout) st = MXM_ERR_TIMEOUT;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(status);
  if (st == MXM_OK) *tflops = ops / (double(ms) * 1e-3) / 1e12;
  return st;
}

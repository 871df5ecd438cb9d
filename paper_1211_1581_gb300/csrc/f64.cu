// f64.cu -- native FP64 product C = A.B (mod2am, Sec. 3.1) on the FP64
// tensor path (DMMA, mma.sync m16n8k4 .f64), fed by bulk copies.
//
// The paper's k-blocked rank-u update (arbb_mxm2b, Sec. 3.1) becomes the K
// loop over 16-wide k-blocks here; every block is a rank-16 update of a
// 128 x 128 C tile held in FP64 registers.
//
// Data path:
//   f64_pack_a / f64_pack_b  copy A and B once into zero-padded 128 x 16
//       tiles (B transposed, both K-major) with an XOR swizzle that makes the
//       DMMA fragment loads bank-conflict free; one tile = 16 KiB, moved by a
//       single cp.async.bulk.
//   f64_gemm  warp 0 streams tiles into a 4-stage shared-memory ring
//       (mbarrier full/empty pairs); warps 1..8 each own a 32 x 64 piece of
//       the C tile and issue DMMA; the epilogue stores C with edge masks.
#include <cuda_runtime.h>

#include <cstdint>

#include "mxm_internal.h"
#include "ptx.cuh"

namespace mxm {
namespace {

constexpr int BM = kF64BM, BN = kF64BN, BK = kF64BK;
constexpr int kStages = 4;
constexpr int kConsumerWarps = 8;
constexpr int kThreads = 32 * (1 + kConsumerWarps);

// element (r, c) of a 128 x 16 tile -> word offset (8-byte words)
__host__ __device__ __forceinline__ int swz(int r, int c) { return r * BK + (c ^ ((r & 3) << 2)); }

// A (m x k) -> [Mt][Kt] tiles, element (r, c) = A[tm*128 + r][tk*16 + c].
__global__ void f64_pack_a_kernel(const double* __restrict__ A, int64_t m, int64_t k, int64_t Kt,
                                  double* __restrict__ out) {
  const int64_t tk = blockIdx.x, tm = blockIdx.y;
  double* tile = out + (tm * Kt + tk) * (BM * BK);
  for (int p = threadIdx.x; p < BM * BK; p += blockDim.x) {
    const int r = p / BK, c = p % BK;
    const int64_t row = tm * BM + r, col = tk * BK + c;
    tile[swz(r, c)] = (row < m && col < k) ? __ldg(A + row * k + col) : 0.0;
  }
}

// B (k x n) -> [Nt][Kt] tiles of B^T, element (r, c) = B[tk*16 + c][tn*128 + r].
__global__ void f64_pack_b_kernel(const double* __restrict__ B, int64_t k, int64_t n, int64_t Kt,
                                  double* __restrict__ out) {
  __shared__ double t[BK][BN + 1];
  const int64_t tk = blockIdx.x, tn = blockIdx.y;
  for (int p = threadIdx.x; p < BK * BN; p += blockDim.x) {
    const int c = p / BN, r = p % BN;  // coalesced along n
    const int64_t kr = tk * BK + c, col = tn * BN + r;
    t[c][r] = (kr < k && col < n) ? __ldg(B + kr * n + col) : 0.0;
  }
  __syncthreads();
  double* tile = out + (tn * Kt + tk) * (BN * BK);
  for (int p = threadIdx.x; p < BN * BK; p += blockDim.x) {
    const int r = p / BK, c = p % BK;
    tile[swz(r, c)] = t[c][r];
  }
}

struct __align__(128) F64Smem {
  double a[kStages][BM * BK];
  double b[kStages][BN * BK];
  uint64_t full[kStages];
  uint64_t empty[kStages];
  int abort_flag;
};

__device__ __forceinline__ void dmma_16x8x4(double (&d)[4], double a0, double a1, double b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};"
      : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
      : "d"(a0), "d"(a1), "d"(b0));
}

__device__ __forceinline__ void tile_coords(int64_t tile, int64_t Mt, int64_t Nt, int64_t& tm,
                                            int64_t& tn) {
  constexpr int64_t G = 8;
  const int64_t per_group = G * Nt;
  const int64_t grp = tile / per_group;
  const int64_t first = grp * G;
  const int64_t gsz = (Mt - first) < G ? (Mt - first) : G;
  const int64_t in = tile - grp * per_group;
  tm = first + in % gsz;
  tn = in / gsz;
}

__global__ void __launch_bounds__(kThreads, 1) f64_gemm_kernel(
    const double* __restrict__ apack, const double* __restrict__ bpack, double* __restrict__ C,
    int64_t m, int64_t n, int64_t Mt, int64_t Nt, int64_t Kt, int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  F64Smem& sm = *reinterpret_cast<F64Smem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t tm, tn;
  tile_coords(blockIdx.x, Mt, Nt, tm, tn);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], kConsumerWarps);
    }
    sm.abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  volatile int* abort_flag = &sm.abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      const double* a_src = apack + tm * Kt * (BM * BK);
      const double* b_src = bpack + tn * Kt * (BN * BK);
      int stage = 0;
      uint32_t phase = 0;
      for (int64_t kb = 0; kb < Kt; ++kb) {
        if (!mbar_wait_bounded(&sm.empty[stage], phase ^ 1u, abort_flag, status)) break;
        mbar_arrive_expect_tx(&sm.full[stage], 2 * kF64TileBytes);
        bulk_g2s(sm.a[stage], a_src + kb * (BM * BK), kF64TileBytes, &sm.full[stage]);
        bulk_g2s(sm.b[stage], b_src + kb * (BN * BK), kF64TileBytes, &sm.full[stage]);
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
      for (int i = 0; i < kStages; ++i) {  // drain: no copy in flight at exit
        if (!mbar_wait_bounded(&sm.empty[stage], phase ^ 1u, abort_flag, status)) break;
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    return;
  }

  // consumers: warp w (1..8) owns rows wm*32 .. +32, columns wn*64 .. +64
  const int cw = warp - 1;
  const int wm = cw >> 1, wn = cw & 1;
  const int g = lane >> 2, t = lane & 3;
  double acc[2][8][4];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 8; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mi][ni][q] = 0.0;

  int stage = 0;
  uint32_t phase = 0;
  for (int64_t kb = 0; kb < Kt; ++kb) {
    if (!mbar_wait_bounded(&sm.full[stage], phase, abort_flag, status)) break;
    const double* As = sm.a[stage];
    const double* Bs = sm.b[stage];
#pragma unroll
    for (int kk = 0; kk < BK / 4; ++kk) {
      const int c = kk * 4 + t;
      double a[2][2], b[8];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r0 = wm * 32 + mi * 16 + g;
        a[mi][0] = As[swz(r0, c)];
        a[mi][1] = As[swz(r0 + 8, c)];
      }
#pragma unroll
      for (int ni = 0; ni < 8; ++ni) b[ni] = Bs[swz(wn * 64 + ni * 8 + g, c)];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 8; ++ni) dmma_16x8x4(acc[mi][ni], a[mi][0], a[mi][1], b[ni]);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[stage]);
    if (++stage == kStages) {
      stage = 0;
      phase ^= 1u;
    }
  }

  // epilogue: D fragment (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)
#pragma unroll
  for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t row = tm * BM + wm * 32 + mi * 16 + g + half * 8;
      if (row >= m) continue;
      double* crow = C + row * n;
#pragma unroll
      for (int ni = 0; ni < 8; ++ni) {
        const int64_t col = tn * BN + wn * 64 + ni * 8 + 2 * t;
        if (col < n) crow[col] = acc[mi][ni][half * 2];
        if (col + 1 < n) crow[col + 1] = acc[mi][ni][half * 2 + 1];
      }
    }
  }
}

constexpr size_t kF64SmemBytes = sizeof(F64Smem) + 128;

}  // namespace

cudaError_t launch_f64_pack(const double* A, const double* B, const F64Dims& d, uint8_t* ws,
                            cudaStream_t s) {
  if (d.Kt == 0) return cudaSuccess;
  double* apack = reinterpret_cast<double*>(ws);
  double* bpack = apack + d.Mt * d.Kt * (BM * BK);
  if (d.Mt > 0)
    f64_pack_a_kernel<<<dim3(static_cast<unsigned>(d.Kt), static_cast<unsigned>(d.Mt)), 256, 0,
                        s>>>(A, d.m, d.k, d.Kt, apack);
  if (d.Nt > 0)
    f64_pack_b_kernel<<<dim3(static_cast<unsigned>(d.Kt), static_cast<unsigned>(d.Nt)), 256, 0,
                        s>>>(B, d.k, d.n, d.Kt, bpack);
  return cudaGetLastError();
}

cudaError_t launch_f64_gemm(const uint8_t* ws, double* C, const F64Dims& d, int* status,
                            cudaStream_t s) {
  if (d.Mt == 0 || d.Nt == 0) return cudaSuccess;
  const double* apack = reinterpret_cast<const double*>(ws);
  const double* bpack = apack + d.Mt * d.Kt * (BM * BK);
  cudaError_t e = cudaFuncSetAttribute(f64_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kF64SmemBytes));
  if (e != cudaSuccess) return e;
  f64_gemm_kernel<<<static_cast<unsigned>(d.Mt * d.Nt), kThreads, kF64SmemBytes, s>>>(
      apack, bpack, C, d.m, d.n, d.Mt, d.Nt, d.Kt, status);
  return cudaGetLastError();
}

}  // namespace mxm

// mxm_internal.h -- declarations shared by the translation units of
// libmxm.so (not part of the public C ABI in include/mxm.h).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace mxm {

// Bits of the sticky device status word (OR-ed by kernels).
constexpr int kStatusNonFinite = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusWorkspace = 4;
constexpr int kStatusBounds = 8;

// Every bounded wait inside a kernel gives up after this long.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

// ---------------------------------------------------------------- Ozaki
// Operand tiles of the slice GEMM: 128 rows x 64 bf16 (128 bytes per row),
// 16 KiB, stored pre-swizzled (128-byte swizzle) so one bulk copy moves a
// tile into shared memory in the layout tcgen05.mma reads.
constexpr int kOzTileRows = 128;
constexpr int kOzTileK = 64;
constexpr int kOzTileBytes = kOzTileRows * kOzTileK * 2;
constexpr int kOzMaxSlices = 12;

struct OzakiDims {
  int64_t m, k, n;
  int64_t Mt, Nt, Kt;  // tiles of 128 rows of A, 128 columns of B, 64 of k
  int S, beta;
};

inline OzakiDims ozaki_dims(int64_t m, int64_t k, int64_t n, int S, int beta) {
  OzakiDims d;
  d.m = m; d.k = k; d.n = n;
  d.Mt = (m + kOzTileRows - 1) / kOzTileRows;
  d.Nt = (n + kOzTileRows - 1) / kOzTileRows;
  d.Kt = (k + kOzTileK - 1) / kOzTileK;
  d.S = S; d.beta = beta;
  return d;
}

// Workspace layout of one emulated product (offsets in bytes, 1 KiB aligned).
struct OzakiLayout {
  size_t rowbits, colbits, aslices, bslices, total;
};

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline OzakiLayout ozaki_layout(const OzakiDims& d) {
  OzakiLayout L;
  size_t off = 0;
  L.rowbits = off; off = align_up(off + sizeof(uint64_t) * (size_t)(d.m > 0 ? d.m : 1), 1024);
  L.colbits = off; off = align_up(off + sizeof(uint64_t) * (size_t)(d.n > 0 ? d.n : 1), 1024);
  L.aslices = off; off = align_up(off + (size_t)d.S * d.Mt * d.Kt * kOzTileBytes, 1024);
  L.bslices = off; off = align_up(off + (size_t)d.S * d.Nt * d.Kt * kOzTileBytes, 1024);
  L.total = off;
  return L;
}

// Largest number of K=16 MMAs whose integer products can be summed in an
// FP32 accumulator without rounding: every product is at most (2^beta-1)^2
// in magnitude and 16 of them enter per MMA, so the running sum stays within
// 2^24 (all integers up to 2^24 are exact in FP32).
inline int ozaki_window_mmas(int beta) {
  const long long dmax = (1ll << beta) - 1;
  const long long per_mma = dmax * dmax * 16;
  return static_cast<int>((1ll << 24) / per_mma);
}

cudaError_t launch_ozaki_scale(const double* A, const double* B, const OzakiDims& d,
                               uint64_t* rowbits, uint64_t* colbits, int* status,
                               cudaStream_t s);
cudaError_t launch_ozaki_split(const double* A, const double* B, const OzakiDims& d,
                               const uint64_t* rowbits, const uint64_t* colbits,
                               uint8_t* aslices, uint8_t* bslices, cudaStream_t s);
cudaError_t launch_ozaki_gemm(const uint8_t* aslices, const uint8_t* bslices,
                              const uint64_t* rowbits, const uint64_t* colbits, double* C,
                              const OzakiDims& d, int* status, cudaStream_t s);

// ---------------------------------------------------------------- FP64
constexpr int kF64BM = 128, kF64BN = 128, kF64BK = 16;
constexpr int kF64TileBytes = kF64BM * kF64BK * 8;  // 16 KiB (BM == BN)

struct F64Dims {
  int64_t m, k, n, Mt, Nt, Kt;
};

inline F64Dims f64_dims(int64_t m, int64_t k, int64_t n) {
  F64Dims d;
  d.m = m; d.k = k; d.n = n;
  d.Mt = (m + kF64BM - 1) / kF64BM;
  d.Nt = (n + kF64BN - 1) / kF64BN;
  d.Kt = (k + kF64BK - 1) / kF64BK;
  return d;
}

inline size_t f64_workspace(const F64Dims& d) {
  return align_up((size_t)(d.Mt + d.Nt) * d.Kt * kF64TileBytes, 1024);
}

cudaError_t launch_f64_pack(const double* A, const double* B, const F64Dims& d, uint8_t* ws,
                            cudaStream_t s);
cudaError_t launch_f64_gemm(const uint8_t* ws, double* C, const F64Dims& d, int* status,
                            cudaStream_t s);

cudaError_t launch_zero_fill(double* C, int64_t count, cudaStream_t s);

}  // namespace mxm

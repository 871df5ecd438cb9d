// noalloc.cu -- the FP64-accurate product for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need the product: code running inside a memory-budgeted host
// process whose allocator owns the whole device, real-time loops that must
// not hit the driver's allocator, or plugins that are handed device pointers
// but no allocator.  mxm_f64_emul itself needs scratch for the row / column
// maxima and the digit planes, which the library normally takes from a
// workspace it grows with cudaMalloc.  mxm_f64_emul_noalloc runs the same
// kernels with that scratch taken from a fixed array in the library's own
// device memory instead: it allocates nothing, at the price of a size limit.
//
// The array lives in every GPU that loads the library, until the process
// exits.  Every call shares it, so calls that overlap on the GPU (different
// streams, or several host threads) race; the array keeps the previous
// call's contents, and the launch sequence clears what must start at zero
// (the column maxima, reduced with atomicMax) before using it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "mxm.h"
#include "mxm_internal.h"

namespace mxm {

// Largest scratch one call may use (64 MiB; e.g. m = k = n = 1024 with up to
// 12 slices, or m = k = n = 1280 with 7).
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

int* device_status_word();  // abi.cu

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
uint8_t* g_noalloc_ptr[kMaxDevices] = {};  // device address of the array, per device

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is asked of
// the runtime once per device, with that device current.
mxm_status noalloc_scratch(uint8_t** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MXM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return MXM_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<uint8_t*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return MXM_OK;
}

bool ranges_overlap(const void* a, size_t an, const void* b, size_t bn) {
  if (an == 0 || bn == 0) return false;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  return a0 < b0 + bn && b0 < a0 + an;
}

}  // namespace
}  // namespace mxm

using namespace mxm;

extern "C" mxm_status mxm_f64_emul_noalloc(const double* A, const double* B, double* C,
                                           int64_t m, int64_t k, int64_t n, int slices,
                                           void* stream) {
  NvtxRange nvtx_range("mxm_f64_emul_noalloc");
  if (slices < 1 || slices > kOzMaxSlices) return MXM_ERR_UNSUPPORTED;
  if (m < 0 || k < 0 || n < 0) return MXM_ERR_INVALID_ARG;
  // the same size limits as mxm_f64_emul: beyond them the byte counts below
  // could wrap around in 64 bits
  if (m > (int64_t(1) << 31) || n > (int64_t(1) << 31) || k > (int64_t(1) << 31))
    return MXM_ERR_UNSUPPORTED;
  if (m == 0 || n == 0) return MXM_OK;
  if (C == nullptr || (k > 0 && (A == nullptr || B == nullptr))) return MXM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) |
       reinterpret_cast<uintptr_t>(C)) & 7)
    return MXM_ERR_ALIGNMENT;
  const size_t cb = sizeof(double) * size_t(m) * size_t(n);
  if (ranges_overlap(C, cb, A, sizeof(double) * size_t(m) * size_t(k)) ||
      ranges_overlap(C, cb, B, sizeof(double) * size_t(k) * size_t(n)))
    return MXM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (k == 0) {
    // the empty sum: zeros, no scratch needed
    return launch_zero_fill(C, m * n, s) == cudaSuccess ? MXM_OK : MXM_ERR_CUDA;
  }
  // the plan of mxm_f64_emul when its scratch fits, else the same product
  // without split-k (same bits); refused when neither fits
  const OzakiDims d = ozaki_dims_capped(m, k, n, slices, 7, kNoAllocScratchBytes);
  const OzakiLayout L = ozaki_layout(d);
  if (L.total > kNoAllocScratchBytes) return MXM_ERR_WORKSPACE_TOO_SMALL;

  uint8_t* ws = nullptr;
  mxm_status st = noalloc_scratch(&ws);
  if (st != MXM_OK) return st;
  int* status = device_status_word();
  if (status == nullptr) return MXM_ERR_CUDA;

  uint64_t* rowbits = reinterpret_cast<uint64_t*>(ws + L.rowbits);
  uint64_t* colbits = reinterpret_cast<uint64_t*>(ws + L.colbits);
  // launch_ozaki_scale zeroes the column maxima before reducing into them;
  // the row maxima, every digit-plane byte (padding included), the running
  // sums and the split-k partials are written before they are read.
  cudaError_t e = launch_ozaki_scale(A, B, d, rowbits, colbits, status, s);
  if (e == cudaSuccess)
    e = launch_ozaki_split(A, B, d, rowbits, colbits, ws + L.aslices, ws + L.bslices,
                             status, s);
  if (e == cudaSuccess)
    e = launch_ozaki_gemm(ws + L.aslices, ws + L.bslices, rowbits, colbits, C, d,
                            reinterpret_cast<uint64_t*>(ws + L.sums), status, s);
  return e == cudaSuccess ? MXM_OK : MXM_ERR_CUDA;
}

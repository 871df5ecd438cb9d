// spmv.cu -- the mod2as sparse product y = A x (Sec. 3.2) with A in the
// paper's 3-array CSR form (matvals, indx, rowp).
//
// One group of G lanes (G a power of two from 2 to 32, chosen from the
// average row length so that short rows do not leave most of a warp idle)
// takes one row: the lanes stride over the row's values (consecutive lanes,
// consecutive values: the loads of matvals and indx are contiguous), each
// keeps an FP64 partial sum built with fused multiply-adds, and a shuffle
// tree adds the G partials; the group's first lane writes y_i.  The gather
// x[indx[j]] goes through the read-only path.  The streamed bytes are those
// of matvals and indx (12 per value); on this GPU the FP64 pipe (one fused
// multiply-add per value plus the shuffle tree) and the L1 work of the
// random gathers bound the rate as much as HBM does.
//
// Rows are taken warp by warp (a warp holds 32 / G rows), so every lane of
// a warp runs the same number of loop rounds and the shuffles are always
// full-warp.  A row whose rowp entries, or a value whose column, fall
// outside the arrays is skipped (its y is left unwritten) and sets the
// bounds bit of the device status word: bad structure is reported, never
// read through.
#include <cuda_runtime.h>

#include <cstdint>

#include "mxm.h"
#include "mxm_internal.h"

namespace mxm {

int* device_status_word();  // abi.cu

namespace {

constexpr int kSpmvThreads = 256;

template <int G, int K>
__global__ void __launch_bounds__(kSpmvThreads) csr_spmv_kernel(
    const double* __restrict__ vals, const int32_t* __restrict__ indx,
    const int32_t* __restrict__ rowp, const double* __restrict__ x, double* __restrict__ y,
    int64_t nrows, int64_t ncols, int64_t nnz, int* __restrict__ status) {
  constexpr int kRowsPerWarp = 32 / G;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);    // lane within the row's group
  const int grp = lane / G;          // the warp's row slot
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kSpmvThreads + threadIdx.x) >> 5;
  const int64_t warps = (static_cast<int64_t>(gridDim.x) * kSpmvThreads) >> 5;
  bool bad = false;
  for (int64_t base = warp * kRowsPerWarp; base < nrows; base += warps * kRowsPerWarp) {
    const int64_t row = base + grp;
    int64_t b = 0, e = 0;
    if (row < nrows) {
      b = __ldg(rowp + row);
      e = __ldg(rowp + row + 1);
      if (b < 0 || e < b || e > nnz) {
        bad = true;
        e = b;  // nothing of this row is read
      }
    }
    double t = 0.0;
    // K values per lane per round (positions j0, j0 + G, ...): all value
    // and column loads first, then the gathers, then the fused
    // multiply-adds in storage order, so that 3K loads are in flight
    for (int64_t j0 = b + sub; j0 < e; j0 += G * K) {
      int32_t c[K];
      double v[K], xv[K];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int64_t j = j0 + static_cast<int64_t>(u) * G;
        c[u] = j < e ? __ldg(indx + j) : 0;
        v[u] = j < e ? __ldg(vals + j) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const bool ok = c[u] >= 0 && c[u] < ncols;  // an absent value has c = 0, v = 0
        bad |= !ok;
        xv[u] = ok ? __ldg(x + c[u]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < K; ++u) t = fma(v[u], xv[u], t);
    }
    // tree over the G lanes of each group (full-warp shuffles)
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    const unsigned bad_lanes = __ballot_sync(0xFFFFFFFFu, bad);
    const bool row_bad = ((bad_lanes >> (grp * G)) & static_cast<unsigned>((1ull << G) - 1)) != 0;
    if (row < nrows && sub == 0) {
      if (row_bad)
        atomicOr(status, kStatusBounds);
      else
        y[row] = t;
    }
    bad = false;
  }
}

template <int G, int K>
cudaError_t launch_spmv_g(const double* vals, const int32_t* indx, const int32_t* rowp,
                          const double* x, double* y, int64_t nrows, int64_t ncols, int64_t nnz,
                          int* status, cudaStream_t s) {
  const int64_t warps_needed = (nrows + (32 / G) - 1) / (32 / G);
  int64_t blocks = (warps_needed * 32 + kSpmvThreads - 1) / kSpmvThreads;
  const int64_t cap = static_cast<int64_t>(sm_count()) * (2048 / kSpmvThreads);
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  csr_spmv_kernel<G, K><<<static_cast<unsigned>(blocks), kSpmvThreads, 0, s>>>(
      vals, indx, rowp, x, y, nrows, ncols, nnz, status);
  return cudaGetLastError();
}

}  // namespace

// Lanes per row from the average row length.  FP64 arithmetic is scarce on
// this GPU (about one fused multiply-add per SM sub-partition every two
// clocks), so the choice weighs the log2(G) shuffle-adds a row costs against
// coalescing: about 4-8 values per lane.  A matrix with too few rows to give
// every resident warp of the GPU a row group takes wider groups instead.
int spmv_group(int64_t nrows, int64_t nnz) {
  const double avg = nrows > 0 ? static_cast<double>(nnz) / static_cast<double>(nrows) : 0.0;
  int g = avg <= 6 ? 2 : avg <= 24 ? 4 : avg <= 96 ? 8 : avg <= 384 ? 16 : 32;
  const int64_t warp_slots = static_cast<int64_t>(sm_count()) * (2048 / 32);
  while (g < 32 && nrows * g < 32 * warp_slots) g *= 2;
  return g;
}

cudaError_t launch_spmv(const double* vals, const int32_t* indx, const int32_t* rowp,
                        const double* x, double* y, int64_t nrows, int64_t ncols, int64_t nnz,
                        int* status, cudaStream_t s) {
  switch (spmv_group(nrows, nnz)) {
    case 2: return launch_spmv_g<2, 2>(vals, indx, rowp, x, y, nrows, ncols, nnz, status, s);
    case 4: return launch_spmv_g<4, 2>(vals, indx, rowp, x, y, nrows, ncols, nnz, status, s);
    case 8: return launch_spmv_g<8, 4>(vals, indx, rowp, x, y, nrows, ncols, nnz, status, s);
    case 16: return launch_spmv_g<16, 4>(vals, indx, rowp, x, y, nrows, ncols, nnz, status, s);
    default: return launch_spmv_g<32, 2>(vals, indx, rowp, x, y, nrows, ncols, nnz, status, s);
  }
}

}  // namespace mxm

using namespace mxm;

extern "C" mxm_status mxm_spmv(const double* matvals, const int32_t* indx, const int32_t* rowp,
                               const double* x, double* y, int64_t nrows, int64_t ncols,
                               int64_t nnz, void* stream) {
  NvtxRange nvtx_range("mxm_spmv");
  if (nrows < 0 || ncols < 0 || nnz < 0) return MXM_ERR_INVALID_ARG;
  if (nrows > INT32_MAX || ncols > INT32_MAX || nnz > INT32_MAX) return MXM_ERR_UNSUPPORTED;
  if (nrows == 0) return MXM_OK;
  if (y == nullptr || rowp == nullptr || (nnz > 0 && (matvals == nullptr || indx == nullptr)) ||
      (ncols > 0 && x == nullptr))
    return MXM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(matvals) | reinterpret_cast<uintptr_t>(x) |
       reinterpret_cast<uintptr_t>(y)) & 7 ||
      (reinterpret_cast<uintptr_t>(indx) | reinterpret_cast<uintptr_t>(rowp)) & 3)
    return MXM_ERR_ALIGNMENT;
  int* status = device_status_word();
  if (status == nullptr) return MXM_ERR_CUDA;
  const cudaError_t e = launch_spmv(matvals, indx, rowp, x, y, nrows, ncols, nnz, status,
                                    static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? MXM_OK : MXM_ERR_CUDA;
}

// grouped.cu -- many independent products C_p = A_p.B_p (mod2am, Sec. 3.1)
// of uneven sizes in one launch sequence whose problem table lives on the
// device: nothing is read back to the host, nothing is allocated, so the
// whole call can be captured in a CUDA graph and replayed.
//
// grouped_plan_kernel (one block) turns the table into a plan at the start of
// the caller's workspace: per problem its tile counts and the prefix sums of
// every count (C tiles, operand tiles, rows, columns), and from the totals
// the byte offsets of the data regions.  Every later kernel is persistent
// (a fixed grid walking items with a grid stride) and finds the problem of an
// item by binary search over these prefixes.  A plan that does not fit the
// workspace is marked invalid: the later kernels do nothing and the device
// status reports MXM_ERR_WORKSPACE_TOO_SMALL.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "mxm.h"
#include "mxm_internal.h"

namespace mxm {
namespace {

constexpr int kPlanThreads = 1024;
// C tiles, A tiles, B tiles, rows, columns, A tile-rows, B tile-columns, C tiles of the
// long-k problems, C tiles of the short-k problems
constexpr int kCounts = 9;

struct PlanGeometry {
  int64_t tile_rows;  // rows of A (or columns of B) per tile
  int64_t tile_k;     // k per operand tile
  int64_t short_kt;   // emulated: problems with at most this many k-blocks are "short"
};

__host__ __device__ inline void problem_counts(int64_t m, int64_t k, int64_t n,
                                               const PlanGeometry& g, int64_t (&Mt_Nt_Kt)[3],
                                               int64_t (&c)[kCounts]) {
  int64_t Mt = 0, Nt = 0, Kt = 0;
  if (m > 0 && n > 0 && k >= 0) {
    Mt = (m + g.tile_rows - 1) / g.tile_rows;
    Nt = (n + g.tile_rows - 1) / g.tile_rows;
    Kt = (k + g.tile_k - 1) / g.tile_k;
  }
  Mt_Nt_Kt[0] = Mt;
  Mt_Nt_Kt[1] = Nt;
  Mt_Nt_Kt[2] = Kt;
  const bool live = Mt > 0 && Nt > 0;
  c[0] = Mt * Nt;
  c[1] = Mt * Kt;
  c[2] = Nt * Kt;
  c[3] = live ? m : 0;
  c[4] = live ? n : 0;
  c[5] = live ? Mt : 0;
  c[6] = live ? Nt : 0;
  c[7] = Kt > g.short_kt ? c[0] : 0;
  c[8] = Kt > g.short_kt ? 0 : c[0];
}

// Exclusive prefix sum over the block (1024 threads = 32 warps).
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* warp_sums, int64_t& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t w = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int64_t res = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
  total = warp_sums[31];
  __syncthreads();
  return res;
}

__global__ void __launch_bounds__(kPlanThreads) grouped_plan_kernel(
    const mxm_problem* __restrict__ table, int64_t count, PlanGeometry geo, int planes,
    size_t tile_bytes, int bits, size_t ws_bytes, uint8_t* __restrict__ ws,
    int* __restrict__ status) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t carry[kCounts];
  __shared__ int64_t max_kt;
  __shared__ int bad;
  GroupedHeader* hdr = reinterpret_cast<GroupedHeader*>(ws);
  GroupedProblem* recs = reinterpret_cast<GroupedProblem*>(ws + kGroupedRecordsOff);
  if (threadIdx.x < kCounts) carry[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    max_kt = 0;
    bad = (bits && count > 2147483647) ? 1 : 0;  // the owner map holds int32 problem indices
  }
  __syncthreads();
  for (int64_t base = 0; base < count; base += kPlanThreads) {
    const int64_t i = base + threadIdx.x;
    mxm_problem pr{nullptr, nullptr, nullptr, 0, 0, 0};
    if (i < count) pr = table[i];
    if (i < count && (pr.m < 0 || pr.k < 0 || pr.n < 0)) {
      bad = 1;
      pr.m = pr.k = pr.n = 0;
    }
    int64_t mnk[3], c[kCounts];
    problem_counts(pr.m, pr.k, pr.n, geo, mnk, c);
    if (mnk[2] > 0) atomicMax(reinterpret_cast<unsigned long long*>(&max_kt),
                              static_cast<unsigned long long>(mnk[2]));
    int64_t begin[kCounts];
#pragma unroll
    for (int q = 0; q < kCounts; ++q) {
      int64_t tot = 0;
      begin[q] = carry[q] + block_exclusive_scan(c[q], warp_sums, tot);
      if (threadIdx.x == 0) carry[q] += tot;
      __syncthreads();
    }
    if (i < count) {
      GroupedProblem r;
      r.A = pr.A;
      r.B = pr.B;
      r.C = pr.C;
      r.m = pr.m;
      r.k = pr.k;
      r.n = pr.n;
      r.Mt = mnk[0];
      r.Nt = mnk[1];
      r.Kt = mnk[2];
      r.tile_begin = begin[0];
      r.atile_begin = begin[1];
      r.btile_begin = begin[2];
      r.row_begin = begin[3];
      r.col_begin = begin[4];
      r.trow_begin = begin[5];
      r.tcol_begin = begin[6];
      r.ltile_begin = begin[7];
      r.stile_begin = begin[8];
      recs[i] = r;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    GroupedHeader h;
    h.count = count;
    h.tiles = carry[0];
    h.atiles = carry[1];
    h.btiles = carry[2];
    h.rows = carry[3];
    h.cols = carry[4];
    h.trows = carry[5];
    h.tcols = carry[6];
    h.ltiles = carry[7];
    h.stiles = carry[8];
    h.max_kt = max_kt;
    h.cursor = 0;
    h.cursor_max = 0;
    grouped_offsets(h, planes, tile_bytes, bits != 0);
    h.valid = (h.total <= ws_bytes && !bad) ? 1 : 0;
    if (!h.valid) atomicOr(status, bad ? kStatusBounds : kStatusWorkspace);
    *hdr = h;
  }
}

bool grouped_mode_ok(int mode, int slices) {
  if (mode == MXM_MODE_F64) return true;
  if (mode == MXM_MODE_EMUL_I8 || mode == MXM_MODE_EMUL_BF16)
    return slices >= 1 && slices <= kOzMaxSlices;
  if (mode == MXM_MODE_EMUL_RN8) return slices >= 1 && slices <= kOzMaxSlicesRn8;
  return false;
}

// The plan's short-k boundary (k-blocks of 128): the caller's, or the default.
int64_t plan_short_kt(const mxm_group_plan* plan) {
  return (plan != nullptr && plan->short_kt >= 0) ? plan->short_kt : kGroupedShortKt;
}

bool group_plan_ok(const mxm_group_plan* plan) {
  if (plan == nullptr) return true;
  return plan->short_kt >= -1 && plan->reserved[0] == 0 && plan->reserved[1] == 0 &&
         plan->reserved[2] == 0;
}

void mode_geometry(int mode, int slices, int64_t short_kt, PlanGeometry& g, int& planes,
                   size_t& tile_bytes, int& bits) {
  if (mode == MXM_MODE_F64) {
    // warp units of 32 x 32; operands read in place (no packed copies)
    g = PlanGeometry{kF64GroupedTile, kF64GroupedK, 0};
    planes = 0;
    tile_bytes = 0;
    bits = 0;
  } else {
    g = PlanGeometry{kOzTileRows, kOzTileK, short_kt};
    planes = slices;
    tile_bytes = kOzTileBytes;
    bits = 1;
  }
}

}  // namespace
}  // namespace mxm

using namespace mxm;

extern "C" mxm_status mxm_grouped_workspace_size_plan(int64_t count,
                                                      const mxm_problem* h_problems, int mode,
                                                      int slices, const mxm_group_plan* plan,
                                                      size_t* bytes) {
  if (bytes == nullptr || count < 0 || (count > 0 && h_problems == nullptr))
    return MXM_ERR_INVALID_ARG;
  if (!grouped_mode_ok(mode, slices)) return MXM_ERR_UNSUPPORTED;
  if (!group_plan_ok(plan)) return MXM_ERR_INVALID_ARG;
  PlanGeometry g;
  int planes, bits;
  size_t tile_bytes;
  mode_geometry(mode, slices, plan_short_kt(plan), g, planes, tile_bytes, bits);
  GroupedHeader h{};
  h.count = count;
  int64_t tot[kCounts] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = 0; i < count; ++i) {
    const mxm_problem& p = h_problems[i];
    if (p.m < 0 || p.k < 0 || p.n < 0) return MXM_ERR_INVALID_ARG;
    int64_t mnk[3], c[kCounts];
    problem_counts(p.m, p.k, p.n, g, mnk, c);
    for (int q = 0; q < kCounts; ++q) tot[q] += c[q];
  }
  h.tiles = tot[0];
  h.atiles = tot[1];
  h.btiles = tot[2];
  h.rows = tot[3];
  h.cols = tot[4];
  h.trows = tot[5];
  h.tcols = tot[6];
  h.ltiles = tot[7];
  h.stiles = tot[8];
  grouped_offsets(h, planes, tile_bytes, bits != 0);
  *bytes = h.total;
  return MXM_OK;
}

extern "C" mxm_status mxm_grouped_workspace_size(int64_t count, const mxm_problem* h_problems,
                                                 int mode, int slices, size_t* bytes) {
  return mxm_grouped_workspace_size_plan(count, h_problems, mode, slices, nullptr, bytes);
}

// defined in abi.cu: the current device's status word
namespace mxm {
int* device_status_word();
}

extern "C" mxm_status mxm_grouped_plan(int64_t count, const mxm_problem* d_problems, int mode,
                                       int slices, const mxm_group_plan* plan, void* d_ws,
                                       size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("mxm_grouped");
  if (count < 0 || (count > 0 && d_problems == nullptr)) return MXM_ERR_INVALID_ARG;
  if (!grouped_mode_ok(mode, slices)) return MXM_ERR_UNSUPPORTED;
  if (!group_plan_ok(plan)) return MXM_ERR_INVALID_ARG;
  if (count == 0) return MXM_OK;
  if (d_ws == nullptr) return MXM_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_ws) & 255) return MXM_ERR_ALIGNMENT;
  if (ws_bytes < grouped_data_begin(count)) return MXM_ERR_WORKSPACE_TOO_SMALL;
  int* status = device_status_word();
  if (status == nullptr) return MXM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PlanGeometry g;
  int planes, bits;
  size_t tile_bytes;
  mode_geometry(mode, slices, plan_short_kt(plan), g, planes, tile_bytes, bits);
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  grouped_plan_kernel<<<1, kPlanThreads, 0, s>>>(d_problems, count, g, planes, tile_bytes, bits,
                                                 ws_bytes, ws, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return MXM_ERR_CUDA;
  if (mode == MXM_MODE_F64)
    e = launch_f64_grouped(ws, status, s);
  else
    e = launch_ozaki_grouped(ws, slices, mode == MXM_MODE_EMUL_I8 ? 7 : 8, plan_short_kt(plan),
                             status, s, mode == MXM_MODE_EMUL_RN8);
  return e == cudaSuccess ? MXM_OK : MXM_ERR_CUDA;
}

extern "C" mxm_status mxm_grouped(int64_t count, const mxm_problem* d_problems, int mode,
                                  int slices, void* d_ws, size_t ws_bytes, void* stream) {
  return mxm_grouped_plan(count, d_problems, mode, slices, nullptr, d_ws, ws_bytes, stream);
}

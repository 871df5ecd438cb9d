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

// Tile (tm, tk) of A (m x k): element (r, c) = A[tm*128 + r][tk*16 + c].
__device__ __forceinline__ void pack_a_tile(const double* __restrict__ A, int64_t m, int64_t k,
                                            int64_t tm, int64_t tk, double* __restrict__ tile) {
  for (int p = threadIdx.x; p < BM * BK; p += blockDim.x) {
    const int r = p / BK, c = p % BK;
    const int64_t row = tm * BM + r, col = tk * BK + c;
    tile[swz(r, c)] = (row < m && col < k) ? __ldg(A + row * k + col) : 0.0;
  }
}

// Tile (tn, tk) of B^T: element (r, c) = B[tk*16 + c][tn*128 + r], staged
// through shared memory so that both the reads and the writes are coalesced.
__device__ __forceinline__ void pack_b_tile(const double* __restrict__ B, int64_t k, int64_t n,
                                            int64_t tn, int64_t tk, double* __restrict__ tile,
                                            double (*t)[BN + 1]) {
  for (int p = threadIdx.x; p < BK * BN; p += blockDim.x) {
    const int c = p / BN, r = p % BN;
    const int64_t kr = tk * BK + c, col = tn * BN + r;
    t[c][r] = (kr < k && col < n) ? __ldg(B + kr * n + col) : 0.0;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < BN * BK; p += blockDim.x) {
    const int r = p / BK, c = p % BK;
    tile[swz(r, c)] = t[c][r];
  }
  __syncthreads();
}

__global__ void f64_pack_a_kernel(const double* __restrict__ A, int64_t m, int64_t k, int64_t Kt,
                                  double* __restrict__ out) {
  const int64_t tk = blockIdx.x, tm = blockIdx.y;
  pack_a_tile(A, m, k, tm, tk, out + (tm * Kt + tk) * (BM * BK));
}

__global__ void f64_pack_b_kernel(const double* __restrict__ B, int64_t k, int64_t n, int64_t Kt,
                                  double* __restrict__ out) {
  __shared__ double t[BK][BN + 1];
  const int64_t tk = blockIdx.x, tn = blockIdx.y;
  pack_b_tile(B, k, n, tn, tk, out + (tn * Kt + tk) * (BN * BK), t);
}

// Every operand tile of a grouped call (A tiles, then B tiles).
__global__ void f64_grouped_pack_kernel(uint8_t* __restrict__ ws) {
  __shared__ double t[BK][BN + 1];
  const GroupedHeader* hdr = reinterpret_cast<const GroupedHeader*>(ws);
  if (!hdr->valid) return;
  const GroupedProblem* recs = reinterpret_cast<const GroupedProblem*>(ws + kGroupedRecordsOff);
  double* apack = reinterpret_cast<double*>(ws + hdr->off_a);
  double* bpack = reinterpret_cast<double*>(ws + hdr->off_b);
  const int64_t na = hdr->atiles, nb = hdr->btiles;
  for (int64_t i = blockIdx.x; i < na + nb; i += gridDim.x) {
    if (i < na) {
      const GroupedProblem& p = recs[grouped_find(recs, hdr->count, i, &GroupedProblem::atile_begin)];
      const int64_t local = i - p.atile_begin;
      pack_a_tile(p.A, p.m, p.k, local / p.Kt, local % p.Kt, apack + i * (BM * BK));
    } else {
      const int64_t j = i - na;
      const GroupedProblem& p = recs[grouped_find(recs, hdr->count, j, &GroupedProblem::btile_begin)];
      const int64_t local = j - p.btile_begin;
      pack_b_tile(p.B, p.k, p.n, local / p.Kt, local % p.Kt, bpack + j * (BN * BK), t);
    }
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

__device__ __forceinline__ void tile_coords(int64_t tile, int64_t Mt, int64_t Nt, int64_t G,
                                            int64_t& tm, int64_t& tn) {
  // groups of G tile-rows, column-major inside a group (L2 reuse of the
  // operand tiles of the CTAs working at the same time)
  const int64_t per_group = G * Nt;
  const int64_t grp = tile / per_group;
  const int64_t first = grp * G;
  const int64_t gsz = (Mt - first) < G ? (Mt - first) : G;
  const int64_t in = tile - grp * per_group;
  tm = first + in % gsz;
  tn = in / gsz;
}

struct F64Tile {
  const double* a;   // packed A tile-row, first k-block of this unit
  const double* b;   // packed B^T tile-row, first k-block of this unit
  int64_t Kt;        // k-blocks of this unit
  double* C;         // output (C, or a partial tile under split-k)
  int64_t m, n, ldc, row0, col0;
};

// Work unit t: C tile t / splits, k range t % splits (consecutive CTAs take
// the k ranges of one tile).  Without split-k the unit writes C with edge
// masks; with it, a full 128 x 128 partial tile (the packed operands are
// zero-padded, so the padding rows and columns are zeros).
struct F64Single {
  const double* apack;
  const double* bpack;
  double* C;
  double* partials;
  int64_t m, n, Mt, Nt, Kt, splits;
  int64_t raster;
  __device__ __forceinline__ int64_t count() const { return Mt * Nt * splits; }
  __device__ __forceinline__ F64Tile tile(int64_t t) const {
    const int64_t tile = t / splits, sp = t - tile * splits;
    int64_t tm, tn;
    tile_coords(tile, Mt, Nt, raster, tm, tn);
    const int64_t kb0 = Kt * sp / splits, kb1 = Kt * (sp + 1) / splits;
    const double* a = apack + (tm * Kt + kb0) * (BM * BK);
    const double* b = bpack + (tn * Kt + kb0) * (BN * BK);
    if (splits == 1) return F64Tile{a, b, kb1 - kb0, C, m, n, n, tm * BM, tn * BN};
    double* p = partials + ((sp * Mt + tm) * Nt + tn) * (BM * BN);
    return F64Tile{a, b, kb1 - kb0, p, BM, BN, BN, 0, 0};
  }
};

// C[row][col] = sum over splits s (in order) of the partial tiles.
__global__ void __launch_bounds__(256) f64_splitk_reduce_kernel(const double* __restrict__ P,
                                                                double* __restrict__ C,
                                                                int64_t m, int64_t n, int64_t Mt,
                                                                int64_t Nt, int64_t splits) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= m * n) return;
  const int64_t row = idx / n, col = idx - (idx / n) * n;
  const int64_t off = ((row / BM) * Nt + col / BN) * (BM * BN) + (row % BM) * BN + col % BN;
  const int64_t stride = Mt * Nt * (BM * BN);
  double acc = 0.0;
  for (int64_t s = 0; s < splits; ++s) acc += __ldcs(P + s * stride + off);
  C[idx] = acc;
}

struct F64Grouped {
  const uint8_t* ws;
  __device__ __forceinline__ int64_t count() const {
    const GroupedHeader* hdr = reinterpret_cast<const GroupedHeader*>(ws);
    return hdr->valid ? hdr->tiles : 0;
  }
  __device__ __forceinline__ F64Tile tile(int64_t t) const {
    const GroupedHeader* hdr = reinterpret_cast<const GroupedHeader*>(ws);
    const GroupedProblem* recs = reinterpret_cast<const GroupedProblem*>(ws + kGroupedRecordsOff);
    const GroupedProblem& p = recs[grouped_find(recs, hdr->count, t, &GroupedProblem::tile_begin)];
    const int64_t local = t - p.tile_begin;
    const int64_t tm = local / p.Nt, tn = local - (local / p.Nt) * p.Nt;
    const double* apack = reinterpret_cast<const double*>(ws + hdr->off_a);
    const double* bpack = reinterpret_cast<const double*>(ws + hdr->off_b);
    return F64Tile{apack + (p.atile_begin + tm * p.Kt) * (BM * BK),
                   bpack + (p.btile_begin + tn * p.Kt) * (BN * BK), p.Kt, p.C, p.m, p.n, p.n,
                   tm * BM, tn * BN};
  }
};

// Persistent: every CTA walks tiles blockIdx.x, +gridDim.x, ...; the producer
// and the consumers walk the same sequence and keep the stage ring running
// across tiles.
template <typename Tiles>
__global__ void __launch_bounds__(kThreads, 1)
    f64_gemm_kernel(const Tiles tiles, int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  F64Smem& sm = *reinterpret_cast<F64Smem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

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
  const int64_t ntiles = tiles.count();

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const F64Tile j = tiles.tile(t);
        for (int64_t kb = 0; kb < j.Kt; ++kb) {
          if (!mbar_wait_bounded(&sm.empty[stage], phase ^ 1u, abort_flag, status)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&sm.full[stage], 2 * kF64TileBytes);
          bulk_g2s(sm.a[stage], j.a + kb * (BM * BK), kF64TileBytes, &sm.full[stage]);
          bulk_g2s(sm.b[stage], j.b + kb * (BN * BK), kF64TileBytes, &sm.full[stage]);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
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
  const int g = lane >> 2, t4 = lane & 3;
  int stage = 0;
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const F64Tile j = tiles.tile(t);
    double acc[2][8][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 8; ++ni)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[mi][ni][q] = 0.0;

    for (int64_t kb = 0; kb < j.Kt; ++kb) {
      if (!mbar_wait_bounded(&sm.full[stage], phase, abort_flag, status)) {
        ok = false;
        break;
      }
      const double* As = sm.a[stage];
      const double* Bs = sm.b[stage];
#pragma unroll
      for (int kk = 0; kk < BK / 4; ++kk) {
        const int c = kk * 4 + t4;
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
    if (!ok) break;

    // epilogue: D fragment (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int64_t row = j.row0 + wm * 32 + mi * 16 + g + half * 8;
        if (row >= j.m) continue;
        double* crow = j.C + row * j.ldc;
#pragma unroll
        for (int ni = 0; ni < 8; ++ni) {
          const int64_t col = j.col0 + wn * 64 + ni * 8 + 2 * t4;
          if (col < j.n) crow[col] = acc[mi][ni][half * 2];
          if (col + 1 < j.n) crow[col + 1] = acc[mi][ni][half * 2 + 1];
        }
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

template <typename Tiles>
static cudaError_t launch_f64_gemm_t(const Tiles& tiles, int64_t grid, int* status,
                                     cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  auto kern = f64_gemm_kernel<Tiles>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kF64SmemBytes));
  if (e != cudaSuccess) return e;
  kern<<<static_cast<unsigned>(grid), kThreads, kF64SmemBytes, s>>>(tiles, status);
  return cudaGetLastError();
}

cudaError_t launch_f64_gemm(uint8_t* ws, double* C, const F64Dims& d, int* status,
                            cudaStream_t s) {
  if (d.Mt == 0 || d.Nt == 0) return cudaSuccess;
  const double* apack = reinterpret_cast<const double*>(ws);
  const double* bpack = apack + d.Mt * d.Kt * (BM * BK);
  double* partials = reinterpret_cast<double*>(ws + f64_partials_offset(d));
  F64Single tiles{apack, bpack, C, partials, d.m, d.n, d.Mt, d.Nt, d.Kt, d.splits,
                  d.raster > 0 ? d.raster : kDefaultRaster};
  const int64_t count = d.Mt * d.Nt * d.splits;
  const int64_t grid = count < sm_count() ? count : sm_count();
  cudaError_t e = launch_f64_gemm_t(tiles, grid, status, s);
  if (e != cudaSuccess || d.splits == 1) return e;
  const int64_t total = d.m * d.n;
  f64_splitk_reduce_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(
      partials, C, d.m, d.n, d.Mt, d.Nt, d.splits);
  return cudaGetLastError();
}

cudaError_t launch_f64_grouped(uint8_t* ws, int* status, cudaStream_t s) {
  const int sms = sm_count();
  f64_grouped_pack_kernel<<<sms * 8, 256, 0, s>>>(ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_f64_gemm_t(F64Grouped{ws}, sms, status, s);
}

}  // namespace mxm

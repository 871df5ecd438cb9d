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
#include <type_traits>

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
#ifdef MXM_DEBUG_BOUNDS
  // the packed operand tiles (bounds checks of the debug build)
  __device__ __forceinline__ const double* a_begin() const { return apack; }
  __device__ __forceinline__ const double* a_end() const { return apack + Mt * Kt * (BM * BK); }
  __device__ __forceinline__ const double* b_begin() const { return bpack; }
  __device__ __forceinline__ const double* b_end() const { return bpack + Nt * Kt * (BN * BK); }
#endif
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

// ---------------------------------------------------------------- grouped
// Many small products of uneven sizes: the work is cut into 32 x 32 pieces
// of the C matrices (the plan's tiles), one warp each, handed out by an
// atomic cursor in the plan header (dynamic scheduling: pieces of long-k
// problems cost more).  The FP64 pipe of this GPU (~3.5 flops per clock per
// SM) is the limit, so the operands are read straight from the caller's
// arrays (L1/L2 serve the reuse) with no packed copies, and the pieces are
// small enough that padding wastes little: every product is cut at 32 rows,
// 32 columns and 4 k, and the DMMA blocks of an edge piece that lie wholly
// past the last row (16) or column (8) are not issued.  Each warp holds its
// 32 x 32 piece as 2 x 4 DMMA m16n8 accumulators and reads the fragments of
// the next k step while the current ones multiply.
constexpr int kGroupedF64Threads = 256;

__device__ __forceinline__ void load_frags(const double* __restrict__ A,
                                           const double* __restrict__ B, int64_t k, int64_t n,
                                           const int64_t (&arow)[4], const int64_t (&bcol)[4],
                                           uint32_t rmask, uint32_t cmask, int64_t kk,
                                           double (&a)[4], double (&b)[4]) {
  const bool kv = kk < k;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    a[i] = (kv && ((rmask >> i) & 1u)) ? __ldg(A + arow[i] * k + kk) : 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    b[i] = (kv && ((cmask >> i) & 1u)) ? __ldg(B + kk * n + bcol[i]) : 0.0;
}

__global__ void __launch_bounds__(kGroupedF64Threads, 2)
    f64_grouped_kernel(uint8_t* __restrict__ ws, int* __restrict__ status) {
  GroupedHeader* hdr = reinterpret_cast<GroupedHeader*>(ws);
  if (!hdr->valid) return;
  const GroupedProblem* recs = reinterpret_cast<const GroupedProblem*>(ws + kGroupedRecordsOff);
  unsigned long long* cursor = reinterpret_cast<unsigned long long*>(&hdr->cursor);
  const int64_t total = hdr->tiles;
  const int64_t count = hdr->count;
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t4 = lane & 3;
  constexpr int T = kF64GroupedTile;
  for (;;) {
    int64_t unit = 0;
    if (lane == 0) unit = static_cast<int64_t>(atomicAdd(cursor, 1ull));
    unit = __shfl_sync(0xFFFFFFFFu, unit, 0);
    if (unit >= total) break;
    const GroupedProblem& r = recs[grouped_find(recs, count, unit, &GroupedProblem::tile_begin)];
    const int64_t local = unit - r.tile_begin;
    const int64_t tm = local / r.Nt, tn = local - (local / r.Nt) * r.Nt;
    const int64_t row0 = tm * T, col0 = tn * T;
    MXM_BOUNDS(row0 < r.m && col0 < r.n && local < r.Mt * r.Nt, status);
    const double* A = r.A;
    const double* B = r.B;
    const int64_t m = r.m, k = r.k, n = r.n;
    // this lane's A rows (mi = 0, 1; halves g, g + 8) and B columns (ni = 0..3)
    int64_t arow[4], bcol[4];
    uint32_t rmask = 0, cmask = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      arow[i] = row0 + (i >> 1) * 16 + (i & 1) * 8 + g;
      if (arow[i] < m) rmask |= 1u << i;
      bcol[i] = col0 + i * 8 + g;
      if (bcol[i] < n) cmask |= 1u << i;
    }
    double acc[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[mi][ni][q] = 0.0;
    // the m16 / n8 blocks holding any row / column of C (warp-uniform)
    const bool mlive1 = row0 + 16 < m;
    const int nlive = static_cast<int>((n - col0 + 7) / 8 < 4 ? (n - col0 + 7) / 8 : 4);
    double a[4], b[4], an[4], bn[4];
    load_frags(A, B, k, n, arow, bcol, rmask, cmask, t4, a, b);
    for (int64_t k0 = 0; k0 < k; k0 += kF64GroupedK) {
      load_frags(A, B, k, n, arow, bcol, rmask, cmask, k0 + kF64GroupedK + t4, an, bn);
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
          if ((mi == 0 || mlive1) && ni < nlive)
            dmma_16x8x4(acc[mi][ni], a[2 * mi], a[2 * mi + 1], b[ni]);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = an[i];
        b[i] = bn[i];
      }
    }
    // D fragment of m16n8: (g, 2 t4), (g, 2 t4 + 1), (g + 8, 2 t4), (g + 8, 2 t4 + 1)
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t row = row0 + mi * 16 + h * 8 + g;
        if (row >= m) continue;
        double* crow = r.C + row * n;
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
          const int64_t col = col0 + ni * 8 + 2 * t4;
          if (col < n) crow[col] = acc[mi][ni][2 * h];
          if (col + 1 < n) crow[col + 1] = acc[mi][ni][2 * h + 1];
        }
      }
    }
  }
}

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
          MXM_BOUNDS(in_range(j.a + kb * (BM * BK), kF64TileBytes, tiles.a_begin(),
                              tiles.a_end()) &&
                         in_range(j.b + kb * (BN * BK), kF64TileBytes, tiles.b_begin(),
                                  tiles.b_end()),
                     status);
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
    // the m16 / n8 blocks of this warp's 32 x 64 region that hold any row /
    // column of C (warp-uniform); the others are not issued (edge tiles)
    const int64_t rows_left = j.m - (j.row0 + wm * 32);
    const int64_t cols_left = j.n - (j.col0 + wn * 64);
    const int mlive = rows_left <= 0 ? 0 : (rows_left > 16 ? 2 : 1);
    const int nlive =
        cols_left <= 0 ? 0 : (cols_left >= 64 ? 8 : static_cast<int>((cols_left + 7) / 8));
    double acc[2][8][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 8; ++ni)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[mi][ni][q] = 0.0;

    // kEdge: the predicated form for a region only partly inside C; whole
    // regions keep the plain loop
    auto kloop = [&](auto edge) {
      constexpr bool kEdge = decltype(edge)::value;
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
            for (int ni = 0; ni < 8; ++ni)
              if (!kEdge || (mi < mlive && ni < nlive))
                dmma_16x8x4(acc[mi][ni], a[mi][0], a[mi][1], b[ni]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.empty[stage]);
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    };
    if (mlive == 2 && nlive == 8)
      kloop(std::false_type{});
    else
      kloop(std::true_type{});
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
  // two resident CTAs of 8 warps per SM, every warp pulling pieces until the
  // cursor passes the last one
  f64_grouped_kernel<<<static_cast<unsigned>(2 * sm_count()), kGroupedF64Threads, 0, s>>>(ws,
                                                                                          status);
  return cudaGetLastError();
}

}  // namespace mxm

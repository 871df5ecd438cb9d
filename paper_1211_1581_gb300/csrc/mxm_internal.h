// mxm_internal.h -- declarations shared by the translation units of
// libmxm.so (not part of the public C ABI in include/mxm.h).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace mxm {

// A named NVTX range around one ABI call (scope-bound), so that a profiler's
// timeline shows which call launched which kernels.  Without a profiler
// attached NVTX calls return at once.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Bits of the sticky device status word (OR-ed by kernels).
constexpr int kStatusNonFinite = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusWorkspace = 4;
constexpr int kStatusBounds = 8;
constexpr int kStatusBreakdown = 16;

// Every bounded wait inside a kernel gives up after this long.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

// Split-k for products with fewer C tiles than SMs: the k-blocks of every
// tile are cut into `splits` contiguous ranges, each computed by its own
// CTA into a partial tile; a second kernel adds the partials in split order
// (a fixed order: the result does not depend on timing).  The number of
// work units aimed at is a constant (two per SM of a 152-SM GB300), not the
// device's SM count, so that a product's rounding does not depend on the
// device it runs on; every range keeps at least `min_blocks` k-blocks.
constexpr int64_t kSplitKUnits = 304;

inline int64_t splitk_count(int64_t tiles, int64_t Kt, int64_t min_blocks) {
  if (tiles <= 0 || tiles >= kSplitKUnits / 2) return 1;
  int64_t s = kSplitKUnits / tiles;
  const int64_t cap = Kt / min_blocks;
  if (s > cap) s = cap;
  return s > 1 ? s : 1;
}

// ---------------------------------------------------------------- Ozaki
// Operand tiles of the slice GEMM: 128 rows x 128 bf16, 32 KiB, stored
// pre-swizzled so that one bulk copy moves a tile into shared memory in the
// layout tcgen05.mma reads: two 128-byte-swizzle atoms along k (k 0..63 and
// 64..127, 16 KiB each), each with rows of 128 bytes in which the 16-byte
// chunk c of row r sits at chunk position c ^ (r % 8).  (Bulk copies of
// 32 KiB stream about twice as fast per SM as copies of 16 KiB.)
constexpr int kOzTileRows = 128;
constexpr int kOzTileK = 128;
constexpr int kOzAtomK = 64;
constexpr int kOzAtomBytes = kOzTileRows * kOzAtomK * 2;
constexpr int kOzTileBytes = kOzTileRows * kOzTileK * 2;
constexpr int kOzChunksPerRow = kOzTileK / 8;

// Byte offset of 16-byte chunk c (k = 8c .. 8c+7) of row r inside a tile.
__host__ __device__ inline int oz_chunk_offset(int r, int c) {
  return (c >> 3) * kOzAtomBytes + r * 128 + (((c & 7) ^ (r & 7)) << 4);
}
constexpr int kOzMaxSlices = 12;

// B tiles for the CTA-pair product (cta_group::2, M = 256): the tile's rows
// (columns of B) in two halves of 64, each half contiguous (16 KiB: its two
// atoms along k of 64 rows x 128 bytes, 8 KiB each), so that each CTA of a
// pair fetches its half with one bulk copy.  Same swizzle: chunk c of row r
// at chunk position c ^ (r % 8).
__host__ __device__ inline int oz_chunk_offset_halves(int r, int c) {
  return (r >> 6) * (kOzTileBytes / 2) + (c >> 3) * (kOzAtomBytes / 2) + (r & 63) * 128 +
         (((c & 7) ^ (r & 7)) << 4);
}

// The 4-bit-digit engine: digits |d| <= 15 carried in FP8 E4M3 (every
// integer up to 16 is exact there) through tcgen05 kind::f8f6f4.  A tile is
// 128 rows x 128 k of one byte: a single 128-byte-swizzle atom of 16 KiB, the
// 16-byte chunk c (k = 16c .. 16c+15) of row r at chunk position c ^ (r % 8).
constexpr int kOzTileBytesE4m3 = kOzTileRows * kOzTileK;
constexpr int kOzMaxSlicesE4m3 = 16;
constexpr int kOzMaxSlicesRn8 = 7;
__host__ __device__ inline int oz_chunk_offset_e4m3(int r, int c) {
  return r * 128 + ((c ^ (r & 7)) << 4);
}

struct OzakiDims {
  int64_t m, k, n;
  int64_t Mt, Nt, Kt;  // tiles of 128 rows of A, 128 columns of B, 128 of k
  int S, beta;
  int64_t splits;      // k ranges per C tile (1: no split-k)
  int fp8;             // 1: digits carried in E4M3 (beta = 4), 0: in bf16
  int rn;              // 1: balanced 8-bit digits, the value rounded once to
                       //    nearest (beta = 8, scale exponent + 1, |d| <= 128)
  int pair;            // 1: the slice GEMM runs on CTA pairs (cta_group::2) and
                       //    the B digit tiles are written in the halves layout
  int raster;          // tile-rows (pair-rows on CTA pairs) per group of the
                       //    persistent walk over C tiles
  int kb_alt;          // 1: alternate the k-block direction from one diagonal
                       //    (pair) to the next
};

// Default walk: groups of 8 tile-rows (4 pair-rows on CTA pairs); the
// emulated modes alternate the k-block direction between diagonal pairs.
constexpr int kDefaultRaster = 8;
constexpr int kPairRaster = 4;

inline OzakiDims ozaki_dims(int64_t m, int64_t k, int64_t n, int S, int beta, bool rn = false) {
  OzakiDims d;
  d.m = m; d.k = k; d.n = n;
  d.Mt = (m + kOzTileRows - 1) / kOzTileRows;
  d.Nt = (n + kOzTileRows - 1) / kOzTileRows;
  d.Kt = (k + kOzTileK - 1) / kOzTileK;
  d.S = S; d.beta = beta;
  d.splits = 1;
  d.fp8 = 0;
  d.rn = rn ? 1 : 0;
  d.pair = d.Mt >= 2 ? 1 : 0;
  d.raster = kDefaultRaster;
  d.kb_alt = 0;
  return d;
}

// Largest digit magnitude of a split.
inline int ozaki_dmax(const OzakiDims& d) { return d.rn ? 128 : (1 << d.beta) - 1; }

// The 4-bit-digit E4M3 engine (paired kernel only: no split-k).
inline OzakiDims ozaki_dims_fp8(int64_t m, int64_t k, int64_t n, int S) {
  OzakiDims d = ozaki_dims(m, k, n, S, 4);
  d.fp8 = 1;
  d.pair = 0;
  return d;
}

inline size_t ozaki_tile_bytes(const OzakiDims& d) {
  return d.fp8 ? kOzTileBytesE4m3 : kOzTileBytes;
}

// The same with split-k where the product has fewer C tiles than SMs (each
// k range at least 4 k-blocks of 128): the per-range digit-pair sums D_g
// are exact integers, added exactly, so the result is bit-identical to the
// unsplit product.
inline OzakiDims ozaki_dims_splitk(int64_t m, int64_t k, int64_t n, int S, int beta,
                                   bool rn = false) {
  OzakiDims d = ozaki_dims(m, k, n, S, beta, rn);
  d.splits = splitk_count(d.Mt * d.Nt, d.Kt, 4);
  if (d.splits > 1) d.pair = 0;
  return d;
}

// Whether the B digit tiles are written in the halves layout above, and
// whether the paired slice GEMM runs on CTA pairs (cta_group::2, 256-row C
// tiles): bf16 digits without split-k, chosen where the dims are made (two
// or more tile-rows of A; products that share B planes share the choice,
// a single tile-row then leaving the second CTA of its pairs idle).
inline bool ozaki_b_halves(const OzakiDims& d) { return d.pair != 0 && !d.fp8; }
inline bool ozaki_cta2(const OzakiDims& d) {
  return ozaki_b_halves(d) && d.splits <= 1 && d.Mt >= 1;
}

// Workspace layout of one emulated product (offsets in bytes, 1 KiB aligned).
struct OzakiLayout {
  size_t rowbits, colbits, aslices, bslices, sums, total;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Whether the per-diagonal integer sums of a tile with Kt k-blocks fit in
// int32, the condition of the paired slice GEMM without spills: every digit
// product is at most (2^beta - 1)^2 and a diagonal has at most S of them
// per k.
__host__ __device__ inline bool ozaki_narrow(int S, int beta, int64_t Kt) {
  const double dmax = static_cast<double>((1 << beta) - 1);
  return static_cast<double>(S) * dmax * dmax * kOzTileK * static_cast<double>(Kt) <
         2147483647.0;
}

// The same for the dims of a product (the digit bound of its split).
inline bool ozaki_narrow(const OzakiDims& d) {
  const double dmax = static_cast<double>(d.rn ? 128 : (1 << d.beta) - 1);
  return static_cast<double>(d.S) * dmax * dmax * kOzTileK * static_cast<double>(d.Kt) <
         2147483647.0;
}

// CTAs of the paired slice GEMM that keep a spill area (the grid is capped
// there when spills are on).
constexpr int64_t kOzSpillCtas = 256;

// Bytes of the running sums of a product (per C tile 128 x 128 x 8 bytes),
// or under split-k the partial sums D_g of every k range.
inline size_t ozaki_sums_bytes(const OzakiDims& d) {
  const size_t tile8 = (size_t)kOzTileRows * kOzTileRows * 8;
  return d.splits > 1 ? (size_t)d.splits * d.Mt * d.Nt * d.S * tile8
                      : (size_t)d.Mt * d.Nt * tile8;
}

// Spill area of the paired slice GEMM when a diagonal's integer sum can
// outgrow int32 over all of k (long k, 8-bit digits): per CTA the int64
// partial sums of the two diagonals in work, 2 x 128 x 128 x 8 bytes.
inline size_t ozaki_spill_bytes(const OzakiDims& d) {
  if (d.fp8 || d.splits > 1 || ozaki_narrow(d)) return 0;
  const int64_t ctas = d.Mt * d.Nt < kOzSpillCtas ? d.Mt * d.Nt : kOzSpillCtas;
  return (size_t)ctas * 2 * kOzTileRows * kOzTileRows * 8;
}

inline OzakiLayout ozaki_layout(const OzakiDims& d) {
  OzakiLayout L;
  size_t off = 0;
  L.rowbits = off; off = align_up(off + sizeof(uint64_t) * (size_t)(d.m > 0 ? d.m : 1), 1024);
  L.colbits = off; off = align_up(off + sizeof(uint64_t) * (size_t)(d.n > 0 ? d.n : 1), 1024);
  L.aslices = off; off = align_up(off + (size_t)d.S * d.Mt * d.Kt * ozaki_tile_bytes(d), 1024);
  L.bslices = off; off = align_up(off + (size_t)d.S * d.Nt * d.Kt * ozaki_tile_bytes(d), 1024);
  // running sums of the recombination between diagonal pairs: per C tile
  // 128 x 128 x 8 bytes, column-major inside the tile (so that a warp, which
  // owns 32 consecutive rows, touches 256 contiguous bytes per column).
  // Under split-k the region holds instead the int64 partial sums D_g of
  // every k range: [splits][Mt x Nt tiles][S diagonals] x 128 x 128,
  // column-major inside the tile.  The spill area (if any) follows the sums.
  L.sums = off; off = align_up(off + ozaki_sums_bytes(d), 1024);
  off = align_up(off + ozaki_spill_bytes(d), 1024);
  L.total = off;
  return L;
}


// The plan of ozaki_dims_splitk when its workspace fits `cap` bytes, else
// the same product without split-k (the split-k partials are exact integers
// added exactly, so both plans give the same bits).  The caller checks
// whether the returned plan fits.
inline OzakiDims ozaki_dims_capped(int64_t m, int64_t k, int64_t n, int S, int beta,
                                   size_t cap) {
  OzakiDims d = ozaki_dims_splitk(m, k, n, S, beta);
  if (d.splits > 1 && ozaki_layout(d).total > cap) d = ozaki_dims(m, k, n, S, beta);
  return d;
}

// Largest number of K=16 MMAs whose integer products can be summed in an
// FP32 accumulator without rounding: every product is at most (2^beta-1)^2
// in magnitude and 16 of them enter per MMA, so the running sum stays within
// 2^24 (all integers up to 2^24 are exact in FP32).
inline int ozaki_window_mmas(int beta, bool rn = false) {
  const long long dmax = rn ? 128 : (1ll << beta) - 1;
  const long long per_mma = dmax * dmax * 16;
  return static_cast<int>((1ll << 24) / per_mma);
}

// The same bound in whole k-blocks (kOzTileK / 16 MMAs each), as the kernel
// counts.
inline int ozaki_window_stages(int beta, bool rn = false) {
  return ozaki_window_mmas(beta, rn) / (kOzTileK / 16);
}

cudaError_t launch_ozaki_scale(const double* A, const double* B, const OzakiDims& d,
                               uint64_t* rowbits, uint64_t* colbits, int* status,
                               cudaStream_t s);
// Splits A and B into digit planes.  For bf16 digits with k up to 24576 the
// row maxima of A are found here too (one pass over A: launch_ozaki_scale then
// does B only), so rowbits is written and status takes a non-finite A.
cudaError_t launch_ozaki_split(const double* A, const double* B, const OzakiDims& d,
                               uint64_t* rowbits, const uint64_t* colbits,
                               uint8_t* aslices, uint8_t* bslices, int* status, cudaStream_t s);
cudaError_t launch_ozaki_gemm(const uint8_t* aslices, const uint8_t* bslices,
                              const uint64_t* rowbits, const uint64_t* colbits, double* C,
                              const OzakiDims& d, uint64_t* sums, int* status, cudaStream_t s);

// ---------------------------------------------------------------- FP64
constexpr int kF64BM = 128, kF64BN = 128, kF64BK = 16;
constexpr int kF64TileBytes = kF64BM * kF64BK * 8;  // 16 KiB (BM == BN)

struct F64Dims {
  int64_t m, k, n, Mt, Nt, Kt;
  int64_t splits;  // k ranges per C tile (1: no split)
  int raster;      // tile-rows per group of the persistent walk over C tiles
};

inline F64Dims f64_dims(int64_t m, int64_t k, int64_t n) {
  F64Dims d;
  d.m = m; d.k = k; d.n = n;
  d.Mt = (m + kF64BM - 1) / kF64BM;
  d.Nt = (n + kF64BN - 1) / kF64BN;
  d.Kt = (k + kF64BK - 1) / kF64BK;
  d.splits = splitk_count(d.Mt * d.Nt, d.Kt, 8);
  d.raster = kDefaultRaster;
  return d;
}

// Packed operand tiles, then (split-k only) the partial C tiles:
// splits x Mt x Nt tiles of 128 x 128 doubles, row-major inside a tile.
inline size_t f64_partials_offset(const F64Dims& d) {
  return align_up((size_t)(d.Mt + d.Nt) * d.Kt * kF64TileBytes, 1024);
}
inline size_t f64_workspace(const F64Dims& d) {
  const size_t partials =
      d.splits > 1 ? (size_t)d.splits * d.Mt * d.Nt * kF64BM * kF64BN * sizeof(double) : 0;
  return align_up(f64_partials_offset(d) + partials, 1024);
}

cudaError_t launch_f64_pack(const double* A, const double* B, const F64Dims& d, uint8_t* ws,
                            cudaStream_t s);
cudaError_t launch_f64_gemm(uint8_t* ws, double* C, const F64Dims& d, int* status,
                            cudaStream_t s);

cudaError_t launch_zero_fill(double* C, int64_t count, cudaStream_t s);

// ---------------------------------------------------------------- grouped
// Device plan of a grouped call, written by grouped_plan_kernel at the start
// of the caller's workspace: a header, one record per problem (with prefix
// sums of every per-problem count), then the data regions.
struct GroupedProblem {
  const double* A;
  const double* B;
  double* C;
  int64_t m, k, n;
  int64_t Mt, Nt, Kt;      // 128-row tiles of A, 128-column tiles of B, k-blocks
  int64_t tile_begin;      // first C tile (prefix of Mt*Nt)
  int64_t atile_begin;     // first A operand tile (prefix of Mt*Kt)
  int64_t btile_begin;     // first B operand tile (prefix of Nt*Kt)
  int64_t row_begin;       // first row maximum (prefix of m)
  int64_t col_begin;       // first column maximum (prefix of n)
  int64_t trow_begin;      // first tile-row of A (prefix of Mt)
  int64_t tcol_begin;      // first tile-column of B (prefix of Nt)
  int64_t ltile_begin;     // emulated: first C tile among the long-k problems
  int64_t stile_begin;     // emulated: first C tile among the short-k problems
};

struct GroupedHeader {
  int64_t valid;           // 0: workspace too small, every later kernel does nothing
  int64_t count;           // problems
  int64_t tiles, atiles, btiles, rows, cols, trows, tcols, ltiles, stiles, max_kt;
  int64_t off_rowbits, off_colbits, off_a, off_b, total;  // byte offsets in the workspace
  int64_t cursor;          // next work unit of a dynamically scheduled kernel (zeroed by
                           // the plan kernel on every call)
  int64_t off_sums, off_spill;  // emulated: running sums of every C tile, spill areas
  int64_t cursor_max;      // next unit of the emulated maxima pass (zeroed like cursor)
  int64_t off_owner;       // emulated: the problem (int32) owning each A tile, B tile,
                           // short-k C tile, long-k C tile, A tile-row and B
                           // tile-column, in that order
};

constexpr size_t kGroupedRecordsOff = 256;
static_assert(sizeof(GroupedHeader) <= kGroupedRecordsOff, "the header precedes the records");

__host__ __device__ inline size_t grouped_data_begin(int64_t count) {
  return align_up(kGroupedRecordsOff + sizeof(GroupedProblem) * static_cast<size_t>(count), 1024);
}

// Byte offsets of the data regions from the totals (same on host and device).
__host__ __device__ inline void grouped_offsets(GroupedHeader& h, int planes, size_t tile_bytes,
                                                bool bits) {
  size_t off = grouped_data_begin(h.count);
  h.off_rowbits = off;
  if (bits) off = align_up(off + 8 * static_cast<size_t>(h.rows > 0 ? h.rows : 1), 1024);
  h.off_colbits = off;
  if (bits) off = align_up(off + 8 * static_cast<size_t>(h.cols > 0 ? h.cols : 1), 1024);
  h.off_a = off;
  off = align_up(off + static_cast<size_t>(planes) * h.atiles * tile_bytes, 1024);
  h.off_b = off;
  off = align_up(off + static_cast<size_t>(planes) * h.btiles * tile_bytes, 1024);
  // emulated: the running sums of the diagonal-pair slice GEMM (128 x 128 x 8
  // bytes per C tile of the long-k problems) and the int64 spill areas of its
  // CTAs (long k)
  h.off_sums = off;
  if (bits) off = align_up(off + static_cast<size_t>(h.ltiles) * kOzTileRows * kOzTileRows * 8, 1024);
  h.off_spill = off;
  if (bits) off = align_up(off + static_cast<size_t>(kOzSpillCtas) * 2 * kOzTileRows * kOzTileRows * 8,
                           1024);
  h.off_owner = off;
  if (bits)
    off = align_up(off + 4 * static_cast<size_t>(h.atiles + h.btiles + h.stiles + h.ltiles +
                                                 h.trows + h.tcols + 1),
                   1024);
  h.total = off;
}

// Index of the problem owning item t of the prefix field `begin`: the last
// record whose begin is <= t (problems with no items share their begin with
// the next one and are skipped by "last").
template <typename Rec>
__device__ __forceinline__ int64_t grouped_find(const Rec* recs, int64_t count, int64_t t,
                                                int64_t Rec::*begin) {
  int64_t lo = 0, hi = count - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (recs[mid].*begin <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Problems of a grouped emulated call with at most this many k-blocks run on
// the one-diagonal slice GEMM (running sums in tensor memory), the others on
// the diagonal-pair GEMM.
// Measured on 2000 problems of dims log-uniform in [16, 1024] (k <= 8 blocks):
// all on the one-diagonal kernel is fastest (11.0 ms at S = 8 against 14.4 ms
// all on the pair kernel), so the default takes every problem up to 8 blocks.
constexpr int kGroupedShortKt = 8;
// short_kt: the plan's boundary (k-blocks) between the short-k problems (the
// one-diagonal kernel) and the long-k ones (the diagonal-pair kernel).
cudaError_t launch_ozaki_grouped(uint8_t* ws, int S, int beta, int64_t short_kt, int* status,
                                 cudaStream_t s, bool rn = false);
// Native grouped products: work units of 32 x 32 C elements (one warp each,
// operands loaded straight from the caller's arrays, k in steps of 4).
constexpr int kF64GroupedTile = 32;
constexpr int kF64GroupedK = 4;
cudaError_t launch_f64_grouped(uint8_t* ws, int* status, cudaStream_t s);
int sm_count();

// Comparison modes (not FP64-accurate).
cudaError_t launch_bf16_gemm(const double* A, const double* B, double* C, const OzakiDims& d,
                             uint8_t* aplane, uint8_t* bplane, int* status, cudaStream_t s);
cudaError_t launch_f32_gemm(const double* A, const double* B, double* C, int64_t m, int64_t k,
                            int64_t n, cudaStream_t s);

}  // namespace mxm

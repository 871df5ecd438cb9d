// ozaki.cu -- FP64-accurate product C = A.B by the Ozaki split, on tcgen05.
//
// The method (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012; in the
// integer-slice form of Ootomo, Ozaki, Yokota, IJHPCA 2024) applied to the
// mod2am product c_ij = sum_l a_il b_lj (Sec. 3.1):
//   1. scale  e_i = frexp exponent of max_l |a_il|, f_j the same for column
//             j of B (an all-zero row/column gets 0);
//   2. split  r = x 2^-e, then S times: t = r 2^beta, d = trunc(t), r = t - d,
//             giving integer digits |d| <= 2^beta - 1 (beta = 7: int8 range,
//             beta = 8: the full 8-bit significand of bf16);
//   3. exact slice products D_g = sum_{s+t=g} A_s B_t for g = 2..S+1;
//   4. recombine acc = 0; for g = S+1 down to 2: acc += D_g 2^{-beta g};
//             c_ij = acc 2^{e_i + f_j}.
//
// GB300 mapping.  tcgen05 has no integer MMA kind on sm_103a, so the integer
// digits ride in bf16 (every integer of magnitude <= 256 is exact in bf16)
// through tcgen05.mma kind::f16 with FP32 accumulation in tensor memory.
// Products are integers of magnitude <= (2^beta - 1)^2; an accumulator that
// receives at most `window` MMAs (16 products per row each) stays below 2^24
// and is therefore exact.  The epilogue warps drain each window into exact
// integer registers, so D_g is exact over all of k, and then fold D_g into a
// running sum in the order of step 4 (exactly in int64 while the partial sum
// stays below 2^52, in FP64 after).
//
// Kernels: oz_rowmax / oz_colmax (step 1, HBM-bound), oz_split_a / oz_split_b
// (step 2; write pre-swizzled bf16 tiles), oz_gemm2 (steps 3-4: diagonals in
// pairs sharing operand tiles, int32 window sums, running sums in a
// workspace scratch; the main kernel), oz_gemm (steps 3-4 one diagonal at a
// time with int64 sums and the running sum in tensor memory: long k, split-k
// units, grouped calls, the BF16 comparison mode), oz_splitk_fold (step 4
// after a split-k product), and the grouped variants of steps 1-2.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "mxm_internal.h"
#include "ptx.cuh"

namespace mxm {
namespace {

constexpr uint64_t kAbsMask = 0x7FFFFFFFFFFFFFFFull;
constexpr uint64_t kInfBits = 0x7FF0000000000000ull;

// ---------------------------------------------------------------- step 1
// The maxima keep what the split and the final scaling read of max |x|: its
// exponent (exponent_from_absbits) and whether it is inf or NaN.  Ordering
// non-negative doubles equals ordering their bit patterns (NaN patterns sort
// above +inf), and the high word of |x| (exponent field, top 20 mantissa
// bits) fixes both properties unless every high word is zero (all
// |x| < 2^-1042), when the low words give the exponent.  So the maxima run
// on 32-bit high words (an integer max; the 64-bit form runs on the FP64
// pipe, the slowest of this GPU), a second pass over the low words covers
// the rows or columns whose high words are all zero, and the stored pattern
// is max_bits(hi, lo): hi 2^32, or lo when hi = 0 -- the exponent of the true
// maximum, and >= kInfBits exactly when the true maximum is.
__device__ __forceinline__ uint32_t abs_hi(double x) {
  return static_cast<uint32_t>(__double2hiint(x)) & 0x7FFFFFFFu;
}
__device__ __forceinline__ uint32_t lo_word(double x) {
  return static_cast<uint32_t>(__double2loint(x));
}
__device__ __forceinline__ uint64_t max_bits(uint32_t hi, uint32_t lo) {
  return hi ? (static_cast<uint64_t>(hi) << 32) : static_cast<uint64_t>(lo);
}
__device__ __forceinline__ uint32_t warp_max_u32(uint32_t v) {
  return __reduce_max_sync(0xFFFFFFFFu, v);
}

// Maximum of one row of k values (a warp; lanes stride the row): max_bits.
__device__ __forceinline__ uint64_t warp_row_max(const double* __restrict__ a, int64_t k,
                                                 int lane) {
  uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
  int64_t l = lane;
  for (; l + 96 < k; l += 128) {
    m0 = max(m0, abs_hi(__ldg(a + l)));
    m1 = max(m1, abs_hi(__ldg(a + l + 32)));
    m2 = max(m2, abs_hi(__ldg(a + l + 64)));
    m3 = max(m3, abs_hi(__ldg(a + l + 96)));
  }
  for (; l < k; l += 32) m0 = max(m0, abs_hi(__ldg(a + l)));
  const uint32_t hi = warp_max_u32(max(max(m0, m1), max(m2, m3)));
  uint32_t lo = 0;
  if (hi == 0) {  // warp-uniform
    for (l = lane; l < k; l += 32) lo = max(lo, lo_word(__ldg(a + l)));
    lo = warp_max_u32(lo);
  }
  return max_bits(hi, lo);
}

// max_l |a_il| per row, a warp per row.
__global__ void oz_rowmax_kernel(const double* __restrict__ A, int64_t m, int64_t k,
                                 uint64_t* __restrict__ rowbits, int* __restrict__ status) {
  const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= m) return;
  const int lane = threadIdx.x & 31;
  const uint64_t mx = warp_row_max(A + row * k, k, lane);
  if (lane == 0) {
    rowbits[row] = mx;
    if (mx >= kInfBits) atomicOr(status, kStatusNonFinite);
  }
}

// max_l |b_lj| for 32 columns per block, rows split over blockIdx.y; the
// per-block maxima meet in colbits by atomicMax (colbits zeroed first).
constexpr int kColRowsPerBlock = 256;
__global__ void oz_colmax_kernel(const double* __restrict__ B, int64_t k, int64_t n,
                                 unsigned long long* __restrict__ colbits,
                                 int* __restrict__ status) {
  __shared__ uint32_t red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t col = static_cast<int64_t>(blockIdx.x) * 32 + tx;
  const int64_t l0 = static_cast<int64_t>(blockIdx.y) * kColRowsPerBlock;
  const int64_t l1 = l0 + kColRowsPerBlock < k ? l0 + kColRowsPerBlock : k;
  uint32_t mh = 0;
  if (col < n)
    for (int64_t l = l0 + ty; l < l1; l += 8) mh = max(mh, abs_hi(__ldg(B + l * n + col)));
  red[ty][tx] = mh;
  __syncthreads();
  if (ty == 0 && col < n) {
#pragma unroll
    for (int y = 1; y < 8; ++y) mh = max(mh, red[y][tx]);
    uint32_t lo = 0;
    if (mh == 0)  // every high word of this block's rows is zero
      for (int64_t l = l0; l < l1; ++l) lo = max(lo, lo_word(__ldg(B + l * n + col)));
    // the block maxima of a column meet in the same form: hi 2^32 beats any lo
    const uint64_t mx = max_bits(mh, lo);
    atomicMax(colbits + col, static_cast<unsigned long long>(mx));
    if (mx >= kInfBits) atomicOr(status, kStatusNonFinite);
  }
}

// ---------------------------------------------------------------- step 2
// Digits of 8 consecutive k-values of one operand row, written as 16-byte
// chunks of bf16 into the pre-swizzled tile image (chunk c of tile row r at
// chunk position c ^ (r % 8)).
// bf16 bit pattern of the integer sign * mag, 0 < mag <= 255 (exact: at most
// 8 significant bits), built from the bits: exponent floor(log2 mag).
__device__ __forceinline__ uint32_t bf16_of_digit(uint32_t mag, uint32_t sign) {
  if (mag == 0) return 0u;
  const int ex = 31 - __clz(static_cast<int>(mag));
  const uint32_t frac = (mag << (7 - ex)) & 0x7Fu;
  return (sign << 15) | (static_cast<uint32_t>(127 + ex) << 7) | frac;
}

// Digits of 8 consecutive values of one operand row, written as 16-byte
// chunks of bf16 into the pre-swizzled tile image, one chunk per slice.
//
// The truncating split r = x 2^-e; t = r 2^beta; d = trunc(t); r = t - d is
// exact in FP64 (every step is exact for |r| < 1), so digit s is simply the
// s-th beta-bit field below the binary point of |x| 2^-e, with the sign of x.
// With |x| = M 2^E2 (M the integer significand), digit s is bits
// [beta (S - s) - sh, + beta) of M, sh = E2 - e + beta S: integer shifts, no
// FP64 arithmetic (FP64 is the slow pipe on this GPU).  When x 2^-e is below
// 2^-1022 every digit is 0 either way.
__device__ __forceinline__ void split_chunk_store(const double (&x)[8], int e, int S, int beta,
                                                  uint8_t* dst, size_t slice_stride) {
  uint64_t M[8];
  int sh[8];
  uint32_t sg[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x[j]));
    const int be = static_cast<int>((b >> 52) & 0x7FF);
    const uint64_t mant = b & 0x000FFFFFFFFFFFFFull;
    M[j] = be ? (mant | 0x0010000000000000ull) : mant;
    const int E2 = be ? be - 1075 : -1074;
    sh[j] = E2 - e + beta * S;
    sg[j] = static_cast<uint32_t>(b >> 63);
  }
  const uint64_t mask = (1ull << beta) - 1;
  for (int s = 1; s <= S; ++s) {
    uint32_t packed[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      uint32_t bits2[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = beta * (S - s) - sh[j + h];  // lowest bit of the field in M
        uint64_t dg;
        if (p >= 0) dg = p < 64 ? (M[j + h] >> p) & mask : 0;
        else dg = -p < 64 ? (M[j + h] << -p) & mask : 0;
        bits2[h] = bf16_of_digit(static_cast<uint32_t>(dg), sg[j + h]);
      }
      packed[j >> 1] = bits2[0] | (bits2[1] << 16);
    }
    *reinterpret_cast<uint4*>(dst + static_cast<size_t>(s - 1) * slice_stride) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
}

// The same for beta * S <= 64: the fraction |x| 2^-e is first put in one
// 64-bit fixed-point word F = floor(|x| 2^{beta S - e}) (one shift), then
// digit s is the field F >> beta (S - s) (a shift uniform over the warp, of
// the high word or a funnel shift of both).  V values per 16-byte chunk:
// V = 8 bf16 digits, or V = 16 E4M3 digits (|d| <= 15, from a 16-entry table
// of the E4M3 codes of 0..15).
//
// A bf16 digit is the upper half of the FP32 pattern of the integer +-mag
// (exact: at most 8 significant bits), made without a conversion
// instruction: the pattern of 2^23 + mag (mag in the low mantissa bits of
// 2^23, with the sign of x) plus -+2^23 is exactly +-mag, and +0 for mag = 0
// (x + (-x) rounds to +0).
__device__ __forceinline__ uint32_t bf16_pair(uint32_t q0, uint32_t q1, uint32_t a0,
                                              uint32_t a1) {
  const float f0 = __uint_as_float(q0) + __uint_as_float(a0);
  const float f1 = __uint_as_float(q1) + __uint_as_float(a1);
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);  // the upper halves
}

template <int V>
__device__ __forceinline__ void split_chunk_store_w64(const double (&x)[V], int e, int S,
                                                      int beta, uint8_t* dst,
                                                      size_t slice_stride) {
  uint32_t Fh[V], Fl[V], mg[V];
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x[j]));
    const int be = static_cast<int>((b >> 52) & 0x7FF);
    const uint64_t mant = b & 0x000FFFFFFFFFFFFFull;
    const uint64_t M = be ? (mant | 0x0010000000000000ull) : mant;
    const int sh = (be ? be - 1075 : -1074) - e + beta * S;
    const uint64_t F = sh >= 0 ? (sh < 64 ? M << sh : 0ull) : (-sh < 64 ? M >> -sh : 0ull);
    Fh[j] = static_cast<uint32_t>(F >> 32);
    Fl[j] = static_cast<uint32_t>(F);
    mg[j] = V == 8 ? (0x4B000000u | (static_cast<uint32_t>(b >> 63) << 31))  // +-2^23
                   : static_cast<uint32_t>(b >> 63);
  }
  const uint32_t mask = (1u << beta) - 1u;
  for (int s = 1; s <= S; ++s) {
    const int p = beta * (S - s);
    auto field = [&](int j) -> uint32_t {
      return (p >= 32 ? (Fh[j] >> (p - 32)) : __funnelshift_r(Fl[j], Fh[j], p)) & mask;
    };
    uint32_t packed[4];
    if constexpr (V == 8) {
#pragma unroll
      for (int j = 0; j < 8; j += 2)
        packed[j >> 1] = bf16_pair(field(j) | mg[j], field(j + 1) | mg[j + 1],
                                   mg[j] ^ 0x80000000u, mg[j + 1] ^ 0x80000000u);
    } else {
      // E4M3 codes of 0..7 and 8..15, one byte each
      constexpr uint64_t kLo = 0x4E4C4A4844403800ull, kHi = 0x5756555453525150ull;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        uint32_t word = 0;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int j = 4 * w + h;
          const uint32_t mag = field(j);
          const uint64_t tbl = mag < 8 ? kLo : kHi;
          uint32_t code = static_cast<uint32_t>(tbl >> (8 * (mag & 7))) & 0xFFu;
          if (mag) code |= mg[j] << 7;
          word |= code << (8 * h);
        }
        packed[w] = word;
      }
    }
    *reinterpret_cast<uint4*>(dst + static_cast<size_t>(s - 1) * slice_stride) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
}

// Balanced 8-bit digits (the round-to-nearest split): with e1 = e + 1,
// V = round(x 2^(8S - e1)) (ties to even; |V| <= 2^(8S-1), S <= 7), and the
// digits of V in base 256 with every lower digit in [-128, 127] and the top
// one in [-128, 128]: with W = V + sum_{i < S-1} 128 256^i, lower digit i is
// byte i of W minus 128 and the top digit is W >> 8(S-1) (floor) -- the
// same digits as taking V mod 256 in [-128, 127] from the bottom up.  Each
// digit is an integer of at most 8 bits, exact in bf16.
__device__ __forceinline__ void split_chunk_store_rn8(const double (&x)[8], int e1, int S,
                                                      uint8_t* dst, size_t slice_stride) {
  long long W[8];
  const long long Boff =
      S > 1 ? static_cast<long long>(0x8080808080808080ull >> (8 * (9 - S))) : 0ll;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x[j]));
    const int be = static_cast<int>((b >> 52) & 0x7FF);
    const uint64_t mant = b & 0x000FFFFFFFFFFFFFull;
    const uint64_t M = be ? (mant | 0x0010000000000000ull) : mant;
    const int sh = (be ? be - 1075 : -1074) - e1 + 8 * S;  // x 2^(8S - e1) = M 2^sh
    uint64_t q;
    if (sh >= 0) {
      q = M << sh;  // |x 2^(8S - e1)| < 2^(8S-1) <= 2^55: no bit leaves the word
    } else if (-sh >= 64) {
      q = 0;        // M < 2^53 <= half of 2^64: rounds to 0
    } else {
      const int nsh = -sh;
      q = M >> nsh;
      const uint64_t rem = M & ((1ull << nsh) - 1ull), half = 1ull << (nsh - 1);
      if (rem > half || (rem == half && (q & 1ull))) ++q;
    }
    const long long V = (b >> 63) ? -static_cast<long long>(q) : static_cast<long long>(q);
    W[j] = V + Boff;
  }
  // digit dg (|dg| <= 128) as an exact float without a conversion
  // instruction: the pattern of 1.5 2^23 + dg minus 1.5 2^23 (+0 for dg = 0)
  constexpr uint32_t kMagic = 0x4B400000u;  // 1.5 2^23 = 12582912
  const uint32_t kNegMagic = 0xCB400000u;
  for (int s = 1; s <= S; ++s) {
    const int p = 8 * (S - s);
    uint32_t packed[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      uint32_t q[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int dg = s == 1 ? static_cast<int>(W[j + h] >> p)
                              : static_cast<int>((W[j + h] >> p) & 255) - 128;
        q[h] = kMagic + static_cast<uint32_t>(dg);
      }
      packed[j >> 1] = bf16_pair(q[0], q[1], kNegMagic, kNegMagic);
    }
    *reinterpret_cast<uint4*>(dst + static_cast<size_t>(s - 1) * slice_stride) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
}

__device__ __forceinline__ void split_chunk(const double (&x)[8], int e, int S, int beta,
                                            uint8_t* dst, size_t slice_stride, bool rn = false) {
  if (rn)
    split_chunk_store_rn8(x, e + 1, S, dst, slice_stride);
  else if (beta * S <= 64)
    split_chunk_store_w64<8>(x, e, S, beta, dst, slice_stride);
  else
    split_chunk_store(x, e, S, beta, dst, slice_stride);
}
__device__ __forceinline__ void split_chunk(const double (&x)[16], int e, int S, int beta,
                                            uint8_t* dst, size_t slice_stride, bool = false) {
  split_chunk_store_w64<16>(x, e, S, beta, dst, slice_stride);  // beta = 4, S <= 16
}

// Tile geometry of the two digit carriers: V digits per 16-byte chunk.
template <int V>
struct SplitGeo {
  static constexpr int kChunksPerRow = kOzTileK / V;
  static constexpr int kTileBytes = V == 8 ? kOzTileBytes : kOzTileBytesE4m3;
  __device__ static int offset(int r, int c) {
    return V == 8 ? oz_chunk_offset(r, c) : oz_chunk_offset_e4m3(r, c);
  }
};

// One 128 x 128 tile (tm, tk) of A (m x k, row-major) -> its S digit tiles,
// `slice_stride` bytes apart.  A thread takes V consecutive k of one row
// (consecutive threads: consecutive chunks of a row, so the loads and the
// 16-byte stores are contiguous); rows of even k are read as 16-byte pairs.
// (row_lim, chunk_lim: only rows < row_lim and chunks < chunk_lim of the
// tile are written -- the rest is never read by the edge-tile copies.)
template <int V>
__device__ __forceinline__ void split_a_tile(const double* __restrict__ A, int64_t m, int64_t k,
                                             const uint64_t* __restrict__ rowbits, int S,
                                             int beta, int64_t tm, int64_t tk, uint8_t* tile,
                                             size_t slice_stride, bool rn = false,
                                             int row_lim = kOzTileRows,
                                             int chunk_lim = SplitGeo<V>::kChunksPerRow) {
  using G = SplitGeo<V>;
  const bool pairs = ((k & 1) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  const int total = row_lim * chunk_lim;
  // two chunks per thread and step, both loaded before either is split
  for (int p0 = threadIdx.x; p0 < total; p0 += 2 * blockDim.x) {
    double v[2][V];
    int e[2], rr[2], cc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int p = p0 + h * static_cast<int>(blockDim.x);
      const bool live = p < total;
      const int c = live ? p % chunk_lim : 0, r = live ? p / chunk_lim : 0;
      rr[h] = r;
      cc[h] = c;
      const int64_t row = tm * kOzTileRows + r;
      const int64_t k0 = tk * kOzTileK + c * V;
      const bool in = live && row < m;
      e[h] = in ? exponent_from_absbits(rowbits[row]) : 0;
      const double* src = A + (in ? row : 0) * k + k0;
      if (in && pairs && k0 + V <= k) {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
          const double2 t = __ldg(reinterpret_cast<const double2*>(src + j));
          v[h][j] = t.x;
          v[h][j + 1] = t.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j) v[h][j] = (in && k0 + j < k) ? __ldg(src + j) : 0.0;
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (p0 + h * static_cast<int>(blockDim.x) < total)
        split_chunk(v[h], e[h], S, beta, tile + G::offset(rr[h], cc[h]), slice_stride, rn);
  }
}

// One tile (tn, tk) of B^T, i.e. 128 columns j x 128 k of B (k x n,
// row-major) -> its S digit tiles: both MMA operands are K-major.  The tile
// is read in four passes of 32 rows of B (coalesced along the rows) through
// shared memory, then every thread takes V consecutive k of one column.
constexpr int kSplitBRows = 32;
constexpr int kSplitThreads = 256;  // the block size of the split launches
template <int V>
__device__ __forceinline__ void split_b_tile(const double* __restrict__ B, int64_t k, int64_t n,
                                             const uint64_t* __restrict__ colbits, int S,
                                             int beta, int64_t tn, int64_t tk, uint8_t* tile,
                                             size_t slice_stride,
                                             double (*sb)[kOzTileRows + 1], bool rn = false,
                                             bool halves = false, int row_lim = kOzTileRows,
                                             int chunk_lim = SplitGeo<V>::kChunksPerRow) {
  using G = SplitGeo<V>;
  const int64_t col0 = tn * kOzTileRows;
  constexpr int kChunksPerPass = kSplitBRows / V;
  for (int pass = 0; pass < kOzTileK / kSplitBRows; ++pass) {
    if (pass * kChunksPerPass >= chunk_lim) break;  // block-uniform
    const int64_t l0 = tk * kOzTileK + pass * kSplitBRows;
    if (blockDim.x == kSplitThreads) {  // every launch: all of a thread's loads in flight at once
      constexpr int kPer = kSplitBRows * kOzTileRows / kSplitThreads;
      double v[kPer];
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int p = threadIdx.x + i * kSplitThreads;
        const int64_t l = l0 + p / kOzTileRows, col = col0 + p % kOzTileRows;
        v[i] = (l < k && col < n) ? __ldg(B + l * n + col) : 0.0;
      }
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int p = threadIdx.x + i * kSplitThreads;
        sb[p / kOzTileRows][p % kOzTileRows] = v[i];
      }
    } else {
      for (int p = threadIdx.x; p < kSplitBRows * kOzTileRows; p += blockDim.x) {
        const int lr = p / kOzTileRows, cc = p % kOzTileRows;
        const int64_t l = l0 + lr, col = col0 + cc;
        sb[lr][cc] = (l < k && col < n) ? __ldg(B + l * n + col) : 0.0;
      }
    }
    __syncthreads();
    constexpr int kChunks = kSplitBRows / V;  // chunks of V k per column in a pass
    // consecutive threads take the consecutive chunks of one tile row (a
    // row's chunks of a pass are one aligned group under the swizzle, so
    // their 16-byte stores are contiguous)
    for (int p = threadIdx.x; p < kOzTileRows * kChunks; p += blockDim.x) {
      const int r = p / kChunks, cl = p % kChunks;
      if (r >= row_lim || pass * kChunks + cl >= chunk_lim) continue;
      const int64_t col = col0 + r;
      const int f = col < n ? exponent_from_absbits(colbits[col]) : 0;
      double v[V];
#pragma unroll
      for (int j = 0; j < V; ++j) v[j] = sb[cl * V + j][r];
      const int c = pass * kChunks + cl;
      const int off = (V == 8 && halves) ? oz_chunk_offset_halves(r, c) : G::offset(r, c);
      split_chunk(v, f, S, beta, tile + off, slice_stride, rn);
    }
    __syncthreads();
  }
}

// A -> A_s tiles [S][Mt][Kt].
template <int V>
__global__ void __launch_bounds__(256) oz_split_a_kernel(
    const double* __restrict__ A, int64_t m, int64_t k, const uint64_t* __restrict__ rowbits,
    int S, int beta, int64_t Mt, int64_t Kt, uint8_t* __restrict__ aslices, bool rn) {
  constexpr size_t kTile = SplitGeo<V>::kTileBytes;
  const int64_t tk = blockIdx.x, tm = blockIdx.y;
  split_a_tile<V>(A, m, k, rowbits, S, beta, tm, tk,
                  aslices + (static_cast<size_t>(tm) * Kt + tk) * kTile,
                  static_cast<size_t>(Mt) * Kt * kTile, rn);
}

// Steps 1 and 2 for A in one pass: one block per row of A (and per padding
// row of the last tile-row) holds the row in shared memory, zero-padded to
// whole k-blocks, takes its maximum and writes its digits into every k-block
// tile from there -- A is read from memory once.  The row's 16-byte chunks of
// a tile atom fill one 128-byte line (the swizzle permutes chunks inside the
// row), so the stores stay whole lines.  Padding rows (i >= m) get zero
// digits and no maximum.
constexpr int64_t kFusedRowMaxK = 24576;  // k doubles held in shared memory (192 KiB)

__global__ void __launch_bounds__(256) oz_scale_split_a_kernel(
    const double* __restrict__ A, int64_t m, int64_t k, uint64_t* __restrict__ rowbits, int S,
    int beta, int64_t Mt, int64_t Kt, uint8_t* __restrict__ aslices, bool rn,
    int* __restrict__ status) {
  extern __shared__ double row[];
  __shared__ uint32_t wmax[32];
  __shared__ uint64_t rmax;
  const int64_t i = blockIdx.x;
  const int64_t kp = Kt * kOzTileK;
  const bool real = i < m;
  const double* a = A + (real ? i : 0) * k;
  uint32_t mh = 0;
  // eight loads of a thread in flight before they go to shared memory
  // (few blocks fit an SM with a whole row in shared memory)
  for (int64_t l0 = threadIdx.x; l0 < kp; l0 += 8 * static_cast<int64_t>(blockDim.x)) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t l = l0 + u * static_cast<int64_t>(blockDim.x);
      v[u] = (real && l < k) ? __ldg(a + l) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t l = l0 + u * static_cast<int64_t>(blockDim.x);
      if (l < kp) {
        row[l] = v[u];
        mh = max(mh, abs_hi(v[u]));
      }
    }
  }
  mh = warp_max_u32(mh);
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mh;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t w = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0;
    w = warp_max_u32(w);
    uint32_t lo = 0;
    if (w == 0) {  // every high word is zero: the low words (row in shared memory)
      for (int64_t l = threadIdx.x; l < kp; l += 32) lo = max(lo, lo_word(row[l]));
      lo = warp_max_u32(lo);
    }
    if (threadIdx.x == 0) {
      const uint64_t mx = max_bits(w, lo);
      rmax = mx;
      if (real) {
        rowbits[i] = mx;
        if (mx >= kInfBits) atomicOr(status, kStatusNonFinite);
      }
    }
  }
  __syncthreads();
  const int e = exponent_from_absbits(rmax < kInfBits ? rmax : 0);
  const int64_t tm = i / kOzTileRows;
  const int r = static_cast<int>(i - tm * kOzTileRows);
  const size_t slice_stride = static_cast<size_t>(Mt) * Kt * kOzTileBytes;
  uint8_t* base = aslices + static_cast<size_t>(tm) * Kt * kOzTileBytes;
  for (int64_t p = threadIdx.x; p < Kt * kOzChunksPerRow; p += blockDim.x) {
    const int64_t tk = p / kOzChunksPerRow;
    const int c = static_cast<int>(p - tk * kOzChunksPerRow);
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = row[tk * kOzTileK + c * 8 + j];
    split_chunk(v, e, S, beta, base + tk * kOzTileBytes + oz_chunk_offset(r, c), slice_stride,
                rn);
  }
}

// Whether A's scale and split run fused (bf16 digits, k short enough for a
// row in shared memory).
__host__ __device__ inline bool oz_fused_a(const OzakiDims& d) {
  return !d.fp8 && d.Kt * kOzTileK <= kFusedRowMaxK;
}

// B -> B_t tiles [S][Nt][Kt]; halves: the CTA-pair layout of each tile.
template <int V>
__global__ void __launch_bounds__(256) oz_split_b_kernel(
    const double* __restrict__ B, int64_t k, int64_t n, const uint64_t* __restrict__ colbits,
    int S, int beta, int64_t Nt, int64_t Kt, uint8_t* __restrict__ bslices, bool rn,
    bool halves) {
  constexpr size_t kTile = SplitGeo<V>::kTileBytes;
  __shared__ double sb[kSplitBRows][kOzTileRows + 1];
  const int64_t tk = blockIdx.x, tn = blockIdx.y;
  split_b_tile<V>(B, k, n, colbits, S, beta, tn, tk,
                  bslices + (static_cast<size_t>(tn) * Kt + tk) * kTile,
                  static_cast<size_t>(Nt) * Kt * kTile, sb, rn, halves);
}

// ---------------------------------------------------------------- grouped steps 1-2
// The scale and the split of a grouped call, in two passes over the operands,
// after oz_grouped_owner_kernel has written the owner map (each unit's
// problem).  oz_grouped_max_kernel (step 1) takes units of 32 rows of A or 32
// columns of B of one problem, their cost following k, from a cursor in the
// plan's header (zeroed by the plan kernel on every call).
// oz_grouped_split_kernel (step 2) takes the 128 x 128 operand tiles, A's
// then B's, round robin over the blocks.  Only what the edge-tile copies of the slice
// GEMM read is written: rows up to the tile's rows rounded up to 8 (A) or
// columns up to 16 (B, the MMA's N step), and in the last k-block the
// 16-byte chunks up to k rounded up to 16 (with zeros past k).

// Chunks of 8 k written in k-block tk of a problem with Kt k-blocks.
__device__ __forceinline__ int grouped_chunk_lim(int64_t k, int64_t Kt, int64_t tk) {
  if (tk < Kt - 1) return kOzChunksPerRow;
  const int64_t klast = k - (Kt - 1) * kOzTileK;
  return static_cast<int>((klast + 15) / 16 * 2);
}

constexpr int kMaxUnit = 32;  // rows of A or columns of B per unit of the maxima pass

// The owner map of a grouped call: for every A tile, B tile, short-k C tile,
// long-k C tile, A tile-row and B tile-column the index of its problem (the
// later kernels look a unit's problem up instead of searching the problem
// table).  A warp per problem.
__global__ void __launch_bounds__(256) oz_grouped_owner_kernel(uint8_t* __restrict__ ws) {
  const GroupedHeader* hdr = reinterpret_cast<const GroupedHeader*>(ws);
  if (!hdr->valid) return;
  const GroupedProblem* recs = reinterpret_cast<const GroupedProblem*>(ws + kGroupedRecordsOff);
  int32_t* owner = reinterpret_cast<int32_t*>(ws + hdr->off_owner);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t count = hdr->count;
  const int64_t tot[6] = {hdr->atiles, hdr->btiles, hdr->stiles, hdr->ltiles, hdr->trows,
                          hdr->tcols};
  int64_t base[6];
  base[0] = 0;
  for (int f = 1; f < 6; ++f) base[f] = base[f - 1] + tot[f - 1];
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * nwarps + warp; q < count;
       q += static_cast<int64_t>(gridDim.x) * nwarps) {
    const GroupedProblem& r = recs[q];
    const GroupedProblem* nx = q + 1 < count ? &recs[q + 1] : nullptr;
    const int64_t b0[6] = {r.atile_begin, r.btile_begin, r.stile_begin, r.ltile_begin,
                           r.trow_begin, r.tcol_begin};
    const int64_t b1[6] = {nx ? nx->atile_begin : tot[0], nx ? nx->btile_begin : tot[1],
                           nx ? nx->stile_begin : tot[2], nx ? nx->ltile_begin : tot[3],
                           nx ? nx->trow_begin : tot[4], nx ? nx->tcol_begin : tot[5]};
#pragma unroll
    for (int f = 0; f < 6; ++f)
      for (int64_t t = b0[f] + lane; t < b1[f]; t += 32)
        owner[base[f] + t] = static_cast<int32_t>(q);
  }
}

__global__ void __launch_bounds__(256) oz_grouped_max_kernel(uint8_t* __restrict__ ws,
                                                             int* __restrict__ status) {
  GroupedHeader* hdr = reinterpret_cast<GroupedHeader*>(ws);
  if (!hdr->valid) return;
  const GroupedProblem* recs = reinterpret_cast<const GroupedProblem*>(ws + kGroupedRecordsOff);
  uint64_t* rowbits = reinterpret_cast<uint64_t*>(ws + hdr->off_rowbits);
  uint64_t* colbits = reinterpret_cast<uint64_t*>(ws + hdr->off_colbits);
  unsigned long long* cursor = reinterpret_cast<unsigned long long*>(&hdr->cursor_max);
  constexpr int kPer = kOzTileRows / kMaxUnit;  // units per tile-row (tile-column)
  const int64_t aunits = hdr->trows * kPer, total = aunits + hdr->tcols * kPer;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // the problem of each A tile-row and B tile-column (the owner map)
  const int32_t* rowowner = reinterpret_cast<const int32_t*>(ws + hdr->off_owner) +
                            hdr->atiles + hdr->btiles + hdr->stiles + hdr->ltiles;
  const int32_t* colowner = rowowner + hdr->trows;
  __shared__ int64_t unit;
  __shared__ uint32_t red[8][kMaxUnit];
  for (;;) {
    if (threadIdx.x == 0) unit = static_cast<int64_t>(atomicAdd(cursor, 1ull));
    __syncthreads();
    const int64_t u = unit;
    __syncthreads();  // every thread has read the unit before thread 0 takes the next
    if (u >= total) break;  // block-uniform
    if (u < aunits) {
      // 32 rows of A
      const int64_t it = u / kPer;
      const GroupedProblem& p = recs[rowowner[it]];
      const int64_t r0 = (it - p.trow_begin) * kOzTileRows + (u - it * kPer) * kMaxUnit;
      // a warp takes four rows at once (their loads in flight together:
      // most rows are short)
      for (int rb = warp; rb < kMaxUnit; rb += 4 * nwarps) {
        const double* ar[4];
        bool live[4];
        uint32_t mh[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t row = r0 + rb + i * nwarps;
          live[i] = rb + i * nwarps < kMaxUnit && row < p.m;
          ar[i] = p.A + (live[i] ? row : 0) * p.k;
          mh[i] = 0;
        }
        for (int64_t l = lane; l < p.k; l += 32) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (live[i]) mh[i] = max(mh[i], abs_hi(__ldg(ar[i] + l)));
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (!live[i]) continue;  // warp-uniform
          const uint32_t hi = warp_max_u32(mh[i]);
          uint32_t lo = 0;
          if (hi == 0) {  // every high word of the row is zero: the low words
            for (int64_t l = lane; l < p.k; l += 32) lo = max(lo, lo_word(__ldg(ar[i] + l)));
            lo = warp_max_u32(lo);
          }
          const uint64_t mx = max_bits(hi, lo);
          if (lane == 0) {
            rowbits[p.row_begin + r0 + rb + i * nwarps] = mx;
            if (mx >= kInfBits) atomicOr(status, kStatusNonFinite);
          }
        }
      }
    } else {
      // 32 columns of B: thread (h, c) takes column c of the rows l = h mod 8
      // (a warp reads 256 contiguous bytes of a row), four rows in flight
      const int64_t ic = (u - aunits) / kPer;
      const GroupedProblem& p = recs[colowner[ic]];
      const int64_t c0 =
          (ic - p.tcol_begin) * kOzTileRows + (u - aunits - ic * kPer) * kMaxUnit;
      const int c = threadIdx.x & (kMaxUnit - 1), h = threadIdx.x >> 5;
      uint32_t mh = 0;
      if (c0 + c < p.n) {
        const double* bc = p.B + c0 + c;
        uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
        int64_t l = h;
        for (; l + 3 * 8 < p.k; l += 4 * 8) {
          m0 = max(m0, abs_hi(__ldg(bc + l * p.n)));
          m1 = max(m1, abs_hi(__ldg(bc + (l + 8) * p.n)));
          m2 = max(m2, abs_hi(__ldg(bc + (l + 16) * p.n)));
          m3 = max(m3, abs_hi(__ldg(bc + (l + 24) * p.n)));
        }
        for (; l < p.k; l += 8) m0 = max(m0, abs_hi(__ldg(bc + l * p.n)));
        mh = max(max(m0, m1), max(m2, m3));
      }
      red[h][c] = mh;
      __syncthreads();
      if (threadIdx.x < kMaxUnit && c0 + threadIdx.x < p.n) {
        uint32_t hi = red[0][threadIdx.x];
#pragma unroll
        for (int q = 1; q < 8; ++q) hi = max(hi, red[q][threadIdx.x]);
        uint32_t lo = 0;
        if (hi == 0)  // every high word of the column is zero
          for (int64_t l = 0; l < p.k; ++l)
            lo = max(lo, lo_word(__ldg(p.B + l * p.n + c0 + threadIdx.x)));
        const uint64_t m = max_bits(hi, lo);
        colbits[p.col_begin + c0 + threadIdx.x] = m;
        if (m >= kInfBits) atomicOr(status, kStatusNonFinite);
      }
    }
  }
}

// Step 2: tile u of A's (u < atiles) or of B's operand tiles, dealt round
// robin over the blocks (tiles of one problem go to neighbouring blocks, so
// every block gets a like mix of large and small tiles); the owner map gives
// each tile's problem.
__global__ void __launch_bounds__(256, 3) oz_grouped_split_kernel(uint8_t* __restrict__ ws,
                                                                  int S, int beta, bool rn) {
  const GroupedHeader* hdr = reinterpret_cast<const GroupedHeader*>(ws);
  if (!hdr->valid) return;
  const GroupedProblem* recs = reinterpret_cast<const GroupedProblem*>(ws + kGroupedRecordsOff);
  const uint64_t* rowbits = reinterpret_cast<const uint64_t*>(ws + hdr->off_rowbits);
  const uint64_t* colbits = reinterpret_cast<const uint64_t*>(ws + hdr->off_colbits);
  const int32_t* owner = reinterpret_cast<const int32_t*>(ws + hdr->off_owner);
  __shared__ double sb[kSplitBRows][kOzTileRows + 1];
  const int64_t atiles = hdr->atiles, total = atiles + hdr->btiles;
  for (int64_t u = blockIdx.x; u < total; u += gridDim.x) {  // block-uniform
    const bool in_b = u >= atiles;
    const int64_t t = in_b ? u - atiles : u;
    const GroupedProblem& r = recs[owner[u]];
    const int64_t local = t - (in_b ? r.btile_begin : r.atile_begin);
    const int64_t tr = local / r.Kt, tk = local - tr * r.Kt;
    const int lim = grouped_chunk_lim(r.k, r.Kt, tk);
    if (!in_b) {
      const int64_t rows = r.m - tr * kOzTileRows;
      const int row_lim = rows >= kOzTileRows ? kOzTileRows : static_cast<int>((rows + 7) / 8 * 8);
      split_a_tile<8>(r.A, r.m, r.k, rowbits + r.row_begin, S, beta, tr, tk,
                      ws + hdr->off_a + static_cast<size_t>(t) * kOzTileBytes,
                      static_cast<size_t>(atiles) * kOzTileBytes, rn, row_lim, lim);
    } else {
      const int64_t cols = r.n - tr * kOzTileRows;
      const int row_lim =
          cols >= kOzTileRows ? kOzTileRows : static_cast<int>((cols + 15) / 16 * 16);
      split_b_tile<8>(r.B, r.k, r.n, colbits + r.col_begin, S, beta, tr, tk,
                      ws + hdr->off_b + static_cast<size_t>(t) * kOzTileBytes,
                      static_cast<size_t>(hdr->btiles) * kOzTileBytes, sb, rn, false, row_lim,
                      lim);
    }
  }
}

// ---------------------------------------------------------------- BF16 mode
// Comparison mode (not part of the Ozaki method): x rounded to the nearest
// bf16 (ties to even), computed on the binary64 bit pattern.
__device__ __forceinline__ uint32_t bf16_rne_bits(double x) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const uint32_t sign = static_cast<uint32_t>(b >> 48) & 0x8000u;
  const uint64_t ab = b & kAbsMask;
  if (ab > kInfBits) return sign | 0x7FC0u;   // nan
  if (ab == kInfBits) return sign | 0x7F80u;  // inf
  const int be = static_cast<int>(ab >> 52);
  if (be == 0) return sign;                   // |x| < 2^-1022: rounds to zero in bf16
  const int E = be - 1023;                    // |x| in [2^E, 2^{E+1})
  if (E >= 128) return sign | 0x7F80u;
  const int Eq = E < -126 ? -126 : E;         // bf16 spacing 2^{Eq-7}
  const uint64_t sig = (ab & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;  // 2^{E-52} units
  const int shift = 45 + (Eq - E);
  if (shift >= 63) return sign;
  uint64_t q = sig >> shift;
  const uint64_t rem = sig & ((1ull << shift) - 1);
  const uint64_t half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (q & 1))) ++q;
  uint32_t bits;
  if (E < -126) bits = static_cast<uint32_t>(q);  // subnormal (q = 128 is the least normal)
  else bits = (static_cast<uint32_t>(Eq + 127) << 7) + static_cast<uint32_t>(q - 128);
  if (bits >= 0x7F80u) bits = 0x7F80u;
  return sign | bits;
}

// A (m x k) or B (k x n, transposed) -> one plane of 128 x 64 bf16 tiles,
// same layout as a slice plane.
__global__ void __launch_bounds__(256) bf16_tiles_kernel(const double* __restrict__ X,
                                                         int64_t rows, int64_t cols, int trans,
                                                         int64_t Kt, uint8_t* __restrict__ out) {
  const int64_t tk = blockIdx.x, tr = blockIdx.y;
  uint8_t* tile = out + (static_cast<size_t>(tr) * Kt + tk) * kOzTileBytes;
  for (int p = threadIdx.x; p < kOzTileRows * kOzChunksPerRow; p += blockDim.x) {
    const int c = p % kOzChunksPerRow, r = p / kOzChunksPerRow;
    const int64_t row = tr * kOzTileRows + r;   // row of A, or column of B
    const int64_t k0 = tk * kOzTileK + c * 8;
    uint32_t packed[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      double x0 = 0.0, x1 = 0.0;
      if (!trans) {
        if (row < rows && k0 + j < cols) x0 = __ldg(X + row * cols + k0 + j);
        if (row < rows && k0 + j + 1 < cols) x1 = __ldg(X + row * cols + k0 + j + 1);
      } else {  // X is k x n: element (k0 + j, row)
        if (row < cols && k0 + j < rows) x0 = __ldg(X + (k0 + j) * cols + row);
        if (row < cols && k0 + j + 1 < rows) x1 = __ldg(X + (k0 + j + 1) * cols + row);
      }
      packed[j >> 1] = bf16_rne_bits(x0) | (bf16_rne_bits(x1) << 16);
    }
    *reinterpret_cast<uint4*>(tile + oz_chunk_offset(r, c)) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
}

// ---------------------------------------------------------------- steps 3-4
constexpr int kStages = 3;
// The slice GEMMs: warp 0 copies, warp 1 issues MMAs, warps 2-3 idle, warps
// 4.. run the epilogue (8, or 16 in the short-k grouped GEMM).
constexpr int kBN = 128;            // MMA N (columns of the C tile)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccCol = 256;   // FP64 running sums: 2 columns per value
// The window accumulators of the one-diagonal kernel: four slots of 64
// columns below kAccCol; a window of a tile with more than 64 MMA columns
// takes two neighbouring slots (0-1 or 2-3), a narrower one a single slot,
// so narrow tiles get four windows in flight instead of two.
constexpr int kAccSlotCols = 64;
constexpr int kMmaK = 16;           // K per tcgen05.mma kind::f16
constexpr int kMmaPerStage = kOzTileK / kMmaK;

__device__ __forceinline__ void tile_coords(int64_t tile, int64_t Mt, int64_t Nt, int64_t G,
                                            int64_t& tm, int64_t& tn) {
  // groups of G tile-rows, column-major inside a group: CTAs working at the
  // same time share A tiles and B tiles in L2
  const int64_t per_group = G * Nt;
  const int64_t grp = tile / per_group;
  const int64_t first = grp * G;
  const int64_t gsz = (Mt - first) < G ? (Mt - first) : G;
  const int64_t in = tile - grp * per_group;
  tm = first + in % gsz;
  tn = in / gsz;
}

// One 128 x 128 tile of C and where its operand tiles live.
struct OzTile {
  const uint8_t* a;          // slice 1 of A tile-row tm, k-block 0
  const uint8_t* b;          // slice 1 of B^T tile-row tn, k-block 0
  size_t a_slice, b_slice;   // bytes from one slice plane to the next
  int64_t Kt;                // k-blocks of kOzTileK
  const uint64_t* rowbits;   // |A| row maxima of this problem
  const uint64_t* colbits;   // |B| column maxima of this problem
  double* C;
  int64_t m, n;              // C is m x n, row-major
  int64_t row0, col0;        // origin of the tile in C
  uint64_t* sums;            // 128 x 128 running sums, column-major (paired kernel)
  uint64_t* partial;         // split-k: this range's D_g, [S - 1 diagonals][128 x 128]
  int eoff;                  // added to e_i + f_j in the final scaling (2: balanced digits)
  // Edge tiles (one-diagonal kernel): the MMAs compute n_eff columns (the
  // tile's columns rounded up to 16, the MMA's N step), only the first
  // a_rows rows of each A atom and n_eff rows of each B atom are copied (the
  // rest of the slot holds older digits, which reach only rows and columns of
  // D that are never stored), and the unit's last k-block issues last_mmas
  // MMAs of K = 16 (k rounded up to 16; the digit planes hold zeros there).
  int n_eff;
  int a_rows;
  int last_mmas;
};

// The one-diagonal kernel's shared memory.  The producer resolves every
// tile it takes (its place in the digit planes, its edges) once and hands it
// to the MMA issuer and the epilogue warps through a ring of kTileRing
// entries: tfull completes when an entry is written, tempty when the issuer
// and every epilogue warp have copied it.  An entry with tile_live == 0 ends
// the CTA's work.
constexpr int kTileRing = 4;
struct __align__(1024) GemmSmem {
  uint8_t a[kStages][kOzTileBytes];
  uint8_t b[kStages][kOzTileBytes];
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t accfull[4];   // per 64-column accumulator slot
  uint64_t accempty[4];
  uint64_t tfull[kTileRing];
  uint64_t tempty[kTileRing];
  OzTile tiles[kTileRing];
  int tile_live[kTileRing];
  uint32_t tmem_base;
  int abort_flag;
};

constexpr size_t kGemmSmemBytes = sizeof(GemmSmem) + 1024;

// Edge geometry of a tile: rows of A left from row0, columns of B from
// col0, and whether the unit's k range ends with the product's last k-block.
__device__ __forceinline__ void oz_edges(OzTile& j, int64_t k, bool ends_at_k) {
  const int64_t rn = j.n - j.col0, rm = j.m - j.row0;
  j.n_eff = rn >= kOzTileRows ? kOzTileRows : static_cast<int>((rn + 15) / 16 * 16);
  j.a_rows = rm >= kOzTileRows ? kOzTileRows : (rm > 0 ? static_cast<int>((rm + 7) / 8 * 8) : 0);
  const int64_t klast = k - (k - 1) / kOzTileK * kOzTileK;  // 1 .. 128 (k > 0)
  j.last_mmas = (ends_at_k && k > 0) ? static_cast<int>((klast + 15) / 16) : kOzTileK / 16;
}

// Tiles of one product.
struct OzSingle {
  const uint8_t* aslices;
  const uint8_t* bslices;
  const uint64_t* rowbits;
  const uint64_t* colbits;
  double* C;
  int64_t m, n, Mt, Nt, Kt;
  uint64_t* sums;     // running sums (paired kernel), or the split-k partials
  int64_t splits;     // k ranges per C tile; > 1: units write partials
  int S;
  int64_t tile_bytes; // operand tile size of the digit carrier
  long long* spill = nullptr;  // paired kernel: per-CTA int64 partials of the two diagonals
  int spill_every = 0;         // window drains after which a diagonal's int32 sum spills
  int eoff = 0;                // added to e_i + f_j in the final scaling (2: balanced digits)
  int64_t k = 0;               // the product's k (edge tiles)
  __device__ __forceinline__ long long* spill_area() const { return spill; }
#ifdef MXM_DEBUG_BOUNDS
  // the digit planes and the running sums (bounds checks of the debug build)
  __device__ __forceinline__ const uint8_t* a_end() const {
    return aslices + static_cast<size_t>(S) * Mt * Kt * tile_bytes;
  }
  __device__ __forceinline__ const uint8_t* b_end() const {
    return bslices + static_cast<size_t>(S) * Nt * Kt * tile_bytes;
  }
  __device__ __forceinline__ const uint8_t* a_begin() const { return aslices; }
  __device__ __forceinline__ const uint8_t* b_begin() const { return bslices; }
  __device__ __forceinline__ const uint64_t* sums_begin() const { return sums; }
  __device__ __forceinline__ const uint64_t* sums_end() const {
    return sums + (splits > 1 ? static_cast<size_t>(splits) * Mt * Nt * S
                              : static_cast<size_t>(Mt) * Nt) * (kOzTileRows * kOzTileRows);
  }
#endif
  int64_t raster = kDefaultRaster;  // tile-rows (pair-rows) per group of the tile walk
  bool kb_alt = false;         // alternate the k-block direction between diagonal (pair)s
  // Address k-block of the it-th k-block of diagonal (pair) q: every other
  // one walks k backwards, so it starts on the tiles the previous one read
  // last (still in L2).  The exact integer sums do not depend on the order.
  __device__ __forceinline__ int64_t kblock(int q, int64_t it, int64_t Kt_) const {
    return (kb_alt && (q & 1)) ? Kt_ - 1 - it : it;
  }
  __device__ __forceinline__ int64_t count() const { return Mt * Nt * splits; }
  // The it-th unit a CTA of the one-diagonal kernel takes: a fixed stride
  // over the grid (equal units; neighbouring CTAs share operand tiles in L2).
  __device__ __forceinline__ int64_t claim(int64_t it) const {
    return static_cast<int64_t>(blockIdx.x) + it * gridDim.x;
  }
  // Unit t: C tile t / splits, k range t % splits.
  __device__ __forceinline__ OzTile tile(int64_t t) const {
    const int64_t tt = t / splits, sp = t - tt * splits;
    int64_t tm, tn;
    tile_coords(tt, Mt, Nt, raster, tm, tn);
    return tile_at(tm, tn, sp);
  }
  // CTA pairs (no split-k): unit t is the 256 x 128 C tile of tile-rows
  // 2 tp, 2 tp + 1; CTA `rank` of the pair takes tile-row 2 tp + rank, which
  // lies past the last one (row0 >= m: nothing to load or store) when Mt is
  // odd.
  __device__ __forceinline__ int64_t pair_count() const { return (Mt + 1) / 2 * Nt; }
  __device__ __forceinline__ OzTile pair_tile(int64_t t, uint32_t rank) const {
    int64_t tp, tn;
    tile_coords(t, (Mt + 1) / 2, Nt, raster, tp, tn);
    return tile_at(2 * tp + rank, tn, 0);
  }
  __device__ __forceinline__ OzTile tile_at(int64_t tm, int64_t tn, int64_t sp) const {
    const int64_t kb0 = Kt * sp / splits, kb1 = Kt * (sp + 1) / splits;
    OzTile j;
    j.a_slice = static_cast<size_t>(Mt) * Kt * tile_bytes;
    j.b_slice = static_cast<size_t>(Nt) * Kt * tile_bytes;
    j.a = aslices + static_cast<size_t>(tm * Kt + kb0) * tile_bytes;
    j.b = bslices + static_cast<size_t>(tn * Kt + kb0) * tile_bytes;
    j.Kt = kb1 - kb0;
    j.rowbits = rowbits;
    j.colbits = colbits;
    j.C = C;
    j.m = m;
    j.n = n;
    j.row0 = tm * kOzTileRows;
    j.col0 = tn * kOzTileRows;
    j.eoff = eoff;
    oz_edges(j, k, kb1 == Kt);
    const size_t tile_words = kOzTileRows * kOzTileRows;
    if (splits > 1) {
      j.sums = nullptr;
      j.partial = sums + (static_cast<size_t>(sp * Mt + tm) * Nt + tn) * S * tile_words;
    } else {
      j.sums = sums ? sums + static_cast<size_t>(tm * Nt + tn) * tile_words : nullptr;
      j.partial = nullptr;
    }
    return j;
  }
};

// Tiles of a grouped call: the device plan (grouped_plan_kernel) lists every
// problem with prefix sums of its tile counts; the owner map (written by
// oz_grouped_owner_kernel) gives the problem of C tile t.
struct OzGrouped {
  const GroupedHeader* hdr;
  const GroupedProblem* recs;
  const uint8_t* ws;
  int eoff;  // 2 for balanced 8-bit digits
  bool long_k;  // the tiles of the long-k problems (else those of the short-k ones)
  int spill_every = 0;         // window drains after which a diagonal's int32 sum spills
  // paired kernel: per-CTA int64 partials of the two diagonals (long k)
  __device__ __forceinline__ long long* spill_area() const {
    return reinterpret_cast<long long*>(const_cast<uint8_t*>(ws) + hdr->off_spill);
  }
  __device__ __forceinline__ int64_t count() const {
    return hdr->valid ? (long_k ? hdr->ltiles : hdr->stiles) : 0;
  }
  // The next tile for the one-diagonal kernel, from the header's cursor
  // (zeroed by the plan kernel on every call): tiles differ in k and in their
  // edges, so CTAs take them as they finish the previous one.
  __device__ __forceinline__ int64_t claim(int64_t) const {
    GroupedHeader* h = const_cast<GroupedHeader*>(hdr);
    return static_cast<int64_t>(
        atomicAdd(reinterpret_cast<unsigned long long*>(&h->cursor), 1ull));
  }
#ifdef MXM_DEBUG_BOUNDS
  // the digit planes and the running sums (bounds checks of the debug build)
  __device__ __forceinline__ const uint8_t* a_begin() const { return ws + hdr->off_a; }
  __device__ __forceinline__ const uint8_t* a_end() const { return ws + hdr->off_b; }
  __device__ __forceinline__ const uint8_t* b_begin() const { return ws + hdr->off_b; }
  __device__ __forceinline__ const uint8_t* b_end() const { return ws + hdr->off_sums; }
  __device__ __forceinline__ const uint64_t* sums_begin() const {
    return reinterpret_cast<const uint64_t*>(ws + hdr->off_sums);
  }
  __device__ __forceinline__ const uint64_t* sums_end() const {
    return reinterpret_cast<const uint64_t*>(ws + hdr->off_spill);
  }
#endif
  __device__ __forceinline__ int64_t kblock(int, int64_t it, int64_t) const { return it; }
  __device__ __forceinline__ OzTile tile(int64_t t) const {
    int64_t GroupedProblem::*begin = long_k ? &GroupedProblem::ltile_begin
                                            : &GroupedProblem::stile_begin;
    const int32_t* owner = reinterpret_cast<const int32_t*>(ws + hdr->off_owner) + hdr->atiles +
                           hdr->btiles + (long_k ? hdr->stiles : 0);
    const GroupedProblem& r = recs[owner[t]];
    const int64_t local = t - r.*begin;
    const int64_t tm = local / r.Nt, tn = local - (local / r.Nt) * r.Nt;
    OzTile j;
    j.a_slice = static_cast<size_t>(hdr->atiles) * kOzTileBytes;
    j.b_slice = static_cast<size_t>(hdr->btiles) * kOzTileBytes;
    j.a = ws + hdr->off_a + static_cast<size_t>(r.atile_begin + tm * r.Kt) * kOzTileBytes;
    j.b = ws + hdr->off_b + static_cast<size_t>(r.btile_begin + tn * r.Kt) * kOzTileBytes;
    j.Kt = r.Kt;
    j.rowbits = reinterpret_cast<const uint64_t*>(ws + hdr->off_rowbits) + r.row_begin;
    j.colbits = reinterpret_cast<const uint64_t*>(ws + hdr->off_colbits) + r.col_begin;
    j.C = r.C;
    j.m = r.m;
    j.n = r.n;
    j.row0 = tm * kOzTileRows;
    j.col0 = tn * kOzTileRows;
    j.sums = reinterpret_cast<uint64_t*>(const_cast<uint8_t*>(ws) + hdr->off_sums) +
             static_cast<size_t>(t) * (kOzTileRows * kOzTileRows);
    j.partial = nullptr;
    j.eoff = eoff;
    oz_edges(j, r.k, true);
    return j;
  }
};

// First diagonal of the FP64 phase of the fold: diagonals g >= the returned
// value are combined exactly in int64 (the partial sum
// Y = sum_g D_g 2^{beta (S+1-g)} stays below 2^52 by the bound
// |D_g| <= (g-1)(2^beta-1)^2 128 Kt, so the FP64 fold of those steps is
// exact and doing them in integers gives the same bits).
__device__ __forceinline__ int oz_exact_from(int S, int beta, int64_t Kt) {
  const double dmax = static_cast<double>((1 << beta) - 1);
  int gx = S + 1;
  double yb = 0.0;
  for (int g = S + 1; g >= 2; --g) {
    yb += (g - 1) * dmax * dmax * static_cast<double>(kOzTileK) * static_cast<double>(Kt) *
          pow2_normal(beta * (S + 1 - g));
    if (yb >= 4503599627370496.0) break;  // 2^52
    gx = g;
  }
  return gx;
}

// The final scaling of one result.  Inline: the folds that call it are
// rolled loops over a few columns at a time, so the code stays small (the
// out-of-line form cost the grouped short-k GEMM ~1 % in call overhead and
// the 8192^3 product nothing).
__device__ __forceinline__ double final_scale(uint64_t st, int e) {
  return ldexp_rn(__longlong_as_double(static_cast<long long>(st)), e);
}

__device__ __noinline__ uint64_t fold_step(uint64_t st, long long dval, int g, int gx, int S,
                                           int beta) {
  if (g >= gx) {
    long long y = (g == S + 1) ? 0ll : static_cast<long long>(st);
    y += dval * (1ll << (beta * (S + 1 - g)));
    if (g == gx)
      return static_cast<uint64_t>(__double_as_longlong(i64_times_pow2(y, -beta * (S + 1))));
    return static_cast<uint64_t>(y);
  }
  const double acc = __longlong_as_double(static_cast<long long>(st));
  const double term = i64_times_pow2(dval, -beta * g);  // exact
  return static_cast<uint64_t>(__double_as_longlong(__dadd_rn(acc, term)));
}

// The kind of a diagonal's fold step: exact int64 partial while g > gx, the
// last exact step and the conversion to FP64 at g == gx, an FP64 addition
// below.  fold_kind is fold_step with the kind fixed by the caller (inline:
// the paired kernel folds 8 elements at a time with one kind per diagonal
// pair, straight-line code); on the first diagonal st is 0.
constexpr int kFoldInt = 0, kFoldConv = 1, kFoldFp = 2, kFoldNone = 3;
__device__ __forceinline__ int fold_kind_of(int g, int gx) {
  return g > gx ? kFoldInt : (g == gx ? kFoldConv : kFoldFp);
}
template <int K>
__device__ __forceinline__ uint64_t fold_kind(uint64_t st, long long d, int g, int S, int beta) {
  if constexpr (K == kFoldFp) {
    const double acc = __longlong_as_double(static_cast<long long>(st));
    return static_cast<uint64_t>(
        __double_as_longlong(__dadd_rn(acc, i64_times_pow2(d, -beta * g))));  // term exact
  } else {
    const long long y = static_cast<long long>(st) + d * (1ll << (beta * (S + 1 - g)));
    if constexpr (K == kFoldConv)
      return static_cast<uint64_t>(__double_as_longlong(i64_times_pow2(y, -beta * (S + 1))));
    else
      return static_cast<uint64_t>(y);
  }
}

// Bring the line holding p into this SM's L1 ahead of a load.
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Register split of the 384-thread slice GEMMs (setmaxnreg acts per
// warpgroup): 384 threads x 168 registers at launch = 128 x 80 (warpgroup 0) + 256 x 208
__device__ __forceinline__ void regs_dec_80() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 80;" ::: "memory");
}
__device__ __forceinline__ void regs_inc_208() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 208;" ::: "memory");
}
// The 640-thread form (16 epilogue warps): 640 threads x 96 registers at
// launch = 128 x 64 (warpgroup 0) + 512 x 104 = 61,440, all of them.
__device__ __forceinline__ void regs_dec_64() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 64;" ::: "memory");
}
__device__ __forceinline__ void regs_inc_104() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 104;" ::: "memory");
}

// Persistent slice GEMM: every CTA walks tiles blockIdx.x, +gridDim.x, ...;
// the three roles walk the same sequence and keep their pipeline state
// (stage ring, accumulator double buffer) from one tile to the next, so the
// epilogue of one tile overlaps the main loop of the next.
//
// Acc: type of the exact per-diagonal running sums (int or long long).
// window: k-blocks (stages of 8 MMAs) per accumulation window.
// Under split-k (OzSingle with splits > 1) a unit is one k range of a C
// tile and the epilogue stores each diagonal's exact D_g instead of folding.
// kFloat (BF16 comparison mode only): one slice of bf16-rounded values, the
// FP32 accumulator covers all of k in one window and is converted to FP64
// without scaling.
//
// kEpiW: epilogue warps, 8 (each of 64 columns of the tile) or 16 (each of 32
// columns; 32-bit digit sums only): with 16 the folds, which wait on tensor
// memory round trips, run on twice as many warps.
template <typename Acc, bool kFloat, typename Tiles, int kEpiW = 8>
__global__ void __launch_bounds__(128 + 32 * kEpiW, 1)
    oz_gemm_kernel(const Tiles tiles, int S, int beta, int window, int* __restrict__ status) {
  static_assert(kEpiW == 8 || (kEpiW == 16 && sizeof(Acc) == 4 && !kFloat),
                "16 epilogue warps need 32-bit digit sums");
  constexpr int kCPW = kOzTileRows / (kEpiW / 4);  // tile columns per epilogue warp
  extern __shared__ uint8_t smem_raw[];
  GemmSmem& sm = *reinterpret_cast<GemmSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int b = 0; b < 4; ++b) {
      mbar_init(&sm.accfull[b], 1);
      mbar_init(&sm.accempty[b], kEpiW);
    }
    for (int b = 0; b < kTileRing; ++b) {
      mbar_init(&sm.tfull[b], 1);
      mbar_init(&sm.tempty[b], 1 + kEpiW);
    }
    sm.abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&sm.tmem_base, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  volatile int* abort_flag = &sm.abort_flag;
  const int64_t ntiles = tiles.count();

  if (warp < 4) {  // warps 2, 3 idle
    if constexpr (kEpiW == 8) regs_dec_80(); else regs_dec_64();
  }
  if (warp == 0) {
    // ------------------------------------------------ producer (bulk copies)
    // Full tiles move as one 32 KiB copy per operand; edge tiles copy the
    // rows the MMAs read, atom by atom, and in the last k-block only the
    // atoms its MMAs reach.
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      // Publish the it-th tile of this CTA in the ring: 1 a tile, 0 the end
      // of the work, -1 a wait that gave up.  Tile it + 1 is published
      // before the copies of tile it are issued, so that its lookup (a
      // search of the problem table in a grouped call) is off the MMA
      // issuer's path.
      auto publish = [&](int64_t it) -> int {
        const int64_t t = tiles.claim(it);
        const int ts = static_cast<int>(it % kTileRing);
        if (!mbar_wait_bounded(&sm.tempty[ts], (static_cast<uint32_t>(it / kTileRing) & 1u) ^ 1u,
                               abort_flag, status))
          return -1;
        const bool live = t < ntiles;
        if (live) sm.tiles[ts] = tiles.tile(t);
        sm.tile_live[ts] = live ? 1 : 0;
        mbar_arrive(&sm.tfull[ts]);  // release: the entry is visible to its waiters
        return live ? 1 : 0;
      };
      int next = publish(0);
      for (int64_t it = 0; ok && next == 1; ++it) {
        next = publish(it + 1);
        if (next < 0) break;
        // the entry stays in place until tile it + kTileRing is published
        const OzTile& j = sm.tiles[it % kTileRing];
        const uint32_t arow_bytes = static_cast<uint32_t>(j.a_rows) * 128u;
        const uint32_t brow_bytes = static_cast<uint32_t>(j.n_eff) * 128u;
        for (int g = S + 1; g >= 2 && ok; --g) {
          for (int64_t kb = 0; kb < j.Kt && ok; ++kb) {
            const int64_t kbx = tiles.kblock(S + 1 - g, kb, j.Kt);
            const int atoms = (kbx == j.Kt - 1 && j.last_mmas <= kOzAtomK / kMmaK) ? 1 : 2;
            const bool whole = atoms == 2 && j.a_rows == kOzTileRows && j.n_eff == kOzTileRows;
            for (int s = 1; s <= g - 1; ++s) {
              if (!mbar_wait_bounded(&sm.empty[stage], phase ^ 1u, abort_flag, status)) {
                ok = false;
                break;
              }
              const uint8_t* asrc = j.a + (s - 1) * j.a_slice + kbx * kOzTileBytes;
              const uint8_t* bsrc = j.b + (g - s - 1) * j.b_slice + kbx * kOzTileBytes;
              MXM_BOUNDS(in_range(asrc, kOzTileBytes, tiles.a_begin(), tiles.a_end()), status);
              MXM_BOUNDS(in_range(bsrc, kOzTileBytes, tiles.b_begin(), tiles.b_end()), status);
              MXM_BOUNDS(j.row0 < j.m && j.col0 < j.n && kbx >= 0 && kbx < j.Kt, status);
              if (whole) {
                mbar_arrive_expect_tx(&sm.full[stage], 2 * kOzTileBytes);
                bulk_g2s(sm.a[stage], asrc, kOzTileBytes, &sm.full[stage]);
                bulk_g2s(sm.b[stage], bsrc, kOzTileBytes, &sm.full[stage]);
              } else {
                mbar_arrive_expect_tx(&sm.full[stage], atoms * (arow_bytes + brow_bytes));
                for (int at = 0; at < atoms; ++at) {
                  bulk_g2s(sm.a[stage] + at * kOzAtomBytes, asrc + at * kOzAtomBytes, arow_bytes,
                           &sm.full[stage]);
                  bulk_g2s(sm.b[stage] + at * kOzAtomBytes, bsrc + at * kOzAtomBytes, brow_bytes,
                           &sm.full[stage]);
                }
              }
              if (++stage == kStages) {
                stage = 0;
                phase ^= 1u;
              }
            }
          }
        }
      }
      // tail: let every outstanding stage be consumed (or time out) so no
      // copy or commit lands after the block has exited
      for (int i = 0; i < kStages; ++i) {
        if (!mbar_wait_bounded(&sm.empty[stage], phase ^ 1u, abort_flag, status)) break;
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    // Kept lean: one wait per stage, the tile's MMAs with precomputed
    // descriptors (stage s of the ring is s * 16 KiB further, i.e. +1024 in
    // the descriptor's address field; K steps of 16 bf16 = 32 bytes are +2),
    // N = the tile's n_eff, and windows counted in whole stages.
    if (lane == 0) {
      const uint64_t adesc0 = sw128_kmajor_desc(smem_u32(sm.a[0]));
      const uint64_t bdesc0 = sw128_kmajor_desc(smem_u32(sm.b[0]));
      int stage = 0;
      uint32_t phase = 0;
      int sc = 0;            // next accumulator slot (of four of 64 columns)
      int first = 0;         // the current window's first slot
      uint32_t uses[4] = {0u, 0u, 0u, 0u};  // windows started in each slot
      bool acquired = false;
      int wcnt = 0;
      bool ok = true;
      bool next_full = false;  // the next stage was seen full (mbar_test) during this one
      for (int64_t it = 0; ok; ++it) {
        const int ts = static_cast<int>(it % kTileRing);
        if (!mbar_wait_bounded(&sm.tfull[ts], static_cast<uint32_t>(it / kTileRing) & 1u,
                               abort_flag, status))
          break;
        if (!sm.tile_live[ts]) break;
        const OzTile j = sm.tiles[ts];
        mbar_arrive(&sm.tempty[ts]);
        const int64_t Kt = j.Kt;
        const uint32_t idesc = idesc_bf16_f32(128, j.n_eff);
        const int wslots = j.n_eff > kAccSlotCols ? 2 : 1;  // slots per window
        for (int g = S + 1; g >= 2 && ok; --g) {
          const int64_t nst = Kt * (g - 1);
          int64_t kb = 0;
          int s = 1;
          for (int64_t st = 0; st < nst; ++st) {
            if (!next_full && !mbar_wait_bounded(&sm.full[stage], phase, abort_flag, status)) {
              ok = false;
              break;
            }
            next_full = false;
            tc_fence_after();
            if (!acquired) {
              // a window of two slots starts on an even slot
              if (wslots == 2 && (sc & 1)) sc = (sc + 1) & 3;
              first = sc;
              for (int i = 0; i < wslots && ok; ++i) {
                const uint32_t u = uses[first + i];
                if (u > 0 && !mbar_wait_bounded(&sm.accempty[first + i], (u - 1u) & 1u,
                                                 abort_flag, status))
                  ok = false;
                ++uses[first + i];
              }
              if (!ok) break;
              sc = (sc + wslots) & 3;
              tc_fence_after();
              acquired = true;
              wcnt = 0;
            }
            const int nmma =
                tiles.kblock(S + 1 - g, kb, Kt) == Kt - 1 ? j.last_mmas : kMmaPerStage;
            const uint64_t da = adesc0 + static_cast<uint64_t>(stage) * (kOzTileBytes >> 4);
            const uint64_t db = bdesc0 + static_cast<uint64_t>(stage) * (kOzTileBytes >> 4);
            const uint32_t d = tmem + static_cast<uint32_t>(first * kAccSlotCols);
            MXM_BOUNDS(first * kAccSlotCols + j.n_eff <= static_cast<int>(kAccCol) && nmma >= 1 &&
                           nmma <= kMmaPerStage, status);
            const int nstage = stage + 1 == kStages ? 0 : stage + 1;
            const uint32_t nphase = stage + 1 == kStages ? phase ^ 1u : phase;
#pragma unroll
            for (int kk = 0; kk < kMmaPerStage; ++kk) {
              // k step kk: atom kk / 4 (16 KiB = +1024), 32 bytes per step inside it (+2)
              const uint64_t off = static_cast<uint64_t>((kk >> 2) * (kOzAtomBytes >> 4) + (kk & 3) * 2);
              if (kk < nmma)
                mma_bf16_ss(d, da + off, db + off, idesc, (kk > 0 || wcnt > 0) ? 1u : 0u);
              // half-way: look at the next stage while these MMAs run
              if (kk == kMmaPerStage / 2 - 1) next_full = mbar_test(&sm.full[nstage], nphase);
            }
            mma_commit(&sm.empty[stage]);
            ++wcnt;
            if (wcnt == window || st + 1 == nst) {
              mma_commit(&sm.accfull[first]);
              acquired = false;
            }
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
            }
            if (++s == g) {
              s = 1;
              ++kb;
            }
          }
        }
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------ epilogue (kEpiW warps)
    // A warp whose 32 rows all lie past the tile's last row, and a group of
    // columns past its last column, skip their tensor-memory reads and their
    // share of the fold (the running sums there are never stored).
    if constexpr (kEpiW == 8) regs_inc_208(); else regs_inc_104();
    const int ew = warp - 4;
    const int quarter = warp & 3;          // TMEM lanes this warp may access
    const int cg = ew >> 2;                // which kCPW columns of the tile
    const int row_in_tile = quarter * 32 + lane;
    const uint32_t t_lane = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
    const uint32_t t_acc = t_lane + kAccCol + static_cast<uint32_t>(cg * 2 * kCPW);
    int sc = 0;                             // next accumulator slot, as the issuer
    uint32_t fulls[4] = {0u, 0u, 0u, 0u};   // windows drained that started in each slot
    bool ok = true;
    Acc D[kCPW];
    using FInt = std::integral_constant<int, kFoldInt>;
    using FConv = std::integral_constant<int, kFoldConv>;
    using FFp = std::integral_constant<int, kFoldFp>;
    for (int64_t it = 0; ok; ++it) {
      const int ts = static_cast<int>(it % kTileRing);
      if (!mbar_wait_bounded(&sm.tfull[ts], static_cast<uint32_t>(it / kTileRing) & 1u,
                             abort_flag, status))
        break;
      if (!sm.tile_live[ts]) break;
      const OzTile j = sm.tiles[ts];
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.tempty[ts]);
      const int gx = oz_exact_from(S, beta, j.Kt);
      const bool rows_live = j.row0 + quarter * 32 < j.m;
      const int64_t row = j.row0 + row_in_tile;
      const bool row_ok = row < j.m;
      const int64_t ncols = j.n - j.col0;    // columns of C in this tile (may exceed 128)
      const int wslots = j.n_eff > kAccSlotCols ? 2 : 1;  // slots per window
      for (int g = S + 1; g >= 2 && ok; --g) {
#pragma unroll
        for (int i = 0; i < kCPW; ++i) D[i] = 0;
        const int64_t nst = j.Kt * (g - 1);
        const int64_t nwin = (nst + window - 1) / window;
        for (int64_t w = 0; w < nwin; ++w) {
          if (wslots == 2 && (sc & 1)) sc = (sc + 1) & 3;
          const int first = sc;
          sc = (sc + wslots) & 3;
          if (!mbar_wait_bounded(&sm.accfull[first], fulls[first] & 1u, abort_flag, status)) {
            ok = false;
            break;
          }
          ++fulls[first];
          tc_fence_after();
          const uint32_t t_win =
              t_lane + static_cast<uint32_t>(first * kAccSlotCols + cg * kCPW);
#pragma unroll
          for (int h = 0; h < kCPW / 32; ++h) {
            if (!rows_live || cg * kCPW + h * 32 >= j.n_eff) continue;  // warp-uniform
            uint32_t r[32];
            tmem_ld32(t_win + h * 32, r);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              if constexpr (kFloat)
                D[h * 32 + i] += static_cast<Acc>(__uint_as_float(r[i]));
              else
                D[h * 32 + i] += static_cast<Acc>(__float2int_rz(__uint_as_float(r[i])));
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0)
            for (int i = 0; i < wslots; ++i) mbar_arrive(&sm.accempty[first + i]);
        }
        if (!ok) break;
        if (!kFloat && j.partial != nullptr) {
          // split-k: this range's exact D_g, column-major in the tile (a
          // warp's 32 lanes store 256 contiguous bytes per column)
          if (!rows_live) continue;
          uint64_t* p = j.partial + static_cast<size_t>(g - 2) * (kOzTileRows * kOzTileRows) +
                        static_cast<size_t>(cg * kCPW) * kOzTileRows + row_in_tile;
#pragma unroll
          for (int i = 0; i < kCPW; ++i)
            if (cg * kCPW + i < ncols)
              __stcg(reinterpret_cast<unsigned long long*>(p + i * kOzTileRows),
                     static_cast<unsigned long long>(static_cast<long long>(D[i])));
          continue;
        }
        if (!rows_live) continue;
        const bool first = (g == S + 1);
        const bool last = (g == 2);
        int er = 0;
        if (!kFloat && last && row_ok) er = exponent_from_absbits(j.rowbits[row]);
        // E columns per step of a rolled loop (8 with 64-bit digit sums or
        // with 16 epilogue warps, 32 with 32-bit ones and 8 warps: one
        // tensor-memory round trip per 32 running sums instead of four); D is
        // rotated down by E after each step so the
        // body only names D[0..E-1] (compact code).  The kind of the fold
        // step (int64 partial, the conversion to FP64, an FP64 addition) is
        // fixed per diagonal, so the E elements of a step are straight-line
        // code.
        auto fold_pass = [&](auto kc) {
          [[maybe_unused]] constexpr int K = decltype(kc)::value;
          constexpr int E = (sizeof(Acc) == 4 && !kFloat && kEpiW == 8) ? 32 : 8;
#pragma unroll 1
          for (int ch = 0; ch < kCPW / E; ++ch) {
            if (cg * kCPW + ch * E < ncols) {  // warp-uniform
              uint32_t r[2 * E];
              if (!first) {
                if constexpr (E == 32) {
                  tmem_ld32(t_acc + ch * 64, *reinterpret_cast<uint32_t(*)[32]>(r));
                  tmem_ld32(t_acc + ch * 64 + 32, *reinterpret_cast<uint32_t(*)[32]>(r + 32));
                } else {
                  tmem_ld16(t_acc + ch * 16, r);
                }
                tmem_wait_ld();
              }
              uint64_t st[E];
#pragma unroll
              for (int i = 0; i < E; ++i) {
                if constexpr (kFloat) {
                  st[i] = static_cast<uint64_t>(__double_as_longlong(static_cast<double>(D[i])));
                } else {
                  const uint64_t prev =
                      first ? 0ull : ((static_cast<uint64_t>(r[2 * i + 1]) << 32) | r[2 * i]);
                  st[i] = fold_kind<K>(prev, static_cast<long long>(D[i]), g, S, beta);
                }
              }
              if (last) {
                if (row_ok) {
                  const int64_t col0 = j.col0 + cg * kCPW + ch * E;
                  double* crow = j.C + row * j.n;
#pragma unroll
                  for (int i = 0; i < E; ++i) {
                    const int64_t col = col0 + i;
                    if (col < j.n) {
                      if constexpr (kFloat)
                        crow[col] = __longlong_as_double(static_cast<long long>(st[i]));
                      else
                        crow[col] = final_scale(
                            st[i], er + exponent_from_absbits(j.colbits[col]) + j.eoff);
                    }
                  }
                }
              } else {
#pragma unroll
                for (int i = 0; i < E; ++i) {
                  r[2 * i] = static_cast<uint32_t>(st[i]);
                  r[2 * i + 1] = static_cast<uint32_t>(st[i] >> 32);
                }
                if constexpr (E == 32) {
                  tmem_st32(t_acc + ch * 64, *reinterpret_cast<const uint32_t(*)[32]>(r));
                  tmem_st32(t_acc + ch * 64 + 32,
                            *reinterpret_cast<const uint32_t(*)[32]>(r + 32));
                } else {
                  tmem_st16(t_acc + ch * 16, r);
                }
                tmem_wait_st();
              }
            }
#pragma unroll
            for (int i = 0; i < kCPW - E; ++i) D[i] = D[i + E];
          }
        };
        if constexpr (kFloat) {
          fold_pass(FInt{});
        } else {
          const int kind = fold_kind_of(g, gx);
          if (kind == kFoldInt) fold_pass(FInt{});
          else if (kind == kFoldConv) fold_pass(FConv{});
          else fold_pass(FFp{});
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------- steps 3-4, diagonals in pairs
// The diagonals are taken two at a time, (g, g-1).  In every k-block, step
// s = 1 .. g-1 brings one new A tile A_s and (for s <= g-2) one new B tile
// B_{g-1-s}; A_s meets B_{g-s} (diagonal g, the B tile of the previous step)
// and B_{g-1-s} (diagonal g-1).  So one A tile and one B tile per step feed
// two digit-pair products: half the operand bytes per flop of taking one
// diagonal at a time, which is what the bulk-copy feed of an SM allows.
// Four TMEM accumulators (two diagonals x double buffer, 4 x 128 columns)
// leave no room for the FP64 running sum, so the epilogue keeps it in C
// itself between diagonal pairs (read-modify-write of its own elements).
// An odd diagonal left over (g = 2 when S is odd) runs alone through the
// same code.  Warpgroup 0 (warp 0: bulk copies, warps 1-2: MMA issue) gives
// registers to warpgroups 1-2 (the epilogue: two diagonals of exact int32
// sums).
constexpr int kP2Threads = 384;
// Operand formats of the paired kernel.  Digits carried in bf16: 32 KiB
// tiles (two 64-k atoms), 8 MMAs of K = 16 per k-block, rings of 3 A and 4 B
// tiles (a B tile serves two steps: one more slot of look-ahead).  Digits
// carried in E4M3: 16 KiB tiles (one 128-k atom), 4 MMAs of K = 32, rings
// twice as deep in the same shared memory.
struct FmtBf16 {
  static constexpr bool kPair = false;
  static constexpr bool kEdges = true;   // edge tiles: n_eff, partial copies, short last k-block
  static constexpr int kTileBytes = kOzTileBytes, kBTileBytes = kOzTileBytes;
  static constexpr int kMmas = 8;
  static constexpr int kRingA = 3, kRingB = 4;
  __device__ static uint32_t idesc() { return idesc_bf16_f32(128, kOzTileRows); }
  __device__ static uint64_t koff(int kk) {  // k step kk: atom kk / 4, 32 bytes per step inside it
    return static_cast<uint64_t>((kk >> 2) * (kOzAtomBytes >> 4) + (kk & 3) * 2);
  }
  __device__ static uint64_t kboff(int kk) { return koff(kk); }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    mma_bf16_ss(d, a, b, idesc, acc);
  }
};
struct FmtE4m3 {
  static constexpr bool kPair = false;
  static constexpr bool kEdges = false;
  static constexpr int kTileBytes = kOzTileBytesE4m3, kBTileBytes = kOzTileBytesE4m3;
  static constexpr int kMmas = 4;
  static constexpr int kRingA = 6, kRingB = 8;
  __device__ static uint32_t idesc() { return idesc_e4m3_f32(128, kOzTileRows); }
  __device__ static uint64_t koff(int kk) { return static_cast<uint64_t>(kk * 2); }
  __device__ static uint64_t kboff(int kk) { return koff(kk); }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    mma_e4m3_ss(d, a, b, idesc, acc);
  }
};
// Digits carried in bf16 on a CTA pair (cta_group::2): 256 x 128 C tiles,
// each CTA with its own 128-row A tile (32 KiB) and one 64-row half of the B
// tile (16 KiB: two 8 KiB atoms along k), so an SM takes in 48 KiB per step
// instead of 64 for the same MMA work.  Rings of 4 A tiles and 6 B halves.
struct FmtBf16Pair {
  static constexpr bool kPair = true;
  static constexpr bool kEdges = false;
  static constexpr int kTileBytes = kOzTileBytes, kBTileBytes = kOzTileBytes / 2;
  static constexpr int kMmas = 8;
  static constexpr int kRingA = 4, kRingB = 6;
  __device__ static uint32_t idesc() { return idesc_bf16_f32(256, kOzTileRows); }
  __device__ static uint64_t koff(int kk) { return FmtBf16::koff(kk); }
  __device__ static uint64_t kboff(int kk) {  // B half: atoms of 64 rows, 8 KiB apart
    return static_cast<uint64_t>((kk >> 2) * ((kOzAtomBytes / 2) >> 4) + (kk & 3) * 2);
  }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    mma_bf16_ss_pair(d, a, b, idesc, acc);
  }
};
constexpr int kP2EpiWarps = 8;

template <typename Fmt>
struct __align__(1024) Gemm2Smem {
  uint8_t a[Fmt::kRingA][Fmt::kTileBytes];
  uint8_t b[Fmt::kRingB][Fmt::kBTileBytes];
  uint64_t a_full[Fmt::kRingA], a_empty[Fmt::kRingA];
  uint64_t b_full[Fmt::kRingB], b_empty[Fmt::kRingB];
  uint64_t accfull[4], accempty[4];  // accumulator 2x + buffer; x = 0: diagonal g, 1: g-1
  uint32_t tmem_base;
  int abort_flag;
};

template <typename Fmt>
constexpr size_t gemm2_smem_bytes() { return sizeof(Gemm2Smem<Fmt>) + 1024; }
// every form fits the 227 KiB of shared memory a CTA may have on this GPU
static_assert(gemm2_smem_bytes<FmtBf16>() <= 232448, "paired kernel: shared memory");
static_assert(gemm2_smem_bytes<FmtE4m3>() <= 232448, "paired kernel (E4M3): shared memory");
static_assert(gemm2_smem_bytes<FmtBf16Pair>() <= 232448, "paired kernel (pairs): shared memory");
// slots stay 1024-byte aligned for the 128-byte-swizzle descriptors
static_assert(FmtBf16Pair::kBTileBytes % 1024 == 0 && FmtBf16Pair::kTileBytes % 1024 == 0,
              "pair tiles: alignment");

// One ring of N shared-memory slots with full/empty barriers.
template <int N>
struct Ring {
  int slot = 0;
  uint32_t phase = 0;
  __device__ __forceinline__ void advance() {
    if (++slot == N) {
      slot = 0;
      phase ^= 1u;
    }
  }
};

// The fold of one diagonal g into a running sum held as 64 bits: an exact
// int64 partial (units of 2^{-beta (S+1)}) while g >= gx, an FP64 value after.
// kSpill: long k, a diagonal's int32 sums spill to an int64 area (below).
//
// kPair (FmtBf16Pair): the kernel runs on clusters of two CTAs, one per SM,
// with the MMAs of cta_group::2.  Both CTAs copy their operand tiles (rank
// r: A of tile-row 2 tp + r, half r of the B tile) and run the epilogue of
// their own 128 rows; rank 0's two issuers issue every MMA.  A tile is ready
// for rank 0 when its own copy has landed and rank 1 (warp 1, the relay)
// has seen its copy land and arrived on rank 0's full barrier; MMA commits
// arrive in both CTAs (multicast) and free the slots and windows there;
// rank 1's epilogue warps arrive on rank 0's window barriers.
template <typename Tiles, typename Fmt, bool kSpill = false>
__global__ void __launch_bounds__(kP2Threads, 1)
    oz_gemm2_kernel(const Tiles tiles, int S, int beta, int window, int* __restrict__ status) {
  constexpr int kRingA = Fmt::kRingA, kRingB = Fmt::kRingB, kTile = Fmt::kTileBytes;
  constexpr int kBTile = Fmt::kBTileBytes;
  constexpr bool kPair = Fmt::kPair;
  constexpr bool kEdges = Fmt::kEdges;
  extern __shared__ uint8_t smem_raw[];
  Gemm2Smem<Fmt>& sm = *reinterpret_cast<Gemm2Smem<Fmt>*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = kPair ? cluster_cta_rank() : 0u;
  const bool leader = rank == 0;

  if (threadIdx.x == 0) {
    const uint32_t full_count = (kPair && leader) ? 2 : 1;  // + the relay's arrival
    for (int i = 0; i < kRingA; ++i) {
      mbar_init(&sm.a_full[i], full_count);
      mbar_init(&sm.a_empty[i], 2);  // one arrival per MMA issuer
    }
    for (int i = 0; i < kRingB; ++i) {
      mbar_init(&sm.b_full[i], full_count);
      mbar_init(&sm.b_empty[i], 2);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&sm.accfull[i], 1);
      mbar_init(&sm.accempty[i], kPair ? 2 * kP2EpiWarps : kP2EpiWarps);
    }
    sm.abort_flag = 0;
    fence_mbar_init();
  }
  if constexpr (kPair) cluster_sync_all();  // barriers initialised before any peer arrives
  if (warp == 1) {
    if constexpr (kPair) {
      tmem_alloc_pair(&sm.tmem_base, kTmemCols);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(&sm.tmem_base, kTmemCols);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  volatile int* abort_flag = &sm.abort_flag;
  // work units: C tiles, or (pairs) 256-row C tiles shared by the cluster
  int64_t nunits;
  if constexpr (kPair)
    nunits = tiles.pair_count();
  else
    nunits = tiles.count();
  const int64_t unit0 = kPair ? (blockIdx.x >> 1) : blockIdx.x;
  const int64_t unit_step = kPair ? (gridDim.x >> 1) : gridDim.x;
  auto unit_tile = [&](int64_t t) {
    if constexpr (kPair)
      return tiles.pair_tile(t, rank);
    else
      return tiles.tile(t);
  };
  const int ngroups = (S + 1) / 2;

  if (warp < 4) {
    regs_dec_80();
    if (warp == 0 && lane == 0) {
      // ------------------------------------------------ producer (bulk copies)
      Ring<kRingA> ra;
      Ring<kRingB> rb;
      bool ok = true;
      // src == nullptr: nothing to copy (rank 1 past the last tile-row); the
      // slot is marked full all the same
      auto load = [&](auto& r, auto buf, uint64_t* full, uint64_t* empty, const uint8_t* src,
                      uint32_t bytes) {
        MXM_BOUNDS(src == nullptr || (full == sm.a_full
                                          ? in_range(src, bytes, tiles.a_begin(), tiles.a_end())
                                          : in_range(src, bytes, tiles.b_begin(), tiles.b_end())),
                   status);
        if (!mbar_wait_bounded(&empty[r.slot], r.phase ^ 1u, abort_flag, status))
          return false;
        if (src != nullptr) {
          mbar_arrive_expect_tx(&full[r.slot], bytes);
          bulk_g2s(buf[r.slot], src, bytes, &full[r.slot]);
        } else {
          mbar_arrive(&full[r.slot]);
        }
        r.advance();
        return true;
      };
      // edge tiles (kEdges): the rows the MMAs read, atom by atom; in the
      // last k-block only the atoms its MMAs reach
      auto load_edge = [&](auto& r, auto buf, uint64_t* full, uint64_t* empty,
                           const uint8_t* src, uint32_t row_bytes, int atoms) {
        MXM_BOUNDS(full == sm.a_full
                       ? in_range(src, kOzTileBytes, tiles.a_begin(), tiles.a_end())
                       : in_range(src, kOzTileBytes, tiles.b_begin(), tiles.b_end()),
                   status);
        if (!mbar_wait_bounded(&empty[r.slot], r.phase ^ 1u, abort_flag, status))
          return false;
        mbar_arrive_expect_tx(&full[r.slot], atoms * row_bytes);
        for (int at = 0; at < atoms; ++at)
          bulk_g2s(buf[r.slot] + at * kOzAtomBytes, src + at * kOzAtomBytes, row_bytes,
                   &full[r.slot]);
        r.advance();
        return true;
      };
      for (int64_t t = unit0; t < nunits && ok; t += unit_step) {
        const OzTile j = unit_tile(t);
        const bool live = !kPair || j.row0 < j.m;
        const size_t bhalf = kPair ? static_cast<size_t>(rank) * kBTile : 0;
        const bool edge = kEdges && (j.a_rows < kOzTileRows || j.n_eff < kOzTileRows ||
                                     j.last_mmas < Fmt::kMmas);
        for (int q = 0; q < ngroups && ok; ++q) {
          const int g = S + 1 - 2 * q;
          for (int64_t kb = 0; kb < j.Kt && ok; ++kb) {
            const int64_t kbx = tiles.kblock(q, kb, j.Kt);
            const size_t koff = static_cast<size_t>(kbx) * kTile;
            if (edge) {
              const int atoms = (kbx == j.Kt - 1 && j.last_mmas <= kOzAtomK / kMmaK) ? 1 : 2;
              const uint32_t arb = static_cast<uint32_t>(j.a_rows) * 128u;
              const uint32_t brb = static_cast<uint32_t>(j.n_eff) * 128u;
              ok = load_edge(rb, sm.b, sm.b_full, sm.b_empty, j.b + (g - 2) * j.b_slice + koff,
                             brb, atoms);
              for (int s = 1; s <= g - 1 && ok; ++s) {
                ok = load_edge(ra, sm.a, sm.a_full, sm.a_empty, j.a + (s - 1) * j.a_slice + koff,
                               arb, atoms);
                if (ok && s <= g - 2)
                  ok = load_edge(rb, sm.b, sm.b_full, sm.b_empty,
                                 j.b + (g - 2 - s) * j.b_slice + koff, brb, atoms);
              }
              continue;
            }
            ok = load(rb, sm.b, sm.b_full, sm.b_empty, j.b + (g - 2) * j.b_slice + koff + bhalf,
                      kBTile);
            for (int s = 1; s <= g - 1 && ok; ++s) {
              ok = load(ra, sm.a, sm.a_full, sm.a_empty,
                        live ? j.a + (s - 1) * j.a_slice + koff : nullptr, kTile);
              if (ok && s <= g - 2)
                ok = load(rb, sm.b, sm.b_full, sm.b_empty,
                          j.b + (g - 2 - s) * j.b_slice + koff + bhalf, kBTile);
            }
          }
        }
      }
      // tail: wait until every slot is released so no copy or commit lands
      // after the block has exited
      for (int i = 0; i < kRingA; ++i) {
        if (!mbar_wait_bounded(&sm.a_empty[ra.slot], ra.phase ^ 1u, abort_flag, status))
          break;
        ra.advance();
      }
      for (int i = 0; i < kRingB; ++i) {
        if (!mbar_wait_bounded(&sm.b_empty[rb.slot], rb.phase ^ 1u, abort_flag, status))
          break;
        rb.advance();
      }
    } else if (kPair && !leader && warp == 1 && lane == 0) {
      // ------------------------------------------------ relay (rank 1)
      // Walks the producer's sequence: when a tile of this CTA has landed,
      // arrive on the same slot's full barrier of rank 0.
      Ring<kRingA> ra;
      Ring<kRingB> rb;
      bool ok = true;
      auto relay = [&](auto& r, uint64_t* full) {
        if (!mbar_wait_bounded(&full[r.slot], r.phase, abort_flag, status)) return false;
        mbar_arrive_remote_release(smem_in_cta(&full[r.slot], 0));
        r.advance();
        return true;
      };
      for (int64_t t = unit0; t < nunits && ok; t += unit_step) {
        const int64_t Kt = unit_tile(t).Kt;
        for (int q = 0; q < ngroups && ok; ++q) {
          const int g = S + 1 - 2 * q;
          for (int64_t kb = 0; kb < Kt && ok; ++kb) {
            ok = relay(rb, sm.b_full);
            for (int s = 1; s <= g - 1 && ok; ++s) {
              ok = relay(ra, sm.a_full);
              if (ok && s <= g - 2) ok = relay(rb, sm.b_full);
            }
          }
        }
      }
    } else if ((warp == 1 || warp == 2) && lane == 0 && leader) {
      // ------------------------------------------------ MMA issuers
      // Two issuing threads: warp 1 issues the products of diagonal g (its
      // accumulators 0/1), warp 2 those of diagonal g-1 (accumulators 2/3).
      // One thread cannot issue 128 x 128 x 16 MMAs as fast as the tensor
      // core retires them; two interleave and keep it busy.  Both walk the
      // same stage sequence; every ring slot is released by two arrivals,
      // one per issuer (a commit after its MMAs, or a plain arrival for a
      // tile it does not read).  On a pair both go to both CTAs.
      const int x = warp - 1;
      uint32_t idesc = Fmt::idesc();
      int nmma = Fmt::kMmas;  // MMAs of the current k-block
      const uint64_t adesc0 = sw128_kmajor_desc(smem_u32(sm.a[0]));
      const uint64_t bdesc0 = sw128_kmajor_desc(smem_u32(sm.b[0]));
      Ring<kRingA> ra;
      Ring<kRingB> rb;
      int buf = 0, cnt = 0;
      bool acq = false;
      uint32_t uses0 = 0u, uses1 = 0u;  // windows started in this issuer's two buffers
      bool ok = true;
      // the next A / B ring slot was seen full (mbar_test) during this
      // issuer's last MMAs: its wait is skipped (the acquire fence of the
      // pair form is still taken)
      bool a_seen = false, b_seen = false;
      auto wait_full = [&](uint64_t* bars, int slot, uint32_t phase, bool& seen) -> bool {
        if (seen) {
          seen = false;
          if constexpr (kPair) fence_acquire_cluster_shared();
          return true;
        }
        return mbar_wait_bounded<false, kPair>(&bars[slot], phase, abort_flag, status);
      };
      auto commit = [&](uint64_t* bar) {
        if constexpr (kPair)
          mma_commit_pair(bar, static_cast<uint16_t>(0x3));
        else
          mma_commit(bar);
      };
      auto release = [&](uint64_t* bar) {
        mbar_arrive(bar);
        if constexpr (kPair) mbar_arrive_cluster(smem_in_cta(bar, 1));
      };
      auto acquire = [&]() {
        if (acq) return true;
        const uint32_t u = buf ? uses1 : uses0;
        const int a = 2 * x + buf;
        if (u > 0 &&
            !mbar_wait_bounded<false, kPair>(&sm.accempty[a], (u - 1u) & 1u, abort_flag, status))
          return false;
        tc_fence_after();
        if (buf) ++uses1; else ++uses0;
        acq = true;
        cnt = 0;
        return true;
      };
      auto mma8 = [&](int aslot, int bslot) {
        const uint64_t da = adesc0 + static_cast<uint64_t>(aslot) * (kTile >> 4);
        const uint64_t db = bdesc0 + static_cast<uint64_t>(bslot) * (kBTile >> 4);
        const uint32_t d = tmem + static_cast<uint32_t>((2 * x + buf) * kBN);
        MXM_BOUNDS((2 * x + buf) * kBN + kBN <= static_cast<int>(kTmemCols) && aslot < kRingA &&
                       bslot < kRingB && nmma >= 1 && nmma <= Fmt::kMmas,
                   status);
        const uint32_t acc0 = cnt > 0 ? 1u : 0u;
#pragma unroll
        for (int kk = 0; kk < Fmt::kMmas; ++kk) {
          if (!kEdges || kk < nmma)
            Fmt::mma(d, da + Fmt::koff(kk), db + Fmt::kboff(kk), idesc, kk > 0 ? 1u : acc0);
          if (kk == Fmt::kMmas / 2 - 1) {  // half-way: the slots the next waits are on
            a_seen = mbar_test<kPair>(&sm.a_full[ra.slot], ra.phase);
            b_seen = mbar_test<kPair>(&sm.b_full[rb.slot], rb.phase);
          }
        }
      };
      auto finish = [&](bool last) {
        if (++cnt == window || last) {
          commit(&sm.accfull[2 * x + buf]);
          buf ^= 1;
          acq = false;
        }
      };
      for (int64_t t = unit0; t < nunits && ok; t += unit_step) {
        const OzTile jt = unit_tile(t);
        const int64_t Kt = jt.Kt;
        if constexpr (kEdges) idesc = idesc_bf16_f32(128, jt.n_eff);
        for (int q = 0; q < ngroups && ok; ++q) {
          const int g = S + 1 - 2 * q;
          const bool pair = g - 1 >= 2;
          for (int64_t kb = 0; kb < Kt && ok; ++kb) {
            if constexpr (kEdges)
              nmma = tiles.kblock(q, kb, Kt) == Kt - 1 ? jt.last_mmas : Fmt::kMmas;
            if (!wait_full(sm.b_full, rb.slot, rb.phase, b_seen)) {
              ok = false;
              break;
            }
            int bprev = rb.slot;  // B_{g-1}: read by diagonal g only
            rb.advance();
            if (x == 1) release(&sm.b_empty[bprev]);
            for (int s = 1; s <= g - 1; ++s) {
              if (!wait_full(sm.a_full, ra.slot, ra.phase, a_seen)) {
                ok = false;
                break;
              }
              const int aslot = ra.slot;
              ra.advance();
              int bnew = -1;
              if (s <= g - 2) {
                if (!wait_full(sm.b_full, rb.slot, rb.phase, b_seen)) {
                  ok = false;
                  break;
                }
                bnew = rb.slot;
                rb.advance();
              }
              tc_fence_after();
              if (x == 0) {
                // diagonal g: A_s x B_{g-s}
                if (!acquire()) {
                  ok = false;
                  break;
                }
                mma8(aslot, bprev);
                finish(kb == Kt - 1 && s == g - 1);
                commit(&sm.a_empty[aslot]);
                commit(&sm.b_empty[bprev]);
              } else if (pair && s <= g - 2) {
                // diagonal g-1: A_s x B_{g-1-s}
                if (!acquire()) {
                  ok = false;
                  break;
                }
                mma8(aslot, bnew);
                finish(kb == Kt - 1 && s == g - 2);
                commit(&sm.a_empty[aslot]);
                commit(&sm.b_empty[bnew]);
              } else {
                release(&sm.a_empty[aslot]);
                if (bnew >= 0) release(&sm.b_empty[bnew]);
              }
              bprev = bnew;
            }
          }
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue (8 warps)
    regs_inc_208();
    const int ew = warp - 4;
    const int quarter = warp & 3;          // TMEM lanes this warp may access
    const int half = ew >> 2;              // which 64 columns of the tile
    const int row_in_tile = quarter * 32 + lane;
    const uint32_t t_lane = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
    int buf0 = 0, buf1 = 0, cnt0 = 0, cnt1 = 0;
    uint32_t fulls00 = 0u, fulls01 = 0u, fulls10 = 0u, fulls11 = 0u;
    bool ok = true;
    int D0[64], D1[64];
    // Long k: a diagonal's int32 sum is moved into this CTA's int64 spill
    // area every spill_every drains (before it could pass 2^31), and the
    // fold adds the spilled part back; the integer sum is the same.
    int nd0 = 0, nd1 = 0;
    bool sp0 = false, sp1 = false;
    long long* const spill_base =
        tiles.spill_area() + static_cast<size_t>(blockIdx.x) * 2 * kOzTileRows * kOzTileRows;
    auto spill = [&](int x, int (&Dx)[64]) {
      bool& sp = x ? sp1 : sp0;
      long long* p = spill_base + (static_cast<size_t>(x) * kOzTileRows + half * 64) * kOzTileRows +
                     row_in_tile;
#pragma unroll 1
      for (int ch = 0; ch < 8; ++ch) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          long long* q = p + static_cast<size_t>(ch * 8 + i) * kOzTileRows;
          *q = (sp ? *q : 0ll) + Dx[i];
        }
#pragma unroll
        for (int i = 0; i < 56; ++i) Dx[i] = Dx[i + 8];
#pragma unroll
        for (int i = 56; i < 64; ++i) Dx[i] = 0;
      }
      sp = true;
    };
    // edge tiles: whether this warp's 32 rows hold any row of C, and the
    // MMA columns (warp-uniform; the tile's values)
    bool warp_rows_live = true;
    int tile_neff = kOzTileRows;
    auto drain = [&](int x, int (&Dx)[64]) {
      int& b = x ? buf1 : buf0;
      uint32_t& f = x ? (b ? fulls11 : fulls10) : (b ? fulls01 : fulls00);
      const int a = 2 * x + b;
      if (!mbar_wait_bounded(&sm.accfull[a], f & 1u, abort_flag, status)) return false;
      ++f;
      tc_fence_after();
      const uint32_t t_win = t_lane + static_cast<uint32_t>(a * kBN + half * 64);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (kEdges && (!warp_rows_live || half * 64 + h * 32 >= tile_neff)) continue;
        uint32_t r[32];
        tmem_ld32(t_win + h * 32, r);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; ++i) Dx[h * 32 + i] += __float2int_rz(__uint_as_float(r[i]));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (kPair && !leader)
          mbar_arrive_remote_release(smem_in_cta(&sm.accempty[a], 0));  // the issuers are in rank 0
        else
          mbar_arrive(&sm.accempty[a]);
      }
      b ^= 1;
      if constexpr (kSpill) {
        int& nd = x ? nd1 : nd0;
        if (++nd == tiles.spill_every) {
          nd = 0;
          spill(x, Dx);
        }
      }
      return true;
    };
    for (int64_t t = unit0; t < nunits && ok; t += unit_step) {
      const OzTile j = unit_tile(t);
      // a CTA of a pair past the last tile-row drains its windows (its sums
      // are not used) and touches no memory of the product
      const bool live = !kPair || j.row0 < j.m;
      if constexpr (kEdges) {
        warp_rows_live = j.row0 + quarter * 32 < j.m;
        tile_neff = j.n_eff;
      }
      const int64_t ncols = j.n - j.col0;  // columns of C in this tile (may exceed 128)
      // diagonals g >= gx fold exactly in int64 (see oz_gemm_kernel)
      const int gx = oz_exact_from(S, beta, j.Kt);
      const int64_t row = j.row0 + row_in_tile;
      const bool row_ok = row < j.m;
      const int64_t col0 = j.col0 + half * 64;
      for (int q = 0; q < ngroups && ok; ++q) {
        const int g = S + 1 - 2 * q;
        const bool pair = g - 1 >= 2;
#pragma unroll
        for (int i = 0; i < 64; ++i) {
          D0[i] = 0;
          D1[i] = 0;
        }
        nd0 = nd1 = 0;
        sp0 = sp1 = false;
        for (int64_t kb = 0; kb < j.Kt && ok; ++kb) {
          if (kb == j.Kt - 1 && q > 0 && live && (!kEdges || warp_rows_live)) {
            // the fold at the end of this k-block reads the tile's running
            // sums: bring them into L2 while the last windows finish
            const uint64_t* ps =
                j.sums + static_cast<size_t>(half * 64) * kOzTileRows + row_in_tile;
#pragma unroll 1
            for (int i = 0; i < 64; ++i)
              if (!kEdges || half * 64 + i < ncols) prefetch_l2(ps + i * kOzTileRows);
          }
          for (int s = 1; s <= g - 1; ++s) {
            if (++cnt0 == window || (kb == j.Kt - 1 && s == g - 1)) {
              cnt0 = 0;
              if (!drain(0, D0)) {
                ok = false;
                break;
              }
            }
            if (pair && s <= g - 2) {
              if (++cnt1 == window || (kb == j.Kt - 1 && s == g - 2)) {
                cnt1 = 0;
                if (!drain(1, D1)) {
                  ok = false;
                  break;
                }
              }
            }
          }
        }
        if (!ok) break;
        if (!live) continue;
        // fold D_g (then D_{g-1}) into the running sum kept in C
        const bool first = (q == 0);
        const bool last = (g - (pair ? 1 : 0) == 2);
        int er = 0;
        if (last && row_ok) er = exponent_from_absbits(j.rowbits[row]);
        // the running sums live in the tile's column-major scratch: for each
        // column the warp's 32 lanes (32 consecutive rows) touch 256
        // contiguous bytes.  8 columns per step of a rolled loop (the next 8
        // prefetched into L1 while these fold: prefetched values held in
        // registers instead pushed the epilogue past its register budget);
        // the digit sums are rotated down by 8 after each step so the loop
        // body only names D[0..7]: a compact loop keeps the kernel inside the
        // instruction caches.  The kinds of the two fold steps are fixed per
        // diagonal pair (one loop per combination), so the 8 elements of a
        // step are independent straight-line code.  Each thread reads only
        // the sums it wrote itself.
        uint64_t* tsum = j.sums + static_cast<size_t>(half * 64) * kOzTileRows + row_in_tile;
        MXM_BOUNDS(j.sums >= tiles.sums_begin() &&
                       j.sums + kOzTileRows * kOzTileRows <= tiles.sums_end(),
                   status);
        auto fold_pass = [&](auto k0c, auto k1c) {
          constexpr int K0 = decltype(k0c)::value, K1 = decltype(k1c)::value;
          // diagonal 2 (the last) is never in the int64-only phase
          constexpr bool kMayLast =
              K1 == kFoldConv || K1 == kFoldFp || (K1 == kFoldNone && K0 != kFoldInt);
          uint64_t cur[8];
#pragma unroll 1
          for (int ch = 0; ch < 8; ++ch) {
            if (kEdges && (!warp_rows_live || half * 64 + ch * 8 >= ncols)) {
              // no row or no column of C here: nothing to fold
#pragma unroll
              for (int i = 0; i < 56; ++i) {
                D0[i] = D0[i + 8];
                D1[i] = D1[i + 8];
              }
              continue;
            }
            uint64_t* tch = tsum + static_cast<size_t>(ch * 8) * kOzTileRows;
#pragma unroll
            for (int i = 0; i < 8; ++i) cur[i] = first ? 0ull : __ldca(tch + i * kOzTileRows);
            if (ch < 7 && !first) {
#pragma unroll
              for (int i = 0; i < 8; ++i) prefetch_l1(tch + (8 + i) * kOzTileRows);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              long long d0 = D0[i], d1 = D1[i];
              if constexpr (kSpill) {
                const size_t sc =
                    static_cast<size_t>(half * 64 + ch * 8 + i) * kOzTileRows + row_in_tile;
                if (sp0) d0 += spill_base[sc];
                if (sp1) d1 += spill_base[static_cast<size_t>(kOzTileRows) * kOzTileRows + sc];
              }
              cur[i] = fold_kind<K0>(cur[i], d0, g, S, beta);
              if constexpr (K1 != kFoldNone) cur[i] = fold_kind<K1>(cur[i], d1, g - 1, S, beta);
            }
            if (kMayLast && last) {
              const int64_t cbase = col0 + ch * 8;
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int64_t col = cbase + i;
                if (row_ok && col < j.n)
                  j.C[row * j.n + col] =
                      ldexp_rn(__longlong_as_double(static_cast<long long>(cur[i])),
                               er + exponent_from_absbits(__ldg(j.colbits + col)) + j.eoff);
              }
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) __stcg(tch + i * kOzTileRows, cur[i]);
            }
#pragma unroll
            for (int i = 0; i < 56; ++i) {
              D0[i] = D0[i + 8];
              D1[i] = D1[i + 8];
            }
          }
        };
        using FInt = std::integral_constant<int, kFoldInt>;
        using FConv = std::integral_constant<int, kFoldConv>;
        using FFp = std::integral_constant<int, kFoldFp>;
        using FNone = std::integral_constant<int, kFoldNone>;
        // g > gx: int64 (g - 1 >= gx: int64 or the conversion); g == gx: the
        // conversion (g - 1: FP64); g < gx: FP64 for both
        const int k0 = fold_kind_of(g, gx);
        const int k1 = pair ? fold_kind_of(g - 1, gx) : kFoldNone;
        switch (k0 * 4 + k1) {
          case kFoldInt * 4 + kFoldInt: fold_pass(FInt{}, FInt{}); break;
          case kFoldInt * 4 + kFoldConv: fold_pass(FInt{}, FConv{}); break;
          case kFoldConv * 4 + kFoldFp: fold_pass(FConv{}, FFp{}); break;
          case kFoldFp * 4 + kFoldFp: fold_pass(FFp{}, FFp{}); break;
          case kFoldInt * 4 + kFoldNone: fold_pass(FInt{}, FNone{}); break;
          case kFoldConv * 4 + kFoldNone: fold_pass(FConv{}, FNone{}); break;
          default: fold_pass(FFp{}, FNone{}); break;  // g < gx, alone
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // pairs: neither CTA leaves (nor frees its tensor memory) while the other
  // may still arrive on its barriers or run MMAs into it
  if constexpr (kPair) cluster_sync_all();
  tc_fence_after();
  if (warp == 1) {
    if constexpr (kPair)
      tmem_dealloc_pair(tmem, kTmemCols);
    else
      tmem_dealloc(tmem, kTmemCols);
  }
}

__global__ void zero_fill_kernel(double* __restrict__ C, int64_t count) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    C[i] = 0.0;
}

}  // namespace

cudaError_t launch_ozaki_scale(const double* A, const double* B, const OzakiDims& d,
                               uint64_t* rowbits, uint64_t* colbits, int* status,
                               cudaStream_t s) {
  // A's row maxima come with its split (launch_ozaki_split) when fused
  if (d.m > 0 && !(oz_fused_a(d) && d.Kt > 0)) {
    const int warps = 8;
    const int64_t blocks = (d.m + warps - 1) / warps;
    oz_rowmax_kernel<<<static_cast<unsigned>(blocks), warps * 32, 0, s>>>(A, d.m, d.k, rowbits,
                                                                          status);
  }
  if (d.n > 0) {
    cudaError_t e = cudaMemsetAsync(colbits, 0, sizeof(uint64_t) * d.n, s);
    if (e != cudaSuccess) return e;
    if (d.k > 0) {
      dim3 grid(static_cast<unsigned>((d.n + 31) / 32),
                static_cast<unsigned>((d.k + kColRowsPerBlock - 1) / kColRowsPerBlock));
      oz_colmax_kernel<<<grid, 256, 0, s>>>(B, d.k, d.n,
                                           reinterpret_cast<unsigned long long*>(colbits), status);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_ozaki_split(const double* A, const double* B, const OzakiDims& d,
                               uint64_t* rowbits, const uint64_t* colbits,
                               uint8_t* aslices, uint8_t* bslices, int* status,
                               cudaStream_t s) {
  if (d.Kt == 0) return cudaSuccess;
  if (d.Mt > 0 && oz_fused_a(d)) {
    const size_t smem = static_cast<size_t>(d.Kt) * kOzTileK * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(oz_scale_split_a_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    oz_scale_split_a_kernel<<<static_cast<unsigned>(d.Mt * kOzTileRows), 256, smem, s>>>(
        A, d.m, d.k, rowbits, d.S, d.beta, d.Mt, d.Kt, aslices, d.rn != 0, status);
  } else if (d.Mt > 0) {
    dim3 grid(static_cast<unsigned>(d.Kt), static_cast<unsigned>(d.Mt));
    if (d.fp8)
      oz_split_a_kernel<16><<<grid, 256, 0, s>>>(A, d.m, d.k, rowbits, d.S, d.beta, d.Mt, d.Kt,
                                                 aslices, false);
    else
      oz_split_a_kernel<8><<<grid, 256, 0, s>>>(A, d.m, d.k, rowbits, d.S, d.beta, d.Mt, d.Kt,
                                                aslices, d.rn != 0);
  }
  if (d.Nt > 0) {
    dim3 grid(static_cast<unsigned>(d.Kt), static_cast<unsigned>(d.Nt));
    if (d.fp8)
      oz_split_b_kernel<16><<<grid, 256, 0, s>>>(B, d.k, d.n, colbits, d.S, d.beta, d.Nt, d.Kt,
                                                 bslices, false, false);
    else
      oz_split_b_kernel<8><<<grid, 256, 0, s>>>(B, d.k, d.n, colbits, d.S, d.beta, d.Nt, d.Kt,
                                                bslices, d.rn != 0, ozaki_b_halves(d));
  }
  return cudaGetLastError();
}

int g_sm_count = 0;

int sm_count() {
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (g_sm_count <= 0) g_sm_count = 1;
  }
  return g_sm_count;
}

template <typename Acc, bool kFloat, typename Tiles, int kEpiW = 8>
static cudaError_t launch_oz_gemm_t(const Tiles& tiles, int64_t grid, int S, int beta,
                                    int window, int* status, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  auto kern = oz_gemm_kernel<Acc, kFloat, Tiles, kEpiW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kGemmSmemBytes));
  if (e != cudaSuccess) return e;
  kern<<<static_cast<unsigned>(grid), 128 + 32 * kEpiW, kGemmSmemBytes, s>>>(tiles, S, beta,
                                                                              window, status);
  return cudaGetLastError();
}

// Split-k recombination (steps 3-4 after a split product): D_g of every C
// element is the exact int64 sum of the k ranges' partials, added in range
// order; then the fold and the final scaling of the slice GEMM's epilogue,
// with the exact phase taken from the full k.  Thread idx walks the
// elements column by column (consecutive threads: consecutive rows, i.e.
// contiguous partials in the column-major tiles).
__global__ void __launch_bounds__(256) oz_splitk_fold_kernel(
    const uint64_t* __restrict__ P, const uint64_t* __restrict__ rowbits,
    const uint64_t* __restrict__ colbits, double* __restrict__ C, int64_t m, int64_t n,
    int64_t Mt, int64_t Nt, int64_t Kt, int64_t splits, int S, int beta, int eoff) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= m * n) return;
  const int64_t col = idx / m, row = idx - (idx / m) * m;
  constexpr int64_t kTileWords = kOzTileRows * kOzTileRows;
  const int64_t tile = (row / kOzTileRows) * Nt + col / kOzTileRows;
  const uint64_t* p = P + tile * S * kTileWords + (col % kOzTileRows) * kOzTileRows +
                      row % kOzTileRows;
  const int64_t range_stride = Mt * Nt * S * kTileWords;
  const int gx = oz_exact_from(S, beta, Kt);
  uint64_t st = 0;
  for (int g = S + 1; g >= 2; --g) {
    long long dval = 0;
    const uint64_t* q = p + static_cast<int64_t>(g - 2) * kTileWords;
    for (int64_t sp = 0; sp < splits; ++sp) dval += static_cast<long long>(__ldcs(q + sp * range_stride));
    st = fold_step(st, dval, g, gx, S, beta);
  }
  C[row * n + col] = final_scale(
      st, exponent_from_absbits(rowbits[row]) + exponent_from_absbits(colbits[col]) + eoff);
}


// The paired kernel on clusters of two CTAs (cta_group::2): one cluster per
// 256 x 128 C tile at a time, as many clusters as fit (at most max_ctas / 2).
static cudaError_t launch_gemm2_pairs(const OzSingle& tiles, const OzakiDims& d,
                                      int64_t max_ctas, int window, int* status,
                                      cudaStream_t s) {
  auto kern = tiles.spill != nullptr ? oz_gemm2_kernel<OzSingle, FmtBf16Pair, true>
                                     : oz_gemm2_kernel<OzSingle, FmtBf16Pair, false>;
  const size_t kSmem = gemm2_smem_bytes<FmtBf16Pair>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kSmem));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kP2Threads, 1, 1);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(2, 1, 1);
  int clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (clusters < 1) return cudaErrorLaunchOutOfResources;
  const int64_t units = (d.Mt + 1) / 2 * d.Nt;
  int64_t pairs = units < clusters ? units : clusters;
  if (pairs > max_ctas / 2) pairs = max_ctas / 2;
  if (pairs < 1) pairs = 1;
  cfg.gridDim = dim3(static_cast<unsigned>(2 * pairs), 1, 1);
  return cudaLaunchKernelEx(&cfg, kern, tiles, d.S, d.beta, window, status);
}

cudaError_t launch_ozaki_gemm(const uint8_t* aslices, const uint8_t* bslices,
                              const uint64_t* rowbits, const uint64_t* colbits, double* C,
                              const OzakiDims& d, uint64_t* sums, int* status, cudaStream_t s) {
  if (d.Mt == 0 || d.Nt == 0) return cudaSuccess;
  const int window = ozaki_window_stages(d.beta, d.rn != 0);
  const int64_t splits = d.splits > 1 ? d.splits : 1;
  OzSingle tiles{aslices, bslices, rowbits, colbits, C,      d.m, d.n,
                 d.Mt,    d.Nt,    d.Kt,    sums,    splits, d.S,
                 static_cast<int64_t>(ozaki_tile_bytes(d))};
  tiles.eoff = d.rn ? 2 : 0;
  tiles.k = d.k;
  tiles.raster = d.raster > 0 ? d.raster : kDefaultRaster;
  tiles.kb_alt = d.kb_alt != 0;
  const int64_t count = d.Mt * d.Nt * splits;
  const int64_t grid = count < sm_count() ? count : sm_count();
  if (d.fp8) {
    // the E4M3 engine: paired kernel only (the caller checks ozaki_narrow)
    if (splits > 1 || !ozaki_narrow(d.S, d.beta, d.Kt)) return cudaErrorNotSupported;
    auto kern = oz_gemm2_kernel<OzSingle, FmtE4m3>;
    const size_t kSmem = gemm2_smem_bytes<FmtE4m3>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmem));
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), kP2Threads, kSmem, s>>>(tiles, d.S, d.beta, window,
                                                                status);
    return cudaGetLastError();
  }
  if (splits > 1) {
    // one diagonal at a time, each k range's D_g to the partials, then the fold
    cudaError_t e =
        launch_oz_gemm_t<long long, false>(tiles, grid, d.S, d.beta, window, status, s);
    if (e != cudaSuccess) return e;
    const int64_t total = d.m * d.n;
    oz_splitk_fold_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(
        sums, rowbits, colbits, C, d.m, d.n, d.Mt, d.Nt, d.Kt, splits, d.S, d.beta,
        d.rn ? 2 : 0);
    return cudaGetLastError();
  }
  // the paired kernel; when a diagonal's sum over all of k may pass int32,
  // with the spill area that follows the running sums (grid capped to it)
  int64_t g2 = grid;
  if (!ozaki_narrow(d)) {
    const double dmax = static_cast<double>(ozaki_dmax(d));
    const double per_drain = static_cast<double>(window) * kOzTileK * dmax * dmax;
    tiles.spill_every = static_cast<int>(2147483647.0 / per_drain);
    if (tiles.spill_every < 1) return cudaErrorNotSupported;
    tiles.spill = reinterpret_cast<long long*>(reinterpret_cast<uint8_t*>(sums) +
                                               align_up(ozaki_sums_bytes(d), 1024));
    if (g2 > kOzSpillCtas) g2 = kOzSpillCtas;
  }
  if (ozaki_cta2(d))
    return launch_gemm2_pairs(tiles, d, tiles.spill != nullptr ? kOzSpillCtas : INT64_MAX,
                              window, status, s);
  auto kern = tiles.spill != nullptr ? oz_gemm2_kernel<OzSingle, FmtBf16, true>
                                     : oz_gemm2_kernel<OzSingle, FmtBf16, false>;
  const size_t kSmem = gemm2_smem_bytes<FmtBf16>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kSmem));
  if (e != cudaSuccess) return e;
  kern<<<static_cast<unsigned>(g2), kP2Threads, kSmem, s>>>(tiles, d.S, d.beta, window, status);
  return cudaGetLastError();
}

cudaError_t launch_ozaki_grouped(uint8_t* ws, int S, int beta, int64_t short_kt, int* status,
                                 cudaStream_t s, bool rn) {
  const int sms = sm_count();
  oz_grouped_owner_kernel<<<sms * 2, 256, 0, s>>>(ws);
  oz_grouped_max_kernel<<<sms * 8, 256, 0, s>>>(ws, status);
  oz_grouped_split_kernel<<<sms * 3, 256, 0, s>>>(ws, S, beta, rn);  // 3 resident per SM
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const GroupedHeader* hdr = reinterpret_cast<const GroupedHeader*>(ws);
  const GroupedProblem* recs = reinterpret_cast<const GroupedProblem*>(ws + kGroupedRecordsOff);
  // long-k problems: the diagonals in pairs on single CTAs, edge tiles cut
  // to their rows and columns; the host does not see the table, so the
  // int32 sums spill to int64 when a problem's k is long enough to need it
  OzGrouped lt{hdr, recs, ws, rn ? 2 : 0, true};
  const int window = ozaki_window_stages(beta, rn);
  const double dmax = rn ? 128.0 : static_cast<double>((1 << beta) - 1);
  lt.spill_every = static_cast<int>(2147483647.0 / (static_cast<double>(window) * kOzTileK *
                                                     dmax * dmax));
  if (lt.spill_every < 1) return cudaErrorNotSupported;
  auto kern = oz_gemm2_kernel<OzGrouped, FmtBf16, true>;
  const size_t kSmem = gemm2_smem_bytes<FmtBf16>();
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(kSmem));
  if (e != cudaSuccess) return e;
  const int grid = sms < kOzSpillCtas ? sms : static_cast<int>(kOzSpillCtas);
  kern<<<grid, kP2Threads, kSmem, s>>>(lt, S, beta, window, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // short-k problems: one diagonal at a time, FP64 running sums in tensor
  // memory (64-bit window sums: any k)
  OzGrouped st{hdr, recs, ws, rn ? 2 : 0, false};
  const double dsum = static_cast<double>(S) * dmax * dmax * kOzTileK;
  if (dsum * static_cast<double>(short_kt) < 2147483647.0)  // every short tile's sums fit int32
    return launch_oz_gemm_t<int, false, OzGrouped, 16>(st, sms, S, beta, window, status, s);
  return launch_oz_gemm_t<long long, false>(st, sms, S, beta, window, status, s);
}

cudaError_t launch_bf16_gemm(const double* A, const double* B, double* C, const OzakiDims& d,
                             uint8_t* aplane, uint8_t* bplane, int* status, cudaStream_t s) {
  if (d.Mt == 0 || d.Nt == 0 || d.Kt == 0) return cudaSuccess;
  bf16_tiles_kernel<<<dim3(static_cast<unsigned>(d.Kt), static_cast<unsigned>(d.Mt)), 256, 0, s>>>(
      A, d.m, d.k, 0, d.Kt, aplane);
  bf16_tiles_kernel<<<dim3(static_cast<unsigned>(d.Kt), static_cast<unsigned>(d.Nt)), 256, 0, s>>>(
      B, d.k, d.n, 1, d.Kt, bplane);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  OzSingle tiles{aplane, bplane, nullptr, nullptr, C,       d.m, d.n, d.Mt, d.Nt,
                 d.Kt,   nullptr, 1,     1,       kOzTileBytes};
  tiles.k = d.k;
  const int64_t count = d.Mt * d.Nt;
  const int64_t grid = count < sm_count() ? count : sm_count();
  // one window covers all of k (FP32 accumulation is the mode's semantics)
  const int whole_k = static_cast<int>(d.Kt);
  return launch_oz_gemm_t<float, true>(tiles, grid, 1, 8, whole_k, status, s);
}

cudaError_t launch_zero_fill(double* C, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  zero_fill_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(C, count);
  return cudaGetLastError();
}

}  // namespace mxm

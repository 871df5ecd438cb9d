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
// integer registers, so D_g is exact over all of k, and then fold D_g into an
// FP64 running sum kept in tensor memory, in the order of step 4.
//
// Kernels: oz_rowmax / oz_colmax (step 1, HBM-bound), oz_split_a / oz_split_b
// (step 2, HBM-bound; write pre-swizzled bf16 tiles), oz_gemm (steps 3-4).
#include <cuda_runtime.h>

#include <cstdint>

#include "mxm_internal.h"
#include "ptx.cuh"

namespace mxm {
namespace {

constexpr uint64_t kAbsMask = 0x7FFFFFFFFFFFFFFFull;
constexpr uint64_t kInfBits = 0x7FF0000000000000ull;

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t w = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// ---------------------------------------------------------------- step 1
// max_l |a_il| as a bit pattern (ordering of non-negative doubles equals the
// ordering of their bit patterns; NaN patterns sort above +inf).
__global__ void oz_rowmax_kernel(const double* __restrict__ A, int64_t m, int64_t k,
                                 uint64_t* __restrict__ rowbits, int* __restrict__ status) {
  const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= m) return;
  const int lane = threadIdx.x & 31;
  const double* a = A + row * k;
  uint64_t mx = 0;
  int64_t l = lane;
  for (; l + 96 < k; l += 128) {
    uint64_t b0 = static_cast<uint64_t>(__double_as_longlong(__ldg(a + l))) & kAbsMask;
    uint64_t b1 = static_cast<uint64_t>(__double_as_longlong(__ldg(a + l + 32))) & kAbsMask;
    uint64_t b2 = static_cast<uint64_t>(__double_as_longlong(__ldg(a + l + 64))) & kAbsMask;
    uint64_t b3 = static_cast<uint64_t>(__double_as_longlong(__ldg(a + l + 96))) & kAbsMask;
    b0 = b0 > b1 ? b0 : b1;
    b2 = b2 > b3 ? b2 : b3;
    b0 = b0 > b2 ? b0 : b2;
    mx = mx > b0 ? mx : b0;
  }
  for (; l < k; l += 32) {
    uint64_t b = static_cast<uint64_t>(__double_as_longlong(__ldg(a + l))) & kAbsMask;
    mx = mx > b ? mx : b;
  }
  mx = warp_max_u64(mx);
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
  __shared__ uint64_t red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t col = static_cast<int64_t>(blockIdx.x) * 32 + tx;
  const int64_t l0 = static_cast<int64_t>(blockIdx.y) * kColRowsPerBlock;
  const int64_t l1 = l0 + kColRowsPerBlock < k ? l0 + kColRowsPerBlock : k;
  uint64_t mx = 0;
  if (col < n) {
    for (int64_t l = l0 + ty; l < l1; l += 8) {
      uint64_t b = static_cast<uint64_t>(__double_as_longlong(__ldg(B + l * n + col))) & kAbsMask;
      mx = mx > b ? mx : b;
    }
  }
  red[ty][tx] = mx;
  __syncthreads();
  if (ty == 0 && col < n) {
#pragma unroll
    for (int y = 1; y < 8; ++y) mx = mx > red[y][tx] ? mx : red[y][tx];
    atomicMax(colbits + col, static_cast<unsigned long long>(mx));
    if (mx >= kInfBits) atomicOr(status, kStatusNonFinite);
  }
}

// ---------------------------------------------------------------- step 2
// Digits of 8 consecutive k-values of one operand row, written as 16-byte
// chunks of bf16 into the pre-swizzled tile image (chunk c of tile row r at
// chunk position c ^ (r % 8)).
__device__ __forceinline__ uint32_t bf16_bits_of_digit(int d) {
  // |d| <= 255: exact in fp32 and in bf16 (at most 8 significant bits), so
  // the bf16 pattern is the top half of the fp32 pattern.
  return __float_as_uint(static_cast<float>(d)) >> 16;
}

__device__ __forceinline__ void split_chunk_store(double (&r)[8], int S, int beta,
                                                  uint8_t* dst, size_t slice_stride) {
  const double scale = pow2_normal(beta);
  for (int s = 0; s < S; ++s) {
    uint32_t packed[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      double t0 = __dmul_rn(r[j], scale);
      double t1 = __dmul_rn(r[j + 1], scale);
      int d0 = __double2int_rz(t0);
      int d1 = __double2int_rz(t1);
      r[j] = __dsub_rn(t0, static_cast<double>(d0));
      r[j + 1] = __dsub_rn(t1, static_cast<double>(d1));
      packed[j >> 1] = bf16_bits_of_digit(d0) | (bf16_bits_of_digit(d1) << 16);
    }
    *reinterpret_cast<uint4*>(dst + static_cast<size_t>(s) * slice_stride) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
}

// A (m x k, row-major) -> A_s tiles [S][Mt][Kt] of 128 x 64 bf16.
__global__ void __launch_bounds__(256) oz_split_a_kernel(
    const double* __restrict__ A, int64_t m, int64_t k, const uint64_t* __restrict__ rowbits,
    int S, int beta, int64_t Mt, int64_t Kt, uint8_t* __restrict__ aslices) {
  const int64_t tk = blockIdx.x, tm = blockIdx.y;
  const size_t slice_stride = static_cast<size_t>(Mt) * Kt * kOzTileBytes;
  uint8_t* tile = aslices + (static_cast<size_t>(tm) * Kt + tk) * kOzTileBytes;
  for (int p = threadIdx.x; p < kOzTileRows * 8; p += blockDim.x) {
    const int c = p & 7, r = p >> 3;
    const int64_t row = tm * kOzTileRows + r;
    const int64_t k0 = tk * kOzTileK + c * 8;
    double v[8];
    int e = 0;
    if (row < m) e = exponent_from_absbits(rowbits[row]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      double x = (row < m && k0 + j < k) ? __ldg(A + row * k + k0 + j) : 0.0;
      v[j] = ldexp_rn(x, -e);
    }
    split_chunk_store(v, S, beta, tile + r * 128 + ((c ^ (r & 7)) << 4), slice_stride);
  }
}

// B (k x n, row-major) -> B_t tiles [S][Nt][Kt] of 128 (columns j) x 64 (k)
// bf16, i.e. B transposed so that both MMA operands are K-major.
__global__ void __launch_bounds__(256) oz_split_b_kernel(
    const double* __restrict__ B, int64_t k, int64_t n, const uint64_t* __restrict__ colbits,
    int S, int beta, int64_t Nt, int64_t Kt, uint8_t* __restrict__ bslices) {
  const int64_t tk = blockIdx.x, tn = blockIdx.y;
  const size_t slice_stride = static_cast<size_t>(Nt) * Kt * kOzTileBytes;
  uint8_t* tile = bslices + (static_cast<size_t>(tn) * Kt + tk) * kOzTileBytes;
  for (int p = threadIdx.x; p < kOzTileRows * 8; p += blockDim.x) {
    const int c = p & 7, r = p >> 3;
    const int64_t col = tn * kOzTileRows + r;
    const int64_t k0 = tk * kOzTileK + c * 8;
    double v[8];
    int f = 0;
    if (col < n) f = exponent_from_absbits(colbits[col]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      double x = (col < n && k0 + j < k) ? __ldg(B + (k0 + j) * n + col) : 0.0;
      v[j] = ldexp_rn(x, -f);
    }
    split_chunk_store(v, S, beta, tile + r * 128 + ((c ^ (r & 7)) << 4), slice_stride);
  }
}

// ---------------------------------------------------------------- steps 3-4
constexpr int kStages = 6;
constexpr int kThreads = 320;       // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int kEpiWarps = 8;
constexpr int kBN = 128;            // MMA N (columns of the C tile)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccCol = 256;   // FP64 running sums: 2 columns per value
constexpr int kMmaK = 16;           // K per tcgen05.mma kind::f16
constexpr int kMmaPerStage = kOzTileK / kMmaK;

struct __align__(1024) GemmSmem {
  uint8_t a[kStages][kOzTileBytes];
  uint8_t b[kStages][kOzTileBytes];
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t accfull[2];
  uint64_t accempty[2];
  uint32_t tmem_base;
  int abort_flag;
};

constexpr size_t kGemmSmemBytes = sizeof(GemmSmem) + 1024;

__device__ __forceinline__ void tile_coords(int64_t tile, int64_t Mt, int64_t Nt, int64_t& tm,
                                            int64_t& tn) {
  // groups of 8 tile-rows, column-major inside a group: neighbouring CTAs
  // share A tiles and B tiles in L2
  constexpr int64_t G = 8;
  const int64_t per_group = G * Nt;
  const int64_t grp = tile / per_group;
  const int64_t first = grp * G;
  const int64_t gsz = (Mt - first) < G ? (Mt - first) : G;
  const int64_t in = tile - grp * per_group;
  tm = first + in % gsz;
  tn = in / gsz;
}

template <typename Acc>
__global__ void __launch_bounds__(kThreads, 1) oz_gemm_kernel(
    const uint8_t* __restrict__ aslices, const uint8_t* __restrict__ bslices,
    const uint64_t* __restrict__ rowbits, const uint64_t* __restrict__ colbits,
    double* __restrict__ C, int64_t m, int64_t n, int64_t Mt, int64_t Nt, int64_t Kt, int S,
    int beta, int window, int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  GemmSmem& sm = *reinterpret_cast<GemmSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  int64_t tm, tn;
  tile_coords(blockIdx.x, Mt, Nt, tm, tn);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm.accfull[b], 1);
      mbar_init(&sm.accempty[b], kEpiWarps);
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

  const size_t a_slice = static_cast<size_t>(Mt) * Kt * kOzTileBytes;
  const size_t b_slice = static_cast<size_t>(Nt) * Kt * kOzTileBytes;
  const uint8_t* a_rowtiles = aslices + static_cast<size_t>(tm) * Kt * kOzTileBytes;
  const uint8_t* b_coltiles = bslices + static_cast<size_t>(tn) * Kt * kOzTileBytes;

  if (warp == 0) {
    // ------------------------------------------------ producer (bulk copies)
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int g = S + 1; g >= 2 && ok; --g) {
        for (int64_t kb = 0; kb < Kt && ok; ++kb) {
          for (int s = 1; s <= g - 1; ++s) {
            const int t = g - s;
            if (!mbar_wait_bounded(&sm.empty[stage], phase ^ 1u, abort_flag, status)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&sm.full[stage], 2 * kOzTileBytes);
            bulk_g2s(sm.a[stage], a_rowtiles + (s - 1) * a_slice + kb * kOzTileBytes,
                     kOzTileBytes, &sm.full[stage]);
            bulk_g2s(sm.b[stage], b_coltiles + (t - 1) * b_slice + kb * kOzTileBytes,
                     kOzTileBytes, &sm.full[stage]);
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
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
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(128, kBN);
      int stage = 0;
      uint32_t phase = 0;
      int buf = 0;
      uint32_t uses0 = 0u, uses1 = 0u;  // windows started in accumulator 0 / 1
      bool acquired = false;
      int cnt = 0;
      bool ok = true;
      for (int g = S + 1; g >= 2 && ok; --g) {
        const int64_t nmma = Kt * kMmaPerStage * (g - 1);
        int64_t done = 0;
        for (int64_t kb = 0; kb < Kt && ok; ++kb) {
          for (int s = 1; s <= g - 1; ++s) {
            if (!mbar_wait_bounded(&sm.full[stage], phase, abort_flag, status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(sm.a[stage]);
            const uint32_t b_addr = smem_u32(sm.b[stage]);
#pragma unroll
            for (int kk = 0; kk < kMmaPerStage; ++kk) {
              if (!acquired) {
                const uint32_t u = buf ? uses1 : uses0;
                if (u > 0 &&
                    !mbar_wait_bounded(&sm.accempty[buf], (u - 1u) & 1u, abort_flag, status)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                if (buf) ++uses1; else ++uses0;
                acquired = true;
                cnt = 0;
              }
              mma_bf16_ss(tmem + static_cast<uint32_t>(buf * kBN),
                          sw128_kmajor_desc(a_addr + kk * 32), sw128_kmajor_desc(b_addr + kk * 32),
                          idesc, cnt > 0 ? 1u : 0u);
              ++cnt;
              ++done;
              if (cnt == window || done == nmma) {
                mma_commit(&sm.accfull[buf]);
                buf ^= 1;
                acquired = false;
              }
            }
            mma_commit(&sm.empty[stage]);
            if (!ok) break;
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue (8 warps)
    const int ew = warp - 2;
    const int quarter = warp & 3;          // TMEM lanes this warp may access
    const int half = ew >> 2;              // which 64 columns of the tile
    const int row_in_tile = quarter * 32 + lane;
    const uint32_t t_lane = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
    const uint32_t t_acc = t_lane + kAccCol + static_cast<uint32_t>(half * 128);
    int buf = 0;
    uint32_t fulls0 = 0u, fulls1 = 0u;  // windows drained from accumulator 0 / 1
    bool ok = true;
    Acc D[64];
    for (int g = S + 1; g >= 2 && ok; --g) {
#pragma unroll
      for (int i = 0; i < 64; ++i) D[i] = 0;
      const int64_t nmma = Kt * kMmaPerStage * (g - 1);
      const int64_t nwin = (nmma + window - 1) / window;
      for (int64_t w = 0; w < nwin; ++w) {
        if (!mbar_wait_bounded(&sm.accfull[buf], (buf ? fulls1 : fulls0) & 1u, abort_flag,
                               status)) {
          ok = false;
          break;
        }
        if (buf) ++fulls1; else ++fulls0;
        tc_fence_after();
        const uint32_t t_win = t_lane + static_cast<uint32_t>(buf * kBN + half * 64);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t r[32];
          tmem_ld32(t_win + h * 32, r);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 32; ++i) D[h * 32 + i] += static_cast<Acc>(__float2int_rz(__uint_as_float(r[i])));
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.accempty[buf]);
        buf ^= 1;
      }
      if (!ok) break;
      // fold D_g into the FP64 running sum: acc = acc + D_g * 2^{-beta g}
      const double wgt = pow2_normal(-beta * g);
      const bool first = (g == S + 1);
      const bool last = (g == 2);
      const int64_t row = tm * kOzTileRows + row_in_tile;
      int er = 0;
      if (last && row < m) er = exponent_from_absbits(rowbits[row]);
#pragma unroll
      for (int ch = 0; ch < 8; ++ch) {
        uint32_t r[16];
        if (!first) {
          tmem_ld16(t_acc + ch * 16, r);
          tmem_wait_ld();
        }
        double v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const double term = __dmul_rn(static_cast<double>(D[ch * 8 + i]), wgt);  // exact
          if (first) {
            v[i] = term;
          } else {
            const double prev =
                __hiloint2double(static_cast<int>(r[2 * i + 1]), static_cast<int>(r[2 * i]));
            v[i] = __dadd_rn(prev, term);
          }
        }
        if (last) {
          if (row < m) {
            const int64_t col0 = tn * kBN + half * 64 + ch * 8;
            double* crow = C + row * n;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int64_t col = col0 + i;
              if (col < n) crow[col] = ldexp_rn(v[i], er + exponent_from_absbits(colbits[col]));
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            r[2 * i] = static_cast<uint32_t>(__double2loint(v[i]));
            r[2 * i + 1] = static_cast<uint32_t>(__double2hiint(v[i]));
          }
          tmem_st16(t_acc + ch * 16, r);
          tmem_wait_st();
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
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
  if (d.m > 0) {
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
                               const uint64_t* rowbits, const uint64_t* colbits,
                               uint8_t* aslices, uint8_t* bslices, cudaStream_t s) {
  if (d.Kt == 0) return cudaSuccess;
  if (d.Mt > 0) {
    dim3 grid(static_cast<unsigned>(d.Kt), static_cast<unsigned>(d.Mt));
    oz_split_a_kernel<<<grid, 256, 0, s>>>(A, d.m, d.k, rowbits, d.S, d.beta, d.Mt, d.Kt,
                                           aslices);
  }
  if (d.Nt > 0) {
    dim3 grid(static_cast<unsigned>(d.Kt), static_cast<unsigned>(d.Nt));
    oz_split_b_kernel<<<grid, 256, 0, s>>>(B, d.k, d.n, colbits, d.S, d.beta, d.Nt, d.Kt,
                                           bslices);
  }
  return cudaGetLastError();
}

cudaError_t launch_ozaki_gemm(const uint8_t* aslices, const uint8_t* bslices,
                              const uint64_t* rowbits, const uint64_t* colbits, double* C,
                              const OzakiDims& d, int* status, cudaStream_t s) {
  if (d.Mt == 0 || d.Nt == 0) return cudaSuccess;
  const int window = ozaki_window_mmas(d.beta);
  // int32 running sums suffice while (S)(2^beta - 1)^2 * 64 Kt < 2^31
  const long long dmax = (1ll << d.beta) - 1;
  const bool narrow = static_cast<double>(d.S) * dmax * dmax * 64.0 * d.Kt < 2147483647.0;
  const int64_t tiles = d.Mt * d.Nt;
  cudaError_t e;
  if (narrow) {
    e = cudaFuncSetAttribute(oz_gemm_kernel<int>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kGemmSmemBytes));
    if (e != cudaSuccess) return e;
    oz_gemm_kernel<int><<<static_cast<unsigned>(tiles), kThreads, kGemmSmemBytes, s>>>(
        aslices, bslices, rowbits, colbits, C, d.m, d.n, d.Mt, d.Nt, d.Kt, d.S, d.beta, window,
        status);
  } else {
    e = cudaFuncSetAttribute(oz_gemm_kernel<long long>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kGemmSmemBytes));
    if (e != cudaSuccess) return e;
    oz_gemm_kernel<long long><<<static_cast<unsigned>(tiles), kThreads, kGemmSmemBytes, s>>>(
        aslices, bslices, rowbits, colbits, C, d.m, d.n, d.Mt, d.Nt, d.Kt, d.S, d.beta, window,
        status);
  }
  return cudaGetLastError();
}

cudaError_t launch_zero_fill(double* C, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  zero_fill_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(C, count);
  return cudaGetLastError();
}

}  // namespace mxm

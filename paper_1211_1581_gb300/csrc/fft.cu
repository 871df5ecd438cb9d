// fft.cu -- the mod2f transform (Sec. 3.3): the 1-D complex DFT of Eq. 1,
// F(k) = sum_n f(n) W_N^{kn}, W_N = exp(-2 pi i / N), N a power of two,
// FP64 complex data interleaved (re, im).
//
// The radix-2 decimation in frequency of Eqs. 2-3 is the butterfly of every
// stage: a block of length L becomes f_e(n) = f(n) + f(n + L/2) in its first
// half and f_o(n) = (f(n) - f(n + L/2)) W_L^n in its second; after log2 L
// stages position i holds F(bitrev(i)).  The paper's split-stream form
// (tangle once, then every stage reads even / odd streams and concatenates
// up / down streams) is a layout for stream processors; here the stages of
// one sub-transform run in a CTA's shared memory instead, and a transform
// too large for one CTA is cut in two passes over global memory (the
// "four-step" factorisation N = N1 N2, n = N2 n1 + n2, k = k1 + N1 k2):
//
//   pass 1: for every n2, the N1-point transform over n1 of x(N2 n1 + n2),
//           times the twiddle W_N^{n2 k1}, stored as Y[k1][n2];
//   pass 2: for every k1, the N2-point transform over n2 of Y[k1][.],
//           stored at X(k1 + N1 k2).
//
// A CTA takes C neighbouring columns, so every global access moves C
// consecutive complex values.  Small transforms (N <= 1024) are one pass of
// one CTA.  FP64 is scarce on this GPU (~4 G fused multiply-adds per second
// per SM): the stages go two at a time (radix 4, 28 FP64 operations per 4
// points and 2 stages against 32 for radix 2; none in the last, whose
// twiddles are 1 and -i).  Twiddles come from a caller-owned table of
// W_T^j, j < T/2, for a power of two T that N divides (one table serves
// every smaller order), expanded per CTA into shared memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "mxm.h"
#include "mxm_internal.h"

namespace mxm {

int sm_count();

namespace {

constexpr int kFftThreads = 256;
constexpr int64_t kFftMaxN = int64_t{1} << 22;
constexpr int64_t kFftSingleMax = 1024;

__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
// (a + bi)(c + di) with one rounding per component after a fused multiply-add
__device__ __forceinline__ double2 cmul(double2 a, double2 w) {
  return make_double2(fma(a.x, w.x, -(a.y * w.y)), fma(a.x, w.y, a.y * w.x));
}

__device__ __forceinline__ uint32_t bitrev(uint32_t i, int bits) {
  return bits == 0 ? 0u : __brev(i) >> (32 - bits);
}

// W_T^j for 0 <= j < T from the half table (W_T^{j + T/2} = -W_T^j).
__device__ __forceinline__ double2 table_w(const double2* __restrict__ table, int64_t T,
                                           int64_t j) {
  const int64_t h = T >> 1;
  if (j < h) return __ldg(table + j);
  const double2 w = __ldg(table + (j - h));
  return make_double2(-w.x, -w.y);
}

struct FftPass {
  const double2* src;
  double2* dst;
  const double2* table;  // W_T^j, j < T/2
  int64_t T;             // table order
  int64_t N;             // transform order
  int64_t N1, N2;        // N = N1 N2; this pass transforms along L = N1 (pass 1) or N2
  int C;                 // columns per CTA
  int stage;             // 1 or 2
};

// One CTA: C columns of an L-point transform in shared memory.
//   stage 1: column n2 = c0 + c reads x(N2 n1 + n2), n1 < L = N1; writes
//            Y[k1][n2] = Z(k1) W_N^{n2 k1} (with N2 = 1 this is the whole
//            transform, written in natural order, no twiddle);
//   stage 2: column k1 = c0 + c reads Y[k1][n2], n2 < L = N2; writes
//            X(k1 + N1 k2).
__global__ void __launch_bounds__(kFftThreads) fft_pass_kernel(const FftPass a) {
  extern __shared__ double2 sm[];
  const int C = a.C;
  const int64_t L = a.stage == 1 ? a.N1 : a.N2;
  const int64_t cols = a.stage == 1 ? a.N2 : a.N1;  // columns of this pass
  int lbits = 0;
  while ((int64_t{1} << lbits) < L) ++lbits;
  double2* data = sm;             // [C][L]
  double2* tw = sm + C * L;       // W_L^m, m < L
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * C;
  const int tid = threadIdx.x;

  // twiddles of the L-point transform: W_L^m = W_T^{m T / L}
  const int64_t tstride = a.T / (L > 0 ? L : 1);
  for (int64_t m = tid; m < L; m += kFftThreads) tw[m] = table_w(a.table, a.T, m * tstride);
  // load: C consecutive columns per row, c fastest
  for (int64_t t = tid; t < L * C; t += kFftThreads) {
    const int64_t r = t / C, c = t - r * C;
    const int64_t col = c0 + c;
    double2 v = make_double2(0.0, 0.0);
    if (col < cols) v = a.src[a.stage == 1 ? a.N2 * r + col : col * a.N2 + r];
    data[c * L + r] = v;
  }
  __syncthreads();

  // decimation-in-frequency stages two at a time (radix 4): a block of
  // length B = 4q with a_m = x(j + m q), W = W_B, j < q, becomes
  //   x(j)      = (a0 + a2) + (a1 + a3)
  //   x(j + q)  = ((a0 + a2) - (a1 + a3)) W^{2j}
  //   x(j + 2q) = ((a0 - a2) - i (a1 - a3)) W^j
  //   x(j + 3q) = ((a0 - a2) + i (a1 - a3)) W^{3j}
  // which is the two radix-2 stages of lengths B and B/2 (Eqs. 2-3) with
  // W_B^{j + q} = -i W_B^j folded in: 3 complex products per 4 points
  // instead of 4, and one barrier per two stages.  An odd stage count ends
  // with the twiddle-free radix-2 stage of length 2.
  int64_t B = L;
  for (; B >= 4; B >>= 2) {
    const int64_t q = B >> 2;
    const int64_t ts = L / B;  // W_B^m = W_L^{m L / B}
    for (int64_t t = tid; t < C * (L >> 2); t += kFftThreads) {
      const int64_t c = t / (L >> 2), u = t - c * (L >> 2);
      const int64_t grp = u / q, j = u - grp * q;
      double2* p = data + c * L + grp * B + j;
      const double2 a0 = p[0], a1 = p[q], a2 = p[2 * q], a3 = p[3 * q];
      const double2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
      const double2 s13 = cadd(a1, a3), d13 = csub(a1, a3);
      const double2 nd13 = make_double2(d13.y, -d13.x);  // -i (a1 - a3)
      p[0] = cadd(s02, s13);
      const double2 y1 = csub(s02, s13), y2 = cadd(d02, nd13), y3 = csub(d02, nd13);
      if (q == 1) {  // j = 0: every twiddle is 1
        p[q] = y1;
        p[2 * q] = y2;
        p[3 * q] = y3;
      } else {
        p[q] = cmul(y1, tw[2 * j * ts]);
        p[2 * q] = cmul(y2, tw[j * ts]);
        p[3 * q] = cmul(y3, tw[3 * j * ts]);
      }
    }
    __syncthreads();
  }
  if (B == 2) {  // the last stage, length 2: W_2^0 = 1
    for (int64_t t = tid; t < C * (L >> 1); t += kFftThreads) {
      double2* p = data + 2 * t;
      const double2 x0 = p[0], x1 = p[1];
      p[0] = cadd(x0, x1);
      p[1] = csub(x0, x1);
    }
    __syncthreads();
  }

  // store: position i of column c holds the transform at bitrev(i)
  for (int64_t t = tid; t < L * C; t += kFftThreads) {
    const int64_t kk = t / C, c = t - kk * C;
    const int64_t col = c0 + c;
    if (col >= cols) continue;
    double2 v = data[c * L + bitrev(static_cast<uint32_t>(kk), lbits)];
    if (a.stage == 1) {
      if (a.N2 > 1) {
        v = cmul(v, table_w(a.table, a.T, ((col * kk) & (a.N - 1)) * (a.T / a.N)));
        a.dst[kk * a.N2 + col] = v;  // Y[k1][n2]
      } else {
        a.dst[kk] = v;
      }
    } else {
      a.dst[col + a.N1 * kk] = v;  // X(k1 + N1 k2)
    }
  }
}

__global__ void fft_twiddle_kernel(double2* table, int64_t T) {
  const int64_t h = T >> 1;
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < h;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double s, c;
    sincospi(static_cast<double>(j) / static_cast<double>(h), &s, &c);  // angle 2 pi j / T
    table[j] = make_double2(c, -s);
  }
}

bool pow2(int64_t v) { return v >= 1 && (v & (v - 1)) == 0; }

// Columns per CTA: as many as keep at least two CTAs per SM, at most 8,
// within 96 KiB of shared memory (C columns and the L twiddles).
int fft_columns(int64_t L, int64_t cols) {
  int C = 8;
  while (C > 1 && (cols / C < 2 * static_cast<int64_t>(sm_count()) || (C * L + L) * 16 > 96 * 1024))
    C /= 2;
  return C;
}

cudaError_t launch_pass(FftPass a, cudaStream_t s) {
  const int64_t L = a.stage == 1 ? a.N1 : a.N2;
  const int64_t cols = a.stage == 1 ? a.N2 : a.N1;
  a.C = fft_columns(L, cols);
  const size_t smem = static_cast<size_t>(a.C * L + L) * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int64_t blocks = (cols + a.C - 1) / a.C;
  fft_pass_kernel<<<static_cast<unsigned>(blocks), kFftThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

}  // namespace mxm

using namespace mxm;

extern "C" int64_t mxm_fft_max_n(void) { return kFftMaxN; }

extern "C" mxm_status mxm_fft_twiddles(double* table, int64_t n, void* stream) {
  if (!pow2(n) || n > kFftMaxN) return MXM_ERR_INVALID_ARG;
  if (n < 2) return MXM_OK;  // no twiddle
  if (table == nullptr) return MXM_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(table) & 15) return MXM_ERR_ALIGNMENT;
  const int64_t h = n / 2;
  int64_t blocks = (h + 255) / 256;
  if (blocks > 4 * sm_count()) blocks = 4 * sm_count();
  fft_twiddle_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<double2*>(table), n);
  return cudaGetLastError() == cudaSuccess ? MXM_OK : MXM_ERR_CUDA;
}

extern "C" mxm_status mxm_fft(const double* in, double* out, double* work, const double* table,
                              int64_t table_n, int64_t n, void* stream) {
  if (!pow2(n) || n > kFftMaxN) return MXM_ERR_INVALID_ARG;
  if (in == nullptr || out == nullptr) return MXM_ERR_INVALID_ARG;
  if (n >= 2 && (table == nullptr || !pow2(table_n) || table_n < n || table_n > kFftMaxN))
    return MXM_ERR_INVALID_ARG;
  const bool two_pass = n > kFftSingleMax;
  if (two_pass && work == nullptr) return MXM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out) |
       reinterpret_cast<uintptr_t>(work) | reinterpret_cast<uintptr_t>(table)) & 15)
    return MXM_ERR_ALIGNMENT;
  const size_t bytes = static_cast<size_t>(n) * 16;
  const auto overlap = [](const void* p, const void* q, size_t b) {
    const auto a0 = reinterpret_cast<uintptr_t>(p), b0 = reinterpret_cast<uintptr_t>(q);
    return a0 < b0 + b && b0 < a0 + b;
  };
  // out may be in (the passes read all of their source before the next
  // pass writes); work must be apart from both; a one-pass transform
  // reads and writes the same CTA's data but must not be in place across CTAs
  if (two_pass && (overlap(work, in, bytes) || overlap(work, out, bytes)))
    return MXM_ERR_INVALID_ARG;
  if (!two_pass && in != out && overlap(in, out, bytes)) return MXM_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 1) {
    return cudaMemcpyAsync(out, in, 16, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? MXM_OK
                                                                                    : MXM_ERR_CUDA;
  }
  FftPass a;
  a.table = reinterpret_cast<const double2*>(table);
  a.T = table_n;
  a.N = n;
  a.C = 1;
  cudaError_t e;
  if (!two_pass) {
    a.src = reinterpret_cast<const double2*>(in);
    a.dst = reinterpret_cast<double2*>(out);
    a.N1 = n;
    a.N2 = 1;
    a.stage = 1;
    e = launch_pass(a, s);
  } else {
    int p = 0;
    while ((int64_t{1} << p) < n) ++p;
    a.N1 = int64_t{1} << ((p + 1) / 2);
    a.N2 = n / a.N1;
    a.src = reinterpret_cast<const double2*>(in);
    a.dst = reinterpret_cast<double2*>(work);
    a.stage = 1;
    e = launch_pass(a, s);
    if (e == cudaSuccess) {
      a.src = reinterpret_cast<const double2*>(work);
      a.dst = reinterpret_cast<double2*>(out);
      a.stage = 2;
      e = launch_pass(a, s);
    }
  }
  return e == cudaSuccess ? MXM_OK : MXM_ERR_CUDA;
}

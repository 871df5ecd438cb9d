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
constexpr int64_t kFftClusterMin = 16, kFftClusterMax = 8192;

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

// The decimation-in-frequency stages of C columns of L points in shared
// memory (data[c L + i]), two at a time (radix 4): a block of length B = 4q
// with a_m = x(j + m q), W = W_B, j < q, becomes
//   x(j)      = (a0 + a2) + (a1 + a3)
//   x(j + q)  = ((a0 + a2) - (a1 + a3)) W^{2j}
//   x(j + 2q) = ((a0 - a2) - i (a1 - a3)) W^j
//   x(j + 3q) = ((a0 - a2) + i (a1 - a3)) W^{3j}
// which is the two radix-2 stages of lengths B and B/2 (Eqs. 2-3) with
// W_B^{j + q} = -i W_B^j folded in: 3 complex products per 4 points instead
// of 4, and one barrier per two stages.  An odd stage count ends with the
// twiddle-free radix-2 stage of length 2.  tw[m] = W_L^m, m < L.  Position i
// of a column then holds its transform at bitrev(i).  All threads of the
// block call it; it ends with a barrier.
__device__ void smem_fft(double2* data, const double2* tw, int64_t L, int C) {
  const int tid = threadIdx.x, nth = blockDim.x;
  int64_t B = L;
  for (; B >= 4; B >>= 2) {
    const int64_t q = B >> 2;
    const int64_t ts = L / B;  // W_B^m = W_L^{m L / B}
    for (int64_t t = tid; t < C * (L >> 2); t += nth) {
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
    for (int64_t t = tid; t < C * (L >> 1); t += nth) {
      double2* p = data + 2 * t;
      const double2 x0 = p[0], x1 = p[1];
      p[0] = cadd(x0, x1);
      p[1] = csub(x0, x1);
    }
    __syncthreads();
  }
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

  smem_fft(data, tw, L, C);

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


// ---------------------------------------------------------------- one launch
// Transforms of up to kFftClusterMax points: both passes of the four-step
// factorisation in one launch of a thread-block cluster of C CTAs.  CTA r
// transforms the columns n2 in [r N2/C, (r + 1) N2/C) over n1, multiplies by
// W_N^{n2 k1} and writes each Y[k1][n2] straight into the shared memory of
// the CTA that owns row k1 in the second pass (rows [r N1/C, (r + 1) N1/C));
// after a cluster barrier every CTA transforms its rows over n2 and stores
// X(k1 + N1 k2).  The cluster barriers are hardware barriers; the only
// distributed-shared-memory writes come between the two, so no CTA can exit
// while a peer still writes to it.
struct FftCluster {
  const double2* src;
  double2* dst;
  const double2* table;
  int64_t T, N, N1, N2;
};

__device__ __forceinline__ uint32_t fft_cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t fft_cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void fft_cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kFftThreads) fft_cluster_kernel(const FftCluster a) {
  extern __shared__ double2 sm[];
  const int64_t N1 = a.N1, N2 = a.N2;
  const uint32_t rank = fft_cluster_rank(), C = fft_cluster_size();
  const int64_t cols = N2 / C, rows = N1 / C;  // columns of pass 1, rows of pass 2 per CTA
  double2* b1 = sm;                  // [cols][N1]
  double2* b2 = b1 + cols * N1;      // [rows][N2], written by every CTA of the cluster
  double2* tw1 = b2 + rows * N2;     // W_N1^m, m < N1
  double2* tw2 = tw1 + N1;           // W_N2^m, m < N2
  const int tid = threadIdx.x;
  for (int64_t m = tid; m < N1; m += kFftThreads) tw1[m] = table_w(a.table, a.T, m * (a.T / N1));
  for (int64_t m = tid; m < N2; m += kFftThreads) tw2[m] = table_w(a.table, a.T, m * (a.T / N2));
  const int64_t c0 = static_cast<int64_t>(rank) * cols;
  for (int64_t t = tid; t < N1 * cols; t += kFftThreads) {
    const int64_t r = t / cols, c = t - r * cols;
    b1[c * N1 + r] = a.src[N2 * r + c0 + c];
  }
  fft_cluster_barrier();  // every CTA runs (and has its tables) before any peer writes to it
  smem_fft(b1, tw1, N1, static_cast<int>(cols));
  int bits1 = 0;
  while ((int64_t{1} << bits1) < N1) ++bits1;
  // Y[k1][n2] = Z_{n2}(k1) W_N^{n2 k1}, into row k1 % rows of CTA k1 / rows
  const uint32_t b2base = static_cast<uint32_t>(__cvta_generic_to_shared(b2));
  for (int64_t t = tid; t < N1 * cols; t += kFftThreads) {
    const int64_t k1 = t / cols, c = t - k1 * cols;
    const int64_t n2 = c0 + c;
    double2 v = b1[c * N1 + bitrev(static_cast<uint32_t>(k1), bits1)];
    v = cmul(v, table_w(a.table, a.T, ((n2 * k1) & (a.N - 1)) * (a.T / a.N)));
    const uint32_t owner = static_cast<uint32_t>(k1 / rows);
    const uint32_t local = b2base + static_cast<uint32_t>(((k1 - owner * rows) * N2 + n2) * 16);
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(owner));
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(remote), "d"(v.x), "d"(v.y)
                 : "memory");
  }
  fft_cluster_barrier();
  smem_fft(b2, tw2, N2, static_cast<int>(rows));
  int bits2 = 0;
  while ((int64_t{1} << bits2) < N2) ++bits2;
  const int64_t r0 = static_cast<int64_t>(rank) * rows;
  for (int64_t t = tid; t < N2 * rows; t += kFftThreads) {
    const int64_t k2 = t / rows, c = t - k2 * rows;
    a.dst[r0 + c + N1 * k2] = b2[c * N2 + bitrev(static_cast<uint32_t>(k2), bits2)];
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

// One launch on a cluster of C CTAs (the largest power of two <= 16 that
// divides both factors), if the device can place it; cudaErrorNotSupported
// when it cannot, so that the caller takes the two-pass form.
cudaError_t launch_cluster(const FftCluster& a, cudaStream_t s) {
  int64_t C = 16;
  while (C > 1 && (a.N1 % C != 0 || a.N2 % C != 0)) C /= 2;
  for (; C >= 1; C /= 2) {
    const size_t smem = static_cast<size_t>(2 * (a.N / C) + a.N1 + a.N2) * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(fft_cluster_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (C > 8 && (e = cudaFuncSetAttribute(fft_cluster_kernel,
                                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
                     cudaSuccess)
      return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(C), 1, 1);
    cfg.blockDim = dim3(kFftThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&clusters, fft_cluster_kernel, &cfg)) != cudaSuccess)
      return e;
    if (clusters >= 1) return cudaLaunchKernelEx(&cfg, fft_cluster_kernel, a);
  }
  return cudaErrorNotSupported;
}

}  // namespace

}  // namespace mxm

using namespace mxm;

extern "C" int64_t mxm_fft_max_n(void) { return kFftMaxN; }

extern "C" mxm_status mxm_fft_twiddles(double* table, int64_t n, void* stream) {
  NvtxRange nvtx_range("mxm_fft_twiddles");
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
  NvtxRange nvtx_range("mxm_fft");
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
  int p = 0;
  while ((int64_t{1} << p) < n) ++p;
  const int64_t N1 = int64_t{1} << ((p + 1) / 2);
  cudaError_t e = cudaErrorNotSupported;
  if (n >= kFftClusterMin && n <= kFftClusterMax) {
    FftCluster c;
    c.src = reinterpret_cast<const double2*>(in);
    c.dst = reinterpret_cast<double2*>(out);
    c.table = reinterpret_cast<const double2*>(table);
    c.T = table_n;
    c.N = n;
    c.N1 = N1;
    c.N2 = n / N1;
    e = launch_cluster(c, s);
    if (e == cudaSuccess) return MXM_OK;
    if (e != cudaErrorNotSupported) return MXM_ERR_CUDA;
  }
  FftPass a;
  a.table = reinterpret_cast<const double2*>(table);
  a.T = table_n;
  a.N = n;
  a.C = 1;
  if (!two_pass) {
    a.src = reinterpret_cast<const double2*>(in);
    a.dst = reinterpret_cast<double2*>(out);
    a.N1 = n;
    a.N2 = 1;
    a.stage = 1;
    e = launch_pass(a, s);
  } else {
    a.N1 = N1;
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

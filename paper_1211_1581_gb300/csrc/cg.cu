// cg.cu -- conjugate gradients for A x = b, A symmetric positive definite in
// the 3-array CSR form of mod2as (Sec. 3.4: the textbook iteration of Fig. 6
// with the sparse product of Sec. 3.2), the whole solve in one launch.
//
// The paper's loop runs on the device: one thread-block cluster of C CTAs
// (C a power of two up to 16, from the matrix size alone, so that the
// rounding of a solve does not depend on the device) owns the system.  CTA c
// owns the rows [c n / C, (c + 1) n / C); every CTA keeps the whole search
// direction p in its shared memory (two buffers), so the sparse product
// gathers p from shared memory.  One step:
//
//   1. q = A p on the CTA's rows (lane groups of G as in the mod2as kernel);
//      the CTA's share of (p, q) goes to slot c of every CTA's table
//      (distributed shared memory); cluster barrier.
//   2. (p, q) = the C shares added in rank order (the same sum in every
//      CTA); alpha = r2 / (p, q); on the CTA's rows r -= alpha q,
//      x += alpha p; its share of (r, r) to every CTA; cluster barrier.
//   3. r2_new = the shares in rank order; beta = r2_new / r2; on the CTA's
//      rows p' = r + beta p, written into the other p buffer of every CTA;
//      cluster barrier.
//
// Every CTA computes the same scalars from the same shares in the same
// order, so every CTA takes the same branch of the loop test: the barriers
// always match, with no flag to wait on.  The cluster barriers are hardware
// barriers; nothing here spins.  A step with (p, A p) <= 0 is not taken (the
// loop ends and the breakdown bit of the device status word is set); a row
// pointer or column outside the arrays is skipped and sets the bounds bit.
// r and q live in a caller workspace of 2n doubles, x is written in place
// (x0 = 0, so r0 = p0 = b as in the paper's listing).
#include <cuda_runtime.h>

#include <cstdint>

#include "mxm.h"
#include "mxm_internal.h"

namespace mxm {

int* device_status_word();  // abi.cu

namespace {

constexpr int kCgThreads = 512;
constexpr int kCgWarps = kCgThreads / 32;
constexpr int kCgMaxCluster = 16;
constexpr int64_t kCgMaxN = 12288;  // two p buffers of 96 KiB in shared memory

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// All threads of all CTAs of the cluster; orders shared::cluster accesses.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_peer(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// Sum of one double per thread, the same order on every call: each warp's
// xor tree, then warp 0 adds the kCgWarps warp sums by another xor tree.
// Every thread receives the total.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < kCgWarps ? red[lane] : 0.0;
#pragma unroll
    for (int o = kCgWarps / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if (lane == 0) red[kCgWarps] = t;
  }
  __syncthreads();
  const double total = red[kCgWarps];
  __syncthreads();  // red is reused by the next call
  return total;
}

struct CgArgs {
  const double* vals;
  const int32_t* indx;
  const int32_t* rowp;
  const double* b;
  double* x;
  double* r;  // workspace: n
  double* q;  // workspace: n
  int64_t n, nnz;
  double stop;
  int32_t max_iters;
  int32_t* iters_out;  // device, 1
  double* r2_out;      // device, 1
  double* r2_hist;     // device, max_iters, or null
  int* status;
};

template <int G>
__global__ void __launch_bounds__(kCgThreads, 1) cg_cluster_kernel(const CgArgs a) {
  extern __shared__ double pbuf[];  // two buffers of n doubles
  __shared__ double red[kCgWarps + 1];
  __shared__ double shares[2][kCgMaxCluster];
  constexpr int kRowsPerWarp = 32 / G;
  const int64_t n = a.n;
  const uint32_t rank = cluster_rank(), C = cluster_size();
  const int64_t lo = static_cast<int64_t>(rank) * n / C;
  const int64_t hi = static_cast<int64_t>(rank + 1) * n / C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sub = lane & (G - 1), grp = lane / G;

  // x0 = 0, r0 = b on the own rows; p0 = b everywhere; r2 = (b, b), summed
  // by every CTA over all n in the same order
  double bb = 0.0;
  for (int64_t i = tid; i < n; i += kCgThreads) {
    const double bi = a.b[i];
    pbuf[i] = bi;
    bb = fma(bi, bi, bb);
  }
  for (int64_t i = lo + tid; i < hi; i += kCgThreads) {
    a.x[i] = 0.0;
    a.r[i] = a.b[i];
  }
  double r2 = block_sum(bb, red);
  cluster_barrier();  // every CTA's p buffer is filled before any peer writes into it

  const uint32_t shares_pq = smem_addr(&shares[0][rank]);
  const uint32_t shares_rr = smem_addr(&shares[1][rank]);
  bool bad = false, breakdown = false;
  int cur = 0;
  int32_t k = 0;
  while (r2 > a.stop && k < a.max_iters) {
    const double* p = pbuf + cur * n;
    double* pn = pbuf + (cur ^ 1) * n;
    // 1. q = A p on the own rows, and the CTA's share of (p, q)
    double pq = 0.0;
    for (int64_t base = lo + static_cast<int64_t>(warp) * kRowsPerWarp; base < hi;
         base += static_cast<int64_t>(kCgWarps) * kRowsPerWarp) {
      const int64_t row = base + grp;
      int64_t rb = 0, re = 0;
      if (row < hi) {
        rb = __ldg(a.rowp + row);
        re = __ldg(a.rowp + row + 1);
        if (rb < 0 || re < rb || re > a.nnz) {
          bad = true;
          re = rb;
        }
      }
      double t = 0.0;
      for (int64_t j = rb + sub; j < re; j += G) {
        const int32_t c = __ldg(a.indx + j);
        const bool ok = c >= 0 && c < n;
        bad |= !ok;
        if (ok) t = fma(__ldg(a.vals + j), p[c], t);
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
      if (row < hi && sub == 0) {
        a.q[row] = t;
        pq = fma(p[row], t, pq);
      }
    }
    pq = block_sum(pq, red);
    if (tid < static_cast<int>(C)) st_peer(peer_addr(shares_pq, tid), pq);
    cluster_barrier();
    double pAp = 0.0;
    for (uint32_t c = 0; c < C; ++c) pAp += shares[0][c];
    if (!(pAp > 0.0)) {  // the same test in every CTA
      breakdown = true;
      break;
    }
    // 2. alpha, r and x on the own rows, and the CTA's share of (r, r)
    const double alpha = r2 / pAp;
    double rr = 0.0;
    for (int64_t i = lo + tid; i < hi; i += kCgThreads) {
      const double ri = fma(-alpha, a.q[i], a.r[i]);
      a.r[i] = ri;
      a.x[i] = fma(alpha, p[i], a.x[i]);
      rr = fma(ri, ri, rr);
    }
    rr = block_sum(rr, red);
    if (tid < static_cast<int>(C)) st_peer(peer_addr(shares_rr, tid), rr);
    cluster_barrier();
    double r2_new = 0.0;
    for (uint32_t c = 0; c < C; ++c) r2_new += shares[1][c];
    // 3. beta and the next direction, broadcast to every CTA's other buffer
    const double beta = r2_new / r2;
    r2 = r2_new;
    for (int64_t i = lo + tid; i < hi; i += kCgThreads) {
      const double pi = fma(beta, p[i], a.r[i]);
      const uint32_t local = smem_addr(pn + i);
      for (uint32_t c = 0; c < C; ++c) st_peer(peer_addr(local, c), pi);
    }
    if (rank == 0 && tid == 0 && a.r2_hist != nullptr) a.r2_hist[k] = r2;
    ++k;
    cur ^= 1;
    cluster_barrier();
  }
  if (rank == 0 && tid == 0) {
    *a.iters_out = k;
    *a.r2_out = r2;
    if (breakdown) atomicOr(a.status, kStatusBreakdown);
  }
  if (bad) atomicOr(a.status, kStatusBounds);
  cluster_barrier();  // no CTA leaves while a peer may still address its shared memory
}

template <int G>
cudaError_t launch_cg_g(const CgArgs& a, int C, cudaStream_t s) {
  const size_t smem = static_cast<size_t>(2 * a.n) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(cg_cluster_kernel<G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(cg_cluster_kernel<G>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(C), 1, 1);
  cfg.blockDim = dim3(kCgThreads, 1, 1);
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
  e = cudaOccupancyMaxActiveClusters(&clusters, cg_cluster_kernel<G>, &cfg);
  if (e != cudaSuccess) return e;
  if (clusters < 1) return cudaErrorLaunchOutOfResources;
  return cudaLaunchKernelEx(&cfg, cg_cluster_kernel<G>, a);
}

}  // namespace

// Cluster size from the matrix alone: enough CTAs that each has a few
// thousand values per step (FP64 fused multiply-adds are the bound of the
// product), at least 32 rows per CTA, at most 16.
int cg_cluster_size(int64_t n, int64_t nnz) {
  int C = 1;
  while (C < kCgMaxCluster && nnz / (2 * C) >= 4096 && n / (2 * C) >= 32) C *= 2;
  return C;
}

// Lanes per row: about 8 values per lane, and enough row groups for the
// CTA's warps.
int cg_group(int64_t n, int64_t nnz, int C) {
  const double avg = n > 0 ? static_cast<double>(nnz) / static_cast<double>(n) : 0.0;
  int g = avg <= 12 ? 2 : avg <= 24 ? 4 : avg <= 96 ? 8 : avg <= 384 ? 16 : 32;
  const int64_t rows = n / C;
  while (g < 32 && rows * g < 32 * kCgWarps) g *= 2;
  return g;
}

}  // namespace mxm

using namespace mxm;

extern "C" int64_t mxm_cg_max_n(void) { return kCgMaxN; }

extern "C" size_t mxm_cg_workspace_size(int64_t n) {
  return n > 0 ? static_cast<size_t>(2 * n) * sizeof(double) : 0;
}

extern "C" mxm_status mxm_cg(const double* matvals, const int32_t* indx, const int32_t* rowp,
                             const double* b, double* x, int64_t n, int64_t nnz, double stop,
                             int32_t max_iters, double* work, int32_t* iters, double* r2,
                             double* r2_hist, void* stream) {
  if (n < 0 || nnz < 0 || max_iters < 0) return MXM_ERR_INVALID_ARG;
  if (n == 0) return MXM_ERR_INVALID_ARG;
  if (n > kCgMaxN || nnz > INT32_MAX) return MXM_ERR_UNSUPPORTED;
  if (rowp == nullptr || b == nullptr || x == nullptr || work == nullptr || iters == nullptr ||
      r2 == nullptr || (nnz > 0 && (matvals == nullptr || indx == nullptr)))
    return MXM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(matvals) | reinterpret_cast<uintptr_t>(b) |
       reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(work) |
       reinterpret_cast<uintptr_t>(r2) | reinterpret_cast<uintptr_t>(r2_hist)) & 7 ||
      (reinterpret_cast<uintptr_t>(indx) | reinterpret_cast<uintptr_t>(rowp) |
       reinterpret_cast<uintptr_t>(iters)) & 3)
    return MXM_ERR_ALIGNMENT;
  // x and the workspace must not overlap each other or the inputs read while they change
  const auto overlap = [](const void* p, size_t pb, const void* q, size_t qb) {
    const auto a0 = reinterpret_cast<uintptr_t>(p), b0 = reinterpret_cast<uintptr_t>(q);
    return a0 < b0 + qb && b0 < a0 + pb;
  };
  const size_t vb = static_cast<size_t>(n) * sizeof(double);
  if (overlap(x, vb, work, 2 * vb) || overlap(x, vb, b, vb) || overlap(work, 2 * vb, b, vb) ||
      (nnz > 0 && (overlap(x, vb, matvals, nnz * sizeof(double)) ||
                   overlap(work, 2 * vb, matvals, nnz * sizeof(double)))))
    return MXM_ERR_INVALID_ARG;
  int* status = device_status_word();
  if (status == nullptr) return MXM_ERR_CUDA;
  CgArgs a;
  a.vals = matvals;
  a.indx = indx;
  a.rowp = rowp;
  a.b = b;
  a.x = x;
  a.r = work;
  a.q = work + n;
  a.n = n;
  a.nnz = nnz;
  a.stop = stop;
  a.max_iters = max_iters;
  a.iters_out = iters;
  a.r2_out = r2;
  a.r2_hist = r2_hist;
  a.status = status;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaErrorLaunchOutOfResources;
  // the size's cluster, or a smaller one where the device cannot place it
  for (int C = cg_cluster_size(n, nnz); C >= 1 && e == cudaErrorLaunchOutOfResources; C /= 2) {
    switch (cg_group(n, nnz, C)) {
      case 2: e = launch_cg_g<2>(a, C, s); break;
      case 4: e = launch_cg_g<4>(a, C, s); break;
      case 8: e = launch_cg_g<8>(a, C, s); break;
      case 16: e = launch_cg_g<16>(a, C, s); break;
      default: e = launch_cg_g<32>(a, C, s); break;
    }
  }
  return e == cudaSuccess ? MXM_OK : MXM_ERR_CUDA;
}

// cg.cu -- conjugate gradients for A x = b, A symmetric positive definite in
// the 3-array CSR form of mod2as (Sec. 3.4: the textbook iteration of Fig. 6
// with the sparse product of Sec. 3.2), the whole solve in one launch.
//
// The paper's loop runs on the device: one thread-block cluster of C CTAs
// (C a power of two up to 16, from the matrix size alone, so that the
// rounding of a solve does not depend on the device) owns the system.  CTA c
// owns the rows [c n / C, (c + 1) n / C); every CTA keeps the whole search
// direction p in its shared memory (two buffers), so the sparse product
// gathers p from shared memory, and its own rows of q, r and x there too
// (x goes to global memory once, after the loop).  The CTA's rows of A are
// copied to shared memory at the start when the rest of it holds them, so
// that every later product streams them from there rather than from L2
// (the same values in the same order: the rounding does not change).
// One step:
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
// x0 = 0, so r0 = p0 = b as in the paper's listing.
//
// FP64 arithmetic is scarce on this GPU (a warp-wide FP64 instruction holds
// an SM sub-partition's FP64 pipe for tens of clocks), so the scalars alpha
// and beta are computed once per CTA by one thread and read from shared
// memory, and the CTA sums are trees over shared memory in which only the
// warps with work issue FP64 adds.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "mxm.h"
#include "mxm_internal.h"

namespace mxm {

int* device_status_word();  // abi.cu
size_t cg_graph_workspace_bytes(int64_t n);  // cg_graph.cu
mxm_status cg_graph_solve(const double* vals, const int32_t* indx, const int32_t* rowp,
                          const double* b, double* x, double* work, int32_t* iters, double* r2,
                          double* r2_hist, int64_t n, int64_t nnz, double stop,
                          int32_t max_iters, int* status, cudaStream_t s);

namespace {

constexpr int kCgThreads = 512;
constexpr int kCgWarps = kCgThreads / 32;
constexpr int kCgMaxCluster = 16;
constexpr int kCgBatch = 4;  // values per lane per round of the product
constexpr int64_t kCgMaxN = 12288;  // p twice (192 KiB) and 3 x 768 own rows, cluster of 16

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

// Sum of one double per thread in a fixed tree (the same order on every
// call with the same `active`): the values of threads at or beyond `active`
// must be 0 and are not added.  Pairs across halves of the smallest power
// of two >= active in shared memory down to one warp, then that warp's xor
// tree.  Every thread of warp 0 receives the total.  Only warps holding
// values issue FP64 adds: each warp-wide FP64 instruction holds its SM
// sub-partition's FP64 pipe for about 64 clocks on this GPU.
__device__ __forceinline__ double block_sum(double v, double* red, int active) {
  const int tid = threadIdx.x;
  int width = 32;
  while (width < active) width <<= 1;
  if (width > 32) {
    red[tid] = v;
    __syncthreads();
    for (int s = width / 2; s >= 32; s >>= 1) {
      if (tid < s) red[tid] += red[tid + s];
      __syncthreads();
    }
    if (tid < 32) v = red[tid];
  }
  if (tid < 32) {
    // xor butterfly over the smallest power-of-two block of lanes holding
    // values (every lane of the block gets the same sum: each level adds
    // the same two numbers in both lanes), then lane 0's to all
    int P = 1;
    while (P < active && P < 32) P <<= 1;
    for (int o = P / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = __shfl_sync(0xFFFFFFFFu, v, 0);
  }
  return v;
}

// Sum of the C shares of a cluster in rank order pairs (an xor tree over
// lanes 0..C-1 of warp 0); every thread of warp 0 receives it.
__device__ __forceinline__ double shares_sum(const double* sh, uint32_t C) {
  const int lane = threadIdx.x & 31;
  double v = lane < static_cast<int>(C) ? sh[lane] : 0.0;
  for (uint32_t o = 1; o < C; o <<= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

struct CgArgs {
  const double* vals;
  const int32_t* indx;
  const int32_t* rowp;
  const double* b;
  double* x;
  int64_t n, nnz;
  int64_t rows_cap;  // ceil(n / C): own rows of q, r, x in shared memory
  int64_t nnz_cap;   // values of the CTA's rows that fit the shared-memory copy (0: none)
  double stop;
  int32_t max_iters;
  int32_t* iters_out;  // device, 1
  double* r2_out;      // device, 1
  double* r2_hist;     // device, max_iters, or null
  int* status;
};

template <int G>
__global__ void __launch_bounds__(kCgThreads, 1) cg_cluster_kernel(const CgArgs a) {
  // dynamic shared memory: p twice (n each), then q, r, x of the own rows
  extern __shared__ double dsm[];
  __shared__ double red[kCgThreads];
  __shared__ double shares[2][kCgMaxCluster];
  __shared__ double scal[2];  // alpha or beta, and r2, written by thread 0
  __shared__ int stop_flag;   // (p, A p) <= 0, written by thread 0
  constexpr int kRowsPerWarp = 32 / G;
  const int64_t n = a.n;
  double* const qs = dsm + 2 * n;
  double* const rs = qs + a.rows_cap;
  double* const xs = rs + a.rows_cap;
  // the CTA's rows of A, copied once when they fit: the product of every
  // step then reads shared memory instead of L2
  double* const mvals = xs + a.rows_cap;
  int32_t* const mindx = reinterpret_cast<int32_t*>(mvals + a.nnz_cap);
  int32_t* const mrowp = mindx + a.nnz_cap;
  const uint32_t rank = cluster_rank(), C = cluster_size();
  const int64_t lo = static_cast<int64_t>(rank) * n / C;
  const int64_t hi = static_cast<int64_t>(rank + 1) * n / C;
  const int64_t own = hi - lo;
  const int active = own < kCgThreads ? static_cast<int>(own) : kCgThreads;  // threads with rows
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sub = lane & (G - 1), grp = lane / G;
  const int64_t jb = __ldg(a.rowp + lo), je = __ldg(a.rowp + hi);
  const bool cached = a.nnz_cap > 0 && jb >= 0 && je >= jb && je <= a.nnz && je - jb <= a.nnz_cap;
  if (cached) {  // the same for all threads of the CTA
    for (int64_t i = tid; i <= own; i += kCgThreads) {
      const int64_t v = static_cast<int64_t>(__ldg(a.rowp + lo + i)) - jb;
      mrowp[i] = static_cast<int32_t>(v < 0 ? -1 : (v > je - jb ? je - jb + 1 : v));
    }
    for (int64_t j = tid; j < je - jb; j += kCgThreads) {
      mvals[j] = __ldg(a.vals + jb + j);
      mindx[j] = __ldg(a.indx + jb + j);
    }
  }

  // x0 = 0, r0 = b on the own rows; p0 = b everywhere; r2 = (b, b), summed
  // by every CTA over all n in the same order
  double bb = 0.0;
  for (int64_t i = tid; i < n; i += kCgThreads) {
    const double bi = a.b[i];
    dsm[i] = bi;
    bb = fma(bi, bi, bb);
  }
  for (int64_t i = tid; i < own; i += kCgThreads) {
    xs[i] = 0.0;
    rs[i] = a.b[lo + i];
  }
  bb = block_sum(bb, red, kCgThreads);
  if (tid == 0) scal[1] = bb;
  cluster_barrier();  // every CTA's p buffer is filled before any peer writes into it
  double r2 = scal[1];

  const uint32_t shares_pq = smem_addr(&shares[0][rank]);
  const uint32_t shares_rr = smem_addr(&shares[1][rank]);
  bool bad = false, breakdown = false;
  int cur = 0;
  int32_t k = 0;
  while (r2 > a.stop && k < a.max_iters) {
    const double* p = dsm + cur * n;
    double* pn = dsm + (cur ^ 1) * n;
    // 1. q = A p on the own rows, then the CTA's share of (p, q)
    auto product = [&](auto in_smem) {
      constexpr bool kSm = decltype(in_smem)::value;
      const int64_t lim = kSm ? je - jb : a.nnz;
      for (int64_t base = lo + static_cast<int64_t>(warp) * kRowsPerWarp; base < hi;
           base += static_cast<int64_t>(kCgWarps) * kRowsPerWarp) {
        const int64_t row = base + grp;
        int64_t rb = 0, re = 0;
        if (row < hi) {
          if constexpr (kSm) {
            rb = mrowp[row - lo];
            re = mrowp[row - lo + 1];
          } else {
            rb = __ldg(a.rowp + row);
            re = __ldg(a.rowp + row + 1);
          }
          if (rb < 0 || re < rb || re > lim) {
            bad = true;
            re = rb;
          }
        }
        // kCgBatch values per lane per round (positions j0, j0 + G, ...):
        // the loads first, so that many are in flight, then the fused
        // multiply-adds in storage order
        double t = 0.0;
        for (int64_t j0 = rb + sub; j0 < re; j0 += G * kCgBatch) {
          int32_t c[kCgBatch];
          double v[kCgBatch];
#pragma unroll
          for (int u = 0; u < kCgBatch; ++u) {
            const int64_t j = j0 + static_cast<int64_t>(u) * G;
            if constexpr (kSm) {
              c[u] = j < re ? mindx[j] : -1;
              v[u] = j < re ? mvals[j] : 0.0;
            } else {
              c[u] = j < re ? __ldg(a.indx + j) : -1;
              v[u] = j < re ? __ldg(a.vals + j) : 0.0;
            }
          }
#pragma unroll
          for (int u = 0; u < kCgBatch; ++u) {
            const bool ok = c[u] >= 0 && c[u] < n;
            bad |= !ok && j0 + static_cast<int64_t>(u) * G < re;
            if (ok) t = fma(v[u], p[c[u]], t);
          }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
        if (row < hi && sub == 0) qs[row - lo] = t;
      }
    };
    if (cached)
      product(std::true_type{});
    else
      product(std::false_type{});
    __syncthreads();
    double pq = 0.0;
    for (int64_t i = tid; i < own; i += kCgThreads) pq = fma(p[lo + i], qs[i], pq);
    pq = block_sum(pq, red, active);
    if (tid < static_cast<int>(C)) st_peer(peer_addr(shares_pq, tid), pq);
    cluster_barrier();
    if (tid < 32) {
      const double pAp = shares_sum(shares[0], C);
      if (tid == 0) {
        stop_flag = !(pAp > 0.0);
        scal[0] = r2 / pAp;  // alpha
      }
    }
    __syncthreads();
    if (stop_flag) {  // the same in every CTA: the same shares, the same order
      breakdown = true;
      break;
    }
    const double alpha = scal[0];
    // 2. r and x on the own rows, and the CTA's share of (r, r)
    double rr = 0.0;
    for (int64_t i = tid; i < own; i += kCgThreads) {
      const double ri = fma(-alpha, qs[i], rs[i]);
      rs[i] = ri;
      xs[i] = fma(alpha, p[lo + i], xs[i]);
      rr = fma(ri, ri, rr);
    }
    rr = block_sum(rr, red, active);
    if (tid < static_cast<int>(C)) st_peer(peer_addr(shares_rr, tid), rr);
    cluster_barrier();
    if (tid < 32) {
      const double r2n = shares_sum(shares[1], C);
      if (tid == 0) {
        scal[1] = r2n;
        scal[0] = r2n / r2;  // beta
      }
    }
    __syncthreads();
    // 3. the next direction, broadcast to every CTA's other buffer
    const double beta = scal[0];
    r2 = scal[1];
    for (int64_t i = tid; i < own; i += kCgThreads) {
      const double pi = fma(beta, p[lo + i], rs[i]);
      const uint32_t local = smem_addr(pn + lo + i);
      for (uint32_t c = 0; c < C; ++c) st_peer(peer_addr(local, c), pi);
    }
    if (rank == 0 && tid == 0 && a.r2_hist != nullptr) a.r2_hist[k] = r2;
    ++k;
    cur ^= 1;
    cluster_barrier();
  }
  for (int64_t i = tid; i < own; i += kCgThreads) a.x[lo + i] = xs[i];
  if (rank == 0 && tid == 0) {
    *a.iters_out = k;
    *a.r2_out = r2;
    if (breakdown) atomicOr(a.status, kStatusBreakdown);
  }
  if (bad) atomicOr(a.status, kStatusBounds);
  cluster_barrier();  // no CTA leaves while a peer may still address its shared memory
}

// Dynamic shared memory of a CTA of a cluster of C for order n: p twice, q,
// r and x of the own rows, then (nnz_cap > 0) the copy of the CTA's rows of
// A: nnz_cap values and columns and the rows' pointers.
size_t cg_smem_bytes(int64_t n, int C, int64_t nnz_cap) {
  const int64_t rows_cap = (n + C - 1) / C;
  size_t bytes = static_cast<size_t>(2 * n + 3 * rows_cap) * sizeof(double);
  if (nnz_cap > 0)
    bytes += static_cast<size_t>(nnz_cap) * (sizeof(double) + sizeof(int32_t)) +
             static_cast<size_t>(rows_cap + 1) * sizeof(int32_t);
  return bytes;
}

template <int G>
cudaError_t launch_cg_g(CgArgs a, int C, cudaStream_t s) {
  // the copy of A takes what shared memory is left, up to the whole matrix;
  // a CTA whose rows hold more values reads them from L2 instead
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, cg_cluster_kernel<G>);
  if (e != cudaSuccess) return e;
  a.rows_cap = (a.n + C - 1) / C;
  const int64_t room = static_cast<int64_t>(optin) - static_cast<int64_t>(fa.sharedSizeBytes) -
                       static_cast<int64_t>(cg_smem_bytes(a.n, C, 0)) -
                       (a.rows_cap + 1) * static_cast<int64_t>(sizeof(int32_t));
  a.nnz_cap = room > 0 ? room / static_cast<int64_t>(sizeof(double) + sizeof(int32_t)) : 0;
  if (a.nnz_cap > a.nnz) a.nnz_cap = a.nnz;
  const size_t smem = cg_smem_bytes(a.n, C, a.nnz_cap);
  e = cudaFuncSetAttribute(cg_cluster_kernel<G>,
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

// Cluster size from the order alone (so the rounding of a solve depends on
// n and nnz only): 16 CTAs, the most FP64 pipes a cluster reaches, as long
// as each keeps 8 rows; the cluster barrier costs the same for any size.
int cg_cluster_size(int64_t n, int64_t /*nnz*/) {
  int C = kCgMaxCluster;
  while (C > 1 && n / C < 8) C /= 2;
  return C;
}

// Lanes per row: the G in {1, ..., 32} whose product step issues the
// fewest warp-wide FP64 instructions on the busiest SM sub-partition:
// a warp takes 32 / G rows per round, each round costs ceil(L / G) fused
// multiply-adds and log2(G) shuffle-adds (L the average row length), the
// CTA's 16 warps sit four to a sub-partition.  Ties go to the wider group.
// G is at least what keeps all 512 threads on rows when the CTA has fewer
// than 512 rows (the matrix streams from L2 and needs the loads of every
// lane in flight), and at least 8 for rows of 64 values or more (loads of
// consecutive values by 8 lanes fill whole 32-byte sectors).
int cg_group(int64_t n, int64_t nnz, int C) {
  const int64_t rows = (n + C - 1) / C;
  const int64_t L = n > 0 ? (nnz + n - 1) / n : 0;
  int best = 32;
  int64_t best_cost = -1;
  for (int g = 32, lg = 5; g >= 1; g /= 2, --lg) {
    const int64_t groups = (rows + (32 / g) - 1) / (32 / g);  // warp-rounds in all
    const int64_t warps = groups < kCgWarps ? groups : kCgWarps;
    const int64_t rounds = (groups + kCgWarps - 1) / kCgWarps;
    const int64_t per_warp = rounds * ((L + g - 1) / g + lg);
    const int64_t cost = (warps + 3) / 4 * per_warp;
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = g;
    }
  }
  while (best < 32 && rows * best < kCgThreads && best * 2 <= L) best *= 2;
  while (best < 8 && best * 8 <= L) best *= 2;  // long rows: 8 lanes coalesce the loads
  return best;
}

}  // namespace mxm

using namespace mxm;

extern "C" int64_t mxm_cg_max_n(void) { return kCgMaxN; }

extern "C" size_t mxm_cg_workspace_size(int64_t n) {
  return n > 0 ? cg_graph_workspace_bytes(n) : 0;
}

// Matrices whose product has more values than this go to the graph engine
// by default: one cluster's 16 SMs then spend longer on the FP64 work of a
// step than the graph engine's three launches over all SMs cost.
constexpr int64_t kCgClusterMaxNnz = 524288;

extern "C" mxm_status mxm_cg(const double* matvals, const int32_t* indx, const int32_t* rowp,
                             const double* b, double* x, int64_t n, int64_t nnz, double stop,
                             int32_t max_iters, int32_t engine, double* work, int32_t* iters,
                             double* r2, double* r2_hist, void* stream) {
  NvtxRange nvtx_range("mxm_cg");
  if (n < 0 || nnz < 0 || max_iters < 0) return MXM_ERR_INVALID_ARG;
  if (n == 0) return MXM_ERR_INVALID_ARG;
  if (engine != MXM_CG_AUTO && engine != MXM_CG_CLUSTER && engine != MXM_CG_GRAPH)
    return MXM_ERR_INVALID_ARG;
  if (nnz > INT32_MAX || n > INT32_MAX) return MXM_ERR_UNSUPPORTED;
  if (engine == MXM_CG_AUTO)
    engine = (n <= kCgMaxN && (nnz <= kCgClusterMaxNnz || work == nullptr)) ? MXM_CG_CLUSTER
                                                                           : MXM_CG_GRAPH;
  if (engine == MXM_CG_CLUSTER && n > kCgMaxN) return MXM_ERR_UNSUPPORTED;
  if (rowp == nullptr || b == nullptr || x == nullptr || iters == nullptr ||
      r2 == nullptr || (nnz > 0 && (matvals == nullptr || indx == nullptr)) ||
      (engine == MXM_CG_GRAPH && work == nullptr))
    return MXM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(matvals) | reinterpret_cast<uintptr_t>(b) |
       reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(work) |
       reinterpret_cast<uintptr_t>(r2) | reinterpret_cast<uintptr_t>(r2_hist)) & 7 ||
      (reinterpret_cast<uintptr_t>(indx) | reinterpret_cast<uintptr_t>(rowp) |
       reinterpret_cast<uintptr_t>(iters)) & 3)
    return MXM_ERR_ALIGNMENT;
  // x and the workspace must not alias what the loop reads, nor each other
  const auto overlap = [](const void* p, size_t pb, const void* q, size_t qb) {
    const auto a0 = reinterpret_cast<uintptr_t>(p), b0 = reinterpret_cast<uintptr_t>(q);
    return a0 < b0 + qb && b0 < a0 + pb;
  };
  const size_t vb = static_cast<size_t>(n) * sizeof(double);
  const size_t wb = engine == MXM_CG_GRAPH ? cg_graph_workspace_bytes(n) : 0;
  const void* outs[2] = {x, work};
  const size_t outb[2] = {vb, wb};
  for (int o = 0; o < 2; ++o) {
    if (outs[o] == nullptr || outb[o] == 0) continue;
    if (overlap(outs[o], outb[o], b, vb) ||
        (nnz > 0 && (overlap(outs[o], outb[o], matvals, nnz * sizeof(double)) ||
                     overlap(outs[o], outb[o], indx, nnz * sizeof(int32_t)))) ||
        overlap(outs[o], outb[o], rowp, static_cast<size_t>(n + 1) * sizeof(int32_t)))
      return MXM_ERR_INVALID_ARG;
  }
  if (wb > 0 && overlap(x, vb, work, wb)) return MXM_ERR_INVALID_ARG;
  int* status = device_status_word();
  if (status == nullptr) return MXM_ERR_CUDA;
  if (engine == MXM_CG_GRAPH)
    return cg_graph_solve(matvals, indx, rowp, b, x, work, iters, r2, r2_hist, n, nnz, stop,
                          max_iters, status, static_cast<cudaStream_t>(stream));
  CgArgs a;
  a.vals = matvals;
  a.indx = indx;
  a.rowp = rowp;
  a.b = b;
  a.x = x;
  a.n = n;
  a.rows_cap = n;
  a.nnz_cap = 0;
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
      case 1: e = launch_cg_g<1>(a, C, s); break;
      case 2: e = launch_cg_g<2>(a, C, s); break;
      case 4: e = launch_cg_g<4>(a, C, s); break;
      case 8: e = launch_cg_g<8>(a, C, s); break;
      case 16: e = launch_cg_g<16>(a, C, s); break;
      default: e = launch_cg_g<32>(a, C, s); break;
    }
  }
  return e == cudaSuccess ? MXM_OK : MXM_ERR_CUDA;
}

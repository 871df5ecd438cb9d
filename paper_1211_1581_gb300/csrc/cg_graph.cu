// cg_graph.cu -- conjugate gradients (Sec. 3.4) for systems too large for
// one thread-block cluster: the paper's `_while` loop is a conditional WHILE
// node of a CUDA graph, so the loop still runs without a host round trip,
// and every step is three kernels over all SMs:
//
//   cg_spmv_dot   q = A p (the mod2as lane-group product) and per-block
//                 shares of (p, q);
//   cg_update     (p, q) = the shares added in block order (the same sum in
//                 every block); alpha = r2 / (p, q); r -= alpha q,
//                 x += alpha p; per-block shares of (r, r);
//   cg_direction  r2_new = the shares in block order; beta = r2_new / r2;
//                 p = r + beta p; block 0 records r2_new and sets the loop
//                 condition r2_new > stop and k < max_iters.
//
// Before the loop, cg_init sets x = 0, r = p = b with shares of (b, b) and
// cg_start sums them and sets the first condition; after it, cg_finish
// writes the step count and the last r2.  Scalars that kernels of the same
// step both read and write (r2) alternate between two slots by step parity,
// the step counter is advanced by block 0 of cg_spmv_dot (which no other
// block of that kernel reads), so no kernel reads a value that another
// block of the same kernel writes.  The number of blocks and the lane
// groups depend on n and nnz only: the rounding of a solve does not depend
// on the device.  Built graphs are kept (per device, the last few argument
// sets) so a repeated solve costs one graph launch.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "mxm.h"
#include "mxm_internal.h"

namespace mxm {

namespace {

constexpr int kCgGThreads = 256;
constexpr int64_t kCgGMaxBlocks = 1216;  // 8 per SM of a 152-SM GB300, as a constant
constexpr int kCgGBatch = 4;

struct CgState {
  double r2v[2];  // r2 after step k is in slot k & 1; slot 0 starts with (b, b)
  int k;          // steps begun
  int brk;        // (p, A p) <= 0 met
};

struct CgWork {  // layout of the caller's workspace
  double* r;
  double* p;
  double* q;
  double* part_pq;
  double* part_rr;
  CgState* st;
};

size_t cg_graph_workspace(int64_t n) {
  return static_cast<size_t>(3 * n + 2 * kCgGMaxBlocks + 4) * sizeof(double) + 256;
}

CgWork cg_work(double* w, int64_t n) {
  CgWork c;
  c.r = w;
  c.p = w + n;
  c.q = w + 2 * n;
  c.part_pq = w + 3 * n;
  c.part_rr = c.part_pq + kCgGMaxBlocks;
  c.st = reinterpret_cast<CgState*>(c.part_rr + kCgGMaxBlocks);
  return c;
}

// Sum of one double per thread in a fixed tree; thread 0 gets the total.
__device__ __forceinline__ double block_total(double v, double* red) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (tid < 32) {
    t = tid < kCgGThreads / 32 ? red[tid] : 0.0;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
  }
  __syncthreads();
  return t;
}

// The blocks' shares added in a fixed order (thread i takes shares i, i + 256,
// ... in turn, then the tree): every block computes the same value.
__device__ __forceinline__ double shares_total(const double* part, int nb, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += kCgGThreads) v += __ldcg(part + i);
  return block_total(v, red);
}

__global__ void __launch_bounds__(kCgGThreads) cg_init_kernel(const double* __restrict__ b,
                                                             double* __restrict__ x, CgWork w,
                                                             int64_t n) {
  __shared__ double red[kCgGThreads / 32];
  double bb = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * kCgGThreads + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kCgGThreads) {
    const double bi = b[i];
    x[i] = 0.0;
    w.r[i] = bi;
    w.p[i] = bi;
    bb = fma(bi, bi, bb);
  }
  bb = block_total(bb, red);
  if (threadIdx.x == 0) w.part_rr[blockIdx.x] = bb;
}

__global__ void __launch_bounds__(kCgGThreads) cg_start_kernel(CgWork w, int nb, double stop,
                                                              int32_t max_iters,
                                                              cudaGraphConditionalHandle h) {
  __shared__ double red[kCgGThreads / 32];
  const double r2 = shares_total(w.part_rr, nb, red);
  if (threadIdx.x == 0) {
    w.st->r2v[0] = r2;
    w.st->r2v[1] = r2;
    w.st->k = 0;
    w.st->brk = 0;
    cudaGraphSetConditional(h, (r2 > stop && max_iters > 0) ? 1u : 0u);
  }
}

template <int G>
__global__ void __launch_bounds__(kCgGThreads) cg_spmv_dot_kernel(
    const double* __restrict__ vals, const int32_t* __restrict__ indx,
    const int32_t* __restrict__ rowp, CgWork w, int64_t n, int64_t nnz, int* status) {
  __shared__ double red[kCgGThreads / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0) w.st->k += 1;  // read by the later kernels only
  constexpr int kRowsPerWarp = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane & (G - 1), grp = lane / G;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kCgGThreads + threadIdx.x) >> 5;
  const int64_t warps = (static_cast<int64_t>(gridDim.x) * kCgGThreads) >> 5;
  const double* __restrict__ p = w.p;
  bool bad = false;
  double pq = 0.0;
  for (int64_t base = warp * kRowsPerWarp; base < n; base += warps * kRowsPerWarp) {
    const int64_t row = base + grp;
    int64_t rb = 0, re = 0;
    if (row < n) {
      rb = __ldg(rowp + row);
      re = __ldg(rowp + row + 1);
      if (rb < 0 || re < rb || re > nnz) {
        bad = true;
        re = rb;
      }
    }
    double t = 0.0;
    for (int64_t j0 = rb + sub; j0 < re; j0 += G * kCgGBatch) {
      int32_t c[kCgGBatch];
      double v[kCgGBatch];
#pragma unroll
      for (int u = 0; u < kCgGBatch; ++u) {
        const int64_t j = j0 + static_cast<int64_t>(u) * G;
        c[u] = j < re ? __ldg(indx + j) : -1;
        v[u] = j < re ? __ldg(vals + j) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kCgGBatch; ++u) {
        const bool ok = c[u] >= 0 && c[u] < n;
        bad |= !ok && j0 + static_cast<int64_t>(u) * G < re;
        if (ok) t = fma(v[u], __ldcg(p + c[u]), t);
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if (row < n && sub == 0) {
      w.q[row] = t;
      pq = fma(__ldcg(p + row), t, pq);
    }
  }
  pq = block_total(pq, red);
  if (threadIdx.x == 0) w.part_pq[blockIdx.x] = pq;
  if (bad) atomicOr(status, kStatusBounds);
}

__global__ void __launch_bounds__(kCgGThreads) cg_update_kernel(double* __restrict__ x, CgWork w,
                                                               int64_t n, int nb) {
  __shared__ double red[kCgGThreads / 32];
  __shared__ double alpha_s;
  __shared__ int brk_s;
  const double pAp = shares_total(w.part_pq, nb, red);
  if (threadIdx.x == 0) {
    const int k = w.st->k;
    brk_s = !(pAp > 0.0);
    alpha_s = w.st->r2v[(k - 1) & 1] / pAp;
    if (brk_s && blockIdx.x == 0) w.st->brk = 1;
  }
  __syncthreads();
  if (brk_s) return;  // the same in every block: the same shares, the same order
  const double alpha = alpha_s;
  double rr = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * kCgGThreads + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kCgGThreads) {
    const double ri = fma(-alpha, w.q[i], w.r[i]);
    w.r[i] = ri;
    x[i] = fma(alpha, w.p[i], x[i]);
    rr = fma(ri, ri, rr);
  }
  rr = block_total(rr, red);
  if (threadIdx.x == 0) w.part_rr[blockIdx.x] = rr;
}

__global__ void __launch_bounds__(kCgGThreads) cg_direction_kernel(
    CgWork w, int64_t n, int nb, double stop, int32_t max_iters, double* r2_hist,
    cudaGraphConditionalHandle h) {
  __shared__ double red[kCgGThreads / 32];
  __shared__ double beta_s;
  const int k = w.st->k;
  if (w.st->brk) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  const double r2n = shares_total(w.part_rr, nb, red);
  if (threadIdx.x == 0) beta_s = r2n / w.st->r2v[(k - 1) & 1];
  __syncthreads();
  const double beta = beta_s;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * kCgGThreads + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kCgGThreads)
    w.p[i] = fma(beta, w.p[i], w.r[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    w.st->r2v[k & 1] = r2n;  // the other slot from the one this kernel reads
    if (r2_hist != nullptr) r2_hist[k - 1] = r2n;
    cudaGraphSetConditional(h, (r2n > stop && k < max_iters) ? 1u : 0u);
  }
}

__global__ void cg_finish_kernel(CgWork w, int32_t* iters, double* r2, int* status) {
  if (threadIdx.x == 0) {
    const int done = w.st->k - w.st->brk;
    *iters = done;
    *r2 = w.st->r2v[done & 1];
    if (w.st->brk) atomicOr(status, kStatusBreakdown);
  }
}

int cg_graph_group(int64_t n, int64_t nnz) {
  const double avg = n > 0 ? static_cast<double>(nnz) / static_cast<double>(n) : 0.0;
  return avg <= 6 ? 2 : avg <= 24 ? 4 : avg <= 96 ? 8 : avg <= 384 ? 16 : 32;
}

int cg_graph_blocks(int64_t n, int64_t nnz) {
  int64_t nb = (nnz + 4095) / 4096;
  const int64_t by_rows = (n + kCgGThreads - 1) / kCgGThreads;
  if (nb < by_rows) nb = by_rows;
  if (nb > kCgGMaxBlocks) nb = kCgGMaxBlocks;
  return static_cast<int>(nb < 1 ? 1 : nb);
}

struct GraphKey {
  const void* ptr[10];
  int64_t n, nnz;
  double stop;
  int32_t max_iters;
  int device;
  bool operator==(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

struct GraphEntry {
  GraphKey key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

std::mutex g_graph_mutex;
std::vector<GraphEntry> g_graphs;  // most recent last
constexpr size_t kGraphCache = 8;

cudaError_t add_kernel(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* dep, int ndep,
                       void* func, unsigned blocks, unsigned threads, void** args) {
  cudaKernelNodeParams p = {};
  p.func = func;
  p.gridDim = dim3(blocks, 1, 1);
  p.blockDim = dim3(threads, 1, 1);
  p.sharedMemBytes = 0;
  p.kernelParams = args;
  p.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, dep, static_cast<size_t>(ndep), &p);
}

template <int G>
void* spmv_dot_func() {
  return reinterpret_cast<void*>(cg_spmv_dot_kernel<G>);
}

cudaError_t build_graph(GraphEntry& e, const double* vals, const int32_t* indx,
                        const int32_t* rowp, const double* b, double* x, double* work,
                        int32_t* iters, double* r2, double* r2_hist, int64_t n, int64_t nnz,
                        double stop, int32_t max_iters, int* status) {
  cudaError_t err = cudaGraphCreate(&e.graph, 0);
  if (err != cudaSuccess) return err;
  cudaGraphConditionalHandle h;
  if ((err = cudaGraphConditionalHandleCreate(&h, e.graph, 0, 0)) != cudaSuccess) return err;
  CgWork w = cg_work(work, n);
  int nb = cg_graph_blocks(n, nnz);
  const unsigned ub = static_cast<unsigned>(nb);
  cudaGraphNode_t n_init, n_start, n_loop, n_finish, n_spmv, n_upd, n_dir;
  void* a_init[] = {&b, &x, &w, &n};
  if ((err = add_kernel(&n_init, e.graph, nullptr, 0, reinterpret_cast<void*>(cg_init_kernel), ub,
                        kCgGThreads, a_init)) != cudaSuccess)
    return err;
  void* a_start[] = {&w, &nb, &stop, &max_iters, &h};
  if ((err = add_kernel(&n_start, e.graph, &n_init, 1, reinterpret_cast<void*>(cg_start_kernel),
                        1, kCgGThreads, a_start)) != cudaSuccess)
    return err;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if ((err = cudaGraphAddNode(&n_loop, e.graph, &n_start, nullptr, 1, &cp)) != cudaSuccess)
    return err;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  void* f_spmv = nullptr;
  switch (cg_graph_group(n, nnz)) {
    case 2: f_spmv = spmv_dot_func<2>(); break;
    case 4: f_spmv = spmv_dot_func<4>(); break;
    case 8: f_spmv = spmv_dot_func<8>(); break;
    case 16: f_spmv = spmv_dot_func<16>(); break;
    default: f_spmv = spmv_dot_func<32>(); break;
  }
  void* a_spmv[] = {&vals, &indx, &rowp, &w, &n, &nnz, &status};
  if ((err = add_kernel(&n_spmv, body, nullptr, 0, f_spmv, ub, kCgGThreads, a_spmv)) != cudaSuccess)
    return err;
  void* a_upd[] = {&x, &w, &n, &nb};
  if ((err = add_kernel(&n_upd, body, &n_spmv, 1, reinterpret_cast<void*>(cg_update_kernel), ub,
                        kCgGThreads, a_upd)) != cudaSuccess)
    return err;
  void* a_dir[] = {&w, &n, &nb, &stop, &max_iters, &r2_hist, &h};
  if ((err = add_kernel(&n_dir, body, &n_upd, 1, reinterpret_cast<void*>(cg_direction_kernel), ub,
                        kCgGThreads, a_dir)) != cudaSuccess)
    return err;
  void* a_fin[] = {&w, &iters, &r2, &status};
  if ((err = add_kernel(&n_finish, e.graph, &n_loop, 1, reinterpret_cast<void*>(cg_finish_kernel),
                        1, 32, a_fin)) != cudaSuccess)
    return err;
  return cudaGraphInstantiate(&e.exec, e.graph, 0);
}

void destroy(GraphEntry& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.graph) cudaGraphDestroy(e.graph);
  e.exec = nullptr;
  e.graph = nullptr;
}

}  // namespace

size_t cg_graph_workspace_bytes(int64_t n) { return cg_graph_workspace(n); }

// One solve by the graph engine (arguments checked by the caller).
mxm_status cg_graph_solve(const double* vals, const int32_t* indx, const int32_t* rowp,
                          const double* b, double* x, double* work, int32_t* iters, double* r2,
                          double* r2_hist, int64_t n, int64_t nnz, double stop,
                          int32_t max_iters, int* status, cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return MXM_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return MXM_ERR_UNSUPPORTED;
  GraphKey key;
  std::memset(&key, 0, sizeof(key));
  const void* ptrs[10] = {vals, indx, rowp, b, x, work, iters, r2, r2_hist, status};
  for (int i = 0; i < 10; ++i) key.ptr[i] = ptrs[i];
  key.n = n;
  key.nnz = nnz;
  key.stop = stop;
  key.max_iters = max_iters;
  if (cudaGetDevice(&key.device) != cudaSuccess) return MXM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_graph_mutex);
  GraphEntry* use = nullptr;
  for (size_t i = 0; i < g_graphs.size(); ++i)
    if (g_graphs[i].key == key) {
      GraphEntry hit = g_graphs[i];
      g_graphs.erase(g_graphs.begin() + static_cast<std::ptrdiff_t>(i));
      g_graphs.push_back(hit);
      use = &g_graphs.back();
      break;
    }
  if (use == nullptr) {
    GraphEntry e;
    e.key = key;
    if (build_graph(e, vals, indx, rowp, b, x, work, iters, r2, r2_hist, n, nnz, stop, max_iters,
                    status) != cudaSuccess) {
      destroy(e);
      return MXM_ERR_CUDA;
    }
    if (g_graphs.size() == kGraphCache) {
      destroy(g_graphs.front());
      g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back(e);
    use = &g_graphs.back();
  }
  return cudaGraphLaunch(use->exec, s) == cudaSuccess ? MXM_OK : MXM_ERR_CUDA;
}

}  // namespace mxm

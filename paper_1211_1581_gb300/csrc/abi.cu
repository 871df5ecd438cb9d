// abi.cu -- the C ABI of libmxm.so (declared in include/mxm.h): argument
// checks, per-device workspace and status word, and the launch sequences of
// each mode.  No arithmetic of the product happens here.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "mxm.h"
#include "mxm_internal.h"
#include "ptx.cuh"

namespace mxm {

// Sticky status word of each device (bits kStatus*), OR-ed by kernels.
static __device__ int g_device_status;

namespace {

constexpr int kMaxDevices = 64;

struct DeviceState {
  bool init = false;
  int* status = nullptr;       // device address of g_device_status
  void* ws = nullptr;          // workspace base
  size_t ws_bytes = 0;
  bool ws_owned = true;        // allocated by the library
  int sm_count = 0;
};

std::mutex g_mutex;
DeviceState g_dev[kMaxDevices];

// Optional per-phase timing (mxm_profile_enable): four events per call.
constexpr int kPhases = 3;
struct CallEvents {
  cudaEvent_t ev[kPhases + 1];
};
bool g_profile = false;
std::vector<CallEvents> g_pending;
std::vector<CallEvents> g_event_pool;

CallEvents* profile_begin(cudaStream_t s) {
  if (!g_profile) return nullptr;
  CallEvents ce;
  if (!g_event_pool.empty()) {
    ce = g_event_pool.back();
    g_event_pool.pop_back();
  } else {
    for (int i = 0; i <= kPhases; ++i)
      if (cudaEventCreate(&ce.ev[i]) != cudaSuccess) return nullptr;
  }
  g_pending.push_back(ce);
  cudaEventRecord(g_pending.back().ev[0], s);
  return &g_pending.back();
}

void profile_mark(CallEvents* ce, int phase_end, cudaStream_t s) {
  if (ce) cudaEventRecord(ce->ev[phase_end], s);
}

mxm_status cuda_fail() { return MXM_ERR_CUDA; }

// Per-device state of the current device (created on first use).
mxm_status current_state(DeviceState** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return cuda_fail();
  DeviceState& st = g_dev[dev];
  if (!st.init) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return cuda_fail();
    st.status = static_cast<int*>(p);
    if (cudaDeviceGetAttribute(&st.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cuda_fail();
    st.init = true;
  }
  *out = &st;
  return MXM_OK;
}

bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

// Make sure the current device's workspace holds `need` bytes.
mxm_status ensure_workspace(DeviceState* st, size_t need, cudaStream_t s) {
  if (need <= st->ws_bytes) return MXM_OK;
  if (!st->ws_owned) return MXM_ERR_WORKSPACE_TOO_SMALL;
  if (stream_capturing(s)) return MXM_ERR_NO_WORKSPACE;
  if (st->ws) {
    if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail();
    cudaFree(st->ws);
    st->ws = nullptr;
    st->ws_bytes = 0;
  }
  size_t grow = need + need / 8;
  grow = align_up(grow, size_t(2) << 20);
  if (cudaMalloc(&st->ws, grow) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&st->ws, need) != cudaSuccess) {
      cudaGetLastError();
      st->ws = nullptr;
      return cuda_fail();
    }
    grow = need;
  }
  st->ws_bytes = grow;
  return MXM_OK;
}

bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  if (abytes == 0 || bbytes == 0) return false;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  return a0 < b0 + bbytes && b0 < a0 + abytes;
}

mxm_status check_gemm_args(const double* A, const double* B, double* C, int64_t m, int64_t k,
                           int64_t n) {
  if (m < 0 || k < 0 || n < 0) return MXM_ERR_INVALID_ARG;
  if (m > (int64_t(1) << 31) || n > (int64_t(1) << 31) || k > (int64_t(1) << 31))
    return MXM_ERR_UNSUPPORTED;
  if (m == 0 || n == 0) return MXM_OK;
  if (C == nullptr) return MXM_ERR_INVALID_ARG;
  if (k > 0 && (A == nullptr || B == nullptr)) return MXM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(C) & 7) || (reinterpret_cast<uintptr_t>(A) & 7) ||
      (reinterpret_cast<uintptr_t>(B) & 7))
    return MXM_ERR_ALIGNMENT;
  const size_t cb = sizeof(double) * size_t(m) * size_t(n);
  if (overlaps(C, cb, A, sizeof(double) * size_t(m) * size_t(k)) ||
      overlaps(C, cb, B, sizeof(double) * size_t(k) * size_t(n)))
    return MXM_ERR_INVALID_ARG;
  return MXM_OK;
}

bool emul_mode(int mode) { return mode == MXM_MODE_EMUL_I8 || mode == MXM_MODE_EMUL_BF16; }
int mode_beta(int mode) { return mode == MXM_MODE_EMUL_BF16 ? 8 : 7; }

size_t workspace_bytes(int mode, int64_t m, int64_t k, int64_t n, int slices) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  if (mode == MXM_MODE_F64) return f64_workspace(f64_dims(m, k, n));
  if (emul_mode(mode))
    return ozaki_layout(ozaki_dims_splitk(m, k, n, slices, mode_beta(mode))).total;
  if (mode == MXM_MODE_BF16_F32ACC) return ozaki_layout(ozaki_dims(m, k, n, 1, 8)).total;
  return 0;
}

// Launch sequence of one product whose workspace is already in place.
mxm_status run_gemm(int mode, const double* A, const double* B, double* C, int64_t m, int64_t k,
                    int64_t n, int slices, uint8_t* ws, int* status, cudaStream_t s) {
  if (m == 0 || n == 0) return MXM_OK;
  if (k == 0) return launch_zero_fill(C, m * n, s) == cudaSuccess ? MXM_OK : cuda_fail();
  cudaError_t e = cudaSuccess;
  if (mode == MXM_MODE_F64) {
    const F64Dims d = f64_dims(m, k, n);
    CallEvents* ce = profile_begin(s);
    profile_mark(ce, 1, s);
    e = launch_f64_pack(A, B, d, ws, s);
    profile_mark(ce, 2, s);
    if (e == cudaSuccess) e = launch_f64_gemm(ws, C, d, status, s);
    profile_mark(ce, 3, s);
  } else if (emul_mode(mode)) {
    const OzakiDims d = ozaki_dims_splitk(m, k, n, slices, mode_beta(mode));
    const OzakiLayout L = ozaki_layout(d);
    uint64_t* rowbits = reinterpret_cast<uint64_t*>(ws + L.rowbits);
    uint64_t* colbits = reinterpret_cast<uint64_t*>(ws + L.colbits);
    CallEvents* ce = profile_begin(s);
    e = launch_ozaki_scale(A, B, d, rowbits, colbits, status, s);
    profile_mark(ce, 1, s);
    if (e == cudaSuccess)
      e = launch_ozaki_split(A, B, d, rowbits, colbits, ws + L.aslices, ws + L.bslices, s);
    profile_mark(ce, 2, s);
    if (e == cudaSuccess)
      e = launch_ozaki_gemm(ws + L.aslices, ws + L.bslices, rowbits, colbits, C, d,
                            reinterpret_cast<uint64_t*>(ws + L.sums), status, s);
    profile_mark(ce, 3, s);
  } else if (mode == MXM_MODE_BF16_F32ACC) {
    const OzakiDims d = ozaki_dims(m, k, n, 1, 8);
    const OzakiLayout L = ozaki_layout(d);
    CallEvents* ce = profile_begin(s);
    profile_mark(ce, 1, s);
    profile_mark(ce, 2, s);
    e = launch_bf16_gemm(A, B, C, d, ws + L.aslices, ws + L.bslices, status, s);
    profile_mark(ce, 3, s);
  } else if (mode == MXM_MODE_F32) {
    CallEvents* ce = profile_begin(s);
    profile_mark(ce, 1, s);
    profile_mark(ce, 2, s);
    e = launch_f32_gemm(A, B, C, m, k, n, s);
    profile_mark(ce, 3, s);
  } else {
    return MXM_ERR_UNSUPPORTED;
  }
  return e == cudaSuccess ? MXM_OK : cuda_fail();
}

mxm_status check_mode(int mode, int slices) {
  if (mode == MXM_MODE_F64 || mode == MXM_MODE_F32 || mode == MXM_MODE_BF16_F32ACC) return MXM_OK;
  if (emul_mode(mode)) return (slices >= 1 && slices <= kOzMaxSlices) ? MXM_OK : MXM_ERR_UNSUPPORTED;
  return MXM_ERR_UNSUPPORTED;
}

}  // namespace

// The current device's status word (nullptr if CUDA is unusable).
int* device_status_word() {
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState* ds = nullptr;
  if (current_state(&ds) != MXM_OK) return nullptr;
  return ds->status;
}

}  // namespace mxm

using namespace mxm;

extern "C" {

int mxm_version(void) { return 100; }

const char* mxm_status_string(mxm_status s) {
  switch (s) {
    case MXM_OK: return "MXM_OK";
    case MXM_ERR_INVALID_ARG: return "MXM_ERR_INVALID_ARG";
    case MXM_ERR_ALIGNMENT: return "MXM_ERR_ALIGNMENT";
    case MXM_ERR_UNSUPPORTED: return "MXM_ERR_UNSUPPORTED";
    case MXM_ERR_NONFINITE: return "MXM_ERR_NONFINITE";
    case MXM_ERR_TIMEOUT: return "MXM_ERR_TIMEOUT";
    case MXM_ERR_CUDA: return "MXM_ERR_CUDA";
    case MXM_ERR_NO_WORKSPACE: return "MXM_ERR_NO_WORKSPACE";
    case MXM_ERR_WORKSPACE_TOO_SMALL: return "MXM_ERR_WORKSPACE_TOO_SMALL";
  }
  return "MXM_ERR_UNKNOWN";
}

size_t mxm_workspace_size(int mode, int64_t m, int64_t k, int64_t n, int slices) {
  if (check_mode(mode, slices) != MXM_OK) return 0;
  return workspace_bytes(mode, m, k, n, slices);
}

mxm_status mxm_gemm(int mode, const double* A, const double* B, double* C, int64_t m, int64_t k,
                    int64_t n, int slices, void* stream) {
  mxm_status st = check_mode(mode, slices);
  if (st != MXM_OK) return st;
  st = check_gemm_args(A, B, C, m, k, n);
  if (st != MXM_OK || m == 0 || n == 0) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState* ds = nullptr;
  if ((st = current_state(&ds)) != MXM_OK) return st;
  const size_t need = workspace_bytes(mode, m, k, n, slices);
  if ((st = ensure_workspace(ds, need, s)) != MXM_OK) return st;
  return run_gemm(mode, A, B, C, m, k, n, slices, static_cast<uint8_t*>(ds->ws), ds->status, s);
}

mxm_status mxm_f64(const double* A, const double* B, double* C, int64_t m, int64_t k, int64_t n,
                   void* stream) {
  return mxm_gemm(MXM_MODE_F64, A, B, C, m, k, n, 0, stream);
}

mxm_status mxm_f64_emul(const double* A, const double* B, double* C, int64_t m, int64_t k,
                        int64_t n, int slices, void* stream) {
  return mxm_gemm(MXM_MODE_EMUL_I8, A, B, C, m, k, n, slices, stream);
}

mxm_status mxm_gemm_host(int mode, const double* hA, const double* hB, double* hC, int64_t m,
                         int64_t k, int64_t n, int slices, void* stream) {
  mxm_status st = check_mode(mode, slices);
  if (st != MXM_OK) return st;
  if (m < 0 || k < 0 || n < 0) return MXM_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return MXM_OK;
  if (hC == nullptr || (k > 0 && (hA == nullptr || hB == nullptr))) return MXM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState* ds = nullptr;
  if ((st = current_state(&ds)) != MXM_OK) return st;
  const size_t ab = align_up(sizeof(double) * size_t(m) * size_t(k), 1024);
  const size_t bb = align_up(sizeof(double) * size_t(k) * size_t(n), 1024);
  const size_t cb = align_up(sizeof(double) * size_t(m) * size_t(n), 1024);
  const size_t need = ab + bb + cb + workspace_bytes(mode, m, k, n, slices);
  if ((st = ensure_workspace(ds, need, s)) != MXM_OK) return st;
  uint8_t* base = static_cast<uint8_t*>(ds->ws);
  double* dA = reinterpret_cast<double*>(base);
  double* dB = reinterpret_cast<double*>(base + ab);
  double* dC = reinterpret_cast<double*>(base + ab + bb);
  if (k > 0) {
    if (cudaMemcpyAsync(dA, hA, sizeof(double) * size_t(m) * size_t(k), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(dB, hB, sizeof(double) * size_t(k) * size_t(n), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
      return cuda_fail();
  }
  st = run_gemm(mode, dA, dB, dC, m, k, n, slices, base + ab + bb + cb, ds->status, s);
  if (st != MXM_OK) return st;
  if (cudaMemcpyAsync(hC, dC, sizeof(double) * size_t(m) * size_t(n), cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return cuda_fail();
  return cudaStreamSynchronize(s) == cudaSuccess ? MXM_OK : cuda_fail();
}

mxm_status mxm_set_workspace(void* d_ws, size_t bytes) {
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState* ds = nullptr;
  mxm_status st = current_state(&ds);
  if (st != MXM_OK) return st;
  if (d_ws != nullptr && (reinterpret_cast<uintptr_t>(d_ws) & 255)) return MXM_ERR_ALIGNMENT;
  if (ds->ws_owned && ds->ws) {
    if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail();
    cudaFree(ds->ws);
  }
  if (d_ws == nullptr) {
    ds->ws = nullptr;
    ds->ws_bytes = 0;
    ds->ws_owned = true;
  } else {
    ds->ws = d_ws;
    ds->ws_bytes = bytes;
    ds->ws_owned = false;
  }
  return MXM_OK;
}

mxm_status mxm_get_device_status(void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceState* ds = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    mxm_status st = current_state(&ds);
    if (st != MXM_OK) return st;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail();
  int v = 0;
  if (cudaMemcpy(&v, ds->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail();
  const int zero = 0;
  if (cudaMemcpy(ds->status, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_fail();
  if (v & kStatusNonFinite) return MXM_ERR_NONFINITE;
  if (v & kStatusTimeout) return MXM_ERR_TIMEOUT;
  if (v & kStatusWorkspace) return MXM_ERR_WORKSPACE_TOO_SMALL;
  if (v & kStatusBounds) return MXM_ERR_INVALID_ARG;
  return MXM_OK;
}

mxm_status mxm_profile_enable(int on) {
  std::lock_guard<std::mutex> lock(g_mutex);
  g_profile = on != 0;
  return MXM_OK;
}

mxm_status mxm_profile_read(double* ms, int max_phases, int64_t* calls) {
  std::lock_guard<std::mutex> lock(g_mutex);
  double sum[kPhases] = {0, 0, 0};
  mxm_status st = MXM_OK;
  for (CallEvents& ce : g_pending) {
    if (cudaEventSynchronize(ce.ev[kPhases]) != cudaSuccess) st = MXM_ERR_CUDA;
    for (int p = 0; p < kPhases; ++p) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ce.ev[p], ce.ev[p + 1]) == cudaSuccess) sum[p] += t;
    }
    g_event_pool.push_back(ce);
  }
  if (calls) *calls = static_cast<int64_t>(g_pending.size());
  g_pending.clear();
  for (int p = 0; p < max_phases && p < kPhases; ++p)
    if (ms) ms[p] = sum[p];
  return st;
}

}  // extern "C"

// ---------------------------------------------------------------- failure-path hook
namespace mxm {
namespace {
__global__ void debug_wait_timeout_kernel(uint64_t limit_ns, int* status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // nothing ever arrives on `bar`: the wait must give up after limit_ns
    (void)mbar_wait_bounded(&bar, 0u, &abort_flag, status, limit_ns);
  }
  __syncthreads();
}
}  // namespace
}  // namespace mxm

extern "C" mxm_status mxm_debug_wait_timeout(uint64_t limit_ns, void* stream) {
  if (limit_ns == 0 || limit_ns > 10000000000ull) return MXM_ERR_INVALID_ARG;
  DeviceState* ds = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    mxm_status st = current_state(&ds);
    if (st != MXM_OK) return st;
  }
  debug_wait_timeout_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(limit_ns, ds->status);
  return cudaGetLastError() == cudaSuccess ? MXM_OK : MXM_ERR_CUDA;
}

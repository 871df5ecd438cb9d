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
  cudaStream_t h2d = nullptr;  // streams of the pipelined host path: copies in,
  cudaStream_t d2h = nullptr;  // copies out, and a second compute stream
  cudaStream_t c1 = nullptr;
  cudaStream_t c2 = nullptr;   // scale and split of B's column panels
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

bool emul_mode(int mode) {
  return mode == MXM_MODE_EMUL_I8 || mode == MXM_MODE_EMUL_BF16 || mode == MXM_MODE_EMUL_RN8;
}
int mode_beta(int mode) { return mode == MXM_MODE_EMUL_I8 ? 7 : 8; }
bool mode_rn(int mode) { return mode == MXM_MODE_EMUL_RN8; }

// The default plan: every field zero.
constexpr mxm_plan kNoPlan = {0, 0, 0, 0};

bool plan_ok(int mode, const mxm_plan& p) {
  if (p.raster < 0 || p.kb_order < 0 || p.kb_order > 2 || p.cta < 0 || p.cta > 1 ||
      p.splitk < 0)
    return false;
  if (mode == MXM_MODE_EMUL_FP8 && p.splitk > 1) return false;
  return true;
}

// Dims of a native product under a plan.
F64Dims native_dims(int64_t m, int64_t k, int64_t n, const mxm_plan& p) {
  F64Dims d = f64_dims(m, k, n);
  if (p.splitk == 1) d.splits = 1;
  else if (p.splitk > 1) d.splits = p.splitk < d.Kt ? p.splitk : (d.Kt > 0 ? d.Kt : 1);
  if (p.raster > 0) d.raster = p.raster;
  return d;
}

// Dims of an emulated product (bf16 digits) under a plan.
OzakiDims emul_dims(int mode, int64_t m, int64_t k, int64_t n, int slices, const mxm_plan& p) {
  OzakiDims d = ozaki_dims_splitk(m, k, n, slices, mode_beta(mode), mode_rn(mode));
  if (p.splitk == 1) {
    d.splits = 1;
    d.pair = d.Mt >= 2 ? 1 : 0;
  } else if (p.splitk > 1) {
    d.splits = p.splitk < d.Kt ? p.splitk : (d.Kt > 0 ? d.Kt : 1);
    if (d.splits > 1) d.pair = 0;
  }
  if (p.cta == 1) d.pair = 0;
  // measured at m = k = n = 8192, S = 7 on CTA pairs: groups of 4 pair-rows
  // with alternating k-block directions read 47.7 GB from DRAM per product
  // against 73.4 GB for groups of 8 going forwards (same time within 0.5 %)
  d.raster = p.raster > 0 ? p.raster : (d.pair ? kPairRaster : kDefaultRaster);
  d.kb_alt = p.kb_order == 1 ? 0 : 1;
  return d;
}

OzakiDims fp8_dims(int64_t m, int64_t k, int64_t n, int slices, const mxm_plan& p) {
  OzakiDims d = ozaki_dims_fp8(m, k, n, slices);
  if (p.raster > 0) d.raster = p.raster;
  d.kb_alt = p.kb_order == 1 ? 0 : 1;
  return d;
}

size_t workspace_bytes(int mode, int64_t m, int64_t k, int64_t n, int slices,
                       const mxm_plan& p = kNoPlan) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  if (mode == MXM_MODE_F64) return f64_workspace(native_dims(m, k, n, p));
  if (emul_mode(mode)) return ozaki_layout(emul_dims(mode, m, k, n, slices, p)).total;
  if (mode == MXM_MODE_EMUL_FP8) return ozaki_layout(fp8_dims(m, k, n, slices, p)).total;
  if (mode == MXM_MODE_BF16_F32ACC) return ozaki_layout(ozaki_dims(m, k, n, 1, 8)).total;
  return 0;
}

// Launch sequence of one product whose workspace is already in place.
mxm_status run_gemm(int mode, const double* A, const double* B, double* C, int64_t m, int64_t k,
                    int64_t n, int slices, uint8_t* ws, int* status, cudaStream_t s,
                    const mxm_plan& plan = kNoPlan) {
  if (m == 0 || n == 0) return MXM_OK;
  if (k == 0) return launch_zero_fill(C, m * n, s) == cudaSuccess ? MXM_OK : cuda_fail();
  cudaError_t e = cudaSuccess;
  if (mode == MXM_MODE_F64) {
    const F64Dims d = native_dims(m, k, n, plan);
    CallEvents* ce = profile_begin(s);
    profile_mark(ce, 1, s);
    e = launch_f64_pack(A, B, d, ws, s);
    profile_mark(ce, 2, s);
    if (e == cudaSuccess) e = launch_f64_gemm(ws, C, d, status, s);
    profile_mark(ce, 3, s);
  } else if (emul_mode(mode)) {
    const OzakiDims d = emul_dims(mode, m, k, n, slices, plan);
    const OzakiLayout L = ozaki_layout(d);
    uint64_t* rowbits = reinterpret_cast<uint64_t*>(ws + L.rowbits);
    uint64_t* colbits = reinterpret_cast<uint64_t*>(ws + L.colbits);
    CallEvents* ce = profile_begin(s);
    e = launch_ozaki_scale(A, B, d, rowbits, colbits, status, s);
    profile_mark(ce, 1, s);
    if (e == cudaSuccess)
      e = launch_ozaki_split(A, B, d, rowbits, colbits, ws + L.aslices, ws + L.bslices,
                             status, s);
    profile_mark(ce, 2, s);
    if (e == cudaSuccess)
      e = launch_ozaki_gemm(ws + L.aslices, ws + L.bslices, rowbits, colbits, C, d,
                            reinterpret_cast<uint64_t*>(ws + L.sums), status, s);
    profile_mark(ce, 3, s);
  } else if (mode == MXM_MODE_EMUL_FP8) {
    const OzakiDims d = fp8_dims(m, k, n, slices, plan);
    if (!ozaki_narrow(d.S, d.beta, d.Kt)) return MXM_ERR_UNSUPPORTED;
    const OzakiLayout L = ozaki_layout(d);
    uint64_t* rowbits = reinterpret_cast<uint64_t*>(ws + L.rowbits);
    uint64_t* colbits = reinterpret_cast<uint64_t*>(ws + L.colbits);
    CallEvents* ce = profile_begin(s);
    e = launch_ozaki_scale(A, B, d, rowbits, colbits, status, s);
    profile_mark(ce, 1, s);
    if (e == cudaSuccess)
      e = launch_ozaki_split(A, B, d, rowbits, colbits, ws + L.aslices, ws + L.bslices,
                             status, s);
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
  if (mode == MXM_MODE_EMUL_RN8)  // the rounded value 2^(8S-1) must fit int64
    return (slices >= 1 && slices <= kOzMaxSlicesRn8) ? MXM_OK : MXM_ERR_UNSUPPORTED;
  if (emul_mode(mode)) return (slices >= 1 && slices <= kOzMaxSlices) ? MXM_OK : MXM_ERR_UNSUPPORTED;
  if (mode == MXM_MODE_EMUL_FP8)
    return (slices >= 1 && slices <= kOzMaxSlicesE4m3) ? MXM_OK : MXM_ERR_UNSUPPORTED;
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
    case MXM_ERR_BREAKDOWN: return "MXM_ERR_BREAKDOWN";
  }
  return "MXM_ERR_UNKNOWN";
}

size_t mxm_workspace_size(int mode, int64_t m, int64_t k, int64_t n, int slices) {
  if (check_mode(mode, slices) != MXM_OK) return 0;
  return workspace_bytes(mode, m, k, n, slices);
}

mxm_status mxm_gemm_plan(int mode, const double* A, const double* B, double* C, int64_t m,
                         int64_t k, int64_t n, int slices, const mxm_plan* plan, void* stream) {
  NvtxRange nvtx_range("mxm_gemm");
  const mxm_plan p = plan ? *plan : kNoPlan;
  mxm_status st = check_mode(mode, slices);
  if (st != MXM_OK) return st;
  if (!plan_ok(mode, p)) return MXM_ERR_INVALID_ARG;
  st = check_gemm_args(A, B, C, m, k, n);
  if (st != MXM_OK || m == 0 || n == 0) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState* ds = nullptr;
  if ((st = current_state(&ds)) != MXM_OK) return st;
  const size_t need = workspace_bytes(mode, m, k, n, slices, p);
  if ((st = ensure_workspace(ds, need, s)) != MXM_OK) return st;
  return run_gemm(mode, A, B, C, m, k, n, slices, static_cast<uint8_t*>(ds->ws), ds->status, s,
                  p);
}

mxm_status mxm_gemm(int mode, const double* A, const double* B, double* C, int64_t m, int64_t k,
                    int64_t n, int slices, void* stream) {
  return mxm_gemm_plan(mode, A, B, C, m, k, n, slices, nullptr, stream);
}

size_t mxm_workspace_size_plan(int mode, int64_t m, int64_t k, int64_t n, int slices,
                               const mxm_plan* plan) {
  const mxm_plan p = plan ? *plan : kNoPlan;
  if (check_mode(mode, slices) != MXM_OK || !plan_ok(mode, p)) return 0;
  return workspace_bytes(mode, m, k, n, slices, p);
}

mxm_status mxm_f64(const double* A, const double* B, double* C, int64_t m, int64_t k, int64_t n,
                   void* stream) {
  return mxm_gemm(MXM_MODE_F64, A, B, C, m, k, n, 0, stream);
}

mxm_status mxm_f64_emul(const double* A, const double* B, double* C, int64_t m, int64_t k,
                        int64_t n, int slices, void* stream) {
  return mxm_gemm(MXM_MODE_EMUL_I8, A, B, C, m, k, n, slices, stream);
}

// Host-buffer product of the emulated modes, pipelined over blocks: P panels
// of rows of A times Q panels of columns of B.  The copy stream brings B's
// first column panel, then A's panels with B's other column panels after
// the first row panel, so the first block product starts once a 1/Q part of
// B (and one panel of A) has crossed the link; every panel is scaled and
// split once (a column panel of B into its own digit planes; a row panel of
// A for the Q products of that row).  Block products alternate between two
// compute streams (the caller's and the library's) with a workspace each, so
// that the persistent GEMM of one block starts on the SMs the previous one
// frees; each block of C goes back by a 2-D copy on a third stream as soon
// as it is done.  Rows of A and columns of B are scaled independently (the
// scale of row i is its own maximum, that of column j its own), so the
// blocks give the same bits as one call over the whole product.
constexpr int64_t kHostPanels = 8;

// Rows per panel (a multiple of the 128-row tile), or 0 when the product is
// too small for a panel to fill the GPU.
static int64_t host_panel_rows(int64_t m, int64_t n, int sms) {
  const int64_t h = align_up((m + kHostPanels - 1) / kHostPanels, size_t(kOzTileRows));
  const int64_t tiles = (h / kOzTileRows) * ((n + kOzTileRows - 1) / kOzTileRows);
  if (h >= m || tiles < sms) return 0;
  return h;
}

// Columns per panel of B: two panels when each still gives a block of one
// row panel enough tiles for the GPU, else all columns.
static int64_t host_panel_cols(int64_t h, int64_t n, int sms) {
  const int64_t w = align_up((n + 1) / 2, size_t(kOzTileRows));
  const int64_t tiles = (h / kOzTileRows) * (w / kOzTileRows);
  if (w >= n || tiles < sms) return n;
  return w;
}

static mxm_status gemm_host_panels(DeviceState* ds, int mode, const double* hA, const double* hB,
                                   double* hC, int64_t m, int64_t k, int64_t n, int slices,
                                   int64_t h, cudaStream_t s) {
  const int beta = mode_beta(mode);
  const bool rn = mode_rn(mode);
  const int64_t w = host_panel_cols(h, n, ds->sm_count);
  const int64_t P = (m + h - 1) / h, Q = (n + w - 1) / w;
  const OzakiDims dp = ozaki_dims(h, k, w, slices, beta, rn);  // the largest block, no split-k
  const OzakiLayout L = ozaki_layout(dp);
  // per compute stream: row scales, A planes, running sums of one block
  const size_t rb_bytes = align_up(sizeof(uint64_t) * size_t(h), 1024);
  const size_t ap_bytes = L.bslices - L.aslices;
  const size_t sm_bytes = L.total - L.sums;
  const size_t per_buf = rb_bytes + ap_bytes + sm_bytes;
  // per column panel: column scales and B planes
  const size_t per_col = (L.aslices - L.colbits) + (L.sums - L.bslices);
  const size_t ab = align_up(sizeof(double) * size_t(m) * size_t(k), 1024);
  const size_t bb = align_up(sizeof(double) * size_t(k) * size_t(n), 1024);
  const size_t cb = align_up(sizeof(double) * size_t(m) * size_t(n), 1024);
  mxm_status st = ensure_workspace(ds, ab + bb + cb + size_t(Q) * per_col + 2 * per_buf, s);
  if (st != MXM_OK) return st;
  if (ds->h2d == nullptr && cudaStreamCreateWithFlags(&ds->h2d, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_fail();
  if (ds->d2h == nullptr && cudaStreamCreateWithFlags(&ds->d2h, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_fail();
  if (ds->c1 == nullptr && cudaStreamCreateWithFlags(&ds->c1, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_fail();
  if (ds->c2 == nullptr && cudaStreamCreateWithFlags(&ds->c2, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_fail();
  uint8_t* base = static_cast<uint8_t*>(ds->ws);
  double* dA = reinterpret_cast<double*>(base);
  double* dB = reinterpret_cast<double*>(base + ab);  // column panel j at dB + j w k (k x wj)
  double* dC = reinterpret_cast<double*>(base + ab + bb);  // block (i, j) at dC + (i n + j w h)
  uint8_t* cols = base + ab + bb + cb;
  uint8_t* bufs = cols + size_t(Q) * per_col;
  // events: per column panel B copied, B split; per row panel A copied; per
  // block C computed; done
  std::vector<cudaEvent_t> ev(2 * Q + P + P * Q + 2, nullptr);
  mxm_status rc = MXM_OK;
  auto fail = [&]() { rc = cuda_fail(); };
  for (auto& e : ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      e = nullptr;
      fail();
    }
  cudaEvent_t* eBc = ev.data();          // Q
  cudaEvent_t* eBs = ev.data() + Q;      // Q
  cudaEvent_t* eA = ev.data() + 2 * Q;   // P
  cudaEvent_t* eC = eA + P;              // P Q
  cudaEvent_t eDone = ev.back();
  cudaEvent_t eStart = ev[ev.size() - 2];
  cudaStream_t cs[2] = {s, ds->c1};
  auto col0 = [&](int64_t j) { return j * w; };
  auto colw = [&](int64_t j) { return (n - j * w) < w ? (n - j * w) : w; };
  auto row0 = [&](int64_t i) { return i * h; };
  auto rowh = [&](int64_t i) { return (m - i * h) < h ? (m - i * h) : h; };
  auto copy_b = [&](int64_t j) {
    double* dst = dB + j * w * k;
    if (cudaMemcpy2DAsync(dst, sizeof(double) * size_t(colw(j)), hB + col0(j),
                          sizeof(double) * size_t(n), sizeof(double) * size_t(colw(j)),
                          size_t(k), cudaMemcpyHostToDevice, ds->h2d) != cudaSuccess ||
        cudaEventRecord(eBc[j], ds->h2d) != cudaSuccess)
      fail();
  };
  auto copy_a = [&](int64_t i) {
    if (cudaMemcpyAsync(dA + row0(i) * k, hA + row0(i) * k,
                        sizeof(double) * size_t(rowh(i)) * size_t(k), cudaMemcpyHostToDevice,
                        ds->h2d) != cudaSuccess ||
        cudaEventRecord(eA[i], ds->h2d) != cudaSuccess)
      fail();
  };
  // copy order: B_0, A_0, B_1 .. B_{Q-1}, A_1 .. A_{P-1}
  if (rc == MXM_OK) copy_b(0);
  if (rc == MXM_OK) copy_a(0);
  for (int64_t j = 1; j < Q && rc == MXM_OK; ++j) copy_b(j);
  for (int64_t i = 1; i < P && rc == MXM_OK; ++i) copy_a(i);
  // column panels of B: scale and split on their own stream as they arrive
  // (the caller's stream first waits for whatever it had queued)
  if (rc == MXM_OK && (cudaEventRecord(eStart, s) != cudaSuccess ||
                       cudaStreamWaitEvent(ds->c2, eStart, 0) != cudaSuccess))
    fail();
  for (int64_t j = 0; j < Q && rc == MXM_OK; ++j) {
    uint8_t* cw = cols + size_t(j) * per_col;
    uint64_t* colbits = reinterpret_cast<uint64_t*>(cw);
    uint8_t* bplanes = cw + (L.aslices - L.colbits);
    OzakiDims db = ozaki_dims(0, k, colw(j), slices, beta, rn);
    db.pair = dp.pair;  // every block's product reads these B planes
    if (cudaStreamWaitEvent(ds->c2, eBc[j], 0) != cudaSuccess ||
        launch_ozaki_scale(nullptr, dB + j * w * k, db, nullptr, colbits, ds->status, ds->c2) !=
            cudaSuccess ||
        launch_ozaki_split(nullptr, dB + j * w * k, db, nullptr, colbits, nullptr, bplanes,
                           ds->status, ds->c2) != cudaSuccess ||
        cudaEventRecord(eBs[j], ds->c2) != cudaSuccess)
      fail();
  }
  for (int64_t i = 0; i < P && rc == MXM_OK; ++i) {
    const int64_t r0 = row0(i), hp = rowh(i);
    cudaStream_t c = cs[i & 1];
    uint8_t* buf = bufs + (i & 1) * per_buf;
    uint64_t* rowbits = reinterpret_cast<uint64_t*>(buf);
    uint8_t* aplanes = buf + rb_bytes;
    uint64_t* sums = reinterpret_cast<uint64_t*>(buf + rb_bytes + ap_bytes);
    OzakiDims da = ozaki_dims(hp, k, 0, slices, beta, rn);
    da.pair = dp.pair;
    if (cudaStreamWaitEvent(c, eA[i], 0) != cudaSuccess ||
        launch_ozaki_scale(dA + r0 * k, nullptr, da, rowbits, nullptr, ds->status, c) !=
            cudaSuccess ||
        launch_ozaki_split(dA + r0 * k, nullptr, da, rowbits, nullptr, aplanes, nullptr,
                           ds->status, c) !=
            cudaSuccess)
      fail();
    for (int64_t j = 0; j < Q && rc == MXM_OK; ++j) {
      uint8_t* cw = cols + size_t(j) * per_col;
      const uint64_t* colbits = reinterpret_cast<const uint64_t*>(cw);
      const uint8_t* bplanes = cw + (L.aslices - L.colbits);
      const int64_t wj = colw(j);
      double* blk = dC + r0 * n + j * w * hp;  // h x wj, row-major, contiguous
      OzakiDims dg = ozaki_dims(hp, k, wj, slices, beta, rn);
      dg.pair = dp.pair;
      dg.raster = dg.pair ? kPairRaster : kDefaultRaster;
      dg.kb_alt = 1;
      cudaEvent_t done = eC[i * Q + j];
      if (cudaStreamWaitEvent(c, eBs[j], 0) != cudaSuccess ||
          launch_ozaki_gemm(aplanes, bplanes, rowbits, colbits, blk, dg, sums, ds->status, c) !=
              cudaSuccess ||
          cudaEventRecord(done, c) != cudaSuccess ||
          cudaStreamWaitEvent(ds->d2h, done, 0) != cudaSuccess ||
          cudaMemcpy2DAsync(hC + r0 * n + col0(j), sizeof(double) * size_t(n), blk,
                            sizeof(double) * size_t(wj), sizeof(double) * size_t(wj), size_t(hp),
                            cudaMemcpyDeviceToHost, ds->d2h) != cudaSuccess)
        fail();
    }
  }
  // the caller's stream ends after the last copy back; every stream is
  // drained before the events go
  if (rc == MXM_OK && (cudaEventRecord(eDone, ds->d2h) != cudaSuccess ||
                       cudaStreamWaitEvent(s, eDone, 0) != cudaSuccess))
    fail();
  if (cudaStreamSynchronize(s) != cudaSuccess) fail();
  cudaStreamSynchronize(ds->c1);
  cudaStreamSynchronize(ds->c2);
  cudaStreamSynchronize(ds->h2d);
  cudaStreamSynchronize(ds->d2h);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  return rc;
}

mxm_status mxm_gemm_host(int mode, const double* hA, const double* hB, double* hC, int64_t m,
                         int64_t k, int64_t n, int slices, void* stream) {
  NvtxRange nvtx_range("mxm_gemm_host");
  mxm_status st = check_mode(mode, slices);
  if (st != MXM_OK) return st;
  if (m < 0 || k < 0 || n < 0) return MXM_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return MXM_OK;
  if (hC == nullptr || (k > 0 && (hA == nullptr || hB == nullptr))) return MXM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState* ds = nullptr;
  if ((st = current_state(&ds)) != MXM_OK) return st;
  if (emul_mode(mode) && k > 0) {
    const int64_t h = host_panel_rows(m, n, ds->sm_count);
    if (h > 0) return gemm_host_panels(ds, mode, hA, hB, hC, m, k, n, slices, h, s);
  }
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

mxm_status mxm_set_workspace(void* d_ws, size_t bytes, void* stream) {
  NvtxRange nvtx_range("mxm_set_workspace");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState* ds = nullptr;
  mxm_status st = current_state(&ds);
  if (st != MXM_OK) return st;
  if (d_ws != nullptr && (reinterpret_cast<uintptr_t>(d_ws) & 255)) return MXM_ERR_ALIGNMENT;
  // the switch synchronises: not while `stream` is being captured
  if (stream_capturing(s)) return MXM_ERR_UNSUPPORTED;
  // work already queued on `stream` may still use the previous workspace
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail();
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
  NvtxRange nvtx_range("mxm_get_device_status");
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
  if (v & kStatusBreakdown) return MXM_ERR_BREAKDOWN;
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

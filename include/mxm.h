/*
 * mxm.h -- C ABI of libmxm.so: the EuroBen mod2am dense matrix product
 * C = A.B on one NVIDIA GB300 (sm_103a), natively in FP64 and FP64-accurate
 * by the Ozaki split on BF16 tensor cores.
 *
 * The operation (Sec. 3.1 of the paper): c_ij = sum_k a_ik b_kj, with the
 * three matrices held in caller memory and C overwritten.  The paper states
 * the square n x n case; this ABI takes general m, k, n.
 *
 * Conventions shared by every call:
 *   - A is m x k, B is k x n, C is m x n, all dense ROW-MAJOR double,
 *     element (i,j) of an r x c matrix at X[i*c + j] (leading dimension =
 *     number of columns; no strides, no alpha/beta: C is overwritten).
 *   - Pointers are DEVICE pointers (cudaMalloc / torch memory) unless the
 *     function name ends in _host.  The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream; argument errors are
 *     reported synchronously through the return value and launch nothing.
 *   - m == 0 or n == 0 is a no-op; k == 0 writes zeros (the empty sum).
 *   - Negative sizes, NULL pointers with non-empty operands, or C overlapping
 *     A or B return MXM_ERR_INVALID_ARG.
 *   - Errors found on the device (a non-finite input in an emulated mode, a
 *     wait that timed out, a workspace overflow in a grouped call) are
 *     recorded in a sticky per-device status word that mxm_get_device_status
 *     reads and clears; the result C is then unspecified.  There is no CPU
 *     fallback: without a usable GPU every call returns MXM_ERR_CUDA.
 *   - Calls on different streams are independent except that they share the
 *     library-owned workspace; do not run two workspace-using calls
 *     concurrently on different streams unless each has its own caller
 *     workspace set (mxm_set_workspace is per device, so serialise them).
 */
#ifndef MXM_H_
#define MXM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MXM_OK = 0,
  MXM_ERR_INVALID_ARG = 1,        /* bad size, NULL pointer, overlap */
  MXM_ERR_ALIGNMENT = 2,          /* pointer not 8-byte aligned */
  MXM_ERR_UNSUPPORTED = 3,        /* mode or slice count not supported */
  MXM_ERR_NONFINITE = 4,          /* emulated mode met inf/nan (device status) */
  MXM_ERR_TIMEOUT = 5,            /* a bounded device wait gave up (device status) */
  MXM_ERR_CUDA = 6,               /* a CUDA runtime call failed */
  MXM_ERR_NO_WORKSPACE = 7,       /* workspace needed while a stream is capturing */
  MXM_ERR_WORKSPACE_TOO_SMALL = 8, /* caller workspace smaller than required */
  MXM_ERR_BREAKDOWN = 9            /* conjugate gradients met (p, A p) <= 0 (device status) */
} mxm_status;

typedef enum {
  MXM_MODE_F64 = 0,        /* native FP64 on the FP64 tensor path (DMMA) */
  MXM_MODE_EMUL_I8 = 1,    /* Ozaki split, 7-bit digits (int8 range) in BF16 */
  MXM_MODE_EMUL_BF16 = 2,  /* Ozaki split, 8-bit digits (full BF16 significand) */
  MXM_MODE_F32 = 3,        /* comparison: inputs rounded to FP32, FP32 sums */
  MXM_MODE_BF16_F32ACC = 4, /* comparison: inputs rounded to BF16, FP32 sums */
  MXM_MODE_EMUL_FP8 = 5,   /* Ozaki split, 4-bit digits carried in FP8 E4M3 */
  MXM_MODE_EMUL_RN8 = 6    /* Ozaki split rounded to nearest: balanced 8-bit digits in BF16 */
} mxm_mode;

/* One problem of a grouped call (device-resident table of these). */
typedef struct {
  const double* A;
  const double* B;
  double* C;
  int64_t m, k, n;
} mxm_problem;

/* Library version: major*10000 + minor*100 + patch. */
int mxm_version(void);

/* Human-readable name of a status code (static string, never NULL): the
 * enumerator's own name, e.g. "MXM_ERR_ALIGNMENT", or "MXM_ERR_UNKNOWN" for a
 * value outside mxm_status.  The paper has no counterpart: error reporting is
 * the library's contract around the Sec. 3.1 operation. */
const char* mxm_status_string(mxm_status s);

/*
 * mxm_f64 -- C = A.B in native FP64 (Sec. 3.1, c_ij = sum_k a_ik b_kj).
 * Every product and sum is an FP64 operation (fused multiply-add on the FP64
 * tensor path); the summation order over k is unspecified, so results agree
 * with any correct FP64 evaluation within |C - AB|_ij <= 2 k u (|A||B|)_ij,
 * u = 2^-53, and are bit-exact whenever every partial sum is exact (e.g.
 * small-integer matrices).  Uses library workspace (zero-padded tile copies
 * of A and B, mxm_workspace_size(MXM_MODE_F64, ...) bytes).
 */
mxm_status mxm_f64(const double* A, const double* B, double* C, int64_t m, int64_t k,
                   int64_t n, void* stream);

/*
 * mxm_f64_emul -- C = A.B, FP64-accurate, by the Ozaki split into `slices`
 * slices of 7-bit signed digits (int8 range) per row of A and column of B
 * under a per-row / per-column power-of-two scale (Ozaki, Ogita, Oishi,
 * Rump 2012; integer-slice form of Ootomo, Ozaki, Yokota 2024).  The slice
 * products s + t <= slices + 1 are computed exactly on tcgen05 tensor cores
 * and recombined in FP64 in a fixed order, so the result is bit-identical to
 * the CPU emulation of the same algorithm.  slices in 1..12; 7 gives FP64
 * accuracy (the bound above) for entries of similar magnitude, 8 for entries
 * spread over ~2^40.  Non-finite input sets MXM_ERR_NONFINITE in the device
 * status.  Uses library workspace.
 */
mxm_status mxm_f64_emul(const double* A, const double* B, double* C, int64_t m, int64_t k,
                        int64_t n, int slices, void* stream);

/*
 * mxm_gemm -- C = A.B in the given mxm_mode (slices is used by the
 * emulated modes and ignored otherwise).  MXM_MODE_F64 is mxm_f64 and
 * MXM_MODE_EMUL_I8 is mxm_f64_emul; MXM_MODE_EMUL_BF16 takes 8-bit digits
 * (6 slices ~ 7 of the 7-bit form); MXM_MODE_EMUL_FP8 takes 4-bit digits
 * (|d| <= 15, exact in FP8 E4M3) on the FP8 tensor path, 1..16 slices, about
 * twice as many as the 7-bit form for the same accuracy, and returns
 * MXM_ERR_UNSUPPORTED when the per-diagonal sums would not fit int32
 * (S 225 k >= 2^31, i.e. k beyond ~600 000) -- it has no grouped form.
 * MXM_MODE_EMUL_RN8 rounds each value once to nearest on the grid of its
 * last digit (scale exponent e + 1) and writes it in balanced 8-bit digits
 * (|d| <= 128, exact in bf16): the accuracy of 8-bit digits with the long
 * exact windows of 7-bit digits; 1..7 slices, no grouped form.  The
 * FP32 and BF16 modes round A and B to the narrow type and sum in FP32: they
 * are reported beside the FP64 modes, not FP64-accurate.
 */
mxm_status mxm_gemm(int mode, const double* A, const double* B, double* C, int64_t m, int64_t k,
                    int64_t n, int slices, void* stream);

/*
 * mxm_plan -- how one product is laid out on the GPU, for the tuner
 * (paper_1211_1581_gb300/tune.py) and for callers that tune by hand.  A
 * zero-filled plan (or NULL) is the library's own rule.  The result does not
 * depend on the plan except through the summation order of the native FP64
 * path under split-k (within the same bound); every emulated mode gives the
 * same bits whatever the plan (its partial sums are exact integers).  The
 * paper has no counterpart (Sec. 3.1 states the operation, not its layout).
 *   raster    C tiles are walked by the persistent grid in groups of
 *             `raster` tile-rows (tile-row pairs on CTA pairs), column by
 *             column inside a group, so that the CTAs working at the same
 *             time share operand tiles in L2; 0: 8 (4 tile-row pairs).
 *   kb_order  the k-block order of the slice GEMM: 0 the default (2), 1
 *             every diagonal (pair) walks k forwards, 2 every other one
 *             walks k backwards (it starts on the tiles the previous one
 *             read last, still in L2).
 *   cta       the slice GEMM on bf16 digits: 0 the rule (CTA pairs,
 *             cta_group::2 with 256 x 128 C tiles, for two or more tile-rows
 *             of A without split-k), 1 single CTAs (128 x 128 C tiles).
 *   splitk    k ranges per C tile: 0 the rule (products with fewer C tiles
 *             than 152 split k towards 304 work units), 1 never, s > 1 that
 *             many (at most the number of k-blocks: 16-wide for the native
 *             path, 128-wide for the emulated modes; not for MXM_MODE_EMUL_FP8).
 */
typedef struct {
  int32_t raster;
  int32_t kb_order;
  int32_t cta;
  int32_t splitk;
} mxm_plan;

/*
 * mxm_gemm_plan -- mxm_gemm under an explicit plan (NULL: the default).
 * Errors as mxm_gemm, and MXM_ERR_INVALID_ARG for a plan field out of range
 * (negative, kb_order > 2, cta > 1) or split-k asked of MXM_MODE_EMUL_FP8.
 */
mxm_status mxm_gemm_plan(int mode, const double* A, const double* B, double* C, int64_t m,
                         int64_t k, int64_t n, int slices, const mxm_plan* plan, void* stream);

/* mxm_workspace_size_plan -- mxm_workspace_size for a product under `plan`
 * (split-k changes it); 0 also for an invalid plan. */
size_t mxm_workspace_size_plan(int mode, int64_t m, int64_t k, int64_t n, int slices,
                               const mxm_plan* plan);

/*
 * mxm_gemm_host -- mxm_gemm on HOST buffers: copies A and B to the device,
 * computes, copies C back, and returns after C is in host memory (the
 * stream is synchronised).  Device buffers come from the library's
 * workspace.  For the emulated modes, products whose panels of about m/8
 * rows still fill the GPU are pipelined: B first, then the panels of A are
 * copied in, computed and their rows of C copied out while the next panels
 * compute (two library-owned copy streams and a second compute stream);
 * the result is bit-identical to mxm_gemm.  Pinned host memory is needed
 * for the copies to overlap; pageable memory works but serialises them.
 */
mxm_status mxm_gemm_host(int mode, const double* hA, const double* hB, double* hC, int64_t m,
                         int64_t k, int64_t n, int slices, void* stream);

/*
 * mxm_workspace_size -- bytes of device workspace one mxm_gemm call of mode
 * `mode` on an m x k by k x n product (Sec. 3.1 shapes) with `slices` slices
 * needs (the FP64 path: zero-padded tile copies of A and B, plus split-k
 * partials; the emulated modes: row and column scales, the digit planes of
 * the Ozaki split, the running sums or split-k partials).  Host arithmetic
 * only, no device call.  Returns 0 for an empty product (m, n or k <= 0),
 * an unknown mode or a slice count the mode does not take.  The paper has no
 * counterpart; size a buffer for mxm_set_workspace with it.
 */
size_t mxm_workspace_size(int mode, int64_t m, int64_t k, int64_t n, int slices);

/*
 * mxm_set_workspace -- use caller-owned device memory [d_ws, d_ws + bytes)
 * (256-byte aligned) as the workspace of the current device from now on; the
 * library then never allocates for mxm_f64 / mxm_f64_emul / mxm_gemm, which
 * makes them safe to capture in a CUDA graph.  d_ws == NULL returns to the
 * library-owned workspace (grown with cudaMalloc on demand, outside
 * capture).  The paper has no counterpart (its calls take arrays the caller
 * owns and nothing else); this is the library's memory contract.
 *   stream  the stream the caller's next calls run on: the switch waits for
 *           the work already queued there (which may still use the previous
 *           workspace), and frees a library-owned previous workspace after
 *           the device is idle.  Calls on other streams must not be using the
 *           workspace meanwhile.
 * Errors: d_ws misaligned: MXM_ERR_ALIGNMENT; `stream` capturing (the switch
 * synchronises): MXM_ERR_UNSUPPORTED; a failed synchronisation:
 * MXM_ERR_CUDA.  The caller keeps d_ws alive while calls that use it run.
 */
mxm_status mxm_set_workspace(void* d_ws, size_t bytes, void* stream);

/*
 * mxm_group_plan -- how a grouped emulated call splits its problems between
 * the two slice GEMMs (for the tuner; NULL or short_kt = -1: the library's
 * default).  Problems with at most short_kt k-blocks of 128 run on the
 * one-diagonal kernel (its FP64 running sums stay in tensor memory, which
 * suits tiles with little k), the others on the diagonal-pair kernel (half
 * the operand bytes per digit product).  Both give the same bits.  Ignored
 * by MXM_MODE_F64.  reserved[] must be zero.  The default is 8.  The paper
 * has no counterpart.
 */
typedef struct {
  int32_t short_kt;
  int32_t reserved[3];
} mxm_group_plan;

/*
 * mxm_grouped_workspace_size -- bytes of workspace mxm_grouped needs for
 * these problems (host copy of the table; only m, k, n are read).
 */
mxm_status mxm_grouped_workspace_size(int64_t count, const mxm_problem* h_problems, int mode,
                                      int slices, size_t* bytes);

/*
 * mxm_grouped -- `count` independent products C_p = A_p.B_p (each the
 * Sec. 3.1 operation c_ij = sum_k a_ik b_kj on its own operands) of uneven sizes
 * in one persistent launch sequence, from a DEVICE-resident table of
 * mxm_problem.  mode is MXM_MODE_F64 or MXM_MODE_EMUL_I8 / _BF16 / _RN8.  d_ws is
 * caller workspace of ws_bytes (see mxm_grouped_workspace_size); the call
 * allocates nothing and synchronises nothing, so it can be captured in a
 * CUDA graph.  Tile offsets are computed on the device; a table that needs
 * more workspace than ws_bytes sets MXM_ERR_WORKSPACE_TOO_SMALL in the device
 * status and computes nothing.
 */
mxm_status mxm_grouped(int64_t count, const mxm_problem* d_problems, int mode, int slices,
                       void* d_ws, size_t ws_bytes, void* stream);

/* mxm_grouped_plan / mxm_grouped_workspace_size_plan -- the same under an
 * explicit mxm_group_plan (NULL: the default); the workspace depends on the
 * plan (running sums for the long-k problems' tiles).  A plan with
 * short_kt < -1 or a nonzero reserved field: MXM_ERR_INVALID_ARG. */
mxm_status mxm_grouped_plan(int64_t count, const mxm_problem* d_problems, int mode, int slices,
                            const mxm_group_plan* plan, void* d_ws, size_t ws_bytes,
                            void* stream);
mxm_status mxm_grouped_workspace_size_plan(int64_t count, const mxm_problem* h_problems, int mode,
                                           int slices, const mxm_group_plan* plan,
                                           size_t* bytes);

/*
 * mxm_get_device_status -- synchronise `stream`, then read and clear the
 * sticky device status word of the current device: MXM_OK, or the first of
 * MXM_ERR_NONFINITE / MXM_ERR_TIMEOUT / MXM_ERR_WORKSPACE_TOO_SMALL /
 * MXM_ERR_INVALID_ARG (a sparse structure indexing outside its arrays) /
 * MXM_ERR_BREAKDOWN recorded by a kernel since the last read.
 */
mxm_status mxm_get_device_status(void* stream);

/*
 * mxm_peak_probe -- measure one execution unit's peak on the current device
 * with a register-resident (or shared-memory-resident) loop timed by CUDA
 * events: kind 0 = FP64 DFMA, 1 = FP64 DMMA m16n8k4, 2 = tcgen05 BF16
 * 128x128x16, 3 = tcgen05 BF16 128x256x16, 4 = legacy IMMA s8 m16n8k32.
 * Writes TFLOP/s (TOP/s for IMMA) to *tflops.  Used for the roofline
 * denominators the driver does not measure.  Synchronises the device.
 */
mxm_status mxm_peak_probe(int kind, double* tflops);

/*
 * mxm_debug_wait_timeout -- test hook for the failure path: launches one
 * block whose thread waits on an mbarrier that nothing completes, with a
 * wait limit of `limit_ns` nanoseconds.  The wait gives up, records
 * MXM_ERR_TIMEOUT in the device status word and the kernel exits normally.
 */
mxm_status mxm_debug_wait_timeout(uint64_t limit_ns, void* stream);

/*
 * mxm_profile_enable / mxm_profile_read -- per-kernel timing of library
 * calls.  While enabled (on != 0), every mxm_gemm / mxm_f64 / mxm_f64_emul
 * call records CUDA events on its stream around each of its phases: phase 0
 * = scale (row/column maxima), 1 = split / pack (operand tiles), 2 = the
 * product kernel.  mxm_profile_read synchronises on the recorded events,
 * writes the summed milliseconds of each phase since the last read to
 * ms[0..min(max_phases,3)-1], the number of calls to *calls, and resets the
 * sums.  Disabled (the default) nothing is recorded.
 */
mxm_status mxm_profile_enable(int on);
mxm_status mxm_profile_read(double* ms, int max_phases, int64_t* calls);

/*
 * mxm_spmv -- y = A x, the mod2as sparse product (Sec. 3.2).  A is
 * nrows x ncols in the paper's 3-array CSR form, all arrays in device
 * memory and owned by the caller: matvals[nnz] (FP64 values, row by row),
 * indx[nnz] (int32: the column of each value), rowp[nrows + 1] (int32: the
 * position in matvals of each row's first value, rowp[nrows] = nnz); x[ncols]
 * and y[nrows] FP64.  y is overwritten; x and y must not overlap.  Each row
 * is summed in FP64 with fused multiply-adds (a row's values are shared out
 * over 2..32 lanes by stride and their partial sums added by a tree), so
 * |y_i - sum_j a_ij x_j| <= 2 len_i u (|A||x|)_i with len_i the row's length.
 * Asynchronous on `stream`; argument errors are returned (sizes above
 * INT32_MAX: MXM_ERR_UNSUPPORTED; misaligned pointers: MXM_ERR_ALIGNMENT).
 * A row whose rowp entries, or a value whose column, lie outside the arrays
 * is skipped (its y_i is not written) and makes mxm_get_device_status
 * report MXM_ERR_INVALID_ARG.
 */
mxm_status mxm_spmv(const double* matvals, const int32_t* indx, const int32_t* rowp,
                    const double* x, double* y, int64_t nrows, int64_t ncols, int64_t nnz,
                    void* stream);

/* Engines of mxm_cg. */
enum {
  MXM_CG_AUTO = 0,     /* the cluster engine for n <= mxm_cg_max_n() and small nnz
                          (or when work is NULL), else the graph engine */
  MXM_CG_CLUSTER = 1,  /* one launch on a thread-block cluster of up to 16 CTAs */
  MXM_CG_GRAPH = 2     /* a CUDA graph: the loop is a conditional WHILE node over three
                          kernels on all SMs; needs `work`; not inside a stream capture */
};

/*
 * mxm_cg -- conjugate gradients for A x = b (Sec. 3.4, the textbook
 * iteration of Fig. 6 and the ArBB loop beside it), A an n x n symmetric
 * positive definite matrix in the CSR form of mxm_spmv (nrows = ncols = n).
 * x0 = 0, so r0 = p0 = b and r2 = (b, b); while r2 > stop and fewer than
 * max_iters steps were taken: q = A p; alpha = r2 / (p, q); r -= alpha q;
 * r2_new = (r, r); beta = r2_new / r2; x += alpha p; p = r + beta p.
 *
 * The loop test runs on the device in both engines: no host round trip per
 * step.  Arguments, all device memory, FP64 / int32, unaliased:
 *   matvals, indx, rowp   A in CSR (nnz values, nnz columns, n + 1 row
 *                         pointers; columns in [0, n));
 *   b                     the right-hand side, n doubles (read only);
 *   x                     the solution, n doubles (written);
 *   engine                MXM_CG_AUTO, MXM_CG_CLUSTER or MXM_CG_GRAPH;
 *   work                  mxm_cg_workspace_size(n) bytes of scratch for the
 *                         graph engine (may be NULL for the cluster engine);
 *   iters                 one int32: the number of steps taken;
 *   r2                    one double: the last (r, r) (the recursive
 *                         residual, as the paper's loop test uses it);
 *   r2_hist               NULL, or max_iters doubles: r2 after each step.
 * Results: x after the last step.  The dot products are deterministic (the
 * same result on every run for the same n, nnz and engine, on any device).
 * A step with (p, A p) <= 0 is not taken: the loop ends and
 * MXM_ERR_BREAKDOWN is recorded in the device status word.  Bad structure (a
 * row pointer or column outside the arrays) is skipped and recorded as
 * MXM_ERR_INVALID_ARG in the device status word; x is then unspecified.
 * Host-side errors: n <= 0, max_iters < 0, an unknown engine, NULL or
 * overlapping arrays, the graph engine without work: MXM_ERR_INVALID_ARG;
 * the cluster engine with n > mxm_cg_max_n(), n or nnz > INT32_MAX, the graph
 * engine inside a stream capture: MXM_ERR_UNSUPPORTED; misaligned
 * pointers: MXM_ERR_ALIGNMENT; a failed launch: MXM_ERR_CUDA.
 */
mxm_status mxm_cg(const double* matvals, const int32_t* indx, const int32_t* rowp,
                  const double* b, double* x, int64_t n, int64_t nnz, double stop,
                  int32_t max_iters, int32_t engine, double* work, int32_t* iters, double* r2,
                  double* r2_hist, void* stream);

/* mxm_cg_workspace_size -- bytes of `work` the graph engine needs for order n
 * (r, p, q and the blocks' shares of the dot products). */
size_t mxm_cg_workspace_size(int64_t n);

/* mxm_cg_max_n -- the largest n the cluster engine accepts (p is held twice
 * in the shared memory of every CTA). */
int64_t mxm_cg_max_n(void);

/*
 * mxm_fft -- the forward 1-D complex DFT of mod2f (Sec. 3.3, Eq. 1):
 * out(k) = sum_{j<n} in(j) exp(-2 pi i k j / n), 0 <= k < n, computed by
 * radix-2 decimation in frequency (Eqs. 2-3) in shared memory, in one pass
 * (n <= 1024) or two passes through `work` (the four-step factorisation).
 * Arguments (device memory; complex FP64 interleaved re, im; 16-byte
 * aligned):
 *   in      n complex values (read);
 *   out     n complex values (written); may be `in` itself;
 *   work    n complex values of scratch, apart from in and out (unused and
 *           may be NULL when n <= 1024);
 *   table   the twiddles W_T^j = exp(-2 pi i j / T), j < T / 2, written by
 *           mxm_fft_twiddles(table, T) (T / 2 complex values); T a power
 *           of two with n <= T (one table serves every smaller order);
 *           unused when n == 1;
 *   n       a power of two, 1 <= n <= mxm_fft_max_n().
 * Asynchronous on `stream`; no allocation; graph-capturable.  Errors: n not
 * a power of two or too large, T < n or not a power of two, NULL or
 * overlapping arrays: MXM_ERR_INVALID_ARG; misalignment: MXM_ERR_ALIGNMENT;
 * a failed launch: MXM_ERR_CUDA.  Accuracy: within the radix-2 bound
 * ||F' - F|| / ||F|| <= (log2 n + 1) eta / (1 - (log2 n + 1) eta),
 * eta = mu + gamma_4 (sqrt 2 + mu), mu the table's error (about u).
 */
mxm_status mxm_fft(const double* in, double* out, double* work, const double* table,
                   int64_t table_n, int64_t n, void* stream);

/* mxm_fft_twiddles -- write the table of mxm_fft for order T (a power of
 * two, T <= mxm_fft_max_n()): T / 2 complex values W_T^j, j < T / 2, from
 * sincospi.  Asynchronous on `stream`; nothing is written for T = 1. */
mxm_status mxm_fft_twiddles(double* table, int64_t n, void* stream);

/* mxm_fft_max_n -- the largest order mxm_fft accepts (2^22). */
int64_t mxm_fft_max_n(void);

/*
 * mxm_f64_emul_noalloc -- mxm_f64_emul (7-bit digits, `slices` slices) for
 * callers that cannot allocate device memory, e.g. code inside a process
 * whose allocator owns the device, loops that must never reach the driver's
 * allocator, or plugins handed device pointers but no allocator.  The paper
 * has no counterpart: this is a library convenience.  The result is the
 * same as mxm_f64_emul's (bit for bit).  The call allocates nothing: its
 * scratch is a fixed 64 MiB array in the library's device memory, present on
 * every GPU that loads the library until the process exits.  The first call
 * on a device looks up that array's device address (a runtime query, no
 * allocation); make that first call before any stream capture.  A product
 * whose scratch would exceed 64 MiB (e.g. beyond m = k = n = 1024 at 12
 * slices, or 1280 at 7) returns MXM_ERR_WORKSPACE_TOO_SMALL and launches
 * nothing.  All calls share the one array and it keeps the previous call's
 * contents (the launch sequence clears what must start at zero): calls whose
 * work overlaps on the GPU (other streams, other host threads) race, so
 * serialise them.  Other conventions as mxm_f64_emul.
 */
mxm_status mxm_f64_emul_noalloc(const double* A, const double* B, double* C, int64_t m,
                                int64_t k, int64_t n, int slices, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MXM_H_ */

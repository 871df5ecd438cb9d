// ptx.cuh -- inline-PTX helpers for sm_103a: mbarriers, bulk async copies
// (the TMA unit's 1-D form), tcgen05 MMA / tensor-memory access, and the
// bounded waits every kernel in this library uses.
//
// Every wait here gives up after a time limit (read from %globaltimer),
// sets a bit in the device status word and tells the caller, so that a
// lost arrival ends the kernel with MXM_ERR_TIMEOUT instead of hanging.
#pragma once
#include <cstdint>

#include "mxm_internal.h"

namespace mxm {

// ------------------------------------------------------------ bounds checks
// The MXM_DEBUG_BOUNDS build (libmxm_debug.so) checks tile coordinates, the
// sources of bulk copies and tensor-memory column ranges in the kernels; a
// failed check records kStatusBounds in the device status word (reported by
// mxm_get_device_status as MXM_ERR_INVALID_ARG) and the kernel goes on.  It
// never traps.  The release build compiles the checks away.
#ifdef MXM_DEBUG_BOUNDS
#define MXM_BOUNDS(cond, status)                          \
  do {                                                    \
    if (!(cond)) atomicOr((status), ::mxm::kStatusBounds); \
  } while (0)
#else
#define MXM_BOUNDS(cond, status) \
  do {                           \
  } while (0)
#endif

// Whether [p, p + bytes) lies inside [lo, hi).
__device__ __forceinline__ bool in_range(const void* p, size_t bytes, const void* lo,
                                         const void* hi) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p), l = reinterpret_cast<uintptr_t>(lo),
                  h = reinterpret_cast<uintptr_t>(hi);
  return a >= l && a + bytes <= h;
}

// ------------------------------------------------------------ misc
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool elect_lane0() { return (threadIdx.x & 31) == 0; }

// ------------------------------------------------------------ mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// Bring the line holding p into L2 ahead of a load.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// The same with cluster-scope acquire: for a barrier that threads (or the
// tensor cores) of the peer CTA of a pair arrive on.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Cluster-scope handshake on an mbarrier the peer CTA arrives on: the peer
// orders what it has observed with a release fence restricted to its shared
// memory, then arrives relaxed at cluster scope; the waiter polls relaxed at
// cluster scope and, once the phase has completed, takes an acquire fence
// restricted to the cluster's shared memory.
__device__ __forceinline__ void mbar_arrive_remote_release(uint32_t cluster_addr) {
  asm volatile("fence.release.sync_restrict::shared::cta.cluster;" ::: "memory");
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_relaxed_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.relaxed.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void fence_acquire_cluster_shared() {
  asm volatile("fence.acquire.sync_restrict::shared::cluster.cluster;" ::: "memory");
}

// Non-blocking test of a phase (mbarrier.test_wait), for an MMA issuer to
// look at the next stage's barrier while its current MMAs are in flight: one
// thread feeds the tensor core with little queueing, so a blocking wait
// between two stages leaves it idle for the wait's round trip, while a test
// issued in the middle of a stage returns behind the remaining MMAs.  A
// completed phase of a full barrier stays complete until the waiter itself
// releases the slot, so a positive result stays valid until it is used.
// kRemote: relaxed at cluster scope (the caller takes
// fence_acquire_cluster_shared before using the slot, as after
// mbar_try_wait_relaxed_cluster); otherwise acquire at CTA scope.
template <bool kRemote = false>
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  if constexpr (kRemote)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.relaxed.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  return ok != 0;
}

// Wait until the phase with the given parity has completed.  Returns false
// (and raises the abort flag and the status bit) after `limit_ns`, or at once
// if another role of the block has already aborted.  kCluster: cluster-scope
// acquire (arrivals from the peer CTA of a pair).
template <bool kCluster = false, bool kRemote = false>
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  volatile int* abort_flag, int* status,
                                                  uint64_t limit_ns = kWaitLimitNs) {
  auto try_once = [&]() {
    if (kRemote) {
      if (!mbar_try_wait_relaxed_cluster(bar, parity)) return false;
      fence_acquire_cluster_shared();
      return true;
    }
    return kCluster ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity);
  };
  if (try_once()) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t it = 1;; ++it) {
    if (try_once()) return true;
    if ((it & 15u) == 0) {
      if (*abort_flag) return false;
      if (global_timer_ns() - t0 > limit_ns) {
        *abort_flag = 1;
        atomicOr(status, kStatusTimeout);
        return false;
      }
      if (it > 1024) __nanosleep(256);
    }
  }
}

// ------------------------------------------------------------ CTA pairs
// A cluster of two CTAs on two SMs running tcgen05 with cta_group::2: one
// thread of rank 0 issues the MMAs for both, whose A operands (and halves of
// B) sit at the same shared-memory offsets in the two CTAs.
__device__ __forceinline__ uint32_t cluster_cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// All threads of both CTAs; orders shared::cluster accesses.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared::cluster address of the same location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t smem_in_cta(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

// Arrive on an mbarrier given by its shared::cluster address, possibly in
// the peer CTA, with the default semantics (release at CTA scope).  Used
// where the arrival carries no data dependency (an issuer giving back a slot
// it did not read); arrivals that announce data the peer will use go through
// mbar_arrive_remote_release.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// ------------------------------------------------------------ bulk copy
// 1-D bulk copy global -> shared (the TMA unit), completion counted in bytes
// on `bar`.  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Same, with an L2 eviction-priority hint (createpolicy fraction form).
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void bulk_g2s_hint(void* dst_smem, const void* src_gmem,
                                              uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
      "[%1], %2, [%3], %4;" ::"r"(smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

// ------------------------------------------------------------ tcgen05
// Tensor memory: 128 lanes x 512 columns of 32-bit cells per SM; address =
// (lane << 16) | column.  A warp may only touch lanes 32*(warp%4) .. +31.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major operand tile stored with the
// 128-byte swizzle: rows of 128 bytes, 8-row (1024-byte) swizzle atoms, the
// 16-byte chunk c of row r stored at chunk position c ^ (r % 8).  The tile
// base must be 1024-byte aligned; stepping K inside the 128-byte row is done
// by adding the byte offset to the start address.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);          // start address
  d |= static_cast<uint64_t>(0) << 16;                           // LBO (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;                   // SBO: 8 rows x 128 B
  d |= static_cast<uint64_t>(1) << 46;                           // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                           // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                                  // D format: F32
         | (1u << 7)                                // A format: BF16
         | (1u << 10)                               // B format: BF16
         | (static_cast<uint32_t>(N >> 3) << 17)    // N / 8
         | (static_cast<uint32_t>(M >> 4) << 24);   // M / 16
}

// D[tmem] (+)= A[smem] . B[smem]^T, one CTA, issued by a single thread.
__device__ __forceinline__ void mma_bf16_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Instruction descriptor of kind::f8f6f4 with both operands E4M3 (format
// code 0), FP32 accumulation.  A and B always have the same type here.
__host__ __device__ constexpr uint32_t idesc_e4m3_f32(int M, int N) {
  return (1u << 4)                                  // D format: F32
         | (static_cast<uint32_t>(N >> 3) << 17)    // N / 8
         | (static_cast<uint32_t>(M >> 4) << 24);   // M / 16
}

// D[tmem] (+)= A[smem] . B[smem]^T with E4M3 operands (K = 32 per MMA).
__device__ __forceinline__ void mma_e4m3_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// cta_group::2 forms (every tcgen05 instruction of a kernel that uses them
// takes the same cta_group).  Allocation: one warp in each CTA of the pair,
// collectively; the same columns in both tensor memories.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// D (+)= A . B^T over the pair, issued by one thread of rank 0: M = 256 rows,
// rows 0-127 from rank 0's A tile into rank 0's tensor memory, rows 128-255
// from rank 1's into rank 1's; B's N rows half from each CTA.
__device__ __forceinline__ void mma_bf16_ss_pair(uint32_t d_tmem, uint64_t a_desc,
                                                 uint64_t b_desc, uint32_t idesc,
                                                 uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive once on the mbarrier at `bar`'s offset in every CTA of `cta_mask`
// when the pair MMAs issued so far by this thread have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar, uint16_t cta_mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
      "[%0], %1;" ::"r"(smem_u32(bar)),
      "h"(cta_mask)
      : "memory");
}

// Arrive once on `bar` when every tcgen05.mma issued so far by this thread
// has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns -> 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ------------------------------------------------------------ FP64 bits
// Exponent e of |x| in the frexp sense (|x| = mu 2^e, mu in [1/2, 1)) from
// the bit pattern of |x|; 0 for x == 0.  Finite x only.
__device__ __forceinline__ int exponent_from_absbits(uint64_t ab) {
  if (ab == 0) return 0;
  const int be = static_cast<int>(ab >> 52);
  if (be != 0) return be - 1022;
  // subnormal: |x| = mant * 2^-1074
  return (63 - __clzll(static_cast<long long>(ab))) - 1073;
}

// x * 2^E rounded to nearest even, computed on the bit pattern (exact when
// the result is normal; one rounding when it is subnormal; +-inf on
// overflow).  Written from the IEEE 754 binary64 layout.
__device__ __forceinline__ double ldexp_rn(double x, int E) {
  uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const uint64_t sign = b & 0x8000000000000000ull;
  uint64_t ab = b & 0x7FFFFFFFFFFFFFFFull;
  if (ab == 0 || ab >= 0x7FF0000000000000ull) return x;  // zero, inf, nan
  int be = static_cast<int>(ab >> 52);
  uint64_t mant = ab & 0x000FFFFFFFFFFFFFull;
  if (be == 0) {  // normalise a subnormal: mant has its top bit below 2^52
    const int sh = __clzll(static_cast<long long>(mant)) - 11;
    mant <<= sh;
    be = 1 - sh;
    mant &= 0x000FFFFFFFFFFFFFull;
  }
  // value = (2^52 + mant) * 2^(be - 1075)
  long long nbe = static_cast<long long>(be) + E;
  if (nbe >= 2047) return __longlong_as_double(static_cast<long long>(sign | 0x7FF0000000000000ull));
  if (nbe >= 1)
    return __longlong_as_double(
        static_cast<long long>(sign | (static_cast<uint64_t>(nbe) << 52) | mant));
  // subnormal result: significand (53 bits) shifted right by 1 - nbe, RNE
  const uint64_t sig = mant | 0x0010000000000000ull;
  const long long shift = 1 - nbe;
  if (shift > 54) return __longlong_as_double(static_cast<long long>(sign));
  const uint64_t q = sig >> shift;
  const uint64_t rem = sig & ((1ull << shift) - 1);
  const uint64_t half = 1ull << (shift - 1);
  uint64_t r = q;
  if (rem > half || (rem == half && (q & 1))) r = q + 1;
  return __longlong_as_double(static_cast<long long>(sign | r));
}

// y * 2^p exactly, for |y| < 2^53 and a normal result, built from the bits
// (no FP64 arithmetic: int -> double conversion and power-of-two scaling).
__device__ __forceinline__ double i64_times_pow2(long long y, int p) {
  if (y == 0) return 0.0;
  const uint64_t sign = y < 0 ? 0x8000000000000000ull : 0ull;
  const uint64_t mag = y < 0 ? static_cast<uint64_t>(-y) : static_cast<uint64_t>(y);
  const int e = 63 - __clzll(static_cast<long long>(mag));  // mag in [2^e, 2^{e+1})
  const uint64_t mant = mag << (52 - e);
  const uint64_t be = static_cast<uint64_t>(1023 + e + p);
  return __longlong_as_double(
      static_cast<long long>(sign | (be << 52) | (mant & 0x000FFFFFFFFFFFFFull)));
}

// 2^p as a double for -1022 <= p <= 1023.
__device__ __forceinline__ double pow2_normal(int p) {
  return __longlong_as_double(static_cast<long long>(static_cast<uint64_t>(p + 1023) << 52));
}

}  // namespace mxm

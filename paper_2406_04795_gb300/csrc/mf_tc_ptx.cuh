// mf_tc_ptx.cuh -- inline-PTX wrappers for the 5th-generation tensor cores
// (tcgen05: TMEM allocation, MMA, commit, TMEM loads) and shared-memory
// mbarriers on sm_103a.  Every wait is bounded by wall time.
#pragma once
#include <cstdint>

__device__ __forceinline__ uint32_t mf_smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t mf_globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// mbarrier (shared::cta)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mf_mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mf_smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ bool mf_mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(mf_smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity to complete; gives up after
// limit_ns of wall time and returns false.
__device__ __forceinline__ bool mf_mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  if (mf_mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = mf_globaltimer_ns();
  while (!mf_mbar_try_wait(bar, parity))
    if (mf_globaltimer_ns() - t0 > limit_ns) return false;
  return true;
}

// Makes this thread's generic-proxy shared-memory writes visible to the async
// proxy (the tensor cores read operands through it).
__device__ __forceinline__ void mf_fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// tcgen05 (cta_group::1)
// ---------------------------------------------------------------------------
// Whole warp: allocates ncols TMEM columns (power of 2, >= 32); the base
// address is written to *dst (shared memory).
__device__ __forceinline__ void mf_tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   mf_smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Whole warp: frees the columns of mf_tmem_alloc.
__device__ __forceinline__ void mf_tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void mf_tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mf_tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, K-major operand without swizzling: the
// operand is a grid of 8-row x 16-byte core matrices (each 128 contiguous
// bytes); lbo = byte distance between core matrices adjacent in K, sbo =
// byte distance between 8-row groups.  Bits 46-47 hold the descriptor
// version (1) of sm_100-family tensor cores; swizzle mode 0.
__device__ __forceinline__ uint64_t mf_tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 with BF16 A and B (both K-major), FP32
// accumulator, dense, shape M x N.
__host__ __device__ constexpr uint32_t mf_tc_idesc_bf16(int M, int N) {
  return (1u << 4)                      // D: FP32
         | (1u << 7)                    // A: BF16
         | (1u << 10)                   // B: BF16
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

// One thread: D[tmem] (+)= A[smem] x B[smem]^T, K = 16 for BF16.
__device__ __forceinline__ void mf_tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                               uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// One thread: the mbarrier receives one arrival when every MMA this thread
// issued before has completed.
__device__ __forceinline__ void mf_tc_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          mf_smem_u32(bar))
      : "memory");
}

// Whole warp: thread i reads TMEM lane (taddr's lane + i), 32 consecutive
// 32-bit columns from taddr's column; waits for the load before returning.
__device__ __forceinline__ void mf_tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row r, k) of a K-major BF16 operand with K = 32
// columns laid out as core matrices: 4 core matrices per 8-row group
// (lbo = 128 bytes), 8-row groups 512 bytes apart (sbo).
__host__ __device__ constexpr uint32_t mf_tc_off_k32(uint32_t r, uint32_t k) {
  return ((r >> 3) * 4u + (k >> 3)) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

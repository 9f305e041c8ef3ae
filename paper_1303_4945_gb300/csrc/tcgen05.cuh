// tcgen05.cuh -- the pieces the tensor-core Legendre kernels (legendre_tc.cu,
// legendre_tc_ana.cu) share: PTX wrappers for tcgen05 matrix products, TMEM and
// mbarriers (every wait bounded), and the exact bf16 digit helpers of their
// error-free operand split.
#pragma once
#include "mixed_common.cuh"

namespace sht {
namespace tc {

constexpr unsigned long long kWaitNs = 100000000ull;  // bounded mbarrier waits: 100 ms of global time

// ---- PTX wrappers -------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// shared-memory matrix descriptor, no swizzle: LBO = byte stride between core
// matrices along K, SBO = along M / N (checked on the device against CPU products)
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}
// instruction descriptor: D FP32, A and B bf16, M x N; A K-major, B K-major or
// (b_mn) MN-major, whose no-swizzle layout takes LBO along K and SBO along N too
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, bool b_mn = false) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// an mbarrier whose phase completes after `count` arrivals (default: the issuer's commit)
__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count = 1) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// waits for the completion of the barrier phase of the given parity; false once
// kWaitNs have passed (the matrix products take microseconds)
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done = 0;
  const unsigned long long t0 = global_ns();
  for (int it = 0; !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (!done && (it & 63) == 63 && global_ns() - t0 > kWaitNs) return false;
  }
  return true;
}
// as bar_wait, and false as soon as *stop is nonzero (a wait of another warp of the
// CTA gave up).  Each try suspends the thread for up to kSuspendNs (it resumes when
// the phase completes), so a waiting warp takes no issue slots from the others.
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool bar_wait_or(uint64_t *bar, uint32_t parity, const volatile int *stop) {
  uint32_t done = 0;
  const unsigned long long t0 = global_ns();
  for (int it = 0; !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (!done && (*stop || global_ns() - t0 > kWaitNs)) return false;
  }
  return true;
}
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 8 consecutive 32-bit TMEM columns of this thread's lane (warp w reads lanes
// 32w..32w+31); the registers are valid after tmem_wait_ld
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
// 16 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// zeros into 16 consecutive TMEM columns of this thread's lane (complete after tmem_wait_st)
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }


// ---- exact digits ---------------------------------------------------------------
// round x to a multiple of the quantum q whose magic constant is s = 1.5 * 2^23 * q
// (|x| < 2^22 q): the sum's rounding does it, the subtraction is exact
__device__ __forceinline__ float round_to(float x, float s) { return __fsub_rn(__fadd_rn(x, s), s); }
// two digits (each with at most 8 significant bits, so their FP32 patterns end in
// 16 zero bits) packed as bf16 in one word: lo at the lower address
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}
// the bf16 bits of one digit
__device__ __forceinline__ uint16_t bf16_of(float d) { return (uint16_t)(__float_as_uint(d) >> 16); }
// the power of two 2^(e+1) above a non-negative x in [2^e, 2^(e+1)) (2^-126 for 0)
__device__ __forceinline__ float pow2_above(float x) {
  return __int_as_float((__float_as_int(x) & 0x7f800000) + 0x00800000);
}

}  // namespace tc

struct TcArgs {
  MixArgs m;        // tables, work items and phase array of the mixed form
  float lam_bound;  // power of two bounding |Lambda_lm| over the plan
  int *err;         // device status word: bit 0 set when a bounded wait gave up
};

}  // namespace sht

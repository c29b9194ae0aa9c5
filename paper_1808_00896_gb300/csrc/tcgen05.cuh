// tcgen05.cuh -- thin inline-PTX wrappers for the 5th-generation tensor cores
// (tcgen05.mma with TMEM accumulators) and mbarriers, as used by the
// mixed-precision DWT kernels.  sm_100a / sm_103a only.
//
// Operand layout used throughout: K-major, no swizzle.  A tile of R rows x K
// elements is stored as 8-row x 16-byte "core matrices"; element (r, k) sits at
//   (k / kpc) * (R * 16) + (r / 8) * 128 + (r % 8) * 16 + (k % kpc) * elem_bytes,
// kpc = 16 / elem_bytes elements per 16 bytes.  In the shared-memory matrix
// descriptor this is SBO = 128 B (between 8-row groups) and LBO = R * 16 B
// (between core matrices along K).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace softgb {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__host__ __device__ constexpr uint32_t kmajor_offset(int r, int k, int rows, int elem_bytes) {
    return (uint32_t)((k / (16 / elem_bytes)) * (rows * 16) + (r / 8) * 128 + (r % 8) * 16 +
                      (k % (16 / elem_bytes)) * elem_bytes);
}

// Shared-memory matrix descriptor (K-major, no swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for sm_100-class tensor cores
    return d;
}

// Instruction descriptor: F32 accumulate, A/B format fmt (1 = BF16 for
// kind::f16, 2 = TF32 for kind::tf32), both K-major, M x N tile.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int M, int N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// The same with the A operand in tensor memory (taddr of its first column, lane
// 0; row r in lane r, two consecutive K elements per 32-bit column, the lower
// K index in the low half).
__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Arrive on an mbarrier when every tcgen05.mma issued so far by this thread completes.
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(mbar)));
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }
// Make this thread's generic-proxy shared-memory writes visible to the tensor cores.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;"); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

// Bounded wait for the mbarrier phase with the given parity.  Returns false if
// the phase did not complete within `limit` polls (each poll may suspend the
// thread for a hardware-defined time), so a lost completion cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint32_t limit) {
    const uint32_t a = smem_u32(mbar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");  // no load of the guarded data may move above the wait
        if (done) return true;
    }
    return false;
}

// Arrive (release) on an mbarrier from this thread.
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// Arrive on an mbarrier and raise its expected transaction count by `bytes`
// (the bulk copies that complete_tx on it must deliver that many bytes).
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

// TMA: a 4-D tile of the tensor map `map` at coordinates (c0 innermost .. c3)
// into shared memory at dst (128-byte aligned), completing `mbar`'s
// transaction bytes.  Coordinates may lie outside the tensor (zero fill), but
// c0 times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_4d(void *dst, const void *map, int c0, int c1, int c2, int c3,
                                            uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(mbar))
        : "memory");
}

// Named barrier over `nthreads` threads (whole warps) of the CTA.
__device__ __forceinline__ void group_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier with an AND over the participating threads' predicates: every
// thread of the group gets the same verdict, so a timeout seen by some threads
// makes the whole group leave together.
__device__ __forceinline__ bool group_and(int id, int nthreads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.and.pred p, %2, %3, q;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// 32 lanes x 16 columns of 32-bit values from TMEM (this warp's lane quarter).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
}

// 32 lanes x 16 columns of 32-bit values into TMEM (this warp's lane quarter);
// waits until the stores are done.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
    asm volatile("tcgen05.wait::st.sync.aligned;");
}

// 32 lanes x 4 columns of 32-bit values into TMEM (this warp's lane quarter),
// asynchronous: tcgen05.wait::st orders them before their use.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(r0), "r"(r1), "r"(r2),
                 "r"(r3));
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Error-free sum of two FP32 values (Knuth's TwoSum): s + e == a + b exactly,
// s = fl(a + b).  Six FP32 additions, no branch; the compiler may not reorder
// them (no fast-math).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Compensated running sum (hi, lo), |lo| <~ ulp(hi): adds x with the rounding
// error of hi + x carried into lo, so that hi + lo tracks the exact sum of the
// added values to about 2^-48 of their magnitude per step.
__device__ __forceinline__ void comp_add(float &hi, float &lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
}

// ---------------------------------------------------------------------------
// FP64 -> FP32 by integer operations (truncation toward zero, 2^-23 relative;
// underflow below the FP32 normal range gives 0, overflow gives inf).  Used on
// the Wigner-d entries so that the conversion does not occupy the FP64 pipe,
// which the recurrence already saturates.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float f64_to_f32_trunc(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    uint32_t f;
    if (e >= 897 && e <= 1150) f = sign | ((uint32_t)(e - 896) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    else if (e > 1150) f = sign | 0x7F800000u;
    else f = sign;
    return __uint_as_float(f);
}

// Split an FP32 value into BF16 hi = bf16_rn(x) and lo = bf16_rn(x - hi)
// (x - hi is exact in FP32): |lo| <= 2^-8 |x|, so the lo*lo term that the
// three-product scheme drops is <= 2^-16 of the product, and hi + lo carries
// ~17 significant bits.
__device__ __forceinline__ void split_bf16(float x, uint16_t &hi, uint16_t &lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
}

// Round an FP32 value to TF32 (10 explicit mantissa bits, nearest, ties away).
__device__ __forceinline__ float round_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// FP64 -> FP32 round-to-nearest-even by integer operations (normal range;
// results below the FP32 normal range flush to signed 0).
__device__ __forceinline__ float f64_to_f32_rn(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    if (e < 897) return __uint_as_float(sign);
    if (e > 1150) return __uint_as_float(e == 0x7FF && ((hi & 0xFFFFFu) | lo) ? 0x7FC00000u : (sign | 0x7F800000u));
    uint32_t f = ((uint32_t)(e - 896) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1FFFFFFFu;
    if (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) f += 1u;  // carry may round up into the exponent
    return __uint_as_float(sign | f);
}

// FP32 -> FP64 by integer operations (exact for normal numbers, 0 for FP32
// subnormals, inf/nan preserved).
__device__ __forceinline__ double f32_to_f64(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t sign = b & 0x80000000u;
    const uint32_t e = (b >> 23) & 0xFFu;
    uint32_t hi;
    uint32_t lo = 0;
    if (e == 0) hi = sign;
    else if (e == 0xFFu) { hi = sign | 0x7FF00000u | ((b & 0x7FFFFFu) >> 3); lo = b << 29; }
    else { hi = sign | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3); lo = b << 29; }
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

}  // namespace tc
}  // namespace softgb

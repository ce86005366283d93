// tc.cuh -- thin inline-PTX wrappers for the 5th-generation tensor cores (tcgen05),
// tensor memory (TMEM) and shared-memory mbarriers on sm_103a.
#pragma once
#include <stdint.h>
#include <cuda_bf16.h>

namespace phs {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major operand without swizzling.  The canonical
// layout is a grid of core matrices of 8 rows x 16 bytes (8 bf16): element (r, k) of
// a tile sits at (r/8)*sbo + (k/8)*lbo + (r%8)*16 + (k%8)*2 bytes from the start.
// lbo: byte distance between core matrices adjacent along K; sbo: along M/N.
__device__ __forceinline__ uint64_t make_desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for sm_100-family tensor cores
    // base offset 0, absolute LBO mode 0, layout type 0 (no swizzle)
    return d;
}

// Instruction descriptor, kind::f16 with bf16 A/B, fp32 accumulator, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4)                      // D format f32
           | (1u << 7)                    // A format bf16
           | (1u << 10)                   // B format bf16
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// arrive on an mbarrier once all previously issued tcgen05.mma of this thread complete
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes become visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity to complete, giving up after timeout_ns
// nanoseconds of wall time or after timeout_ns / 4 polls, whichever comes first (a poll
// takes more than 4 ns, so the poll cap only binds if %globaltimer does not advance);
// false on timeout.  Each poll is a try_wait, which suspends the warp for up to
// kSuspendNs while the phase is incomplete, so waiting warps leave their issue slots
// to the warps still working.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint64_t timeout_ns) {
    constexpr uint32_t kSuspendNs = 1000;
    const uint32_t a = smem_u32(mbar);
    const uint64_t max_polls = timeout_ns / 4 + 64;
    uint64_t t0 = 0;
    for (uint64_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity), "r"(kSuspendNs)
            : "memory");
        if (done) return true;
        if ((it & 63) == 0) {
            const uint64_t t = globaltimer_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > timeout_ns) return false;
        }
        if (it >= max_polls) return false;
    }
}

// one arrival (release at CTA scope)
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// one arrival on the mbarrier that also expects `bytes` of asynchronous copies
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
// bulk copy global -> shared through the TMA engine, completing on an mbarrier
// (both addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

// 32 lanes x 32-bit, 16 consecutive columns per thread: thread i of warp w reads TMEM
// lane 32*(w%4) + i, columns [col, col + 16)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// same load without the wait; follow a batch of them with tmem_wait_ld()
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
// 32 lanes x 32-bit, 8 consecutive columns per thread, no wait
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// byte offset of element (r, k) in a K-major no-swizzle tile with `kcols` columns
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int r, int k, int kcols) {
    return (uint32_t)((r >> 3) * (kcols / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

}  // namespace tc

// ---- exact fixed point on bf16 digit planes, shared by the tensor-core M2L passes
// (m2l_tc.cu for the log kernel, cheb_tc.cu for the distance kernel)
constexpr int TC_DB = 8;                     // bits per digit
constexpr int TC_NPL = 6;                    // digit planes per operand
constexpr int TC_QB = TC_DB * TC_NPL - 1;    // fixed point: |X| <= 2^47
constexpr int TC_GB = 6;                     // guard bits kept through the frame change
constexpr int TC_NCLS = 49;
constexpr uint64_t TC_TIMEOUT_NS = 2000000000ull;

// round(x * 2^sh) for |x| * 2^sh < 2^62, from the bit pattern (no FP64 arithmetic);
// the caller guarantees a right shift (sh small enough).  Zero and subnormals give 0.
__device__ __forceinline__ long long to_fixed(double x, int sh) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) return 0;
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const int r = 1075 - e - sh;
    long long v;
    if (r >= 64) v = 0;
    else if (r <= 0) v = (long long)(m << (-r));
    else v = (long long)((m + (1ull << (r - 1))) >> r);
    return (long long)bits < 0 ? -v : v;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Balanced base-256 digits of |y| < 2^47 as floats, d[0] the top digit: with
// z = y + 0x808080 the three low digits are the bytes of z minus 128 and the rest
// follow from z >> 24 the same way.  Each byte becomes a float exactly by the
// magic number 2^23 (bits 0x4B000000 | byte), so no integer-to-float conversion.
__device__ __forceinline__ void digits_f(long long y, float *d) {
    const long long z = y + 0x808080ll;
    const unsigned lo = (unsigned)z;
    const unsigned z2 = (unsigned)((int)(z >> 24) + 0x8080);
    constexpr float kBias = 8388736.0f;  // 2^23 + 128
    d[5] = __int_as_float(__byte_perm(lo, 0x4B000000u, 0x7540)) - kBias;
    d[4] = __int_as_float(__byte_perm(lo, 0x4B000000u, 0x7541)) - kBias;
    d[3] = __int_as_float(__byte_perm(lo, 0x4B000000u, 0x7542)) - kBias;
    d[2] = __int_as_float(__byte_perm(z2, 0x4B000000u, 0x7540)) - kBias;
    d[1] = __int_as_float(__byte_perm(z2, 0x4B000000u, 0x7541)) - kBias;
    d[0] = (float)((int)z2 >> 16);
}

// rounding arithmetic right shift, 1 <= s <= 63
__device__ __forceinline__ long long rshift_round(long long x, int s) { return (x + (1ll << (s - 1))) >> s; }


}  // namespace phs

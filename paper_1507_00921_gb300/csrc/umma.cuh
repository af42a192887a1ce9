// tcgen05 (5th-generation tensor core) primitives for the DFT-GEMM kernels: shared-memory
// matrix descriptors, the kind::f16 instruction descriptor, single-thread MMA issue with
// operands in shared memory and the accumulator in tensor memory (TMEM), completion
// through tcgen05.commit on an mbarrier, bounded mbarrier waits, and 32x32b TMEM loads.
//
// Operand layout (no swizzle): core matrices of 8 rows x 16 bytes (8 16-bit elements),
// each stored as 128 contiguous bytes.  The descriptor's leading byte offset (LBO) is
// the distance between core matrices adjacent along K and the stride byte offset (SBO)
// the distance between core matrices adjacent along M (or N); this holds for K-major
// operands (16-byte rows run along K) and for MN-major ones (16-byte rows run along M
// or N), as measured on GB300 with exact integer products.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dbp {
namespace umma {

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory descriptor: start address, LBO, SBO (bytes, multiples of 16), version 1,
// base offset 0, no swizzle.
__device__ __forceinline__ uint64_t desc(uint32_t start, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((start >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of a dense kind::f16 MMA with FP32 accumulation: A and B FP16
// (or both BF16), K-major (0) or MN-major (1) each, shape M x N (x K = 16).
__host__ __device__ constexpr uint32_t idesc_f16(bool bf16, int m, int n, bool a_mn, bool b_mn) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((a_mn ? 1u : 0u) << 15) |
           ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D (TMEM) = A * B (+ D when acc != 0); issued by one thread.
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// The mbarrier receives one arrival once every MMA issued so far by this thread is complete.
__device__ __forceinline__ void commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(saddr(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the completion of phase `parity` of the mbarrier, at most limit_ns
// nanoseconds; returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint64_t limit_ns) {
    const uint32_t a = saddr(mbar);
    const uint64_t t0 = globaltimer();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}

// Four loads of 8 consecutive 32-bit TMEM columns of this thread's lane (columns
// c0..c0+7, c1.., c2.., c3..), then one wait; the wait names the registers so that no
// use is scheduled before the data has arrived.
__device__ __forceinline__ void ld4x8(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t (&r)[32]) {
#define DBP_LD8(ADDR, O)                                                                                   \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"         \
                 : "=r"(r[O + 0]), "=r"(r[O + 1]), "=r"(r[O + 2]), "=r"(r[O + 3]), "=r"(r[O + 4]),          \
                   "=r"(r[O + 5]), "=r"(r[O + 6]), "=r"(r[O + 7])                                           \
                 : "r"(ADDR)                                                                                \
                 : "memory")
    DBP_LD8(c0, 0);
    DBP_LD8(c1, 8);
    DBP_LD8(c2, 16);
    DBP_LD8(c3, 24);
#undef DBP_LD8
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

}  // namespace umma
}  // namespace dbp

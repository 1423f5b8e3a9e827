// tcgen05 building blocks for sm_103a: tensor memory (TMEM) allocation, shared-memory
// matrix descriptors for the K-major no-swizzle canonical layout, the instruction
// descriptor of kind::f16 (BF16 or FP16 operands, FP32 accumulation), MMA issue, commit to
// an mbarrier and TMEM -> register loads.
//
// Canonical K-major layout without swizzle (16-bit elements): the operand tile of R rows x K
// columns is cut into core matrices of 8 rows x 8 elements (16 bytes per row, 128 bytes per
// core matrix, rows at 16-byte stride).  Core matrices adjacent along K are LBO bytes apart,
// core matrices adjacent along the rows SBO bytes apart.  Here: LBO = 128, SBO = K/8 * 128,
// i.e. element (r, k) sits at byte ((r/8) * (K/8) + k/8) * 128 + (r%8) * 16 + (k%8) * 2.
#pragma once

#include <stdint.h>

namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (r, k) of a K-major no-swizzle tile with K columns
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int r, int k, int K) {
    return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor (tcgen05): start address, LBO, SBO (all >> 4), the fixed
// version bits 46-48 = 0b001, base offset 0, swizzle mode 0 (none)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: D = F32, A and B of one type (bf16 = true: BF16,
// else FP16), both K-major, dense, M x N
__host__ __device__ __forceinline__ uint32_t idesc_f16(int M, int N, bool bf16) {
    uint32_t d = 0;
    d |= 1u << 4;                        // D format F32
    d |= (bf16 ? 1u : 0u) << 7;          // A format
    d |= (bf16 ? 1u : 0u) << 10;         // B format
    d |= (uint32_t)(N >> 3) << 17;       // N / 8
    d |= (uint32_t)(M >> 4) << 24;       // M / 16
    return d;
}

// TMEM allocation by one full warp; the base address is written to *smem_dst
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(smem_dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        bool accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate ? 1u : 0u)
        : "memory");
}

// arrive on the mbarrier when every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Accumulator layouts (cta_group::1): an M = 128 accumulator keeps row r in lane r; an
// M = 64 accumulator keeps 16 rows in the first half of each warp's 32-lane quarter, rows
// 16w .. 16w+15 in lanes 32w .. 32w+15, so warp w reads row 16w + lane for lane < 16.  The
// columns are those of D.

// the calling warp reads 8 consecutive 32-bit columns of its 32 TMEM lanes
// (warp w of the CTA owns lanes 32*(w%4) .. 32*(w%4)+31)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// bounded wait for the phase with the given parity; false when the bound was reached
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t max_iter) {
    const uint32_t a = smem_addr(bar);
    for (uint32_t it = 0; it < max_iter; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it > 32) __nanosleep(64);
    }
    return false;
}

}  // namespace tc

// h2_tc.cuh -- 5th-generation tensor-core (tcgen05) helpers for sm_103a.
//
// Operand tiles are K-major with 128 bytes per row (64 bf16 or 32 tf32 K-elements) in the 128-byte
// swizzled canonical layout: byte offset o = r*128 + 2k (bf16; 4k for tf32 within a 32-column
// K-block), stored at o ^ (((o >> 7) & 7) << 4)
// (the 16-byte chunk index is XORed with the row index modulo 8). Eight rows form a 1 KB
// swizzle atom; tiles start on 1 KB boundaries. The layout is produced in HBM once (blocks at
// upload, vectors per product), so a 1-D bulk copy lands the exact shared-memory image that
// the MMA reads.
//
// Accumulators live in tensor memory (TMEM). The streams issue M = 128 with one CTA: row r of D
// is in TMEM lane r, so warp w (w = 0..3) reads rows 32w .. 32w+31 with its 32 lanes, one
// 32-bit column per register.
#pragma once

#include <cstdint>

#include "h2_pipe.cuh"

namespace h2t {

__host__ __device__ inline uint32_t sw128_offset(int r, int k)
{
    const uint32_t o = uint32_t(r) * 128u + uint32_t(k) * 2u;
    return o ^ (((o >> 7) & 7u) << 4);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1 KB apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *tile)
{
    const uint32_t a = h2p::smem_addr(tile);
    uint64_t d = uint64_t((a >> 4) & 0x3FFFu);
    d |= uint64_t(1) << 16;          // leading byte offset (not used by swizzled K-major)
    d |= uint64_t(1024 >> 4) << 32;  // stride byte offset: 8 rows x 128 bytes
    d |= uint64_t(1) << 46;          // descriptor version
    d |= uint64_t(2) << 61;          // 128-byte swizzle
    return d;
}

// Instruction descriptor: bf16 x bf16 -> fp32, both operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// Instruction descriptor: tf32 x tf32 -> fp32, both operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32_f32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(h2p::smem_addr(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T with one K = 16 step; accumulate selects D += vs D =.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]^T with one K = 8 tf32 step; A is 128 lanes x 8 columns of
// tensor memory (one tf32 element per 32-bit column), B a shared-memory descriptor.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on an mbarrier once every earlier tcgen05 operation of this thread has completed.
__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     h2p::smem_addr(bar))
                 : "memory");
}

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes into v[0..15].
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// v[0..15] into 16 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace h2t

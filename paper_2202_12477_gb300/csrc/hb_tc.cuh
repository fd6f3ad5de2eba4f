// Blackwell (sm_100 family) tensor-core primitives as inline PTX: tensor
// memory (TMEM) allocation, shared-memory matrix descriptors, the
// instruction descriptor of tcgen05.mma kind::f16, the MMA itself, its
// completion through an mbarrier, and TMEM loads.
//
// Operand layouts are the "canonical" no-swizzle layouts of the tcgen05
// shared-memory descriptor: an operand tile is built of core matrices of
// 8 rows x 16 bytes (8 half-precision values), each core matrix one
// contiguous 128-byte block, row r of it at byte 16 r.
//   K-major  (the 8 values of a core-matrix row run along K):
//     element (mn, k) at (mn % 8) * 16 + (k % 8) * 2 + (mn / 8) * SBO + (k / 8) * LBO
//   MN-major (the 8 values of a core-matrix row run along M or N):
//     element (mn, k) at (mn % 8) * 2 + (k % 8) * 16 + (mn / 8) * LBO + (k / 8) * SBO
// (LBO: the leading byte offset field; SBO: the stride byte offset field.)
// The accumulator of an M = 128 MMA (one CTA) holds row i of D in TMEM lane
// i, column j in TMEM column j (32-bit values); warp w of the CTA reads lanes
// 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once

#include <stdint.h>

namespace hbtc {

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle: start address, leading and
// stride byte offsets (all multiples of 16 bytes), the fixed 0b001 at bits
// 46-48, base offset 0, relative leading offsets, swizzle mode 0.
__device__ __forceinline__ uint64_t smem_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP16 A and B, FP32
// accumulator, dense, no negation; a_mn / b_mn select MN-major operands;
// M in {64, 128}, N a multiple of 8 (of 16 for M = 128) up to 256.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool a_mn, bool b_mn)
{
    return (1u << 4)                       // D: FP32
           | (0u << 7) | (0u << 10)        // A, B: FP16
           | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16)
           | ((uint32_t)(N >> 3) << 17)
           | ((uint32_t)(M >> 4) << 24);
}

// TMEM allocation by one whole warp: `ncols` (a power of two, 32..512)
// columns; the TMEM address is written to *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(unsigned *dst, unsigned ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Release by the warp that allocated (same column count).
__device__ __forceinline__ void tmem_free(unsigned taddr, unsigned ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (TMEM) = A * B^T (+ D when accumulate), issued by one thread.
__device__ __forceinline__ void mma_f16(unsigned d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate ? 1u : 0u)
        : "memory");
}

// The mbarrier gets one arrival when every MMA this thread issued before it
// has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory writes become visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive 32-bit columns of this thread's TMEM lane, starting at taddr
// (lane in bits 16-31, column in bits 0-15); complete after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld16(unsigned taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
// Waits for this thread's outstanding TMEM loads; the registers of v are
// operands, so no use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                   "+r"(v[15])
                 :
                 : "memory");
}

}  // namespace hbtc

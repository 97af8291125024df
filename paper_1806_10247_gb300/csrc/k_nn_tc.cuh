// Tensor-core (tcgen05) building blocks of the warm-start network's
// convolutions: implicit GEMMs with BF16 operands staged in shared memory and
// FP32 accumulators in tensor memory (TMEM).  Included by k_nn.cu only.
//
// Layout of an operand tile in shared memory: R rows (R a multiple of 8) by
// Kp BF16 values along K (Kp a multiple of 16), K-major, no swizzle, as 8 x 8
// "core matrices" of 128 contiguous bytes (8 rows of 16 bytes): the core
// matrix of rows 8g..8g+7 and K values 8c..8c+7 starts at byte
// (c * R / 8 + g) * 128.  For one MMA over K values 16s..16s+15 the matrix
// descriptor starts at the core matrix (2s, 0), the two core matrices along K
// are R / 8 * 128 bytes apart (leading-dimension offset) and consecutive
// 8-row groups 128 bytes apart (stride-dimension offset).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace nntc {

constexpr int kM = 128;          // rows of one MMA tile (pixels or weight rows)
constexpr int kMaxKp = 512;      // padded K of one tile
constexpr int kMaxNp = 64;       // padded N (output channels) of one tile
// Slack after the operand tiles: even a descriptor read with its two strides
// exchanged (at most 15 * 2048 + 255 bytes past a tile's start) stays inside
// the block's own shared memory.
constexpr int kSlack = 32768;
constexpr unsigned long long kWaitNs = 2000000000ull;  // bound of every wait: 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int core_off(int r, int k, int R)
{
    return ((((k >> 3) * (R >> 3)) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

// Shared-memory matrix descriptor (no swizzle): start address, leading- and
// stride-dimension byte offsets (each >> 4 in 14 bits), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of a dense BF16 x BF16 -> FP32 MMA, both operands
// K-major: D format F32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory stores made visible to the tensor cores.
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t addr)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(addr) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of the barrier, giving up after kWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t parity)
{
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(addr, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

// D[tmem] (+)= A[adesc] * B[bdesc]^T, one instruction of K = 16.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on the barrier when every MMA issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Issue the MMAs of one tile: kM rows of A (Kp values each, at a0) times Np
// rows of B (at b0), into the FP32 accumulators at tmem.
__device__ __forceinline__ void issue_tile(uint32_t tmem, uint32_t a0, uint32_t b0, int Kp, int Np, bool accumulate)
{
    const uint32_t id = idesc_bf16(kM, Np);
    const uint32_t lboA = (kM / 8) * 128, lboB = (uint32_t)(Np / 8) * 128;
    for (int s = 0; s < Kp / 16; s++) {
        const uint64_t ad = smem_desc(a0 + (uint32_t)s * 2u * lboA, lboA, 128);
        const uint64_t bd = smem_desc(b0 + (uint32_t)s * 2u * lboB, lboB, 128);
        mma_bf16(tmem, ad, bd, id, (accumulate || s > 0) ? 1u : 0u);
    }
}

// 16 FP32 accumulator columns c0..c0+15 of this thread's row (warp w reads
// TMEM lanes 32 w .. 32 w + 31; row = lane).
__device__ __forceinline__ void tmem_load16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

__host__ __device__ constexpr int tmem_cols(int Np) { return Np <= 32 ? 32 : (Np <= 64 ? 64 : 128); }

}  // namespace nntc

// Fifth-generation tensor core (tcgen05) helpers for sm_103a: tensor-memory
// allocation, single-thread MMA issue, commit to an mbarrier, bounded mbarrier
// waits and tensor-memory loads, as inline PTX.
//
// Operand layout used by every MMA here: BF16, K-major, no swizzle.  An R x K
// tile (R a multiple of 8, K a multiple of 16) is stored as K/16 blocks of one
// MMA K-step each; inside a block the 8-row groups are 256 B apart, the two
// 8-element K halves of a group are 128 B apart (two 8 x 16 B core matrices),
// and a core matrix row is 16 B.  So the shared-memory descriptor of a K-step
// has leading (K-direction) byte offset 128 and stride (row-direction) byte
// offset 256, and block s starts s * R/8 * 256 bytes after the tile.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace dex {
namespace umma {

// byte offset of element (r, k) in an R-row tile
__host__ __device__ __forceinline__ int tile_offset(int r, int k, int R)
{
    return (k >> 4) * (R >> 3) * 256 + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// bytes of one K-step block of an R-row tile
__host__ __device__ constexpr int kstep_bytes(int R) { return (R >> 3) * 256; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all >> 4), the fixed version bit 46, no swizzle, base offset 0
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(256u >> 4) << 32;
    d |= 1ull << 46;
    return d;
}

// instruction descriptor of kind::f16: F32 accumulator, BF16 A and B, both
// K-major, dense, M x N
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- tensor memory (executed by one full warp) ----
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_slot, uint32_t ncols)
{
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// ---- ordering ----
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- MMA issue and completion (one thread) ----
// D[tmem] (+)= A[smem] * B[smem]^T, both operands K-major
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1u : 0u)
        : "memory");
}

// arrive once on the mbarrier when every MMA this thread issued so far is done
__device__ __forceinline__ void mma_commit(unsigned long long* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// Wait for the phase with the given parity to complete, at most max_iter
// polls; returns false if it did not complete.
__device__ __forceinline__ bool mbar_wait(unsigned long long* mbar, uint32_t parity, int max_iter)
{
    const uint32_t a = smem_u32(mbar);
    for (int it = 0; it < max_iter; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ---- tensor memory -> registers: this warp's 32 lanes, 16 consecutive columns ----
// The load and its wait are one asm statement, so no register is read before
// the data has arrived.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    __syncwarp();  // .sync.aligned: the whole warp, converged
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// TMEM address of lane `lane`, column `col` relative to an allocation base
__device__ __forceinline__ uint32_t tmem_at(uint32_t base, int lane, int col)
{
    return base + ((uint32_t)lane << 16) + (uint32_t)col;
}

}  // namespace umma
}  // namespace dex

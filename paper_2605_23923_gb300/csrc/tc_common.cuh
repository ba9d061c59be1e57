// Tensor-core pieces shared by the stage-2 kernels that run the split-BF16
// contraction on tcgen05 (the per-group kernel and the ragged-batch kernel):
// warp roles, operand layouts in shared memory, descriptors, MMA issue and
// commit, tensor-memory loads and the BF16 hi/lo split.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace su2 {
namespace tc {

constexpr int NP = 4;                       // pairs (consecutive n) per tile
constexpr int KC = 16;                      // beta nodes per chunk = one MMA K step
constexpr int BM = 64;                      // functions per tile (M = 128)
constexpr int NWARPS = 16;
constexpr int THREADS = NWARPS * 32;
constexpr int W_TMA = 0, W_MMA = 1, W_CONV = 2, W_GEN = 6, W_CONV2 = 10, W_EPI = 12;
constexpr int N_CONV = 6;                   // converter warps: 2-5 and 10-11

// Operand layouts (SWIZZLE_NONE canonical; core matrix = 8 rows x 16 bytes):
// A, K-major:  (row, kk) -> (row/8)*SBO_A + (kk/8)*LBO_A + (row%8)*16 + (kk%8)*2
// B, MN-major: (kk, col) -> (col/8)*SBO_B + (kk/8)*LBO_B + (kk%8)*16 + (col%8)*2
// A: the 16 row groups of one K half are contiguous (SBO_A = 128) and the
// second K half follows 16 bytes later than dense (LBO_A = 2064); with a
// 16-byte skew between the eight matrices (OPA) the converters' 8-byte stores
// of one batch row hit 32 different banks, and the eight matrices of a stage
// (33,024 bytes) fit over the 32 KB of staged F2 they are converted from.
constexpr int LBO_A = 2064, SBO_A = 128, LBO_B = 128, SBO_B = 256;
constexpr int OPA = LBO_A + 16 * SBO_A + 16;  // one pair's A matrix (hi or lo), skewed
constexpr int OPB = 16 * SBO_B;             // one pair's B matrix (hi or lo)
constexpr int STAGE_BYTES = BM * KC * NP * 8;       // fp32 staging: 32 KB
constexpr int A_BYTES = 2 * NP * OPA;
constexpr int NSA = 4;                      // F2 / A stages
constexpr int SA = ((A_BYTES > STAGE_BYTES ? A_BYTES : STAGE_BYTES) + 127) / 128 * 128;
constexpr int B_BYTES = 2 * NP * OPB;

__device__ __forceinline__ int a_off(int row, int kk) {
    return (row >> 3) * SBO_A + (kk >> 3) * LBO_A + (row & 7) * 16 + (kk & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
    const uint32_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;    // leading byte offset: K direction
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;    // stride byte offset: M / N direction
    d |= (uint64_t)1 << 46;                        // descriptor version
    return d;                                      // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: BF16 x BF16 -> F32, A K-major, B MN-major, M = 128.
__device__ __forceinline__ uint32_t instr_desc(int nmma) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) |
           ((uint32_t)(nmma >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(ad), "l"(bd), "r"(idesc), "r"((uint32_t)acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// 5-D tensor load with an L2 policy (the planes are read once: evict-first).
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7], %8;"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar)),
          "l"(policy)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);     // a -> low half (lower address)
    return *reinterpret_cast<uint32_t*>(&h);
}
// hi/lo split of two floats, packed as bf16x2 each.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float ha = __low2float(h), hb = __high2float(h);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = pack_bf16(a - ha, b - hb);
}

// Order this thread's earlier generic-proxy accesses of global memory, made
// visible to it by an acquire, before its later async-proxy (bulk copy) reads.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

}  // namespace tc
}  // namespace su2

// Stage 2 on the 5th-generation tensor cores: the beta contraction of Sec. 4
// (<s, P^l_{nm}> for every l, Sec. 6 second-stage Proposition with depth 1) as
// one small GEMM per (m, n) pair with the batch of functions as the M side:
//
//   D_p[b'][r] = sum_k  F2_p[b'][k] * d_p[k][r],     b' = 2 b + (0: re, 1: im),
//   r = l - l0 (row of the tile), d_p[k][r] = d^{l0 + r}_{nm}(beta_k)
//
// A = F2^T (K-major, M = 128 rows = 64 functions x re/im), B = d (MN-major,
// N = rows of l rounded up to 16), K = 16 beta nodes per MMA, FP32
// accumulation in tensor memory.  Split-BF16 ("BF16x3") arithmetic:
// x = x_hi + x_lo with x_hi = bf16(x), x_lo = bf16(x - x_hi) for both
// operands, D += A_hi B_hi + A_hi B_lo + A_lo B_hi.
//
// A CTA (one per SM, persistent) owns 4 consecutive n at fixed (sector, m)
// and 64 functions; per chunk of 16 nodes it
//   * loads the F2 chunk [64 functions][16 nodes][4 n] with one 5-D TMA copy,
//   * converts it to the BF16 hi/lo A operands (threads 0-127),
//   * regenerates the d-values of the 4 pairs x 16 nodes by the three-term
//     recurrence and writes the BF16 hi/lo B operands (threads 128-191),
//   * issues 3 tcgen05.mma per pair from one thread, committed to an mbarrier
//     that frees the stage two chunks later.
// Two stages of every buffer overlap the MMAs and the next TMA with the
// conversion and the recurrence.  The epilogue (warps 0-3 own the 128 TMEM
// lanes) multiplies by i^{n-m} and writes 4 consecutive n of each coefficient
// row with one contiguous store.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "recurrence.cuh"
#include "su2_internal.h"

namespace su2 {
namespace tc {

constexpr int NP = 4;                       // pairs (consecutive n) per tile
constexpr int KC = 16;                      // beta nodes per chunk = one MMA K step
constexpr int BM = 64;                      // functions per tile (M = 128)
constexpr int THREADS = 256;
constexpr int RMAX = 128;                   // rows of l per pair (N <= 256)
constexpr int STAGE_BYTES = BM * KC * NP * 8;       // F2 fp32 staging: 32 KB
constexpr int OPB = 128 * KC * 2;                   // one bf16 operand of one pair: 4 KB
constexpr int A_BYTES = 2 * NP * OPB;               // hi + lo, 4 pairs: 32 KB
constexpr int B_BYTES = 2 * NP * OPB;               // 32 KB
constexpr int OFF_STAGE = 0;
constexpr int OFF_A = OFF_STAGE + 2 * STAGE_BYTES;
constexpr int OFF_B = OFF_A + 2 * A_BYTES;
constexpr int OFF_COEF = OFF_B + 2 * B_BYTES;
constexpr int OFF_BAR = OFF_COEF + NP * RMAX * (int)sizeof(StepCoef<float>);
constexpr int SMEM_BYTES = OFF_BAR + 8 * 8 + 16;
constexpr uint32_t TMEM_COLS = 512;         // 4 pairs x 128 columns

// Canonical SWIZZLE_NONE layouts (core matrix = 8 rows x 16 bytes):
// A, K-major: element (row, kk) -> (row/8)*256 + (kk/8)*128 + (row%8)*16 + (kk%8)*2
//             LBO (K step) = 128, SBO (M step) = 256.
// B, MN-major: element (kk, col) -> (col/8)*256 + (kk/8)*128 + (kk%8)*16 + (col%8)*2
//             LBO (K step) = 128, SBO (N step) = 256.
__device__ __forceinline__ int a_off(int row, int kk) {
    return (row >> 3) * 256 + (kk >> 3) * 128 + (row & 7) * 16 + (kk & 7) * 2;
}
__device__ __forceinline__ int b_off(int kk, int col) {
    return (col >> 3) * 256 + (kk >> 3) * 128 + (kk & 7) * 16 + (col & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    const uint32_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;        // leading byte offset: K direction
    d |= (uint64_t)(256 >> 4) << 32;        // stride byte offset: M / N direction
    d |= (uint64_t)1 << 46;                 // descriptor version
    return d;                               // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: BF16 x BF16 -> F32, A K-major, B MN-major.
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

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
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

template <int N>
__global__ void __launch_bounds__(THREADS, 1)
contract_tc_kernel(BandArgs a, const __grid_constant__ CUtensorMap tmap, float2* __restrict__ coeffs) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int NCH = N / KC;
    StepCoef<float>* coef = reinterpret_cast<StepCoef<float>*>(smem + OFF_COEF);
    uint64_t* bar_full = reinterpret_cast<uint64_t*>(smem + OFF_BAR);        // [2] TMA landed
    uint64_t* bar_mma = bar_full + 2;                                        // [2] MMAs of the stage done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar_full + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tslot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar_full[0], 1);
        mbar_init(&bar_full[1], 1);
        mbar_init(&bar_mma[0], 1);
        mbar_init(&bar_mma[1], 1);
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;

    const int ntiles = 2 * N * (N / NP);
    const int nbb = (a.nfunc + BM - 1) / BM;
    const int nitems = ntiles * nbb;
    uint32_t tma_iss[2] = {0u, 0u}, tma_got[2] = {0u, 0u};
    uint32_t mma_iss[2] = {0u, 0u}, mma_got[2] = {0u, 0u};

    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int t = item / nbb, bb = item % nbb;
        Tile<NP> tl;
        tl.decode(N, t);
        if (!tl.any) continue;
        const int Lt = tl.L;
        const int nmma = (Lt + 15) & ~15;
        const uint32_t idesc = instr_desc(nmma);

        for (int idx = tid; idx < NP * (Lt - 1); idx += THREADS) {
            const int p = idx % NP, r = idx / NP;
            const int J = tl.j0 + 2 * r;
            if (J >= tl.mu2[p]) coef[p * RMAX + r] = step_coef<float>(J, tl.n2[p], tl.m2);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            for (int c = 0; c < 2 && c < NCH; ++c) {
                mbar_arrive_expect_tx(&bar_full[c], (uint32_t)STAGE_BYTES);
                tma_load_5d(smem + OFF_STAGE + c * STAGE_BYTES, &tmap, tl.nb * NP, tl.mi, tl.s, c * KC, bb * BM,
                            &bar_full[c]);
            }
        }
        for (int c = 0; c < 2 && c < NCH; ++c) ++tma_iss[c];

        for (int c = 0; c < NCH; ++c) {
            const int st = c & 1;
            if (mma_iss[st] > mma_got[st]) {         // stage operands still read by earlier MMAs
                mbar_wait_bounded(&bar_mma[st], (mma_iss[st] - 1) & 1, a.err);
                mma_got[st] = mma_iss[st];
            }
            mbar_wait_bounded(&bar_full[st], tma_got[st] & 1, a.err);
            ++tma_got[st];
            unsigned char* Ab = smem + OFF_A + st * A_BYTES;
            unsigned char* Bb = smem + OFF_B + st * B_BYTES;
            if (tid < 128) {
                // ---- F2 (fp32) -> A_hi / A_lo, rows 2b (re) and 2b+1 (im), two nodes per item
                const float2* stg = reinterpret_cast<const float2*>(smem + OFF_STAGE + st * STAGE_BYTES);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = tid + 128 * j;
                    const int b = i >> 3, kp = i & 7;
                    const float4* src = reinterpret_cast<const float4*>(stg + (b * KC + 2 * kp) * NP);
                    const float4 q0 = src[0], q1 = src[1], q2 = src[2], q3 = src[3];
                    // node 2kp: pairs (q0.xy, q0.zw, q1.xy, q1.zw); node 2kp+1: (q2.xy, q2.zw, q3.xy, q3.zw)
                    const float re0[NP] = {q0.x, q0.z, q1.x, q1.z}, im0[NP] = {q0.y, q0.w, q1.y, q1.w};
                    const float re1[NP] = {q2.x, q2.z, q3.x, q3.z}, im1[NP] = {q2.y, q2.w, q3.y, q3.w};
                    const int ore = a_off(2 * b, 2 * kp), oim = a_off(2 * b + 1, 2 * kp);
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        uint32_t hr, lr, hi_, li;
                        split2(re0[p], re1[p], hr, lr);
                        split2(im0[p], im1[p], hi_, li);
                        *reinterpret_cast<uint32_t*>(Ab + p * OPB + ore) = hr;
                        *reinterpret_cast<uint32_t*>(Ab + p * OPB + oim) = hi_;
                        *reinterpret_cast<uint32_t*>(Ab + (NP + p) * OPB + ore) = lr;
                        *reinterpret_cast<uint32_t*>(Ab + (NP + p) * OPB + oim) = li;
                    }
                }
            } else if (tid < 128 + NP * KC) {
                // ---- recurrence for (pair p, node k) -> B_hi / B_lo column kk
                const int g = tid - 128, p = g >> 4, kk = g & 15, k = c * KC + kk;
                unsigned char* Bh = Bb + p * OPB;
                unsigned char* Bl = Bb + (NP + p) * OPB;
                const int colbase = (kk >> 3) * 128 + (kk & 7) * 16;
                if (!tl.valid[p]) {
                    for (int rb = 0; rb < nmma; rb += 8) {
                        *reinterpret_cast<uint4*>(Bh + (rb >> 3) * 256 + colbase) = make_uint4(0, 0, 0, 0);
                        *reinterpret_cast<uint4*>(Bl + (rb >> 3) * 256 + colbase) = make_uint4(0, 0, 0, 0);
                    }
                } else {
                    Rec<float> rc;
                    rc.seed(a, tl.n2[p], tl.m2, k);
                    const int rp = (tl.mu2[p] - tl.j0) / 2;
                    for (int rb = 0; rb < nmma; rb += 8) {
                        float v[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int r = rb + i;
                            if (r < rp || r >= Lt) {
                                v[i] = 0.f;
                            } else {
                                v[i] = rc.value();
                                if (r + 1 < Lt) rc.step(coef[p * RMAX + r]);
                            }
                        }
                        uint4 h, l;
                        split2(v[0], v[1], h.x, l.x);
                        split2(v[2], v[3], h.y, l.y);
                        split2(v[4], v[5], h.z, l.z);
                        split2(v[6], v[7], h.w, l.w);
                        *reinterpret_cast<uint4*>(Bh + (rb >> 3) * 256 + colbase) = h;
                        *reinterpret_cast<uint4*>(Bl + (rb >> 3) * 256 + colbase) = l;
                    }
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0 && c + 2 < NCH) {
                mbar_arrive_expect_tx(&bar_full[st], (uint32_t)STAGE_BYTES);
                tma_load_5d(smem + OFF_STAGE + st * STAGE_BYTES, &tmap, tl.nb * NP, tl.mi, tl.s, (c + 2) * KC,
                            bb * BM, &bar_full[st]);
            }
            if (c + 2 < NCH) ++tma_iss[st];
            if (tid == 32) {
                tc_fence_after();
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    if (!tl.valid[p]) continue;
                    const uint32_t d = taddr + (uint32_t)(p * 128);
                    const uint64_t ah = smem_desc(Ab + p * OPB), al = smem_desc(Ab + (NP + p) * OPB);
                    const uint64_t bh = smem_desc(Bb + p * OPB), bl = smem_desc(Bb + (NP + p) * OPB);
                    mma_bf16(d, ah, bh, idesc, c > 0);
                    mma_bf16(d, ah, bl, idesc, true);
                    mma_bf16(d, al, bh, idesc, true);
                }
                mma_commit(&bar_mma[st]);
            }
            ++mma_iss[st];
        }

        // ---- epilogue: TMEM -> coefficients
        {
            const int st = (NCH - 1) & 1;
            mbar_wait_bounded(&bar_mma[st], (mma_iss[st] - 1) & 1, a.err);
            mma_got[st] = mma_iss[st];
        }
        tc_fence_after();
        if (warp < 4) {
            const int row = 32 * warp + lane;
            const int fb = bb * BM + (row >> 1);
            const bool fok = fb < a.nfunc;
            const int f = fok ? a.fidx[fb] : 0;
            float2* cf = coeffs + (fok ? a.coeff_off[f] : 0);
            const bool even = (row & 1) == 0;
            for (int cc = 0; cc < nmma; cc += 16) {
                uint32_t rv[NP][16];
#pragma unroll
                for (int p = 0; p < NP; ++p)
                    tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)(p * 128 + cc), rv[p]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int r = cc + j;
                    float mine[NP], other[NP];
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        mine[p] = __uint_as_float(rv[p][j]);
                        other[p] = __shfl_xor_sync(0xffffffffu, mine[p], 1);
                    }
                    if (r >= Lt || !even || !fok) continue;
                    const int J = tl.j0 + 2 * r;
                    const size_t rowbase = block_offset(J) + (size_t)((tl.m2 + J) / 2) * (J + 1);
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        if (!tl.valid[p] || J < tl.mu2[p]) continue;
                        const float2 z = cmul_ipow(make_float2(mine[p], other[p]), (tl.n2[p] - tl.m2) / 2);
                        cf[rowbase + (tl.n2[p] + J) / 2] = z;
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    // drain: the last commit of the other stage may still be outstanding
    for (int st = 0; st < 2; ++st)
        if (mma_iss[st] > mma_got[st]) mbar_wait_bounded(&bar_mma[st], (mma_iss[st] - 1) & 1, a.err);
    tc_fence_after();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

template <int N>
static cudaError_t launch_n(const BandArgs& a, const void* ws, void* coeffs, cudaStream_t st) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[5] = {(cuuint64_t)N, (cuuint64_t)N, 2, (cuuint64_t)N, (cuuint64_t)a.nfunc};
    const cuuint64_t strides[4] = {(cuuint64_t)N * 8, (cuuint64_t)N * N * 8, (cuuint64_t)2 * N * N * 8,
                                   (cuuint64_t)2 * N * N * N * 8};
    const cuuint32_t box[5] = {NP, 1, 1, KC, BM};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    void* base = (void*)((const char*)ws + a.ws_group_off * sizeof(float2));
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    auto kern = contract_tc_kernel<N>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nitems = 2 * N * (N / NP) * ((a.nfunc + BM - 1) / BM);
    const int grid = sms < nitems ? sms : nitems;
    kern<<<grid, THREADS, SMEM_BYTES, st>>>(a, map, (float2*)coeffs);
    return cudaGetLastError();
}

}  // namespace tc

bool tc_supported(int N) { return N == 64 || N == 128 || N == 256; }

cudaError_t launch_contract_forward_tc(const BandArgs& a, const void* ws, void* coeffs, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    switch (a.N) {
        case 64: return tc::launch_n<64>(a, ws, coeffs, st);
        case 128: return tc::launch_n<128>(a, ws, coeffs, st);
        case 256: return tc::launch_n<256>(a, ws, coeffs, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace su2

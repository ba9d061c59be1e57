// The FP32 / FP64 forward contraction of one tile (fused recurrence + beta
// contraction, Sec. 4 discrete Legendre transform, Sec. 6 second-stage
// Proposition with depth 1) as a device function, shared by the per-group
// contraction kernel and the ragged-batch kernel.  The arithmetic is described
// at the top of contract.cu.
#pragma once

#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "recurrence.cuh"

namespace su2 {

template <typename T> __device__ __forceinline__ void store4(T* dst, const T (&v)[4]);
template <> __device__ __forceinline__ void store4<float>(float* dst, const float (&v)[4]) {
    *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
}
template <> __device__ __forceinline__ void store4<double>(double* dst, const double (&v)[4]) {
    reinterpret_cast<double2*>(dst)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(dst)[1] = make_double2(v[2], v[3]);
}

// ---------------------------------------------------------------------------
// Forward contraction
// ---------------------------------------------------------------------------
template <typename T, int NB, int BT, int KC, int LW, int ML, int MB>
struct FwdCfg {
    static constexpr int THREADS = NB * (LW / ML) * (BT / MB);
    static constexpr int LDD = LW + 4;
    static size_t smem_bytes(int N) {
        return sizeof(StepCoef<T>) * NB * (N / 2) + sizeof(T) * NB * KC * LDD + sizeof(cplx<T>) * KC * NB * BT +
               sizeof(SeedPair) * NB + sizeof(size_t) * BT;
    }
};

// Asynchronous global -> shared copy of one complex value (8 or 16 bytes), so a
// thread's loads of a chunk are all in flight together; cp_async_wait_all()
// before the barrier that publishes them.
template <typename C>
__device__ __forceinline__ void cp_async_cplx(C* dst, const C* src) {
    static_assert(sizeof(C) == 8 || sizeof(C) == 16, "complex64 or complex128");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "n"((int)sizeof(C)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One CTA's share of the forward contraction: tile `tile` (Tile<NB> numbering),
// function block bb (BT functions), rows of l from r0 (a window of LW).  All
// THREADS threads of the CTA call it; it synchronises them with __syncthreads.
// async_stage: stage F2 with cp.async (large batches), else through registers.
// smem_raw: FwdCfg::smem_bytes(N) bytes of shared memory, 16-byte aligned.
template <typename T, int NB, int BT, int KC, int LW, int ML, int MB>
__device__ __forceinline__ void contract_fwd_tile(const BandArgs& a, const cplx<T>* __restrict__ F2,
                                                  cplx<T>* __restrict__ coeffs, int tile, int bb, int r0,
                                                  bool async_stage, unsigned char* smem_raw) {
    using Cx = cplx<T>;
    using Cfg = FwdCfg<T, NB, BT, KC, LW, ML, MB>;
    constexpr int THREADS = Cfg::THREADS, LDD = Cfg::LDD;
    static_assert(NB * KC <= THREADS, "one generator thread per (pair, node)");
    const int N = a.N;
    Tile<NB> tl;
    tl.decode(N, tile);
    if (!tl.any) return;
    if (r0 >= tl.L) return;
    const int r_end = min(r0 + LW, tl.L);
    const int RS = N / 2;

    StepCoef<T>* coef = reinterpret_cast<StepCoef<T>*>(smem_raw);                 // [NB][RS]
    T* Dsm = reinterpret_cast<T*>(coef + NB * RS);                                 // [NB][KC][LDD]
    Cx* Fsm = reinterpret_cast<Cx*>(Dsm + NB * KC * LDD);                          // [KC][NB][BT]
    SeedPair* spair = reinterpret_cast<SeedPair*>(Fsm + KC * NB * BT);            // [NB] (FP32 seeds)
    size_t* fbase = reinterpret_cast<size_t*>(spair + NB);                         // [BT] (m, n-block) of each function
    const int tid = threadIdx.x;
    constexpr bool F32 = std::is_same<T, float>::value;
    if (F32 && tid < NB) spair[tid] = make_seed_pair(a.lf2, tl.n2[tid], tl.m2);
    constexpr size_t NOFN = ~(size_t)0;                                            // padding slot of the block
    for (int b = tid; b < BT; b += THREADS) {
        const int fb = bb * BT + b;
        fbase[b] = fb < a.nfunc ? a.ws_off[a.fidx[fb]] + (size_t)tl.mi * N + tl.nb * NB : NOFN;
    }

    // Step coefficients for rows r in [0, r_end - 1) of every pair.
    for (int idx = tid; idx < NB * (r_end - 1); idx += THREADS) {
        const int p = idx % NB, r = idx / NB;
        const int J = tl.j0 + 2 * r;
        if (J >= tl.mu2[p]) coef[p * RS + r] = step_coef<T>(J, tl.n2[p], tl.m2);
    }
    __syncthreads();

    constexpr int TPP = THREADS / NB;                 // threads per pair in the contraction
    const int pg = tid / TPP;
    const int lg = (tid % TPP) / (BT / MB);
    const int bg = (tid % TPP) % (BT / MB);
    Cx acc[ML][MB];
#pragma unroll
    for (int i = 0; i < ML; ++i)
#pragma unroll
        for (int j = 0; j < MB; ++j) acc[i][j] = mk<T>(T(0), T(0));
    const bool active = lg * ML < r_end - r0;

    for (int k0 = 0; k0 < N; k0 += KC) {
        if (tid < NB * KC) {
            // ---- recurrence for (pair p, node k), rows r0 .. r0+LW-1 into shared memory
            const int p = tid / KC, kk = tid % KC, k = k0 + kk;
            T* drow = Dsm + (p * KC + kk) * LDD;
            const bool live = tl.valid[p] && k < N;
            Rec<T> rc;
            bool fast = false;
            if constexpr (F32) {
                const int kc = live ? k : 0;
                rc.seed32(spair[p], a.seed32[kc], a.xsplit[kc], kc, N);
                if (!live) { rc.cur = 0.f; rc.E = 0; }
                fast = __all_sync(0xffffffffu, rc.E == 0);       // generator threads are whole warps
            } else if (live) {
                rc.seed(a, tl.n2[p], tl.m2, k);
            }
            if (!live) {
                for (int rb = 0; rb < LW; rb += 4) { const T z[4] = {T(0), T(0), T(0), T(0)}; store4<T>(drow + rb, z); }
            } else {
                auto adv = [&](const StepCoef<T>& c) {
                    if constexpr (F32) { if (fast) rc.step_fast(c); else rc.step(c); }
                    else rc.step(c);
                };
                int r = (tl.mu2[p] - tl.j0) / 2;      // row of the seed
                while (r < r0) { adv(coef[p * RS + r]); ++r; }
                for (int rb = 0; rb < LW; rb += 4) {
                    T v[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int rr = r0 + rb + i;
                        if (rr < r || rr >= r_end) {
                            v[i] = T(0);
                        } else {
                            v[i] = rc.value();
                            if (rr + 1 < r_end) { adv(coef[p * RS + rr]); r = rr + 1; }
                        }
                    }
                    store4<T>(drow + rb, v);
                }
            }
        } else {
            // ---- stage F2[k0 .. k0+KC) for the NB pairs and BT functions
            if (async_stage) {
                // row-class launches (large batches): asynchronous copies, all in flight
                for (int idx = tid - NB * KC; idx < KC * BT; idx += THREADS - NB * KC) {
                    const int kk = idx % KC, b = idx / KC;
                    const int k = k0 + kk;
                    const size_t base = fbase[b];
                    if (base != NOFN && k < N) {
                        const Cx* src = F2 + base + ((size_t)k * 2 + tl.s) * N * N;
#pragma unroll
                        for (int p = 0; p < NB; ++p) cp_async_cplx(&Fsm[(kk * NB + p) * BT + b], src + p);
                    } else {
#pragma unroll
                        for (int p = 0; p < NB; ++p) Fsm[(kk * NB + p) * BT + b] = mk<T>(T(0), T(0));
                    }
                }
                cp_async_wait_all();
            } else {
                // small batches: vector loads through registers (faster there, e.g. at
                // N = 512 with 8 functions per block)
                for (int idx = tid - NB * KC; idx < KC * BT; idx += THREADS - NB * KC) {
                    const int kk = idx % KC, b = idx / KC;
                    const int k = k0 + kk;
                    const size_t base = fbase[b];
                    Cx v[NB];
                    if (base != NOFN && k < N) {
                        const Cx* src = F2 + base + ((size_t)k * 2 + tl.s) * N * N;
#pragma unroll
                        for (int p = 0; p < NB; ++p) v[p] = src[p];
                    } else {
#pragma unroll
                        for (int p = 0; p < NB; ++p) v[p] = mk<T>(T(0), T(0));
                    }
#pragma unroll
                    for (int p = 0; p < NB; ++p) Fsm[(kk * NB + p) * BT + b] = v[p];
                }
            }
        }
        __syncthreads();
        if (active) {
            const int kc = min(KC, N - k0);
            for (int kk = 0; kk < kc; ++kk) {
                T dv[ML];
                const T* dsrc = Dsm + (pg * KC + kk) * LDD + lg * ML;
#pragma unroll
                for (int i = 0; i < ML; ++i) dv[i] = dsrc[i];
                Cx fv[MB];
                const Cx* fsrc = Fsm + (kk * NB + pg) * BT + bg * MB;
#pragma unroll
                for (int j = 0; j < MB; ++j) fv[j] = fsrc[j];
#pragma unroll
                for (int i = 0; i < ML; ++i)
#pragma unroll
                    for (int j = 0; j < MB; ++j) {
                        acc[i][j].x = fma(dv[i], fv[j].x, acc[i][j].x);
                        acc[i][j].y = fma(dv[i], fv[j].y, acc[i][j].y);
                    }
            }
        }
        __syncthreads();
    }

    // ---- epilogue: multiply by i^{n-m} and scatter to the packed layout
    if (!active || !tl.valid[pg]) return;
    const int n2 = tl.n2[pg], m2 = tl.m2;
#pragma unroll
    for (int i = 0; i < ML; ++i) {
        const int r = r0 + lg * ML + i;
        const int J = tl.j0 + 2 * r;
        if (r >= r_end || J < tl.mu2[pg]) continue;
        const size_t idx = block_offset(J) + (size_t)((m2 + J) / 2) * (J + 1) + (n2 + J) / 2;
#pragma unroll
        for (int j = 0; j < MB; ++j) {
            const int fb = bb * BT + bg * MB + j;
            if (fb >= a.nfunc) continue;
            const int f = a.fidx[fb];
            coeffs[a.coeff_off[f] + idx] = cmul_ipow(acc[i][j], (n2 - m2) / 2);
        }
    }
}

}  // namespace su2

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
// One persistent CTA per SM owns tiles of 4 consecutive n at fixed
// (sector, m) and 64 functions.  Warp roles, connected by mbarriers:
//   warp 0      TMA: F2 chunk [64 functions][16 nodes][4 n] into the ring of F2 / A
//               stages (the planes are tile-major, so a function's chunk is 512 B)
//   warp 1      MMA issue (one thread), tensor-memory owner
//   warps 2-5, 10-11  convert a landed F2 chunk (fp32) into the BF16 hi/lo A
//               operands in place: all of it is read into registers, the six
//               warps meet at a named barrier, then the operands are written
//               over the same 32 KB (hi and lo of 4 pairs fill it exactly)
//   warps 6-9 (and 16-17 at N = 256)  two (three) generator groups, chunk g to
//               group g mod 2 (3): the d-values of the 4 pairs x 16 nodes by the
//               three-term recurrence, written as the BF16 hi/lo B operands
//   warps 12-15 epilogue: tensor memory -> i^{n-m} * coefficients
// Four (three at N = 256) stages of F2 / A (a stage is reloaded once the MMAs
// that read it are done) and one B stage per generator group; the MMA commits
// free them.
// The recurrence is the critical path: each chunk's MMAs wait for its d-values,
// and a group can start its next chunk only once the MMAs of its previous one
// are done, so the number of groups (bounded by the B stages that fit in
// shared memory) sets the rate.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "recurrence.cuh"
#include "su2_internal.h"
#include "tc_common.cuh"

namespace su2 {
namespace tc {

constexpr int RMAX = 128;                   // rows of l per pair (N <= 256)
constexpr int NMAX = 256;

constexpr int W_GEN3 = 16;                  // warps 16-17: the third generator group (N = 256)
// Shared-memory layout for NG generator groups (= B stages): three at N = 256,
// where the recurrence over up to 128 rows of l is the critical path, two
// (with a fourth F2 / A stage) at N <= 128, where a third group's warps only
// take issue slots from the others (measured: N = 256 x 64 6.76 -> 6.12 ms,
// N = 128 x 64 0.75 -> 0.85 ms with three).
template <int NG>
struct Lay {
    static constexpr int NSK = NG == 3 ? 3 : 4;        // F2 / A stages
    static constexpr int THREADS = (NWARPS + 2 * (NG - 2)) * 32;
    static constexpr int OFF_STG = 0;                  // stage st at OFF_STG + st * SA (F2, then its A operands)
    static constexpr int OFF_B = OFF_STG + NSK * SA;
    static constexpr int OFF_COEF = OFF_B + NG * B_BYTES;
    static constexpr int OFF_TAB = OFF_COEF + NG * NP * RMAX * (int)sizeof(StepCoef<float>);
    // seed32 (float4) + lf2 (double) + xsplit (float2) + seed parameters of the pairs
    static constexpr int TAB_BYTES = NMAX * 16 + NMAX * 8 + NMAX * 8 + NG * NP * (int)sizeof(SeedPair) + NMAX * 4;
    static constexpr int OFF_BAR = OFF_TAB + TAB_BYTES;
    static constexpr int NBAR = 3 * NSK + 2 * NG + 4;
    static constexpr int SMEM_BYTES = OFF_BAR + NBAR * 8 + 16;
    static_assert(SMEM_BYTES <= 232448, "shared memory budget");
};
template <int N> constexpr int ngroups() { return N >= 256 ? 3 : 2; }
constexpr uint32_t TMEM_COLS = 512;         // 4 pairs x 128 columns, or two halves of 4 x 64
// Accumulator placement: a tile with at most 64 rows of l ("small") takes one
// half of tensor memory (pairs 64 columns apart), alternating halves, so its
// MMAs overlap the epilogue of the previous tile; a larger tile takes both
// (pair p at column 128 p) and its epilogue drains pairs 0, 1 first and frees
// half 0 before it reads pairs 2, 3, so the next tile starts in half 0.
__device__ __forceinline__ void acc_place(int nmma, int& nexth, int& h0, bool& big) {
    big = nmma > 64;
    h0 = big ? 0 : nexth;
    nexth = big ? 0 : (nexth ^ 1);     // after a big tile, half 0 (drained first) comes next
}

template <int N>
__global__ void __launch_bounds__(Lay<ngroups<N>()>::THREADS, 1)
contract_tc_kernel(BandArgs a, const __grid_constant__ CUtensorMap tmap, float2* __restrict__ coeffs) {
    constexpr int NGRP = ngroups<N>();
    using L = Lay<NGRP>;
    constexpr int NSK = L::NSK, THREADS_K = L::THREADS, OFF_STG = L::OFF_STG, OFF_B = L::OFF_B,
                  OFF_COEF = L::OFF_COEF, OFF_TAB = L::OFF_TAB, OFF_BAR = L::OFF_BAR, NBAR = L::NBAR;
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int NCH = N / KC;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OFF_BAR);
    uint64_t* bar_full = bars + 0;               // [NSK] TMA landed              (count 1 + tx)
    uint64_t* bar_afull = bars + NSK;            // [NSK] A operands written      (count N_CONV)
    uint64_t* bar_opa = bars + 2 * NSK;          // [NSK] MMAs of the A stage done (tcgen05.commit)
    uint64_t* bar_bfull = bars + 3 * NSK;        // [NGRP] B operands written     (count 2)
    uint64_t* bar_opb = bar_bfull + NGRP;        // [NGRP] MMAs of the B stage done (tcgen05.commit)
    uint64_t* bar_accfull = bar_opb + NGRP;      // [2] accumulators of a tile in half h final (tcgen05.commit)
    uint64_t* bar_hfree = bar_accfull + 2;       // [2] epilogue drained half h    (count 4)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + NBAR);
    float4* t_seed = reinterpret_cast<float4*>(smem + OFF_TAB);
    double* t_lf2 = reinterpret_cast<double*>(t_seed + NMAX);
    float2* t_xs = reinterpret_cast<float2*>(t_lf2 + NMAX);
    SeedPair* t_gp = reinterpret_cast<SeedPair*>(t_xs + NMAX);      // [NGRP groups][NP]
    uint32_t* t_rowoff = reinterpret_cast<uint32_t*>(t_gp + NGRP * NP); // J(J+1)(2J+1)/6, J = 2l
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int t = tid; t < N; t += THREADS_K) {
        t_seed[t] = a.seed32[t];
        t_lf2[t] = a.lf2[t];
        t_xs[t] = a.xsplit[t];
        t_rowoff[t] = (uint32_t)block_offset(t);
    }
    if (warp == W_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tslot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < NSK; ++i) {
            mbar_init(&bar_full[i], 1);
            mbar_init(&bar_afull[i], N_CONV);
            mbar_init(&bar_opa[i], 1);
        }
        for (int i = 0; i < NGRP; ++i) {
            mbar_init(&bar_bfull[i], 2);
            mbar_init(&bar_opb[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_accfull[i], 1);
            mbar_init(&bar_hfree[i], 4);
        }
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;


    // tiles [tc_t0, tc_t0 + ntiles) of the global numbering (all of them by default)
    const int ntiles = a.tc_ntiles ? a.tc_ntiles : 2 * N * (N / NP);
    const int nbb = (a.nfunc + BM - 1) / BM;
    const int nitems = ntiles * nbb;

    if (warp == W_TMA) {
        // ------------------------------------------------------------------ TMA
        if (lane == 0) {
            uint64_t pol;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
            uint32_t g = 0;
            for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
                Tile<NP> tl;
                tl.decode(N, a.tc_t0 + item / nbb);
                if (!tl.any) continue;
                const int bb = item % nbb;
                for (int c = 0; c < NCH; ++c, ++g) {
                    const int st = g % NSK;
                    const uint32_t u = g / NSK;
                    if (u > 0) mbar_wait_bounded(&bar_opa[st], (u - 1) & 1, a.err);   // its A operands read
                    mbar_arrive_expect_tx(&bar_full[st], (uint32_t)STAGE_BYTES);
                    if (a.xrecv) {        // [source][row][fb][n/4][node][n%4], nk nodes per source
                        const int kg = c * KC;
                        tma_load_5d(smem + OFF_STG + st * SA, &tmap, (kg % a.nk) * NP, tl.nb, bb * BM,
                                    tl.s * N + tl.mi - a.x_row0, kg / a.nk, &bar_full[st], pol);
                    } else {
                        tma_load_5d(smem + OFF_STG + st * SA, &tmap, c * KC * NP, tl.nb, tl.mi, tl.s, bb * BM,
                                    &bar_full[st], pol);
                    }
                }
            }
        }
    } else if (warp == W_MMA) {
        // ------------------------------------------------------------------ MMA
        if (lane == 0) {
            uint32_t g = 0, uses[2] = {0, 0};
            int nexth = 0;
            for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
                Tile<NP> tl;
                tl.decode(N, a.tc_t0 + item / nbb);
                if (!tl.any) continue;
                const int nmma = (tl.L + 15) & ~15;
                const uint32_t idesc = instr_desc(nmma);
                int h0;
                bool big;
                acc_place(nmma, nexth, h0, big);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h != h0 && !big) continue;
                    if (uses[h] > 0) mbar_wait_bounded(&bar_hfree[h], (uses[h] - 1) & 1, a.err);
                    ++uses[h];
                }
                const uint32_t base = taddr + (uint32_t)(h0 * 256);
                const uint32_t pstride = big ? 128u : 64u;
                tc_fence_after();
                for (int c = 0; c < NCH; ++c, ++g) {
                    const int sa = g % NSK, sb = g % NGRP;
                    mbar_wait_bounded(&bar_afull[sa], (g / NSK) & 1, a.err);
                    mbar_wait_bounded(&bar_bfull[sb], (g / NGRP) & 1, a.err);
                    tc_fence_after();
                    unsigned char* Ab = smem + OFF_STG + sa * SA;
                    unsigned char* Bb = smem + OFF_B + sb * B_BYTES;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        if (!tl.valid[p]) continue;
                        const uint32_t d = base + (uint32_t)p * pstride;
                        const uint64_t ah = smem_desc(Ab + p * OPA, LBO_A, SBO_A);
                        const uint64_t al = smem_desc(Ab + (NP + p) * OPA, LBO_A, SBO_A);
                        const uint64_t bh = smem_desc(Bb + p * OPB, LBO_B, SBO_B);
                        const uint64_t bl = smem_desc(Bb + (NP + p) * OPB, LBO_B, SBO_B);
                        mma_bf16(d, ah, bh, idesc, c > 0);
                        mma_bf16(d, ah, bl, idesc, true);
                        mma_bf16(d, al, bh, idesc, true);
                    }
                    mma_commit(&bar_opa[sa]);
                    mma_commit(&bar_opb[sb]);
                }
                mma_commit(&bar_accfull[h0]);
            }
        }
    } else if ((warp >= W_CONV && warp < W_CONV + 4) || warp == W_CONV2 || warp == W_CONV2 + 1) {
        // ------------------------------------------------------------------ F2 -> A (bf16 hi/lo)
        // Item = (function b, node group t, pair p): four staged values (nodes t,
        // t + 4, t + 8, t + 12 at K positions 4t .. 4t + 3 of the chunk) -> two
        // bf16x2 words (8 bytes) per row (re: 2b, im: 2b+1) for hi and lo.  With this
        // K order 16 lanes read 16 consecutive staged values (no bank conflicts) and
        // the stores are 8 bytes; the generators write the d-values in the same order.
        const int cw = (warp < W_CONV + 4) ? warp - W_CONV : 4 + (warp - W_CONV2);
        const int ct = cw * 32 + lane;                     // 0 .. 191
        constexpr int NIT = BM * (KC / 4) * NP;            // 1024 items per chunk
        constexpr int MAXI = (NIT + 32 * N_CONV - 1) / (32 * N_CONV);
        uint32_t g = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
            Tile<NP> tl;
            tl.decode(N, a.tc_t0 + item / nbb);
            if (!tl.any) continue;
            for (int c = 0; c < NCH; ++c, ++g) {
                const int st = g % NSK;
                mbar_wait_bounded(&bar_full[st], (g / NSK) & 1, a.err);   // stage free: TMA waited for the MMAs
                const float2* stg = reinterpret_cast<const float2*>(smem + OFF_STG + st * SA);
                unsigned char* Ab = smem + OFF_STG + st * SA;
                // every converter reads its items of the staged chunk before any of
                // them overwrites the chunk with the operands
                float2 v[MAXI][4];
#pragma unroll
                for (int j = 0; j < MAXI; ++j) {
                    const int i = ct + 32 * N_CONV * j;
                    if (i < NIT) {
                        const int p = i & 3, t = (i >> 2) & 3, b = i >> 4;
#pragma unroll
                        for (int q = 0; q < 4; ++q) v[j][q] = stg[(b * KC + t + 4 * q) * NP + p];
                    }
                }
                named_sync(3, 32 * N_CONV);
#pragma unroll
                for (int j = 0; j < MAXI; ++j) {
                    const int i = ct + 32 * N_CONV * j;
                    if (i < NIT) {
                        const int p = i & 3, t = (i >> 2) & 3, b = i >> 4;
                        uint2 hr, lr, hi_, li;
                        split2(v[j][0].x, v[j][1].x, hr.x, lr.x);
                        split2(v[j][2].x, v[j][3].x, hr.y, lr.y);
                        split2(v[j][0].y, v[j][1].y, hi_.x, li.x);
                        split2(v[j][2].y, v[j][3].y, hi_.y, li.y);
                        const int ore = a_off(2 * b, 4 * t), oim = a_off(2 * b + 1, 4 * t);
                        *reinterpret_cast<uint2*>(Ab + p * OPA + ore) = hr;
                        *reinterpret_cast<uint2*>(Ab + p * OPA + oim) = hi_;
                        *reinterpret_cast<uint2*>(Ab + (NP + p) * OPA + ore) = lr;
                        *reinterpret_cast<uint2*>(Ab + (NP + p) * OPA + oim) = li;
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_afull[st]);
            }
        }
    } else if ((warp >= W_GEN && warp < W_GEN + 4) || warp == W_GEN3 || warp == W_GEN3 + 1) {
        // ------------------------------------------------------------------ recurrence -> B (bf16 hi/lo)
        // Thread (p, kk) runs the chain of pair p at node c*KC + kk/4 + 4*(kk%4) (K
        // position kk, the order the converters use) for the chunks of
        // its group's stage.  Seeds in FP32 from the split logarithms (exact
        // products and sums; only the pair's factorial ratio K is FP64, once per
        // tile).  Range extension: value = cur * 2^(-120 E); while E > 0 the value is
        // below 2^-39 and enters as 0.  A warp whose chains all have E = 0 runs the
        // plain recurrence; otherwise cur is renormalised once per 8 rows when
        // |cur| >= 2^40 (8 steps grow it by less than 2^41, so it stays finite).
        const int grp = warp >= W_GEN3 ? 2 : (warp - W_GEN) >> 1;   // handles the chunks of stage grp
        const int gt = tid - (warp >= W_GEN3 ? W_GEN3 * 32 : W_GEN * 32 + grp * 64);   // 0..63
        const int p = gt >> 4, kk = gt & 15;
        StepCoef<float>* coef = reinterpret_cast<StepCoef<float>*>(smem + OFF_COEF) + grp * NP * RMAX;
        SeedPair* gp = t_gp + grp * NP;
        uint32_t g = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
            Tile<NP> tl;
            tl.decode(N, a.tc_t0 + item / nbb);
            if (!tl.any) continue;
            const int Lt = tl.L, nmma = (Lt + 15) & ~15;
            named_sync(grp == 2 ? 4 : 1 + grp, 64);        // previous tile's tables no longer read
            for (int idx = gt; idx < NP * (Lt - 1); idx += 64) {
                const int pp = idx % NP, r = idx / NP;
                const int J = tl.j0 + 2 * r;
                if (J >= tl.mu2[pp]) coef[pp * RMAX + r] = step_coef<float>(J, tl.n2[pp], tl.m2);
            }
            if (gt < NP) gp[gt] = make_seed_pair(t_lf2, tl.n2[gt], tl.m2);
            named_sync(grp == 2 ? 4 : 1 + grp, 64);
            const bool valid = tl.valid[p];
            const int rp = valid ? (tl.mu2[p] - tl.j0) / 2 : nmma;   // first row of my pair
            const SeedPair q = gp[p];
            const StepCoef<float>* cp = coef + p * RMAX;
            for (int c = 0; c < NCH; ++c, ++g) {
                const int st = g % NGRP;
                if (st != grp) continue;
                const uint32_t u = g / NGRP;
                if (u > 0) mbar_wait_bounded(&bar_opb[st], (u - 1) & 1, a.err);
                unsigned char* Bh = smem + OFF_B + st * B_BYTES + p * OPB + (kk >> 3) * LBO_B + (kk & 7) * 16;
                unsigned char* Bl = Bh + NP * OPB;
                const int k = c * KC + ((kk >> 2) | ((kk & 3) << 2));   // node at K position kk
                // seed
                int E;
                float cur = seed_value32(q, t_seed[k], k, N, E);
                float prev = 0.f;
                const float2 xs = t_xs[k];
                const bool fast = __all_sync(0xffffffffu, E == 0);
                // blocks of 8 rows entirely before my pair's first row: zeros
                int rb = 0;
                for (; rb + 8 <= rp && rb < nmma; rb += 8) {
                    *reinterpret_cast<uint4*>(Bh + (rb >> 3) * SBO_B) = make_uint4(0, 0, 0, 0);
                    *reinterpret_cast<uint4*>(Bl + (rb >> 3) * SBO_B) = make_uint4(0, 0, 0, 0);
                }
                for (; rb < nmma; rb += 8) {
                    float v[8];
                    const bool full_blk = (rb >= rp) && (rb + 8 < Lt);   // 8 active rows, each stepped
                    if (fast && full_blk) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const StepCoef<float> cf = cp[rb + i];
                            v[i] = cur;
                            const float xb = (xs.x - cf.bh) + (xs.y - cf.bl);
                            const float nxt = fmaf(cf.A * xb, cur, -cf.C * prev);
                            prev = cur;
                            cur = nxt;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int r = rb + i;
                            if (r < rp || r >= Lt) {
                                v[i] = 0.f;
                            } else {
                                v[i] = (E == 0) ? cur : 0.f;
                                if (r + 1 < Lt) {
                                    const StepCoef<float> cf = cp[r];
                                    const float xb = (xs.x - cf.bh) + (xs.y - cf.bl);
                                    const float nxt = fmaf(cf.A * xb, cur, -cf.C * prev);
                                    prev = cur;
                                    cur = nxt;
                                }
                            }
                        }
                        if (E > 0 && fabsf(cur) >= 1.099511627776e12f) {   // 2^40
                            cur *= 7.52316384526264e-37f;                    // 2^-120
                            prev *= 7.52316384526264e-37f;
                            --E;
                        }
                    }
                    uint4 h, l;
                    split2(v[0], v[1], h.x, l.x);
                    split2(v[2], v[3], h.y, l.y);
                    split2(v[4], v[5], h.z, l.z);
                    split2(v[6], v[7], h.w, l.w);
                    *reinterpret_cast<uint4*>(Bh + (rb >> 3) * SBO_B) = h;
                    *reinterpret_cast<uint4*>(Bl + (rb >> 3) * SBO_B) = l;
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_bfull[st]);
            }
        }
    } else if (warp >= W_EPI && warp < W_EPI + 4) {
        // ------------------------------------------------------------------ epilogue
        const int q = warp - W_EPI;                          // TMEM lane quadrant (warp % 4)
        uint32_t commits[2] = {0, 0};
        int nexth = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
            Tile<NP> tl;
            tl.decode(N, a.tc_t0 + item / nbb);
            if (!tl.any) continue;
            const int bb = item % nbb;
            const int Lt = tl.L, nmma = (Lt + 15) & ~15;
            int h0;
            bool big;
            acc_place(nmma, nexth, h0, big);
            mbar_wait_bounded(&bar_accfull[h0], commits[h0] & 1, a.err);
            ++commits[h0];
            tc_fence_after();
            const uint32_t base = taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)(h0 * 256);
            const uint32_t pstride = big ? 128u : 64u;
            // After the TMEM load lane l holds row 32q + l (function 16q + l/2; re for
            // even l, im for odd l) of every pair.  Lanes 2f and 2f + 1 complete their
            // values with one exchange per pair they write (shfl.xor 1): the even lane
            // writes the lower pairs of function 16q + l/2, the odd lane the upper ones.
            const int fbl = bb * BM + 16 * q + (lane >> 1);
            const bool okl = fbl < a.nfunc;
            float2* cfl = coeffs + (okl ? a.coeff_off[a.fidx[fbl]] : 0);
            const bool odd = lane & 1;
            if (big) {
                // two halves: pairs 0, 1 (columns 0..255) then pairs 2, 3; half 0 is
                // released as soon as it is drained.  Lane l writes pair 2g + l % 2.
#pragma unroll 1
                for (int g = 0; g < 2; ++g) {
                    const int p2 = 2 * g + (lane & 1);
                    const int n2t = tl.n2[p2], mu2t = tl.mu2[p2];
                    const bool vt = tl.valid[p2] && okl;
                    const int ipw = (n2t - tl.m2) / 2;
                    for (int cc = 0; cc < nmma; cc += 16) {
                        uint32_t rv[2][16];
#pragma unroll
                        for (int pp = 0; pp < 2; ++pp)
                            tmem_ld16(base + (uint32_t)(2 * g + pp) * 128u + (uint32_t)cc, rv[pp]);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int r = cc + j;
                            const int J = tl.j0 + 2 * r;
                            const size_t rowbase =
                                (size_t)t_rowoff[J < N ? J : N - 1] + (size_t)((tl.m2 + J) / 2) * (J + 1);
                            // even lane: re of pair 2g is its own, im comes from the odd lane;
                            // odd lane: im of pair 2g + 1 is its own, re comes from the even lane
                            const float v0 = __uint_as_float(rv[0][j]), v1 = __uint_as_float(rv[1][j]);
                            const float own = odd ? v1 : v0;
                            const float x = __shfl_xor_sync(0xffffffffu, odd ? v0 : v1, 1);
                            const float re = odd ? x : own, im = odd ? own : x;
                            if (r < Lt && vt && J >= mu2t)
                                __stcs(&cfl[rowbase + (n2t + J) / 2], cmul_ipow(make_float2(re, im), ipw));
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar_hfree[g]);
                }
                continue;
            }
            // lane l writes pairs pa = 2 (l % 2) and pa + 1 of its function
            const int pa = odd ? 2 : 0;
            const int n2a = tl.n2[pa], mu2a = tl.mu2[pa], n2b = tl.n2[pa + 1], mu2b = tl.mu2[pa + 1];
            const bool va = tl.valid[pa] && okl, vb = tl.valid[pa + 1] && okl;
            const int ipa = (n2a - tl.m2) / 2, ipb = (n2b - tl.m2) / 2;
            for (int cc = 0; cc < nmma; cc += 16) {
                uint32_t rv[NP][16];
#pragma unroll
                for (int pp = 0; pp < NP; ++pp)
                    tmem_ld16(base + (uint32_t)pp * pstride + (uint32_t)cc, rv[pp]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int r = cc + j;
                    const int J = tl.j0 + 2 * r;
                    const size_t rowbase = (size_t)t_rowoff[J < N ? J : N - 1] + (size_t)((tl.m2 + J) / 2) * (J + 1);
                    // even lane sends re of pairs 2, 3 and receives im of pairs 0, 1;
                    // odd lane sends im of pairs 0, 1 and receives re of pairs 2, 3
                    const float v0 = __uint_as_float(rv[0][j]), v1 = __uint_as_float(rv[1][j]);
                    const float v2 = __uint_as_float(rv[2][j]), v3 = __uint_as_float(rv[3][j]);
                    const float x0 = __shfl_xor_sync(0xffffffffu, odd ? v0 : v2, 1);
                    const float x1 = __shfl_xor_sync(0xffffffffu, odd ? v1 : v3, 1);
                    const float o0 = odd ? v2 : v0, o1 = odd ? v3 : v1;
                    const float2 za = odd ? make_float2(x0, o0) : make_float2(o0, x0);
                    const float2 zb = odd ? make_float2(x1, o1) : make_float2(o1, x1);
                    // the two pairs are adjacent coefficients: one 16-byte store where the
                    // address allows it (a store's cost follows the lines it touches, so
                    // two 8-byte stores of 16 functions each cost about twice one of 16 bytes)
                    const bool wa = r < Lt && va && J >= mu2a, wb = r < Lt && vb && J >= mu2b;
                    float2* pz = &cfl[rowbase + (n2a + J) / 2];
                    const float2 ya = cmul_ipow(za, ipa), yb = cmul_ipow(zb, ipb);
                    if (wa && wb && ((reinterpret_cast<uintptr_t>(pz) & 15) == 0)) {
                        __stcs(reinterpret_cast<float4*>(pz), make_float4(ya.x, ya.y, yb.x, yb.y));   // written once
                    } else {
                        if (wa) __stcs(pz, ya);
                        if (wb) __stcs(pz + 1, yb);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&bar_hfree[h0]);
                if (big) mbar_arrive(&bar_hfree[1]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == W_MMA)
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
    CUtensorMap map;
    if (a.xrecv) {
        // received exchange layout [N/nk sources][x_nrows rows][nfunc][N/4][nk][4]: a chunk
        // (16 nodes x 4 consecutive n) of one function is 512 contiguous bytes (nk % 16 == 0)
        const cuuint64_t nk = (cuuint64_t)a.nk, n = (cuuint64_t)N, nf = (cuuint64_t)a.nfunc;
        const cuuint64_t dims[5] = {nk * NP, n / NP, nf, (cuuint64_t)a.x_nrows, n / nk};
        const cuuint64_t strides[4] = {nk * NP * 8, n * nk * 8, nf * n * nk * 8, (cuuint64_t)a.x_nrows * nf * n * nk * 8};
        const cuuint32_t box[5] = {KC * NP, 1, BM, 1, 1};
        if (!encode_tensor_map_8b(&map, 5, a.xrecv, dims, strides, box)) return cudaErrorNotSupported;
    } else {
        // tile-major planes of a function: [s][mi][ni/4][k][ni%4]; one chunk of a tile
        // (16 nodes x 4 consecutive n) is 512 contiguous bytes per function
        if (!a.ws_tile_major) return cudaErrorInvalidValue;
        const cuuint64_t dims[5] = {(cuuint64_t)N * NP, (cuuint64_t)N / NP, (cuuint64_t)N, 2, (cuuint64_t)a.nfunc};
        const cuuint64_t strides[4] = {(cuuint64_t)N * NP * 8, (cuuint64_t)N * N * 8, (cuuint64_t)N * N * N * 8,
                                       (cuuint64_t)2 * N * N * N * 8};
        const cuuint32_t box[5] = {KC * NP, 1, 1, 1, BM};
        const void* base = (const char*)ws + a.ws_group_off * sizeof(float2);
        if (!encode_tensor_map_8b(&map, 5, base, dims, strides, box)) return cudaErrorNotSupported;
    }
    using L = Lay<ngroups<N>()>;
    auto kern = contract_tc_kernel<N>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nitems = (a.tc_ntiles ? a.tc_ntiles : 2 * N * (N / NP)) * ((a.nfunc + BM - 1) / BM);
    const int grid = sms < nitems ? sms : nitems;
    kern<<<grid, L::THREADS, L::SMEM_BYTES, st>>>(a, map, (float2*)coeffs);
    return cudaGetLastError();
}

}  // namespace tc

bool encode_tensor_map_8b(CUtensorMap* map, int rank, const void* base, const cuuint64_t* dims,
                          const cuuint64_t* strides_bytes, const cuuint32_t* box) {
    tc::EncodeTiledFn enc = tc::encode_fn();
    if (!enc) return false;
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank, const_cast<void*>(base), dims,
                     strides_bytes, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

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

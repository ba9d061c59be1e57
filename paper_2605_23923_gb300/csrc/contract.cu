// Stage 2 of the SU(2) transform: the beta contraction (Sec. 4, discrete
// Legendre transform <s, P^l_{nm}>; Sec. 6 second-stage Proposition, depth 1)
// with the Wigner-d values regenerated on chip by their three-term recurrence
// in l (Sec. 4 Lemma; its Jacobi analogue for general m, n):
//
//   f^(l)_{mn} = i^{n-m} sum_k d^l_{nm}(beta_k) F2_s[k][m][n]      (F2 already carries w_k/(2N^2))
//   d^{l+1} = A_l (x - b_l) d^l - C_l d^{l-1},   x = cos(beta_k),
//   A_l = (l+1)(2l+1) / sqrt(((l+1)^2-n^2)((l+1)^2-m^2)),  b_l = nm / (l(l+1)),
//   C_l = (l+1)/l * sqrt((l^2-n^2)(l^2-m^2)) / sqrt(((l+1)^2-n^2)((l+1)^2-m^2)),
//   seeded at l = mu = max(|n|,|m|) by the closed form of the Rodrigues-type
//   formula there (factorials and half-angle powers summed in FP64 log2 space).
//
// FP32 path details (all arithmetic FP32 except the seed logarithm):
// * x - b_l is formed from double-float splits of x and b_l, so that the
//   difference keeps full relative precision near the turning point;
// * range extension: the recurrence state is d~ = d * 2^(120 E) with an
//   integer E >= 0 per (pair, node); while E > 0 the state is renormalised by
//   2^-120 whenever |d~| reaches 2^60, and a value with E > 0 (|d| < 2^-60)
//   contributes zero.  Seeds far below the FP32 range (1e-41 and smaller at
//   N = 256) are therefore carried exactly.
//
// Tiling: a CTA owns NB = 4 consecutive n at fixed (sector, m), a block of BT
// functions and a window of LW rows of l.  Per chunk of KC beta nodes, half the
// CTA runs the NB*KC recurrences into shared memory while the other half
// stages the F2 chunk; then all threads run the register-tiled contraction
// acc[l][b] += d[l][k] * F2[k][b].
#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "contract_fwd.cuh"
#include "recurrence.cuh"
#include "su2_internal.h"

namespace su2 {

template <typename T, int NB, int BT, int KC, int LW, int ML, int MB>
__global__ void __launch_bounds__(FwdCfg<T, NB, BT, KC, LW, ML, MB>::THREADS)
contract_fwd(BandArgs a, const cplx<T>* __restrict__ F2, cplx<T>* __restrict__ coeffs,
             const int* __restrict__ tiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // tiles: one row class of them (large batches, asynchronous staging)
    contract_fwd_tile<T, NB, BT, KC, LW, ML, MB>(a, F2, coeffs, tiles ? tiles[blockIdx.x] : (int)blockIdx.x,
                                                 (int)blockIdx.y, (int)blockIdx.z * LW, tiles != nullptr, smem_raw);
}

// ---------------------------------------------------------------------------
// Transposed contraction (synthesis / adjoint):
//   G_s[k][m][n] = rho(k) sum_l wl(l) i^{m-n} d^l_{nm}(beta_k) c(l)_{mn}
//   synthesis: wl = 2l+1, rho = 1;  adjoint: wl = 1, rho = w_k/(2N^2).
// A CTA owns NB consecutive n at fixed (sector, m) and BT functions; the whole
// l range is kept in shared memory (weighted coefficients and, per chunk of
// KC nodes, the recurrence values).
// ---------------------------------------------------------------------------
template <typename T, int NB, int BT, int KC, int MK, int MB>
struct TrCfg {
    static constexpr int THREADS = NB * (KC / MK) * (BT / MB);
    static size_t smem_bytes(int N) {
        const int RS = N / 2;
        return sizeof(StepCoef<T>) * NB * RS + sizeof(T) * NB * RS * KC + sizeof(cplx<T>) * NB * RS * BT +
               sizeof(SeedPair) * NB;
    }
};

template <typename T, int NB, int BT, int KC, int MK, int MB>
__global__ void __launch_bounds__(TrCfg<T, NB, BT, KC, MK, MB>::THREADS)
contract_tr(BandArgs a, int mode, const cplx<T>* __restrict__ coeffs, cplx<T>* __restrict__ G) {
    using Cx = cplx<T>;
    using Cfg = TrCfg<T, NB, BT, KC, MK, MB>;
    constexpr int THREADS = Cfg::THREADS;
    static_assert(NB * KC <= THREADS, "one generator thread per (pair, node)");
    const int N = a.N;
    Tile<NB> tl;
    tl.decode(N, blockIdx.x);
    if (!tl.any) return;
    const int bb = blockIdx.y;
    const int RS = N / 2;
    const int L = tl.L;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepCoef<T>* coef = reinterpret_cast<StepCoef<T>*>(smem_raw);   // [NB][RS]
    T* Dsm = reinterpret_cast<T*>(coef + NB * RS);                   // [NB][RS][KC]
    Cx* Csm = reinterpret_cast<Cx*>(Dsm + NB * RS * KC);             // [NB][RS][BT]
    SeedPair* spair = reinterpret_cast<SeedPair*>(Csm + NB * RS * BT); // [NB] (FP32 seeds)
    const int tid = threadIdx.x;
    constexpr bool F32 = std::is_same<T, float>::value;
    if (F32 && tid < NB) spair[tid] = make_seed_pair(a.lf2, tl.n2[tid], tl.m2);

    for (int idx = tid; idx < NB * (L - 1); idx += THREADS) {
        const int p = idx % NB, r = idx / NB;
        const int J = tl.j0 + 2 * r;
        if (J >= tl.mu2[p]) coef[p * RS + r] = step_coef<T>(J, tl.n2[p], tl.m2);
    }
    for (int idx = tid; idx < NB * L * BT; idx += THREADS) {
        const int b = idx % BT, r = (idx / BT) % L, p = idx / (BT * L);
        const int J = tl.j0 + 2 * r;
        const int fb = bb * BT + b;
        Cx v = mk<T>(T(0), T(0));
        if (tl.valid[p] && J >= tl.mu2[p] && fb < a.nfunc) {
            const int f = a.fidx[fb];
            const size_t ci = block_offset(J) + (size_t)((tl.m2 + J) / 2) * (J + 1) + (tl.n2[p] + J) / 2;
            v = cmul_ipow(coeffs[a.coeff_off[f] + ci], (tl.m2 - tl.n2[p]) / 2);
            if (mode == 0) v = cscale(v, T(J + 1));
        }
        Csm[(p * RS + r) * BT + b] = v;
    }
    __syncthreads();

    constexpr int TPP = THREADS / NB;
    const int pg = tid / TPP;
    const int kg = (tid % TPP) / (BT / MB);
    const int bg = (tid % TPP) % (BT / MB);
    const T inv2n2 = T(1) / (T(2) * T(N) * T(N));

    for (int k0 = 0; k0 < N; k0 += KC) {
        if (tid < NB * KC) {
            const int p = tid / KC, kk = tid % KC, k = k0 + kk;
            T* dcol = Dsm + p * RS * KC + kk;
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
                for (int r = 0; r < L; ++r) dcol[r * KC] = T(0);
            } else {
                const int rs = (tl.mu2[p] - tl.j0) / 2;
                for (int r = 0; r < rs; ++r) dcol[r * KC] = T(0);
                if constexpr (F32) {
                    if (fast) {
                        for (int r = rs; r < L; ++r) {
                            dcol[r * KC] = rc.cur;
                            if (r + 1 < L) rc.step_fast(coef[p * RS + r]);
                        }
                    } else {
                        for (int r = rs; r < L; ++r) {
                            dcol[r * KC] = rc.value();
                            if (r + 1 < L) rc.step(coef[p * RS + r]);
                        }
                    }
                } else {
                    for (int r = rs; r < L; ++r) {
                        dcol[r * KC] = rc.value();
                        if (r + 1 < L) rc.step(coef[p * RS + r]);
                    }
                }
            }
        }
        __syncthreads();
        Cx acc[MK][MB];
#pragma unroll
        for (int i = 0; i < MK; ++i)
#pragma unroll
            for (int j = 0; j < MB; ++j) acc[i][j] = mk<T>(T(0), T(0));
        for (int r = 0; r < L; ++r) {
            T dv[MK];
            Cx cv[MB];
#pragma unroll
            for (int i = 0; i < MK; ++i) dv[i] = Dsm[(pg * RS + r) * KC + kg * MK + i];
#pragma unroll
            for (int j = 0; j < MB; ++j) cv[j] = Csm[(pg * RS + r) * BT + bg * MB + j];
#pragma unroll
            for (int i = 0; i < MK; ++i)
#pragma unroll
                for (int j = 0; j < MB; ++j) {
                    acc[i][j].x = fma(dv[i], cv[j].x, acc[i][j].x);
                    acc[i][j].y = fma(dv[i], cv[j].y, acc[i][j].y);
                }
        }
        if (tl.valid[pg]) {
            const int ni = tl.nb * NB + pg;
#pragma unroll
            for (int i = 0; i < MK; ++i) {
                const int k = k0 + kg * MK + i;
                if (k >= N) continue;
                T rho = T(1);
                if (mode == 1) rho = T(a.w64[k]) * inv2n2;
#pragma unroll
                for (int j = 0; j < MB; ++j) {
                    const int fb = bb * BT + bg * MB + j;
                    if (fb >= a.nfunc) continue;
                    const int f = a.fidx[fb];
                    G[a.ws_off[f] + ((size_t)k * 2 + tl.s) * N * N + (size_t)tl.mi * N + ni] = cscale(acc[i][j], rho);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Float-float ("double-FP32") form of the recurrence, for the synthesis near
// the poles.  There the three-term recurrence is badly conditioned (at x = 1
// it adds two terms of size ~l to get d = 1), so the rounding of the FP32
// state and of the FP32 step coefficients each leave errors of ~1e-5 to 1e-4
// in d at l ~ 100 for nodes within a few steps of beta = 0 or pi; the forward
// map does not see them (its weight w_k vanishes like sin beta there) but the
// synthesis (weight 2l + 1 on the coefficients) does.  Carrying value and
// coefficients as unevaluated sums hi + lo of two floats (products and sums
// made exact with FMA-based two-product / two-sum) removes both.
// ---------------------------------------------------------------------------
struct FF { float h, l; };
// a * b = p + e exactly
__device__ __forceinline__ FF ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}
// a + b = s + e exactly (no ordering assumption)
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}
// renormalise (|h| >= |l| assumed)
__device__ __forceinline__ FF ff_fast(float h, float l) {
    const float s = __fadd_rn(h, l);
    return {s, __fsub_rn(l, __fsub_rn(s, h))};
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const FF p = ff_two_prod(a.h, b.h);
    return ff_fast(p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l)));
}
__device__ __forceinline__ FF ff_sub(FF a, FF b) {
    const FF s = ff_two_sum(a.h, -b.h);
    return ff_fast(s.h, __fadd_rn(s.l, __fsub_rn(a.l, b.l)));
}
__device__ __forceinline__ FF ff_div(FF a, FF b) {
    const float q = __fdiv_rn(a.h, b.h);
    const float r = fmaf(-q, b.l, __fadd_rn(fmaf(-q, b.h, a.h), a.l));   // a - q b, to first order
    return ff_fast(q, __fdiv_rn(r, b.h));
}
// sqrt of an integer p < 2^24 (exact in FP32)
__device__ __forceinline__ FF ff_sqrt_int(float p) {
    if (p <= 0.f) return {0.f, 0.f};
    const float s = __fsqrt_rn(p);
    return ff_fast(s, __fdiv_rn(fmaf(-s, s, p), __fmul_rn(2.f, s)));
}

// Step coefficients A, C of the pair (n2, m2) from 2l = J to J + 2 as
// float-float (b keeps its hi/lo split of StepCoef).  All integers involved
// are below 2^24 (J < 2^11).
struct StepCoefFF { FF A, C; float bh, bl; };
__device__ __forceinline__ StepCoefFF step_coef_ff(int J, int n2, int m2) {
    StepCoefFF c;
    const FF rs = ff_mul(ff_sqrt_int((float)((J + 2) * (J + 2) - n2 * n2)),
                         ff_sqrt_int((float)((J + 2) * (J + 2) - m2 * m2)));
    c.A = ff_div({(float)(2 * (J + 2) * (J + 1)), 0.f}, rs);
    if (J == 0) {
        c.C = {0.f, 0.f}; c.bh = 0.f; c.bl = 0.f;
    } else {
        const int ip0 = J * J - n2 * n2, iq0 = J * J - m2 * m2;
        const FF r0 = ff_mul(ff_sqrt_int((float)(ip0 > 0 ? ip0 : 0)), ff_sqrt_int((float)(iq0 > 0 ? iq0 : 0)));
        const FF t = ff_div(r0, rs);                                        // sqrt(p0 q0 / (p1 q1))
        const FF u = ff_mul(t, {(float)(J + 2), 0.f});
        c.C = ff_div(u, {(float)J, 0.f});
        const float num = (float)(n2 * m2), den = (float)(J * (J + 2));
        c.bh = num / den;
        c.bl = fmaf(-c.bh, den, num) / den;
    }
    return c;
}

// Recurrence state in float-float with the same range extension as Rec<float>
// (value = h * 2^(-120 E); while E > 0 the value is below 2^-39 and counts as 0).
struct RecFF {
    FF cur, prev;
    float xh, xl;
    int E;
    __device__ __forceinline__ void seed32(const SeedPair& q, float4 tb, float2 xs, int k, int N) {
        cur = {seed_value32(q, tb, k, N, E), 0.f};
        prev = {0.f, 0.f};
        xh = xs.x;
        xl = xs.y;
    }
    __device__ __forceinline__ float value() const { return E == 0 ? cur.h : 0.f; }
    __device__ __forceinline__ void step(const StepCoefFF& c) {
        const FF xb = ff_sub({xh, xl}, {c.bh, c.bl});
        const FF t = ff_mul(c.A, xb);
        const FF nxt0 = ff_sub(ff_mul(t, cur), ff_mul(c.C, prev));
        FF nxt = nxt0;
        if (E > 0 && fabsf(nxt.h) >= 1.152921504606847e18f) {   // 2^60
            const float sc = 7.52316384526264e-37f;               // 2^-120 (exact scaling)
            nxt = {nxt.h * sc, nxt.l * sc};
            cur = {cur.h * sc, cur.l * sc};
            --E;
        }
        prev = cur;
        cur = nxt;
    }
};


// ---------------------------------------------------------------------------
// Transposed contraction, complex64 (synthesis / adjoint), fused form.
// A CTA owns a tile (sector, m, NB = 4 consecutive n) and BT = 8 functions;
// thread (g, h) runs the recurrence chains of pairs 2h, 2h+1 at the two nodes
// k = 2g, 2g+1 of the current pass and accumulates, while walking l,
//     acc[node][pair][b] += d^l_{nm}(beta_k) * Cw[l][pair][b],
// where Cw = wl(l) i^{m-n} c(l)_{mn} is kept in shared memory for the whole l
// range (one broadcast row per l).  No d values are stored.  Output: the
// workspace planes tile-major, [s][mi][ni/4][k][ni%4], so that the two
// threads of a node group write one 32-byte sector and a warp 512 bytes.
// Synthesis at N >= 128: the warps whose 32 nodes lie within N/8 of a pole
// run the recurrence in float-float (RecFF, coefficients with their low
// parts); there the FP32 recurrence loses ~1e-4 of d at high l, which the
// synthesis (weight 2l + 1, no sin(beta) factor) would show.
// ---------------------------------------------------------------------------
namespace tr32 {
constexpr int NB = 4, BT = 8;
template <int N> struct Cfg {
    static constexpr int THREADS = N < 256 ? N : 256;        // 2 threads per node pair-group
    static constexpr int NODES = THREADS;                     // nodes per pass (2 per node group)
    static constexpr int PASSES = N / NODES;
    static constexpr int RS = N / 2;
    static constexpr bool FF_POLES = N >= 128;                // float-float chains near the poles (synthesis)
    // The two halves of a warp (h = 0, 1) read pairs {0, 1} and {2, 3}: the step
    // coefficients of a pair are CS = RS + 1 entries apart and a row of weighted
    // coefficients is [pairs 0, 1][2 pad][pairs 2, 3][2 pad], so the two halves
    // never hit the same bank.
    static constexpr int CS = RS + 1;
    static constexpr int CROW = NB * BT + 4;                  // complex values per row of l
    static constexpr size_t smem_bytes() {
        return sizeof(StepCoef<float>) * NB * CS + sizeof(float2) * RS * CROW + sizeof(SeedPair) * NB + 16 * NB +
               (FF_POLES ? sizeof(float2) * NB * CS : 0);
    }
};
}  // namespace tr32

// FF: instantiation for the synthesis at N >= 128 (float-float chains near the
// poles); the adjoint and smaller N use the plain one, whose register count
// stays unaffected.
template <int N, bool FF>
__global__ void __launch_bounds__(tr32::Cfg<N>::THREADS, FF ? 2 : 0)
contract_tr32(BandArgs a, int mode, const float2* __restrict__ coeffs, float2* __restrict__ G) {
    using namespace tr32;
    using P = Cfg<N>;
    constexpr int RS = P::RS;
    Tile<NB> tl;
    tl.decode(N, blockIdx.x);
    if (!tl.any) return;
    const int bb = blockIdx.y;
    const int L = tl.L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int CS = P::CS, CROW = P::CROW;
    StepCoef<float>* coef = reinterpret_cast<StepCoef<float>*>(smem_raw);   // [NB][CS]
    float2* Csm = reinterpret_cast<float2*>(coef + NB * CS);               // [RS][CROW]
    SeedPair* spair = reinterpret_cast<SeedPair*>(Csm + RS * CROW);         // [NB]
    int* rstart = reinterpret_cast<int*>(spair + NB);                       // [NB] first row of each pair
    float2* coef_lo = reinterpret_cast<float2*>(rstart + NB);               // [NB][CS] (A, C) low parts
    const int tid = threadIdx.x;
    constexpr bool ff = FF;

    for (int idx = tid; idx < NB * (L - 1); idx += P::THREADS) {
        const int p = idx % NB, r = idx / NB;
        const int J = tl.j0 + 2 * r;
        if (J >= tl.mu2[p]) {
            if (ff) {
                const StepCoefFF c = step_coef_ff(J, tl.n2[p], tl.m2);
                coef[p * CS + r] = StepCoef<float>{c.A.h, c.C.h, c.bh, c.bl};
                coef_lo[p * CS + r] = make_float2(c.A.l, c.C.l);
            } else {
                coef[p * CS + r] = step_coef<float>(J, tl.n2[p], tl.m2);
            }
        }
    }
    for (int idx = tid; idx < L * NB * BT; idx += P::THREADS) {
        const int b = idx % BT, p = (idx / BT) % NB, r = idx / (BT * NB);
        const int J = tl.j0 + 2 * r;
        const int fb = bb * BT + b;
        float2 v = make_float2(0.f, 0.f);
        if (tl.valid[p] && J >= tl.mu2[p] && fb < a.nfunc) {
            const int f = a.fidx[fb];
            const size_t ci = block_offset(J) + (size_t)((tl.m2 + J) / 2) * (J + 1) + (tl.n2[p] + J) / 2;
            v = cmul_ipow(coeffs[a.coeff_off[f] + ci], (tl.m2 - tl.n2[p]) / 2);
            if (mode == 0) v = cscale(v, (float)(J + 1));
        }
        Csm[r * CROW + p * BT + (p >= 2 ? 2 : 0) + b] = v;
    }
    if (tid < NB) {
        spair[tid] = make_seed_pair(a.lf2, tl.n2[tid], tl.m2);
        rstart[tid] = tl.valid[tid] ? (tl.mu2[tid] - tl.j0) / 2 : L;
    }
    __syncthreads();

    const int h = tid & 1, gidx = tid >> 1;
    const int rs0 = rstart[2 * h], rs1 = rstart[2 * h + 1];
    const SeedPair q0 = spair[2 * h], q1 = spair[2 * h + 1];
    const StepCoef<float>* c0p = coef + (2 * h) * CS;
    const StepCoef<float>* c1p = coef + (2 * h + 1) * CS;
    // adjoint prefactor: the grid cell over the Haar measure, 1/(2N^2) on the paper's
    // domain, 1/(4N^2) on the full group (psi over 4 pi), 1/(2(N-1)^2) on the printed grid
    const float NC = a.literal ? (float)(N - 1) : (float)N;
    const float inv2n2 = 1.f / ((a.full_group ? 4.f : 2.f) * NC * NC);
    const int ni0 = tl.nb * NB + 2 * h;

    for (int pass = 0; pass < P::PASSES; ++pass) {
        const int ka = pass * P::NODES + 2 * gidx;           // nodes ka, ka + 1
        // a warp's 32 nodes start at a multiple of 32: float-float chains when any
        // of them is within N/8 of a pole
        const int kw = pass * P::NODES + 32 * (tid >> 5);
        if (ff && (kw < N / 8 || kw + 31 >= N - N / 8)) {     // compile-time false unless FF
            RecFF ch[2][2];                                   // [node][pair]
#pragma unroll
            for (int nd = 0; nd < 2; ++nd) {
                const int k = ka + nd;
                ch[nd][0].seed32(q0, a.seed32[k], a.xsplit[k], k, N);
                ch[nd][1].seed32(q1, a.seed32[k], a.xsplit[k], k, N);
            }
            float2 acc[2][2][BT];
#pragma unroll
            for (int nd = 0; nd < 2; ++nd)
#pragma unroll
                for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                    for (int b = 0; b < BT; ++b) acc[nd][pp][b] = make_float2(0.f, 0.f);
            for (int r = min(rs0, rs1); r < L; ++r) {
                const float4* crow = reinterpret_cast<const float4*>(Csm + r * CROW + 2 * h * (BT + 1));
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    if (r < (pp ? rs1 : rs0)) continue;
                    float2 cv[BT];
#pragma unroll
                    for (int b2 = 0; b2 < BT / 2; ++b2) {
                        const float4 t = crow[pp * (BT / 2) + b2];
                        cv[2 * b2] = make_float2(t.x, t.y);
                        cv[2 * b2 + 1] = make_float2(t.z, t.w);
                    }
                    const StepCoef<float> c32 = (pp ? c1p : c0p)[r];
                    const float2 clo = coef_lo[(2 * h + pp) * CS + r];
                    const StepCoefFF cf{{c32.A, clo.x}, {c32.C, clo.y}, c32.bh, c32.bl};
#pragma unroll
                    for (int nd = 0; nd < 2; ++nd) {
                        RecFF& rc = ch[nd][pp];
                        const float dv = rc.value();
#pragma unroll
                        for (int b = 0; b < BT; ++b) {
                            acc[nd][pp][b].x = fmaf(dv, cv[b].x, acc[nd][pp][b].x);
                            acc[nd][pp][b].y = fmaf(dv, cv[b].y, acc[nd][pp][b].y);
                        }
                        if (r + 1 < L) rc.step(cf);
                    }
                }
            }
#pragma unroll
            for (int nd = 0; nd < 2; ++nd) {
                const int k = ka + nd;
#pragma unroll
                for (int b = 0; b < BT; ++b) {
                    const int fb = bb * BT + b;
                    if (fb >= a.nfunc) continue;
                    const int f = a.fidx[fb];
                    float4* dst = reinterpret_cast<float4*>(G + a.ws_off[f] + (size_t)tl.s * N * N * N +
                                                            (size_t)tl.mi * N * N + (size_t)(ni0 >> 2) * 4 * N +
                                                            (size_t)4 * k + (ni0 & 3));
                    *dst = make_float4(acc[nd][0][b].x, acc[nd][0][b].y, acc[nd][1][b].x, acc[nd][1][b].y);
                }
            }
            continue;
        }
        Rec<float> ch[2][2];                                  // [node][pair]
#pragma unroll
        for (int nd = 0; nd < 2; ++nd) {
            const int k = ka + nd;
            ch[nd][0].seed32(q0, a.seed32[k], a.xsplit[k], k, N);
            ch[nd][1].seed32(q1, a.seed32[k], a.xsplit[k], k, N);
        }
        constexpr unsigned mask = P::THREADS >= 32 ? 0xffffffffu : ((1u << P::THREADS) - 1u);
        const bool fast = __all_sync(mask, (ch[0][0].E | ch[0][1].E | ch[1][0].E | ch[1][1].E) == 0);
        float2 acc[2][2][BT];
#pragma unroll
        for (int nd = 0; nd < 2; ++nd)
#pragma unroll
            for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                for (int b = 0; b < BT; ++b) acc[nd][pp][b] = make_float2(0.f, 0.f);

        for (int r = min(rs0, rs1); r < L; ++r) {
            const float4* crow = reinterpret_cast<const float4*>(Csm + r * CROW + 2 * h * (BT + 1));
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                if (r < (pp ? rs1 : rs0)) continue;           // uniform across the CTA
                float2 cv[BT];
#pragma unroll
                for (int b2 = 0; b2 < BT / 2; ++b2) {
                    const float4 t = crow[pp * (BT / 2) + b2];
                    cv[2 * b2] = make_float2(t.x, t.y);
                    cv[2 * b2 + 1] = make_float2(t.z, t.w);
                }
                const StepCoef<float> cf = (pp ? c1p : c0p)[r];
#pragma unroll
                for (int nd = 0; nd < 2; ++nd) {
                    Rec<float>& rc = ch[nd][pp];
                    const float dv = fast ? rc.cur : rc.value();
#pragma unroll
                    for (int b = 0; b < BT; ++b) {
                        acc[nd][pp][b].x = fmaf(dv, cv[b].x, acc[nd][pp][b].x);
                        acc[nd][pp][b].y = fmaf(dv, cv[b].y, acc[nd][pp][b].y);
                    }
                    if (r + 1 < L) {
                        if (fast) rc.step_fast(cf);
                        else rc.step(cf);
                    }
                }
            }
        }
        // store: element (k, s, mi, ni) at s N^3 + mi N^2 + (ni/4) 4N + 4k + ni%4
#pragma unroll
        for (int nd = 0; nd < 2; ++nd) {
            const int k = ka + nd;
            const float rho = (mode == 1) ? a.w32[k] * inv2n2 : 1.f;
#pragma unroll
            for (int b = 0; b < BT; ++b) {
                const int fb = bb * BT + b;
                if (fb >= a.nfunc) continue;
                const int f = a.fidx[fb];
                float4* dst = reinterpret_cast<float4*>(G + a.ws_off[f] + (size_t)tl.s * N * N * N +
                                                        (size_t)tl.mi * N * N + (size_t)(ni0 >> 2) * 4 * N +
                                                        (size_t)4 * k + (ni0 & 3));
                *dst = make_float4(acc[nd][0][b].x * rho, acc[nd][0][b].y * rho, acc[nd][1][b].x * rho,
                                   acc[nd][1][b].y * rho);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// tile_list / ntiles: launch over the listed tiles only (one row class), else over all
template <typename T, int NB, int BT, int KC, int LW, int ML, int MB>
static cudaError_t launch_fwd_t(const BandArgs& a, const void* ws, void* coeffs, cudaStream_t st,
                                const int* tile_list = nullptr, int ntiles = 0) {
    using Cfg = FwdCfg<T, NB, BT, KC, LW, ML, MB>;
    auto kern = contract_fwd<T, NB, BT, KC, LW, ML, MB>;
    const size_t smem = Cfg::smem_bytes(a.N);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = tile_list ? ntiles : 2 * a.N * (a.N / NB);
    if (tiles <= 0) return cudaSuccess;
    const int windows = (a.N / 2 + LW - 1) / LW;
    dim3 g(tiles, (a.nfunc + BT - 1) / BT, windows);
    kern<<<g, Cfg::THREADS, smem, st>>>(a, (const cplx<T>*)ws, (cplx<T>*)coeffs, tile_list);
    return cudaGetLastError();
}

cudaError_t launch_contract_forward(const BandArgs& a, bool fp64, const void* ws, void* coeffs, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    if (fp64) return launch_fwd_t<double, 4, 8, 32, 64, 4, 2>(a, ws, coeffs, st);
    if (a.s2_tiles && (a.s2_rc > 0 || (a.s2_rc < 0 && a.nfunc >= 48))) {
        // Large batches: one launch per row class, each with a row window that fits
        // its tiles (32, 64, 128 rows of l) and the threads that a window of all 128
        // rows would leave idle on short tiles spent on more functions (64, 32, 16
        // per block; 256 threads each).
        const int* t0 = a.s2_tiles;
        const int* t1 = t0 + a.s2_ntiles[0];
        const int* t2 = t1 + a.s2_ntiles[1];
        cudaError_t e = launch_fwd_t<float, 4, 64, 32, 32, 8, 4>(a, ws, coeffs, st, t0, a.s2_ntiles[0]);
        if (e == cudaSuccess) e = launch_fwd_t<float, 4, 32, 32, 64, 8, 4>(a, ws, coeffs, st, t1, a.s2_ntiles[1]);
        if (e == cudaSuccess) e = launch_fwd_t<float, 4, 16, 32, 128, 8, 4>(a, ws, coeffs, st, t2, a.s2_ntiles[2]);
        return e;
    }
    // 8 or 16 functions per block (chosen by the plan's autotuner, else by batch
    // size: small batches take 8 so that no FMA lane works on padding)
    const int bt = a.s2_bt ? a.s2_bt : (a.nfunc <= 8 ? 8 : 16);
    if (bt == 8) return launch_fwd_t<float, 4, 8, 16, 128, 8, 4>(a, ws, coeffs, st);
    return launch_fwd_t<float, 4, 16, 32, 128, 8, 4>(a, ws, coeffs, st);
}

template <typename T, int NB, int BT, int KC, int MK, int MB>
static cudaError_t launch_tr_t(const BandArgs& a, int mode, const void* coeffs, void* ws, cudaStream_t st) {
    using Cfg = TrCfg<T, NB, BT, KC, MK, MB>;
    auto kern = contract_tr<T, NB, BT, KC, MK, MB>;
    const size_t smem = Cfg::smem_bytes(a.N);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = 2 * a.N * (a.N / NB);
    dim3 g(tiles, (a.nfunc + BT - 1) / BT, 1);
    kern<<<g, Cfg::THREADS, smem, st>>>(a, mode, (const cplx<T>*)coeffs, (cplx<T>*)ws);
    return cudaGetLastError();
}

template <int N>
static cudaError_t launch_tr32_n(const BandArgs& a, int mode, const void* coeffs, void* ws, cudaStream_t st) {
    using P = tr32::Cfg<N>;
    auto kern = (P::FF_POLES && mode == 0) ? contract_tr32<N, P::FF_POLES> : contract_tr32<N, false>;
    const size_t smem = P::smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 g(2 * N * (N / tr32::NB), (a.nfunc + tr32::BT - 1) / tr32::BT, 1);
    kern<<<g, P::THREADS, smem, st>>>(a, mode, (const float2*)coeffs, (float2*)ws);
    return cudaGetLastError();
}

cudaError_t launch_contract_transpose(const BandArgs& a, bool fp64, TransposeMode mode, const void* coeffs,
                                      void* ws, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    const int m = (mode == TransposeMode::Synthesis) ? 0 : 1;
    if (fp64) return launch_tr_t<double, 4, 4, 16, 2, 2>(a, m, coeffs, ws, st);
    if (!a.ws_tile_major) return cudaErrorInvalidValue;      // the complex64 planes are tile-major here
    switch (a.N) {
        case 4: return launch_tr32_n<4>(a, m, coeffs, ws, st);
        case 8: return launch_tr32_n<8>(a, m, coeffs, ws, st);
        case 16: return launch_tr32_n<16>(a, m, coeffs, ws, st);
        case 32: return launch_tr32_n<32>(a, m, coeffs, ws, st);
        case 64: return launch_tr32_n<64>(a, m, coeffs, ws, st);
        case 128: return launch_tr32_n<128>(a, m, coeffs, ws, st);
        case 256: return launch_tr32_n<256>(a, m, coeffs, ws, st);
        case 512: return launch_tr32_n<512>(a, m, coeffs, ws, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace su2

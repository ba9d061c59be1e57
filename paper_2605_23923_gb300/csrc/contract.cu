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

#include "common.cuh"
#include "su2_internal.h"

namespace su2 {

template <typename T> struct StepCoef { T A, C, bh, bl; };

__device__ __forceinline__ size_t block_offset(int J) {
    const size_t j = (size_t)J;
    return j * (j + 1) * (2 * j + 1) / 6;
}

// Step coefficients for advancing from 2l = J to J + 2 for the pair (n2, m2).
template <typename T>
__device__ __forceinline__ StepCoef<T> step_coef(int J, int n2, int m2) {
    StepCoef<T> c;
    const T p1 = T((J + 2) * (J + 2) - n2 * n2), q1 = T((J + 2) * (J + 2) - m2 * m2);
    const T rs = sqrt(p1) * sqrt(q1);
    c.A = T(2 * (J + 2) * (J + 1)) / rs;
    if (J == 0) {
        c.C = T(0); c.bh = T(0); c.bl = T(0);
    } else {
        const int ip0 = J * J - n2 * n2, iq0 = J * J - m2 * m2;
        const T p0 = T(ip0 > 0 ? ip0 : 0), q0 = T(iq0 > 0 ? iq0 : 0);
        c.C = (T(J + 2) / T(J)) * (sqrt(p0) * sqrt(q0)) / rs;
        const T num = T(n2 * m2), den = T(J * (J + 2));
        c.bh = num / den;
        c.bl = fma(-c.bh, den, num) / den;       // exact remainder of the division
    }
    return c;
}

// log2 |d^mu_{nm}(beta_k)| and its sign (Rodrigues-type formula at l = mu).
__device__ __forceinline__ double seed_log2(const BandArgs& a, int n2, int m2, int k, double* sgn) {
    const int mu2 = max(abs(n2), abs(m2));
    int other, pc, ps;
    double sg = 1.0;
    if (abs(n2) == mu2 && (n2 > 0 || mu2 == 0)) {
        other = m2; pc = (mu2 + m2) / 2; ps = (mu2 - m2) / 2;
        if (((mu2 - m2) / 2) & 1) sg = -1.0;
    } else if (n2 == -mu2) {
        other = m2; pc = (mu2 - m2) / 2; ps = (mu2 + m2) / 2;
    } else if (m2 == mu2) {
        other = n2; pc = (mu2 + n2) / 2; ps = (mu2 - n2) / 2;
    } else {
        other = n2; pc = (mu2 - n2) / 2; ps = (mu2 + n2) / 2;
        if (((mu2 + n2) / 2) & 1) sg = -1.0;
    }
    double L = 0.5 * (a.lf2[mu2] - a.lf2[(mu2 + other) / 2] - a.lf2[(mu2 - other) / 2]);
    if (pc) L += (double)pc * a.log2c[k];
    if (ps) L += (double)ps * a.log2s[k];
    *sgn = sg;
    return L;
}

// Recurrence state for one (pair, node).
template <typename T> struct Rec;

template <> struct Rec<float> {
    float cur, prev, xh, xl;
    int E;
    __device__ __forceinline__ void seed(const BandArgs& a, int n2, int m2, int k) {
        double sg;
        const double L = seed_log2(a, n2, m2, k, &sg);
        prev = 0.f;
        const float2 xs = a.xsplit[k];
        xh = xs.x; xl = xs.y;
        if (!(L > -1e300)) { cur = 0.f; E = 0; return; }      // a zero power of a zero base
        int e = 0;
        if (L < -60.0) e = (int)ceil((-L - 60.0) / 120.0);
        const double t = L + 120.0 * e;                        // in [-60, 60)
        const double ti = floor(t);
        const float mant = exp2f((float)(t - ti));
        cur = (float)sg * ldexpf(mant, (int)ti);
        E = e;
    }
    __device__ __forceinline__ float value() const { return E == 0 ? cur : 0.f; }
    __device__ __forceinline__ void step(const StepCoef<float>& c) {
        const float xb = (xh - c.bh) + (xl - c.bl);
        float nxt = fmaf(c.A * xb, cur, -c.C * prev);
        if (E > 0 && fabsf(nxt) >= 1.152921504606847e18f) {   // 2^60
            nxt *= 7.52316384526264e-37f;                        // 2^-120
            cur *= 7.52316384526264e-37f;
            --E;
        }
        prev = cur;
        cur = nxt;
    }
};

template <> struct Rec<double> {
    double cur, prev, x;
    __device__ __forceinline__ void seed(const BandArgs& a, int n2, int m2, int k) {
        double sg;
        const double L = seed_log2(a, n2, m2, k, &sg);
        prev = 0.0;
        x = a.cosb[k];
        cur = (L > -1e300) ? sg * exp2(L) : 0.0;
    }
    __device__ __forceinline__ double value() const { return cur; }
    __device__ __forceinline__ void step(const StepCoef<double>& c) {
        const double nxt = c.A * (x - c.bh) * cur - c.C * prev;
        prev = cur;
        cur = nxt;
    }
};

// Decoded tile: sector s, fixed m, NB consecutive n.
template <int NB>
struct Tile {
    int s, mi, nb, m2, jtop, j0, L;
    int n2[NB], mu2[NB];
    bool valid[NB];
    bool any;
    __device__ __forceinline__ void decode(int N, int t) {
        const int nbk = N / NB;
        nb = t % nbk; t /= nbk;
        mi = t % N; t /= N;
        s = t;
        m2 = 2 * (mi - N / 2) + s;
        jtop = N - 2 + s;
        j0 = 1 << 30;
        any = !(s == 0 && mi == 0);
        bool some = false;
#pragma unroll
        for (int p = 0; p < NB; ++p) {
            const int ni = nb * NB + p;
            n2[p] = 2 * (ni - N / 2) + s;
            valid[p] = any && !(s == 0 && ni == 0);
            mu2[p] = max(abs(n2[p]), abs(m2));
            if (valid[p]) { j0 = min(j0, mu2[p]); some = true; }
        }
        any = some;
        L = any ? (jtop - j0) / 2 + 1 : 0;
    }
};

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
        return sizeof(StepCoef<T>) * NB * (N / 2) + sizeof(T) * NB * KC * LDD + sizeof(cplx<T>) * KC * NB * BT;
    }
};

template <typename T, int NB, int BT, int KC, int LW, int ML, int MB>
__global__ void __launch_bounds__(FwdCfg<T, NB, BT, KC, LW, ML, MB>::THREADS)
contract_fwd(BandArgs a, const cplx<T>* __restrict__ F2, cplx<T>* __restrict__ coeffs) {
    using Cx = cplx<T>;
    using Cfg = FwdCfg<T, NB, BT, KC, LW, ML, MB>;
    constexpr int THREADS = Cfg::THREADS, LDD = Cfg::LDD;
    static_assert(NB * KC <= THREADS, "one generator thread per (pair, node)");
    const int N = a.N;
    Tile<NB> tl;
    tl.decode(N, blockIdx.x);
    if (!tl.any) return;
    const int bb = blockIdx.y;
    const int r0 = blockIdx.z * LW;
    if (r0 >= tl.L) return;
    const int r_end = min(r0 + LW, tl.L);
    const int RS = N / 2;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepCoef<T>* coef = reinterpret_cast<StepCoef<T>*>(smem_raw);                 // [NB][RS]
    T* Dsm = reinterpret_cast<T*>(coef + NB * RS);                                 // [NB][KC][LDD]
    Cx* Fsm = reinterpret_cast<Cx*>(Dsm + NB * KC * LDD);                          // [KC][NB][BT]
    const int tid = threadIdx.x;

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
            if (!tl.valid[p] || k >= N) {
                for (int rb = 0; rb < LW; rb += 4) { const T z[4] = {T(0), T(0), T(0), T(0)}; store4<T>(drow + rb, z); }
            } else {
                Rec<T> rc;
                rc.seed(a, tl.n2[p], tl.m2, k);
                int r = (tl.mu2[p] - tl.j0) / 2;      // row of the seed
                while (r < r0) { rc.step(coef[p * RS + r]); ++r; }
                for (int rb = 0; rb < LW; rb += 4) {
                    T v[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int rr = r0 + rb + i;
                        if (rr < r || rr >= r_end) {
                            v[i] = T(0);
                        } else {
                            v[i] = rc.value();
                            if (rr + 1 < r_end) { rc.step(coef[p * RS + rr]); r = rr + 1; }
                        }
                    }
                    store4<T>(drow + rb, v);
                }
            }
        } else {
            // ---- stage F2[k0 .. k0+KC) for the NB pairs and BT functions
            for (int idx = tid - NB * KC; idx < KC * BT; idx += THREADS - NB * KC) {
                const int kk = idx % KC, b = idx / KC;
                const int fb = bb * BT + b, k = k0 + kk;
                Cx v[NB];
                if (fb < a.nfunc && k < N) {
                    const int f = a.fidx[fb];
                    const Cx* src = F2 + a.ws_off[f] + ((size_t)k * 2 + tl.s) * N * N + (size_t)tl.mi * N + tl.nb * NB;
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
        return sizeof(StepCoef<T>) * NB * RS + sizeof(T) * NB * RS * KC + sizeof(cplx<T>) * NB * RS * BT;
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
    const int tid = threadIdx.x;

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
            if (!tl.valid[p] || k >= N) {
                for (int r = 0; r < L; ++r) dcol[r * KC] = T(0);
            } else {
                Rec<T> rc;
                rc.seed(a, tl.n2[p], tl.m2, k);
                const int rs = (tl.mu2[p] - tl.j0) / 2;
                for (int r = 0; r < rs; ++r) dcol[r * KC] = T(0);
                for (int r = rs; r < L; ++r) {
                    dcol[r * KC] = rc.value();
                    if (r + 1 < L) rc.step(coef[p * RS + r]);
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
// Launchers
// ---------------------------------------------------------------------------
template <typename T, int NB, int BT, int KC, int LW, int ML, int MB>
static cudaError_t launch_fwd_t(const BandArgs& a, const void* ws, void* coeffs, cudaStream_t st) {
    using Cfg = FwdCfg<T, NB, BT, KC, LW, ML, MB>;
    auto kern = contract_fwd<T, NB, BT, KC, LW, ML, MB>;
    const size_t smem = Cfg::smem_bytes(a.N);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = 2 * a.N * (a.N / NB);
    const int windows = (a.N / 2 + LW - 1) / LW;
    dim3 g(tiles, (a.nfunc + BT - 1) / BT, windows);
    kern<<<g, Cfg::THREADS, smem, st>>>(a, (const cplx<T>*)ws, (cplx<T>*)coeffs);
    return cudaGetLastError();
}

cudaError_t launch_contract_forward(const BandArgs& a, bool fp64, const void* ws, void* coeffs, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    if (fp64) return launch_fwd_t<double, 4, 8, 32, 64, 4, 2>(a, ws, coeffs, st);
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

cudaError_t launch_contract_transpose(const BandArgs& a, bool fp64, TransposeMode mode, const void* coeffs,
                                      void* ws, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    const int m = (mode == TransposeMode::Synthesis) ? 0 : 1;
    if (fp64) return launch_tr_t<double, 4, 4, 16, 2, 2>(a, m, coeffs, ws, st);
    return launch_tr_t<float, 4, 8, 16, 2, 2>(a, m, coeffs, ws, st);
}

}  // namespace su2

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
#include "recurrence.cuh"
#include "su2_internal.h"

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

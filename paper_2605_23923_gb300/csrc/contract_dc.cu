// Stage 2 by the divide-and-conquer projection of Sec. 4 (Theorem
// "Divide-and-conquer" with the composition Proposition for A_{r+s}, B_{r+s}),
// at recursion depth k, for complex128 plans.
//
// For one pair (n, m), mu = max(|n|, |m|), s_k = F2[k] (the stage-1 plane
// already carries w_k and the prefactor):
//   l = mu and mu + 1:   <s, d^mu>, <s, d^{mu+1}>  (seed and one recurrence step);
//   base L = mu + 1,     s^L = s d^L, s^{L-1} = s d^mu;
//   l = L + r, r = 1..R: sum over tau_1 in {A, B} and eps in {0,1}^{k-1} of
//                        <s^{L or L-1}, V>,  V = prod_i X_i[sel_i][eps_i],
// with X_i[A|B][e] = A|B^{L_{i-1}}_{n_i - e} the shifted polynomials of level i
// (d^{L'+j} = A_j^{L'} d^{L'} + B_j^{L'} d^{L'-1}; the end of Sec. 4 states the
// (m, n) case is the analogue of the Legendre one, so they follow the Wigner
// recurrence in j from A_0 = 1, A_{-1} = 0, B_0 = 0, B_{-1} = 1), sel_1 = tau_1,
// sel_i = eps_{i-1}, eps_k = 0.  The shift is split into the digits of r in
// base b (b the smallest base with b^k > R): n_i = d_i b^{k-i}, levels
// L_i = L_{i-1} + n_i.  Walking r upwards the digits run like an odometer: the
// level whose digit grows by one advances its (A, A_prev, B, B_prev) state by
// b^{k-i} recurrence steps, the levels below it restart at their new base, so
// the shifted polynomials cost k recurrence steps per r (amortised) and every
// coefficient costs 2^k inner products of length N: the Sec. 6 second-stage cost
// O(2^k k N^4) (Proposition "Second Stage Complexity"), which Theorem "optimal
// k" minimises at k = 1.  This kernel exists to measure that, not for speed.
//
// FP64 throughout: for large mu, d^mu near the poles lies far below the FP32
// range while the shifted polynomials grow, so their product needs FP64.
// One CTA per (sector, m, n) pair and 4 functions, one thread per beta node;
// per coefficient a warp-shuffle then shared-memory reduction over the nodes.
#include <cuda_runtime.h>

#include "common.cuh"
#include "recurrence.cuh"
#include "su2_internal.h"

namespace su2 {
namespace dc {

constexpr int FB = 4;        // functions per CTA
constexpr int MAXT = 256;    // one thread per node (N <= 256)

template <int K>
__global__ void __launch_bounds__(MAXT)
contract_dc(BandArgs a, const double2* __restrict__ ws, double2* __restrict__ coeffs) {
    extern __shared__ double smem[];
    const int N = a.N;
    int p = blockIdx.x;
    const int s = p / (N * N);
    p -= s * N * N;
    const int mi = p / N, ni = p - (p / N) * N;
    if (s == 0 && (mi == 0 || ni == 0)) return;               // Nyquist row / column
    const int m2 = 2 * (mi - N / 2) + s, n2 = 2 * (ni - N / 2) + s;
    const int mu2 = max(abs(n2), abs(m2)), jtop = N - 2 + s;
    if (mu2 > jtop) return;                                   // no coefficient for this pair
    const int rows = (jtop - mu2) / 2 + 1;                    // l = mu .. mu + rows - 1
    const int f0 = blockIdx.y * FB;
    const int nf = min(FB, a.nfunc - f0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = blockDim.x >> 5;
    double* cA = smem;                                        // step coefficients from degree mu + i
    double* cB = smem + N;
    double* cC = smem + 2 * N;
    double* red = smem + 3 * N;                               // [2][NW][FB][2]
    for (int i = tid; i < rows - 1; i += blockDim.x) {
        const StepCoef<double> c = step_coef<double>(mu2 + 2 * i, n2, m2);
        cA[i] = c.A;
        cB[i] = c.bh;
        cC[i] = c.C;
    }
    const bool act = tid < N;
    double x = 0.0, d0 = 0.0, d1 = 0.0;
    if (act) {
        Rec<double> rc;
        rc.seed(a, n2, m2, tid);
        x = rc.x;
        d0 = rc.value();
        if (rows > 1) {
            rc.step(step_coef<double>(mu2, n2, m2));
            d1 = rc.value();
        }
    }
    double2 sv0[FB], sv1[FB];                                 // s^{L-1} = s d^mu, s^L = s d^{mu+1}
#pragma unroll
    for (int q = 0; q < FB; ++q) {
        double2 F = make_double2(0.0, 0.0);
        if (act && q < nf)
            F = ws[a.ws_off[a.fidx[f0 + q]] + ((size_t)(2 * tid + s) * N + mi) * N + ni];
        sv0[q] = make_double2(F.x * d0, F.y * d0);
        sv1[q] = make_double2(F.x * d1, F.y * d1);
    }
    __syncthreads();                                          // step coefficients ready

    int buf = 0;
    // sum acc over all nodes and store coefficient row `row` of every function
    auto emit = [&](int row, double2 (&acc)[FB]) {
#pragma unroll
        for (int q = 0; q < FB; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, o);
                acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, o);
            }
        double* rb = red + (size_t)buf * NW * FB * 2;
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < FB; ++q) {
                rb[(warp * FB + q) * 2] = acc[q].x;
                rb[(warp * FB + q) * 2 + 1] = acc[q].y;
            }
        __syncthreads();
        if (tid < nf) {
            double2 v = make_double2(0.0, 0.0);
            for (int w = 0; w < NW; ++w) {
                v.x += rb[(w * FB + tid) * 2];
                v.y += rb[(w * FB + tid) * 2 + 1];
            }
            const int J = mu2 + 2 * row;
            const size_t idx = block_offset(J) + (size_t)((m2 + J) / 2) * (J + 1) + (n2 + J) / 2;
            coeffs[a.coeff_off[a.fidx[f0 + tid]] + idx] = cmul_ipow(v, (n2 - m2) / 2);
        }
        buf ^= 1;                                             // the next row writes the other buffer
    };

    {
        double2 acc[FB];
#pragma unroll
        for (int q = 0; q < FB; ++q) acc[q] = sv0[q];
        emit(0, acc);
    }
    if (rows < 2) return;
    {
        double2 acc[FB];
#pragma unroll
        for (int q = 0; q < FB; ++q) acc[q] = sv1[q];
        emit(1, acc);
    }
    const int R = rows - 2;
    if (R < 1) return;
    int b = 1;                                                // smallest base with b^K > R
    for (;;) {
        long long pk = 1;
        for (int i = 0; i < K; ++i) pk *= b;
        if (pk >= R + 1) break;
        ++b;
    }
    int pw[K], dg[K], base[K];
    double sA[K], sAp[K], sB[K], sBp[K];
    pw[K - 1] = 1;
#pragma unroll
    for (int i = K - 2; i >= 0; --i) pw[i] = pw[i + 1] * b;
    const int JL = mu2 + 2;                                   // 2L
#pragma unroll
    for (int i = 0; i < K; ++i) {
        dg[i] = 0;
        base[i] = JL;
        sA[i] = 1.0; sAp[i] = 0.0; sB[i] = 0.0; sBp[i] = 1.0;
    }
    for (int r = 1; r <= R; ++r) {
        int rem = r;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int nd = rem / pw[i];
            rem -= nd * pw[i];
            if (nd != dg[i]) {
                if (nd > dg[i]) {
                    // digit up by one: order n_i grows by pw[i]; steps from degree base + 2 * order
                    const int c0 = (base[i] - mu2) / 2 + dg[i] * pw[i];
                    for (int j = 0; j < pw[i]; ++j) {
                        const double ca = cA[c0 + j], cb = cB[c0 + j], cc = cC[c0 + j];
                        const double t = ca * (x - cb);
                        const double nA = t * sA[i] - cc * sAp[i];
                        const double nB = t * sB[i] - cc * sBp[i];
                        sAp[i] = sA[i]; sA[i] = nA;
                        sBp[i] = sB[i]; sB[i] = nB;
                    }
                } else {
                    // digit wrapped to zero: restart at the level's new base
                    base[i] = i == 0 ? JL : base[i - 1] + 2 * dg[i - 1] * pw[i - 1];
                    sA[i] = 1.0; sAp[i] = 0.0; sB[i] = 0.0; sBp[i] = 1.0;
                }
                dg[i] = nd;
            }
        }
        double2 acc[FB];
#pragma unroll
        for (int q = 0; q < FB; ++q) acc[q] = make_double2(0.0, 0.0);
#pragma unroll
        for (int t1 = 0; t1 < 2; ++t1) {
#pragma unroll
            for (int e = 0; e < (1 << (K - 1)); ++e) {
                // level i lowers its order by eps_i = bit i of e (none at the last level);
                // it takes B if the previous level lowered (bit i-1), A otherwise; level 0 takes tau_1
                double V;
                {
                    const int ep = (K > 1) ? (e & 1) : 0;
                    V = t1 ? (ep ? sBp[0] : sB[0]) : (ep ? sAp[0] : sA[0]);
                }
#pragma unroll
                for (int i = 1; i < K; ++i) {
                    const int sel = (e >> (i - 1)) & 1;
                    const int ep = (i < K - 1) ? ((e >> i) & 1) : 0;
                    V *= sel ? (ep ? sBp[i] : sB[i]) : (ep ? sAp[i] : sA[i]);
                }
                const double2* sv = t1 ? sv0 : sv1;           // tau_1 = B pairs with s^{L-1}
#pragma unroll
                for (int q = 0; q < FB; ++q) {
                    acc[q].x = fma(sv[q].x, V, acc[q].x);
                    acc[q].y = fma(sv[q].y, V, acc[q].y);
                }
            }
        }
        emit(r + 1, acc);
    }
}

template <int K>
static cudaError_t launch_k(const BandArgs& a, const void* ws, void* coeffs, cudaStream_t st) {
    const int N = a.N;
    const int threads = N < 32 ? 32 : N;
    const int NW = threads / 32;
    const size_t smem = (size_t)(3 * N + 2 * NW * FB * 2) * sizeof(double);
    dim3 g(2 * N * N, (a.nfunc + FB - 1) / FB, 1);
    contract_dc<K><<<g, threads, smem, st>>>(a, (const double2*)ws, (double2*)coeffs);
    return cudaGetLastError();
}

}  // namespace dc

cudaError_t launch_contract_forward_depth(const BandArgs& a, int depth, const void* ws, void* coeffs,
                                          cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    if (a.N > dc::MAXT || a.ws_tile_major) return cudaErrorInvalidValue;
    switch (depth) {
        case 1: return dc::launch_k<1>(a, ws, coeffs, st);
        case 2: return dc::launch_k<2>(a, ws, coeffs, st);
        case 3: return dc::launch_k<3>(a, ws, coeffs, st);
        case 4: return dc::launch_k<4>(a, ws, coeffs, st);
        case 5: return dc::launch_k<5>(a, ws, coeffs, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace su2

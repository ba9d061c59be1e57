// Wigner-d recurrence pieces shared by the stage-2 kernels: step coefficients,
// log-space seeds, the range-extended FP32 state and the tile decode.
//
//   d^{l+1} = A_l (x - b_l) d^l - C_l d^{l-1},   x = cos(beta_k),
//   A_l = (l+1)(2l+1) / sqrt(((l+1)^2-n^2)((l+1)^2-m^2)),  b_l = nm / (l(l+1)),
//   C_l = (l+1)/l * sqrt((l^2-n^2)(l^2-m^2)) / sqrt(((l+1)^2-n^2)((l+1)^2-m^2)),
//   seeded at l = mu = max(|n|,|m|) by the Rodrigues-type formula evaluated there
//   (Sec. 3), with factorials and half-angle powers summed in FP64 log2 space.
#pragma once

#include <math.h>

#include "common.cuh"

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

// Seed of the pair (n, m) at l = mu = max(|n|, |m|) (Rodrigues-type formula of
// Sec. 3 evaluated there):  d^mu_{nm}(beta) = sg * 2^K * cos(beta/2)^pc * sin(beta/2)^ps
// with K = log2 sqrt((2 mu)! / ((mu + o)! (mu - o)!)), o the index other than the
// one at +-mu.  Doubled indices throughout.
struct SeedParams {
    double K;
    int pc, ps;
    double sg;
};

__device__ __forceinline__ SeedParams seed_params(const double* lf2, int n2, int m2) {
    const int mu2 = max(abs(n2), abs(m2));
    SeedParams p;
    int other;
    p.sg = 1.0;
    if (abs(n2) == mu2 && (n2 > 0 || mu2 == 0)) {
        other = m2; p.pc = (mu2 + m2) / 2; p.ps = (mu2 - m2) / 2;
        if (((mu2 - m2) / 2) & 1) p.sg = -1.0;
    } else if (n2 == -mu2) {
        other = m2; p.pc = (mu2 - m2) / 2; p.ps = (mu2 + m2) / 2;
    } else if (m2 == mu2) {
        other = n2; p.pc = (mu2 + n2) / 2; p.ps = (mu2 - n2) / 2;
    } else {
        other = n2; p.pc = (mu2 - n2) / 2; p.ps = (mu2 + n2) / 2;
        if (((mu2 + n2) / 2) & 1) p.sg = -1.0;
    }
    p.K = 0.5 * (lf2[mu2] - lf2[(mu2 + other) / 2] - lf2[(mu2 - other) / 2]);
    return p;
}

// log2 |d^mu_{nm}(beta_k)| and its sign, in FP64.
__device__ __forceinline__ double seed_log2(const BandArgs& a, int n2, int m2, int k, double* sgn) {
    const SeedParams sp = seed_params(a.lf2, n2, m2);
    double L = sp.K;
    if (sp.pc) L += (double)sp.pc * a.log2c[k];
    if (sp.ps) L += (double)sp.ps * a.log2s[k];
    *sgn = sp.sg;
    return L;
}

// The seed in FP32 for the complex64 paths.  Per pair, K is split as
// K_hi + K_lo with K_hi on the 2^-11 grid; per node the table holds the same
// split of log2 cos(beta_k/2) and log2 sin(beta_k/2) (BandArgs::seed32).  For
// pc, ps < 2^8 every product pc * hi and the sum of the hi terms are exact in
// FP32, so log2 |d| = L_hi + L_lo is carried to ~1e-8 absolute; then
// |d| = 2^frac * 2^e with e an integer, stored as cur * 2^(-120 E) with the
// scaled exponent in [-60, 60).
struct SeedPair {
    float Khi, Klo, pc, ps, sg;
    int zero_c, zero_s, pad;
};

__device__ __forceinline__ SeedPair make_seed_pair(const double* lf2, int n2, int m2) {
    const SeedParams sp = seed_params(lf2, n2, m2);
    const double kh = rint(sp.K * 2048.0) / 2048.0;
    SeedPair q;
    q.Khi = (float)kh;
    q.Klo = (float)(sp.K - kh);
    q.pc = (float)sp.pc;
    q.ps = (float)sp.ps;
    q.sg = (float)sp.sg;
    q.zero_c = sp.pc > 0;             // cos(beta/2) = 0 at the last node
    q.zero_s = sp.ps > 0;             // sin(beta/2) = 0 at the first node
    q.pad = 0;
    return q;
}

__device__ __forceinline__ float seed_value32(const SeedPair& q, float4 tb, int k, int N, int& E) {
    const float Lh = fmaf(q.ps, tb.z, fmaf(q.pc, tb.x, q.Khi));     // exact
    const float Ll = fmaf(q.ps, tb.w, fmaf(q.pc, tb.y, q.Klo));
    const float ti = floorf(Lh);
    int e = (int)ti;
    const float mant = exp2f((Lh - ti) + Ll);
    E = 0;
    if (e < -60) {
        E = (-e - 60 + 119) / 120;
        e += 120 * E;
    }
    const bool zero = (q.zero_c && k == N - 1) || (q.zero_s && k == 0);
    return zero ? 0.f : q.sg * mant * __int_as_float((e + 127) << 23);
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
    __device__ __forceinline__ void seed32(const SeedPair& q, float4 tb, float2 xs, int k, int N) {
        cur = seed_value32(q, tb, k, N, E);
        prev = 0.f;
        xh = xs.x;
        xl = xs.y;
    }
    __device__ __forceinline__ float value() const { return E == 0 ? cur : 0.f; }
    // plain step, for a state known to have E = 0
    __device__ __forceinline__ void step_fast(const StepCoef<float>& c) {
        const float xb = (xh - c.bh) + (xl - c.bl);
        const float nxt = fmaf(c.A * xb, cur, -c.C * prev);
        prev = cur;
        cur = nxt;
    }
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

}  // namespace su2

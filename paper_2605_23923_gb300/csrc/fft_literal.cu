// Stage 1 on the sampling grid as the paper prints it (Sec. 4, definition of
// the sampling grid): alpha_j = gamma_j = -pi + 2 pi j/(N-1), j = 0..N-1, so
// the last node (+pi) is the first one (-pi) again, with weight 1/(8 pi^2) times
// the cell (2 pi/(N-1))^2, i.e. the prefactor 1/(2M^2) with M = N - 1.
//
// One angle's sum, n integer or n = n0 + 1/2:
//   sum_{j=0}^{M} x_j e^{i n alpha_j} = e^{-i pi n} sum_{j<M} x'_j e^{2 pi i n j/M},
// with the repeated node folded onto the first, x'_0 = x_0 + x_M for integer n
// and x_0 - x_M for half-integer n (e^{2 pi i n} = -1 there), the other x'_j = x_j.
// Half-integer n also carries e^{i pi j/M} on x'_j, leaving the frequency n0.
// M is odd and not a power of two (63, 127 (prime), 255, 511), so the M-point
// DFT is a dense product with W[r][t] = e^{2 pi i (r - N/2) t/M} (t < M; the
// column t = M, and the folded row j = M, are zero):
//   T = X W^T   (sum over gamma, j2),      Y = W T   (sum over alpha, j1),
// Y[r][c] the sum at n = r - N/2 (or n0), m = c - N/2 (or m0).  Both phases
// multiply to (-1)^{n+m} (integer sector) and -(-1)^{n0+m0} (half-integer),
// as on the periodic grid.  Output F2_s[k][m][n] = w_k/(2M^2) * phase * Y[n][m];
// the integer sector's row and column of index 0 (m or n = -N/2) stay zero.
//
// N >= 64 (M = 63, 127, 255, 511): each M-point DFT is taken by Bluestein's
// chirp-z identity, q t = (q^2 + t^2 - (q - t)^2)/2, so
//   sum_t x_t w^{q t} = e^{i pi q^2/M} sum_t (x_t e^{i pi t^2/M}) e^{-i pi (q - t)^2/M},
// w = e^{2 pi i/M}: a convolution with the chirp e^{-i pi u^2/M}, taken
// cyclically with length L = 2N (the N outputs q = -N/2 .. N/2 - 1 from M
// inputs touch u in a range of 2N - 2 < L values, so nothing wraps) by two
// L-point FFTs and the filter's spectrum, precomputed in FP64 on the host.
// Launch 1 (rows): per plane, 16 rows j1 (folded), both sectors, convolution
// over j2 -> T_s[j1][c] in a chunk buffer of the workspace (sized to stay in
// L2); launch 2 (columns): 16 columns c of T_s, convolution over j1, scale,
// phase, planes.  Sector 1's twist e^{i pi (j1 + j2)/M} splits into the two
// launches' input chirps, e^{i pi (t^2 + t)/M}.  O(N^3 log N) per function,
// like the periodic grid.
//
// N < 64, dense products: persistent CTAs, one plane (function, k, s) at a
// time; both products are complex FP32 GEMMs on the CUDA cores, 64 x 64
// output blocks, 256 threads with 4 x 4 complex accumulators each, operand
// chunks of 16 staged in shared memory with the next chunk prefetched into
// registers.  T goes to a per-CTA slab of the workspace (N^2 complex; read
// back at once, so it stays in L2).
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "common.cuh"
#include "su2_internal.h"

namespace su2 {
namespace lit {

constexpr int BM = 64;            // output block (rows and columns)
constexpr int BK = 16;            // contraction chunk
constexpr int THREADS = 256;      // 16 x 16 threads, 4 x 4 outputs each
constexpr int PAD = 1;            // shared row padding (conflict-free transposed stores)
constexpr int LDS = BM + PAD;

__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}

// Folded (and, in the half-integer sector, twisted) sample X_s[j1][t] of plane k.
__device__ __forceinline__ float2 folded(const float2* __restrict__ g, int N, int j1, int t, int s,
                                         const float2* __restrict__ twist) {
    const int M = N - 1;
    if (j1 >= M || t >= M) return make_float2(0.f, 0.f);
    const size_t rs = (size_t)N * N;                 // alpha row stride of a grid
    float2 v = __ldg(g + (size_t)j1 * rs + t);
    const float sg = s ? -1.f : 1.f;
    if (j1 == 0) {
        const float2 u = __ldg(g + (size_t)M * rs + t);
        v.x += sg * u.x;
        v.y += sg * u.y;
    }
    if (t == 0) {
        const float2 u = __ldg(g + (size_t)j1 * rs + M);
        v.x += sg * u.x;
        v.y += sg * u.y;
        if (j1 == 0) {                               // corner: both repeated nodes, sign squared
            const float2 c = __ldg(g + (size_t)M * rs + M);
            v.x += c.x;
            v.y += c.y;
        }
    }
    if (s) v = cmul(v, __ldg(twist + j1 + t));
    return v;
}

// One 64 x 64 block of C = A B with K = N (zero-padded), A(row, t) and B(t, col)
// fetched by the two functors; accumulators acc[i][j] for row i*16+ty, col j*16+tx.
template <typename FA, typename FB>
__device__ __forceinline__ void gemm_block(int N, FA fa, FB fb, float2 (*As)[LDS], float2 (*Bs)[LDS],
                                           float2 (&acc)[4][4]) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    float2 ra[4], rb[4];
    // element q of this thread's share of a chunk: A as (row = e/16, tt = e%16),
    // B as returned by the functor's own mapping
    auto fetch = [&](int t0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + THREADS * q;
            ra[q] = fa(e >> 4, t0 + (e & 15));
            rb[q] = fb(e, t0);
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + THREADS * q;
            As[e & 15][e >> 4] = ra[q];
            int tt, col;
            FB::place(e, &tt, &col);
            Bs[tt][col] = rb[q];
        }
    };
    fetch(0);
    for (int t0 = 0; t0 < N; t0 += BK) {
        __syncthreads();                             // previous chunk consumed
        stash();
        __syncthreads();
        if (t0 + BK < N) fetch(t0 + BK);             // next chunk in flight during the products
#pragma unroll
        for (int tt = 0; tt < BK; ++tt) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[tt][i * 16 + ty];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[tt][j * 16 + tx];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cfma(acc[i][j], a[i], b[j]);
        }
    }
}

// B operand read along t from a row-major matrix R[col][t] (W^T in the first product).
struct BFromRowsT {
    const float2* R;
    int N, c0;
    __device__ float2 operator()(int e, int t0) const {
        const int col = c0 + (e >> 4), t = t0 + (e & 15);
        return (col < N && t < N) ? __ldg(R + (size_t)col * N + t) : make_float2(0.f, 0.f);
    }
    __device__ static void place(int e, int* tt, int* col) { *tt = e & 15; *col = e >> 4; }
};
// B operand read along columns from a row-major matrix R[t][col] (T in the second product).
struct BFromRows {
    const float2* R;
    int N, c0;
    __device__ float2 operator()(int e, int t0) const {
        const int col = c0 + (e & 63), t = t0 + (e >> 6);
        return (col < N && t < N) ? R[(size_t)t * N + col] : make_float2(0.f, 0.f);
    }
    __device__ static void place(int e, int* tt, int* col) { *tt = e >> 6; *col = e & 63; }
};

__global__ void __launch_bounds__(THREADS, 2)
fft_fwd_literal(BandArgs a, const float2* __restrict__ grid, float2* __restrict__ ws) {
    __shared__ float2 As[BK][LDS];
    __shared__ float2 Bs[BK][LDS];
    const int N = a.N, M = N - 1;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int nb = (N + BM - 1) / BM;                // blocks per dimension
    const float2* W = a.lit_w;
    float2* T = ws + a.ws_aux_off + (size_t)blockIdx.x * N * N;
    const long total = (long)a.nfunc * N * 2;
    const float inv2m2 = 1.f / (2.f * (float)M * (float)M);
    for (long p = blockIdx.x; p < total; p += gridDim.x) {
        const int fb = (int)(p / (2 * N)), k = (int)((p >> 1) % N), s = (int)(p & 1);
        const int f = a.fidx[fb];
        const float2* g = grid + a.grid_off[f] + (size_t)k * N;     // plane k: g[j1 * N^2 + j2]
        // T[j1][c] = sum_t X_s[j1][t] W[c][t]
        for (int bi = 0; bi < nb; ++bi)
            for (int bc = 0; bc < nb; ++bc) {
                float2 acc[4][4];
                const int r0 = bi * BM, c0 = bc * BM;
                gemm_block(
                    N, [&](int row, int t) { return (r0 + row < N && t < N) ? folded(g, N, r0 + row, t, s, a.lit_twist)
                                                                             : make_float2(0.f, 0.f); },
                    BFromRowsT{W, N, c0}, As, Bs, acc);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int row = r0 + i * 16 + ty, col = c0 + j * 16 + tx;
                        if (row < N && col < N) T[(size_t)row * N + col] = acc[i][j];
                    }
            }
        __syncthreads();                             // T complete (and visible to the CTA)
        // Y[r][c] = sum_j1 W[r][j1] T[j1][c]; plane element (m = c, n = r)
        const float scale = a.w32[k] * inv2m2;
        float2* out = ws + a.ws_off[f];
        for (int bi = 0; bi < nb; ++bi)
            for (int bc = 0; bc < nb; ++bc) {
                float2 acc[4][4];
                const int r0 = bi * BM, c0 = bc * BM;
                gemm_block(
                    N, [&](int row, int t) { return (r0 + row < N && t < N) ? __ldg(W + (size_t)(r0 + row) * N + t)
                                                                             : make_float2(0.f, 0.f); },
                    BFromRows{T, N, c0}, As, Bs, acc);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int ni = r0 + i * 16 + ty, mi = c0 + j * 16 + tx;
                        if (ni >= N || mi >= N) continue;
                        float sc = ((ni + mi) & 1) ? -scale : scale;
                        if (s) sc = -sc;
                        float2 v = make_float2(acc[i][j].x * sc, acc[i][j].y * sc);
                        if (s == 0 && (ni == 0 || mi == 0)) v = make_float2(0.f, 0.f);
                        const size_t off = a.ws_tile_major
                                               ? (size_t)s * N * N * N + (size_t)mi * N * N + (size_t)(ni >> 2) * 4 * N +
                                                     (size_t)4 * k + (ni & 3)
                                               : ((size_t)k * 2 + s) * N * N + (size_t)mi * N + ni;
                        out[off] = v;
                    }
            }
        __syncthreads();                             // T free for the next plane
    }
}

}  // namespace lit

// ---------------------------------------------------------------------------
// Bluestein (chirp-z) form, N >= 64
// ---------------------------------------------------------------------------
namespace litbs {

// Table block (float2 each): chirp_in[2][N] (sector 0: e^{i pi t^2/M}; sector 1:
// e^{i pi (t^2 + t)/M}), chirp_out[N] (e^{i pi q^2/M}, q = c - N/2), filter[L]
// (FFT of the chirp e^{-i pi u^2/M} over one period of L, divided by L, stored in
// the order the forward four-step FFT leaves its output), om[L] (e^{2 pi i t/L}),
// filter_inv[L] (the same for the chirp e^{+i pi u^2/M} on the inverse's range
// of u; the inverse's chirps are the conjugates of chirp_out and chirp_in).
template <int N> struct Cfg {
    static constexpr int M = N - 1, L = 2 * N;
    static constexpr int R1 = Radix<L>::R1, R2 = Radix<L>::R2;
    static constexpr int ROWS = N >= 512 ? 8 : 16;       // rows (launch 1) / columns (launch 2) per item
    // one pad element per R1 block, plus one so that the rows start in different
    // banks (the column launches fill their rows across lanes)
    static constexpr int PITCH = L + L / R1 + 1;
    static constexpr int THREADS = 256;
    static constexpr int TAB = 3 * N + 3 * L;
    // in shared memory: the chirps (3N) and the re-laid filter and twiddles (3L)
    static constexpr int TABX = 3 * N + 3 * L;
    // launch 1 keeps its raw input rows in shared memory below N = 256; from 256 on
    // it rereads them from L2 for the second sector instead, so that two blocks fit
    // per SM (N = 256 x 8: 10.4 -> 9.5 ms; at N = 128 three fit either way)
    static constexpr bool RAW = N < 256;
    static constexpr size_t smem_bytes() { return (size_t)ROWS * PITCH * 8 + (RAW ? (size_t)ROWS * N * 8 : 0) + (size_t)TABX * 8; }
    __host__ __device__ static constexpr int pad(int p) { return p + p / R1; }
};

// Cyclic convolution of each of the ROWS rows of buf (length L, padded) with
// the chirp: forward four-step FFT (R2-point DFTs over stride R1, twiddle,
// R1-point DFTs), filter, and the transposed steps backwards (inverse R1-point
// DFTs, conjugate twiddle, inverse R2-point DFTs), so the permuted frequency
// order of the forward FFT is never undone explicitly.
// The filter and twiddles come re-laid so that consecutive lanes read consecutive
// entries: filtT[qa R2 + qq] = filter[qa + R1 qq], omA[qq R1 + ia] = omB[ia R2 + qq]
// = om[ia qq] (lanes vary ia in the R2-point passes, qq in the R1-point pass).
template <int N>
__device__ __forceinline__ void conv_rows(float2* buf, const float2* __restrict__ filtT, const float2* __restrict__ omA,
                                          const float2* __restrict__ omB) {
    using P = Cfg<N>;
    constexpr int R1 = P::R1, R2 = P::R2;
    const int tid = threadIdx.x;
    for (int task = tid; task < P::ROWS * R1; task += P::THREADS) {
        const int row = task / R1, ia = task % R1;
        float2* x = buf + row * P::PITCH;
        float2 v[R2];
#pragma unroll
        for (int q = 0; q < R2; ++q) v[q] = x[P::pad(ia + R1 * q)];
        dft_reg<R2, -1, float>(v);
#pragma unroll
        for (int qq = 1; qq < R2; ++qq) v[qq] = cmul(v[qq], cconj(omA[qq * R1 + ia]));
#pragma unroll
        for (int qq = 0; qq < R2; ++qq) x[P::pad(ia + R1 * qq)] = v[qq];
    }
    __syncthreads();
    for (int task = tid; task < P::ROWS * R2; task += P::THREADS) {
        const int row = task / R2, qq = task % R2;
        float2* x = buf + row * P::PITCH + qq * (R1 + 1);  // pad(qq R1 + ia) = qq (R1 + 1) + ia
        float2 v[R1];
#pragma unroll
        for (int ia = 0; ia < R1; ++ia) v[ia] = x[ia];
        dft_reg<R1, -1, float>(v);                       // v[qa]: frequency qq + R2 qa
#pragma unroll
        for (int qa = 0; qa < R1; ++qa) v[qa] = cmul(v[qa], filtT[qa * R2 + qq]);
        dft_reg<R1, 1, float>(v);
#pragma unroll
        for (int ia = 1; ia < R1; ++ia) v[ia] = cmul(v[ia], omB[ia * R2 + qq]);
#pragma unroll
        for (int ia = 0; ia < R1; ++ia) x[ia] = v[ia];
    }
    __syncthreads();
    for (int task = tid; task < P::ROWS * R1; task += P::THREADS) {
        const int row = task / R1, ia = task % R1;
        float2* x = buf + row * P::PITCH;
        float2 v[R2];
#pragma unroll
        for (int qq = 0; qq < R2; ++qq) v[qq] = x[P::pad(ia + R1 * qq)];
        dft_reg<R2, 1, float>(v);
#pragma unroll
        for (int q = 0; q < R2; ++q) x[P::pad(ia + R1 * q)] = v[q];
    }
    __syncthreads();
}

// Copies the chirps of the table block to shared memory at byte offset `off`,
// followed by the re-laid filter (the inverse's when inv) and twiddles that
// conv_rows reads (the caller makes them visible with a barrier before the
// first use).
template <int N>
__device__ __forceinline__ float2* load_tables(const BandArgs& a, unsigned char* smem, size_t off, bool inv) {
    using P = Cfg<N>;
    constexpr int L = P::L, R1 = P::R1, R2 = P::R2;
    float2* tab = reinterpret_cast<float2*>(smem + off);
    for (int t = threadIdx.x; t < 3 * N; t += P::THREADS) tab[t] = a.lit_bs[t];   // chirps
    const float2* filt = a.lit_bs + 3 * N + (inv ? 2 * L : 0);
    const float2* om = a.lit_bs + 3 * N + L;
    float2* x = tab + 3 * N;                             // [filtT L][omA L][omB L]
    for (int t = threadIdx.x; t < L; t += P::THREADS) {
        x[t] = filt[(t / R2) + R1 * (t % R2)];           // filtT[qa R2 + qq]
        x[L + t] = om[(t % R1) * (t / R1)];              // omA[qq R1 + ia]
        x[2 * L + t] = om[(t / R2) * (t % R2)];          // omB[ia R2 + qq]
    }
    return tab;
}

// Launch 1: item = (plane p0 + i / NRB, rows j1 in [ROWS rb, ROWS rb + ROWS)).
template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
lit_rows(BandArgs a, const float2* __restrict__ grid, float2* __restrict__ ws, int p0) {
    using P = Cfg<N>;
    constexpr int M = P::M, L = P::L, NRB = N / P::ROWS;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);                        // [ROWS][PITCH]
    float2* raw = buf + P::ROWS * P::PITCH;                               // [ROWS][N] (RAW)
    const float2* tab = load_tables<N>(a, smem, (size_t)P::ROWS * P::PITCH * 8 + (P::RAW ? (size_t)P::ROWS * N * 8 : 0), false);
    const float2 *cin = tab, *cout = tab + 2 * N;
    const int plane = p0 + blockIdx.x / NRB, rb = blockIdx.x % NRB;
    const int fb = plane / N, k = plane % N;
    const float2* g = grid + a.grid_off[a.fidx[fb]] + (size_t)k * N;     // plane k: g[j1 N^2 + j2]
    const size_t rs = (size_t)N * N;
    if constexpr (P::RAW) {
        for (int e = threadIdx.x; e < P::ROWS * N; e += P::THREADS) {
            const int rr = e / N, t = e % N, j1 = rb * P::ROWS + rr;
            raw[e] = (j1 < M) ? g[(size_t)j1 * rs + t] : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    float2* T = ws + a.ws_aux_off + (size_t)(plane - p0) * 2 * N * N;
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
        const float sg = s ? -1.f : 1.f;
        for (int e = threadIdx.x; e < P::ROWS * L; e += P::THREADS) {
            const int rr = e / L, t = e % L, j1 = rb * P::ROWS + rr;
            float2 v = make_float2(0.f, 0.f);
            if (j1 < M && t < M) {
                v = P::RAW ? raw[rr * N + t] : __ldg(g + (size_t)j1 * rs + t);
                if (t == 0) {                                  // repeated gamma node folded
                    const float2 u = P::RAW ? raw[rr * N + M] : __ldg(g + (size_t)j1 * rs + M);
                    v.x += sg * u.x;
                    v.y += sg * u.y;
                }
                if (j1 == 0) {                                 // repeated alpha node folded
                    const float2 u = g[(size_t)M * rs + t];
                    v.x += sg * u.x;
                    v.y += sg * u.y;
                    if (t == 0) {                              // corner: both, sign squared
                        const float2 c = g[(size_t)M * rs + M];
                        v.x += c.x;
                        v.y += c.y;
                    }
                }
                v = cmul(v, cin[s * N + t]);
            }
            buf[rr * P::PITCH + P::pad(t)] = v;
        }
        __syncthreads();
        conv_rows<N>(buf, tab + 3 * N, tab + 3 * N + L, tab + 3 * N + 2 * L);
        for (int e = threadIdx.x; e < P::ROWS * N; e += P::THREADS) {
            const int rr = e / N, c = e % N, j1 = rb * P::ROWS + rr;
            if (j1 >= M) continue;
            const int q = (c - N / 2 + L) % L;
            T[(size_t)s * N * N + (size_t)j1 * N + c] = cmul(buf[rr * P::PITCH + P::pad(q)], cout[c]);
        }
        __syncthreads();
    }
}

// Launch 2: item = (plane p0 + i / (2 NCB), sector, columns c in [ROWS cb, ROWS cb + ROWS)).
template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
lit_cols(BandArgs a, float2* __restrict__ ws, int p0) {
    using P = Cfg<N>;
    constexpr int M = P::M, L = P::L, NCB = N / P::ROWS, R = P::ROWS;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);                        // [ROWS][PITCH]
    const float2* tab = load_tables<N>(a, smem, (size_t)P::ROWS * P::PITCH * 8, false);   // no raw rows here
    __syncthreads();
    const float2 *cin = tab, *cout = tab + 2 * N;
    const int plane = p0 + blockIdx.x / (2 * NCB), s = (blockIdx.x / NCB) & 1, cb = blockIdx.x % NCB;
    const int fb = plane / N, k = plane % N;
    const float2* T = ws + a.ws_aux_off + ((size_t)(plane - p0) * 2 + s) * N * N;
    for (int e = threadIdx.x; e < R * L; e += P::THREADS) {
        const int cc = e % R, j1 = e / R;                        // R consecutive columns of row j1
        float2 v = make_float2(0.f, 0.f);
        if (j1 < M) v = cmul(T[(size_t)j1 * N + cb * R + cc], cin[s * N + j1]);
        buf[cc * P::PITCH + P::pad(j1)] = v;
    }
    __syncthreads();
    conv_rows<N>(buf, tab + 3 * N, tab + 3 * N + L, tab + 3 * N + 2 * L);
    const float scale = a.w32[k] / (2.f * (float)M * (float)M);
    const size_t plane_off = a.ws_off[a.fidx[fb]];
    for (int e = threadIdx.x; e < R * N; e += P::THREADS) {
        const int cc = e / N, ni = e % N, mi = cb * R + cc;
        const int q = (ni - N / 2 + L) % L;
        float sc = ((ni + mi) & 1) ? -scale : scale;
        if (s) sc = -sc;
        float2 v = cmul(buf[cc * P::PITCH + P::pad(q)], cout[ni]);
        v = (s == 0 && (ni == 0 || mi == 0)) ? make_float2(0.f, 0.f) : make_float2(v.x * sc, v.y * sc);
        const size_t off = a.ws_tile_major ? (size_t)s * N * N * N + (size_t)mi * N * N + (size_t)(ni >> 2) * 4 * N +
                                                 (size_t)4 * k + (ni & 3)
                                           : ((size_t)k * 2 + s) * N * N + (size_t)mi * N + ni;
        ws[plane_off + off] = v;
    }
}

// ---------------------------------------------------------------------------
// Synthesis / adjoint on the printed grid: from the tile-major planes G_s[k][mi][ni]
// (the transposed contraction's output) to the grid at every printed node,
//   f[j1,k,j2] = sum_s sum_{n', m'} sg_s G_s e^{-2 pi i (n' j1 + m' j2)/M} e^{-i pi s (j1 + j2)/M}
// for j1, j2 < M (n' = n or n0, the N frequencies of each angle, sg_s the origin
// phase as in the forward), and at the repeated node +pi (j = M) the value at
// -pi with the half-integer sector negated.  The inverse M-point DFTs (N inputs,
// M outputs) by Bluestein with the conjugate chirps and the inverse filter.
// Launch 1: plane, sector, 16 rows mi: DFT over ni -> T_s[mi][j1];
// launch 2: plane, 16 columns j1, both sectors: DFT over mi, untwist, sector
// sum, the repeated gamma node; the item of column j1 = 0 also writes row M.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
lit_inv_rows(BandArgs a, float2* __restrict__ ws, int p0) {
    using P = Cfg<N>;
    constexpr int M = P::M, L = P::L, NRB = N / P::ROWS;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);                        // [ROWS][PITCH]
    const float2* tab = load_tables<N>(a, smem, (size_t)P::ROWS * P::PITCH * 8, true);
    __syncthreads();
    const float2 *cin = tab, *cout = tab + 2 * N;
    const int plane = p0 + blockIdx.x / (2 * NRB), s = (blockIdx.x / NRB) & 1, rb = blockIdx.x % NRB;
    const int fb = plane / N, k = plane % N;
    const float2* G = ws + a.ws_off[a.fidx[fb]] + (size_t)s * N * N * N + (size_t)4 * k;
    for (int e = threadIdx.x; e < P::ROWS * L; e += P::THREADS) {
        const int rr = e / L, ni = e % L, mi = rb * P::ROWS + rr;
        float2 v = make_float2(0.f, 0.f);
        if (ni < N && !(s == 0 && (ni == 0 || mi == 0))) {
            const float2 g = G[(size_t)mi * N * N + (size_t)(ni >> 2) * 4 * N + (ni & 3)];
            float sg = ((ni + mi) & 1) ? -1.f : 1.f;
            if (s) sg = -sg;
            v = cmul(make_float2(g.x * sg, g.y * sg), cconj(cout[ni]));
        }
        buf[rr * P::PITCH + P::pad(ni)] = v;
    }
    __syncthreads();
    conv_rows<N>(buf, tab + 3 * N, tab + 3 * N + L, tab + 3 * N + 2 * L);
    float2* T = ws + a.ws_aux_off + ((size_t)(plane - p0) * 2 + s) * N * N;
    for (int e = threadIdx.x; e < P::ROWS * N; e += P::THREADS) {
        const int rr = e / N, j1 = e % N, mi = rb * P::ROWS + rr;
        if (j1 >= M) continue;
        T[(size_t)mi * N + j1] = cmul(buf[rr * P::PITCH + P::pad(j1 + N / 2)], cconj(cin[s * N + j1]));
    }
}

template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
lit_inv_cols(BandArgs a, const float2* __restrict__ ws, float2* __restrict__ grid, int p0) {
    using P = Cfg<N>;
    constexpr int M = P::M, L = P::L, NCB = N / P::ROWS, R = P::ROWS;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);                        // [ROWS][PITCH]
    float2* Z = buf + R * P::PITCH;                                       // [ROWS][N] sector-0 values
    const float2* tab = load_tables<N>(a, smem, (size_t)R * P::PITCH * 8 + (size_t)R * N * 8, true);
    __syncthreads();
    const float2 *cin = tab, *cout = tab + 2 * N;
    const int plane = p0 + blockIdx.x / NCB, cb = blockIdx.x % NCB;
    const int fb = plane / N, k = plane % N;
    float2* g = grid + a.grid_off[a.fidx[fb]] + (size_t)k * N;          // g[j1 N^2 + j2]
    const size_t rs = (size_t)N * N;
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
        const float2* T = ws + a.ws_aux_off + ((size_t)(plane - p0) * 2 + s) * N * N;
        for (int e = threadIdx.x; e < R * L; e += P::THREADS) {
            const int cc = e % R, mi = e / R, j1 = cb * R + cc;           // R consecutive j1 of row mi
            float2 v = make_float2(0.f, 0.f);
            if (mi < N && j1 < M) v = cmul(T[(size_t)mi * N + j1], cconj(cout[mi]));
            buf[cc * P::PITCH + P::pad(mi)] = v;
        }
        __syncthreads();
        conv_rows<N>(buf, tab + 3 * N, tab + 3 * N + L, tab + 3 * N + 2 * L);
        for (int e = threadIdx.x; e < R * N; e += P::THREADS) {
            const int cc = e / N, j2 = e % N, j1 = cb * R + cc;
            if (j1 >= M || j2 >= M) continue;
            const float2 y = cmul(buf[cc * P::PITCH + P::pad(j2 + N / 2)], cconj(cin[s * N + j2]));
            if (s == 0) {
                Z[cc * N + j2] = y;
                continue;
            }
            const float2 z = Z[cc * N + j2];
            g[(size_t)j1 * rs + j2] = make_float2(z.x + y.x, z.y + y.y);
            if (j2 == 0) g[(size_t)j1 * rs + M] = make_float2(z.x - y.x, z.y - y.y);   // gamma = +pi
            if (j1 == 0) {                                                          // alpha = +pi
                g[(size_t)M * rs + j2] = make_float2(z.x - y.x, z.y - y.y);
                if (j2 == 0) g[(size_t)M * rs + M] = make_float2(z.x + y.x, z.y + y.y);
            }
        }
        __syncthreads();
    }
}

template <int N>
static cudaError_t launch_inv_n(const BandArgs& a, const void* ws, void* grid, cudaStream_t st) {
    using P = Cfg<N>;
    const size_t smem1 = (size_t)P::ROWS * P::PITCH * 8 + (size_t)P::TABX * 8;
    const size_t smem2 = (size_t)P::ROWS * P::PITCH * 8 + (size_t)P::ROWS * N * 8 + (size_t)P::TABX * 8;
    cudaError_t e = cudaFuncSetAttribute(lit_inv_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(lit_inv_cols<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
    const int nplanes = a.nfunc * N, chunk = a.aux_ring;
    for (int p0 = 0; p0 < nplanes; p0 += chunk) {
        const int np = nplanes - p0 < chunk ? nplanes - p0 : chunk;
        lit_inv_rows<N><<<np * 2 * (N / P::ROWS), P::THREADS, smem1, st>>>(a, (float2*)ws, p0);
        lit_inv_cols<N><<<np * (N / P::ROWS), P::THREADS, smem2, st>>>(a, (const float2*)ws, (float2*)grid, p0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// planes per chunk: the chunk's intermediate (2 N^2 complex per plane) stays
// near 64 MB, well inside the L2
inline int chunk_planes(int N) {
    const size_t per = (size_t)2 * N * N * 8;
    const size_t p = ((size_t)64 << 20) / per;
    return (int)(p < 1 ? 1 : (p > 4096 ? 4096 : p));
}

template <int N>
static cudaError_t launch_n(const BandArgs& a, const void* grid, void* ws, cudaStream_t st) {
    using P = Cfg<N>;
    // launch 1: rows (+ raw rows below N = 256) + tables; launch 2: rows + tables
    const size_t smem2 = (size_t)P::ROWS * P::PITCH * 8 + (size_t)P::TABX * 8, smem1 = P::smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(lit_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lit_cols<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
    const int nplanes = a.nfunc * N, chunk = a.aux_ring;
    for (int p0 = 0; p0 < nplanes; p0 += chunk) {
        const int np = nplanes - p0 < chunk ? nplanes - p0 : chunk;
        lit_rows<N><<<np * (N / P::ROWS), P::THREADS, smem1, st>>>(a, (const float2*)grid, (float2*)ws, p0);
        lit_cols<N><<<np * 2 * (N / P::ROWS), P::THREADS, smem2, st>>>(a, (float2*)ws, p0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace litbs

bool fft_literal_bluestein(int N) { return N >= 64 && N <= 512; }

// Host-side Bluestein tables for bandwidth N (FP64, rounded once): see litbs::Cfg.
void fft_literal_bluestein_tables(int N, std::vector<float2>& out) {
    const int M = N - 1, L = 2 * N;
    int R1 = 0;
    switch (L) {
        case 128: R1 = Radix<128>::R1; break;
        case 256: R1 = Radix<256>::R1; break;
        case 512: R1 = Radix<512>::R1; break;
        default: R1 = Radix<1024>::R1; break;
    }
    const int R2 = L / R1;
    const double pi = 3.14159265358979323846;
    auto cis = [&](long num, long den) {             // e^{i pi num/den}, num reduced mod 2 den
        long r = num % (2 * den);
        if (r < 0) r += 2 * den;
        const double ang = pi * (double)r / (double)den;
        return make_float2((float)cos(ang), (float)sin(ang));
    };
    out.assign(3 * N + 3 * L, make_float2(0.f, 0.f));
    for (int t = 0; t < N; ++t) {
        out[t] = cis((long)t * t, M);
        out[N + t] = cis((long)t * t + t, M);
        const long q = t - N / 2;
        out[2 * N + t] = cis(q * q, M);
    }
    // filter spectra: the chirp e^{sg i pi u^2/M} on u in [u0, u1], placed at u mod L,
    // transformed (e^{-2 pi i f n/L}), divided by L, in the four-step output order
    auto filter = [&](double sg, long u0, long u1, int at) {
        std::vector<double> br(L, 0.0), bi(L, 0.0);
        for (long u = u0; u <= u1; ++u) {
            const long r = (u * u) % (2L * M);
            const double ang = sg * pi * (double)r / (double)M;
            const int idx = (int)((u % L + L) % L);
            br[idx] = cos(ang);
            bi[idx] = sin(ang);
        }
        for (int qa = 0; qa < R1; ++qa)
            for (int qq = 0; qq < R2; ++qq) {
                const int f = qq + R2 * qa;              // frequency held at position qa + R1 qq
                double sr = 0.0, si = 0.0;
                for (int n = 0; n < L; ++n) {
                    const long r = ((long)f * n) % L;
                    const double ang = -2.0 * pi * (double)r / (double)L;
                    const double c = cos(ang), sn = sin(ang);
                    sr += br[n] * c - bi[n] * sn;
                    si += br[n] * sn + bi[n] * c;
                }
                out[at + qa + R1 * qq] = make_float2((float)(sr / L), (float)(si / L));
            }
    };
    // forward: outputs q in [-N/2, N/2 - 1] from inputs t in [0, M): u = q - t
    filter(-1.0, -(long)(N / 2) - M + 1, N / 2 - 1, 3 * N);
    // inverse: outputs j in [0, M) from inputs q in [-N/2, N/2 - 1] at position q + N/2:
    // u = j + N/2 - p ranges over [-N/2 + 1, 3N/2 - 2]
    filter(1.0, -(long)(N / 2) + 1, 3L * N / 2 - 2, 3 * N + 2 * L);
    for (int t = 0; t < L; ++t) {
        const double ang = 2.0 * pi * (double)t / (double)L;
        out[3 * N + L + t] = make_float2((float)cos(ang), (float)sin(ang));
    }
}

cudaError_t fft_forward_literal_aux(int N, int device, int* ctas, size_t* elems) {
    if (fft_literal_bluestein(N)) {
        // chunk of planes whose intermediate T_s (2 N^2 complex per plane) stays in L2
        *ctas = litbs::chunk_planes(N);
        *elems = (((size_t)*ctas * 2 * N * N + 31) / 32) * 32;
        return cudaSuccess;
    }
    int sms = 0, per = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lit::fft_fwd_literal, lit::THREADS, 0);
    if (e != cudaSuccess) return e;
    if (per < 1) per = 1;
    *ctas = sms * per;
    // one N x N slab per CTA, rounded to 256 bytes (32 complex64)
    *elems = (((size_t)*ctas * N * N + 31) / 32) * 32;
    return cudaSuccess;
}

cudaError_t launch_fft_inverse_literal(const BandArgs& a, const void* ws, void* grid, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    if (!fft_literal_bluestein(a.N) || a.aux_ring < 1 || !a.lit_bs || !a.ws_tile_major) return cudaErrorInvalidValue;
    switch (a.N) {
        case 64: return litbs::launch_inv_n<64>(a, ws, grid, st);
        case 128: return litbs::launch_inv_n<128>(a, ws, grid, st);
        case 256: return litbs::launch_inv_n<256>(a, ws, grid, st);
        case 512: return litbs::launch_inv_n<512>(a, ws, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fft_forward_literal(const BandArgs& a, const void* grid, void* ws, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    if (fft_literal_bluestein(a.N)) {
        if (a.aux_ring < 1 || !a.lit_bs) return cudaErrorInvalidValue;
        switch (a.N) {
            case 64: return litbs::launch_n<64>(a, grid, ws, st);
            case 128: return litbs::launch_n<128>(a, grid, ws, st);
            case 256: return litbs::launch_n<256>(a, grid, ws, st);
            case 512: return litbs::launch_n<512>(a, grid, ws, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (a.aux_ring < 1 || !a.lit_w || !a.lit_twist) return cudaErrorInvalidValue;
    const long planes = (long)a.nfunc * a.N * 2;
    const int g = planes < a.aux_ring ? (int)planes : a.aux_ring;     // at most one slab per CTA
    lit::fft_fwd_literal<<<g, lit::THREADS, 0, st>>>(a, (const float2*)grid, (float2*)ws);
    return cudaGetLastError();
}

}  // namespace su2

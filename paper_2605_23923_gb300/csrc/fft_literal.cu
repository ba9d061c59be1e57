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
// Kernel: persistent CTAs, one plane (function, k, s) at a time; both products
// are complex FP32 GEMMs on the CUDA cores, 64 x 64 output blocks, 256 threads
// with 4 x 4 complex accumulators each, operand chunks of 16 staged in shared
// memory with the next chunk prefetched into registers.  T goes to a per-CTA
// slab of the workspace (N^2 complex; read back at once, so it stays in L2).
#include <cuda_runtime.h>

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

cudaError_t fft_forward_literal_aux(int N, int device, int* ctas, size_t* elems) {
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

cudaError_t launch_fft_forward_literal(const BandArgs& a, const void* grid, void* ws, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    if (a.aux_ring < 1 || !a.lit_w || !a.lit_twist) return cudaErrorInvalidValue;
    const long planes = (long)a.nfunc * a.N * 2;
    const int g = planes < a.aux_ring ? (int)planes : a.aux_ring;     // at most one slab per CTA
    lit::fft_fwd_literal<<<g, lit::THREADS, 0, st>>>(a, (const float2*)grid, (float2*)ws);
    return cudaGetLastError();
}

}  // namespace su2

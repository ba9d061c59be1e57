// Stage 1 of the SU(2) transform: the 2-D DFT over (alpha, gamma) for every
// beta node (Sec. 4 factorised Riemann sum; Sec. 6 first-stage Proposition),
// and its inverse for the synthesis / adjoint.
//
// Forward, for function f, node k and sector s (0: integer l, 1: half-integer l):
//   F2_s[k][m][n] = w_k/(2N^2) (-1)^{n+m} sum_{j1,j2} f[j1,k,j2] tw_s(j1,j2) omega^{p j1 + q j2}
//   omega = exp(+2 pi i/N), p = n mod N, q = m mod N (sector 0);
//   sector 1 uses n = n0 + 1/2, m = m0 + 1/2, p = n0 mod N, q = m0 mod N and the
//   pre-twist tw_1(j1,j2) = exp(i pi (j1 + j2)/N); tw_0 = 1.
// This equals w_k/(2N^2) sum f exp(i(n alpha_j1 + m gamma_j2)) with
// alpha_j = gamma_j = -pi + 2 pi j/N.  Storage: plane (k, s) of function f at
// ws_off[f] + (2k + s) N^2, row mi = (q + N/2) mod N, column ni = (p + N/2) mod N
// (n fastest).  In sector 0 row/column 0 (the Nyquist bin) is unused and
// written as zero.
//
// Inverse: f[j1,k,j2] = sum_s conj(tw_s(j1,j2)) sum_{p,q} (-1)^{n+m} G_s[k][m][n] omega^{-(p j1 + q j2)}.
//
// Kernel design (N >= 32): one thread-block cluster of C = N/32 CTAs per plane;
// CTA c holds the 32 columns j2 in [32c, 32c+32) of all N rows.  Pass 1 runs
// the column DFTs over j1 (four-step: R2-point then R1-point register DFTs,
// twiddle table in shared memory, padded [N][33] layout, lanes across columns).
// After a cluster barrier, CTA c' gathers the rows p in [32c', 32c'+32) from
// every CTA's shared memory (ld.shared::cluster) and runs the row DFTs over
// j2; the second half of that DFT writes 32 consecutive n per warp store.
#include <string.h>

#include "common.cuh"
#include "su2_internal.h"

namespace su2 {

// Stage-1 plane (k, s) of function f in the workspace and the offset of element
// (mi, ni) from it: [k][s][mi][ni] or, tile-major, [s][mi][ni/4][k][ni%4].
template <typename Cx>
__device__ __forceinline__ const Cx* plane_base(const Cx* ws, const BandArgs& a, int f, int k, int s, int N) {
    if (a.ws_tile_major) return ws + a.ws_off[f] + (size_t)s * N * N * N + (size_t)4 * k;
    return ws + a.ws_off[f] + ((size_t)k * 2 + s) * N * N;
}
__device__ __forceinline__ size_t plane_index(const BandArgs& a, int mi, int ni, int N) {
    if (a.ws_tile_major) return (size_t)mi * N * N + (size_t)(ni >> 2) * 4 * N + (ni & 3);
    return (size_t)mi * N + ni;
}

template <typename T> __device__ __forceinline__ cplx<T> om_at(const BandArgs& a, int t);
template <> __device__ __forceinline__ float2 om_at<float>(const BandArgs& a, int t) { return a.om32[t]; }
template <> __device__ __forceinline__ double2 om_at<double>(const BandArgs& a, int t) { return a.om64[t]; }
template <typename T> __device__ __forceinline__ cplx<T> twist_at(const BandArgs& a, int t);
template <> __device__ __forceinline__ float2 twist_at<float>(const BandArgs& a, int t) { return __ldg(a.twist32 + t); }
template <> __device__ __forceinline__ double2 twist_at<double>(const BandArgs& a, int t) { return __ldg(a.twist64 + t); }
template <typename T> __device__ __forceinline__ T weight_at(const BandArgs& a, int k);
template <> __device__ __forceinline__ float weight_at<float>(const BandArgs& a, int k) { return a.w32[k]; }
template <> __device__ __forceinline__ double weight_at<double>(const BandArgs& a, int k) { return a.w64[k]; }

template <typename T, int N, int C>
struct FftShape {
    static constexpr int W = N / C;
    static constexpr int R1 = Radix<N>::R1;
    static constexpr int R2 = Radix<N>::R2;
    static constexpr int LD1 = W + 1;
    static constexpr int LD2 = N + 1;
    static constexpr int BUF = (N * LD1 > W * LD2) ? N * LD1 : W * LD2;
    static constexpr size_t smem_bytes() { return (size_t)(BUF + N) * sizeof(cplx<T>); }
};

// ---------------------------------------------------------------------------
// Forward, cluster version
// ---------------------------------------------------------------------------
template <typename T, int N, int C, int THREADS>
__global__ void __launch_bounds__(THREADS)
fft_fwd_cluster(BandArgs a, const cplx<T>* __restrict__ grid, cplx<T>* __restrict__ ws) {
    using Cx = cplx<T>;
    using S = FftShape<T, N, C>;
    constexpr int W = S::W, R1 = S::R1, R2 = S::R2, LD1 = S::LD1, LD2 = S::LD2;
    static_assert(W == 32, "one warp of columns per CTA");
    static_assert((W * R1) % THREADS == 0 && (W * R2) % THREADS == 0, "task split");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx* buf = reinterpret_cast<Cx*>(smem_raw);
    Cx* om = buf + S::BUF;

    const int c = (C > 1) ? (int)cluster_ctarank() : 0;
    const int s = blockIdx.x / C;
    const int k = blockIdx.y;
    const int f = a.fidx[blockIdx.z];
    const int tid = threadIdx.x;

    for (int t = tid; t < N; t += THREADS) om[t] = om_at<T>(a, t);
    __syncthreads();

    const Cx* X = grid + a.grid_off[f] + (size_t)k * N;     // X[j1*N*N + j2]

    // Pass 1A: column DFT, stride-R1 part, loaded straight from global memory.
#pragma unroll
    for (int it = 0; it < (W * R1) / THREADS; ++it) {
        const int task = tid + it * THREADS;
        const int jc = task % W, ia = task / W;
        const int j2 = c * W + jc;
        Cx v[R2];
#pragma unroll
        for (int b = 0; b < R2; ++b) v[b] = X[(size_t)(ia + R1 * b) * N * N + j2];
        if (s) {
            const Cx t2 = twist_at<T>(a, j2);
#pragma unroll
            for (int b = 0; b < R2; ++b) v[b] = cmul(v[b], cmul(twist_at<T>(a, ia + R1 * b), t2));
        }
        dft_reg<R2, 1, T>(v);
#pragma unroll
        for (int qb = 0; qb < R2; ++qb)
            buf[(ia + R1 * qb) * LD1 + jc] = (qb == 0) ? v[0] : cmul(v[qb], om[ia * qb]);
    }
    __syncthreads();
    // Pass 1B: contiguous R1-point DFTs; bin p = qb + R2*qa lands in row qa + R1*qb.
#pragma unroll
    for (int it = 0; it < (W * R2) / THREADS; ++it) {
        const int task = tid + it * THREADS;
        const int jc = task % W, qb = task / W;
        Cx v[R1];
#pragma unroll
        for (int ia = 0; ia < R1; ++ia) v[ia] = buf[(ia + R1 * qb) * LD1 + jc];
        dft_reg<R1, 1, T>(v);
#pragma unroll
        for (int qa = 0; qa < R1; ++qa) buf[(qa + R1 * qb) * LD1 + jc] = v[qa];
    }
    if constexpr (C > 1) cluster_sync_all(); else __syncthreads();

    // Pass 2A: gather the owned rows p from all CTAs, stride-R1 part of the row DFT.
    constexpr int NT2 = (W * R1) / THREADS;
    Cx hold[NT2][R2];
#pragma unroll
    for (int it = 0; it < NT2; ++it) {
        const int task = tid + it * THREADS;
        const int pl = task % W, ia = task / W;
        const int p = c * W + pl;
        const int rowp = p / R2 + R1 * (p % R2);
        Cx v[R2];
#pragma unroll
        for (int b = 0; b < R2; ++b) {
            const int j2 = ia + R1 * b;
            const Cx* src = &buf[rowp * LD1 + (j2 % W)];
            if constexpr (C > 1) v[b] = ld_dsmem(map_shared(src, (unsigned)(j2 / W)), Cx());
            else v[b] = *src;
        }
        dft_reg<R2, 1, T>(v);
#pragma unroll
        for (int qb = 0; qb < R2; ++qb) hold[it][qb] = (qb == 0) ? v[0] : cmul(v[qb], om[ia * qb]);
    }
    if constexpr (C > 1) cluster_sync_all(); else __syncthreads();
#pragma unroll
    for (int it = 0; it < NT2; ++it) {
        const int task = tid + it * THREADS;
        const int pl = task % W, ia = task / W;
#pragma unroll
        for (int qb = 0; qb < R2; ++qb) buf[pl * LD2 + ia + R1 * qb] = hold[it][qb];
    }
    __syncthreads();

    // Pass 2B: R1-point DFTs, scale and store F2 rows (n fastest).
    const T scale = weight_at<T>(a, k) / (T(2) * T(N) * T(N));
    Cx* out = ws + a.ws_off[f] + ((size_t)k * 2 + s) * N * N;
#pragma unroll
    for (int it = 0; it < (W * R2) / THREADS; ++it) {
        const int task = tid + it * THREADS;
        const int pl = task % W, qb = task / W;
        const int p = c * W + pl;
        Cx v[R1];
#pragma unroll
        for (int ia = 0; ia < R1; ++ia) v[ia] = buf[pl * LD2 + ia + R1 * qb];
        dft_reg<R1, 1, T>(v);
        const int ni = (p + N / 2) & (N - 1);
#pragma unroll
        for (int qa = 0; qa < R1; ++qa) {
            const int q = qb + R2 * qa;
            const int mi = (q + N / 2) & (N - 1);
            T sg = ((ni + mi) & 1) ? T(-1) : T(1);
            if (s) sg = -sg;
            Cx val = cscale(v[qa], sg * scale);
            if (s == 0 && (ni == 0 || mi == 0)) val = mk<T>(T(0), T(0));
            out[(size_t)mi * N + ni] = val;
        }
    }
}

// ---------------------------------------------------------------------------
// Forward, persistent pipelined version (N = 64, 128, 256; complex64).
// One cluster of C = N/32 CTAs walks over planes (function, beta node); CTA c
// owns the 32 columns j2 in [32c, 32c+32).  The next plane's N x 32 column
// slab is brought into a second shared buffer by 1-D bulk copies (TMA, one
// 256-byte row each, completion on an mbarrier) while the current plane runs
// both sectors through the four DFT passes, so loads overlap compute.
// ---------------------------------------------------------------------------
template <int N>
struct PipeCfg {
    static constexpr int C = N / 32;
    static constexpr int W = 32;
    static constexpr int R1 = Radix<N>::R1, R2 = Radix<N>::R2;
    static constexpr int THREADS = (W * R1 > 512) ? 512 : W * R1;
    static constexpr int LD1 = W + 1, LD2 = N + 1;
    static constexpr int SLAB = N * W;
    static constexpr int WBUF = (N * LD1 > W * LD2) ? N * LD1 : W * LD2;
    static constexpr int F2S = 2 * SLAB + WBUF + N + 2 * N;       // float2 elements
    static constexpr size_t smem_bytes() { return (size_t)F2S * sizeof(float2) + 2 * sizeof(uint64_t); }
};

template <int N>
__global__ void __launch_bounds__(PipeCfg<N>::THREADS, 1)
fft_fwd_pipe(BandArgs a, const float2* __restrict__ grid, float2* __restrict__ ws) {
    using P = PipeCfg<N>;
    constexpr int C = P::C, W = P::W, R1 = P::R1, R2 = P::R2, LD1 = P::LD1, LD2 = P::LD2;
    constexpr int THREADS = P::THREADS, SLAB = P::SLAB;
    static_assert(C >= 2, "cluster of at least two CTAs");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);       // [2][N][W] dense
    float2* Wb = S + 2 * SLAB;                              // work buffer
    float2* om = Wb + P::WBUF;                              // exp(+2 pi i t/N)
    float2* tw2 = om + N;                                   // exp(i pi t/N), t < 2N
    uint64_t* mbar = reinterpret_cast<uint64_t*>(tw2 + 2 * N);

    const int c = (int)cluster_ctarank();
    const int q = blockIdx.x / C, nq = gridDim.x / C;
    const int nplanes = a.nfunc * N;
    const int tid = threadIdx.x, lane = tid & 31;

    for (int t = tid; t < N; t += THREADS) om[t] = a.om32[t];
    for (int t = tid; t < 2 * N; t += THREADS) {
        const float2 z = a.twist32[t & (N - 1)];
        tw2[t] = (t < N) ? z : make_float2(-z.x, -z.y);
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](int plane, int buf) {   // warp 0 only
        const int f = a.fidx[plane / N], k = plane % N;
        const float2* src = grid + a.grid_off[f] + (size_t)k * N + c * W;
        float2* dst = S + buf * SLAB;
        if (lane == 0) mbar_arrive_expect_tx(&mbar[buf], (uint32_t)(N * W * sizeof(float2)));
        __syncwarp();
        for (int j1 = lane; j1 < N; j1 += 32)
            bulk_g2s(dst + j1 * W, src + (size_t)j1 * N * N, (uint32_t)(W * sizeof(float2)), &mbar[buf]);
    };

    if (q < nplanes && tid < 32) issue(q, 0);
    int it = 0;
    for (int plane = q; plane < nplanes; plane += nq, ++it) {
        const int buf = it & 1;
        const int next = plane + nq;
        if (next < nplanes && tid < 32) {
            fence_proxy_async_smem();
            issue(next, buf ^ 1);
        }
        const int f = a.fidx[plane / N], k = plane % N;
        mbar_wait_bounded(&mbar[buf], (uint32_t)((it >> 1) & 1), a.err);
        const float2* Sb = S + buf * SLAB;
        float2* out_plane = ws + a.ws_off[f] + (size_t)k * 2 * N * N;
        const float scale = a.w32[k] / (2.f * (float)N * (float)N);

        for (int s = 0; s < 2; ++s) {
            // Pass 1A: column DFT over j1, stride-R1 part (sector 1 pre-twisted).
#pragma unroll
            for (int task = tid; task < W * R1; task += THREADS) {
                const int jc = task % W, ia = task / W;
                const int j2 = c * W + jc;
                float2 v[R2];
#pragma unroll
                for (int b = 0; b < R2; ++b) v[b] = Sb[(ia + R1 * b) * W + jc];
                if (s) {
#pragma unroll
                    for (int b = 0; b < R2; ++b) v[b] = cmul(v[b], tw2[ia + R1 * b + j2]);
                }
                dft_reg<R2, 1, float>(v);
#pragma unroll
                for (int qb = 0; qb < R2; ++qb)
                    Wb[(ia + R1 * qb) * LD1 + jc] = (qb == 0) ? v[0] : cmul(v[qb], om[ia * qb]);
            }
            __syncthreads();
            // Pass 1B: contiguous R1-point DFTs; bin p = qb + R2*qa in row qa + R1*qb.
#pragma unroll
            for (int task = tid; task < W * R2; task += THREADS) {
                const int jc = task % W, qb = task / W;
                float2 v[R1];
#pragma unroll
                for (int ia = 0; ia < R1; ++ia) v[ia] = Wb[(ia + R1 * qb) * LD1 + jc];
                dft_reg<R1, 1, float>(v);
#pragma unroll
                for (int qa = 0; qa < R1; ++qa) Wb[(qa + R1 * qb) * LD1 + jc] = v[qa];
            }
            cluster_arrive_release();
            cluster_wait_acquire();
            // Pass 2A: gather the owned rows p from every CTA of the cluster.
            constexpr int NT2 = (W * R1 + THREADS - 1) / THREADS;
            float2 hold[NT2][R2];
#pragma unroll
            for (int i2 = 0; i2 < NT2; ++i2) {
                const int task = tid + i2 * THREADS;
                if (task < W * R1) {
                    const int pl = task % W, ia = task / W;
                    const int p = c * W + pl;
                    const int rowp = p / R2 + R1 * (p % R2);
                    float2 v[R2];
#pragma unroll
                    for (int b = 0; b < R2; ++b) {
                        const int j2 = ia + R1 * b;
                        v[b] = ld_dsmem(map_shared(&Wb[rowp * LD1 + (j2 % W)], (unsigned)(j2 / W)), float2());
                    }
                    dft_reg<R2, 1, float>(v);
#pragma unroll
                    for (int qb = 0; qb < R2; ++qb) hold[i2][qb] = (qb == 0) ? v[0] : cmul(v[qb], om[ia * qb]);
                }
            }
            cluster_arrive_release();
            cluster_wait_acquire();
#pragma unroll
            for (int i2 = 0; i2 < NT2; ++i2) {
                const int task = tid + i2 * THREADS;
                if (task < W * R1) {
                    const int pl = task % W, ia = task / W;
#pragma unroll
                    for (int qb = 0; qb < R2; ++qb) Wb[pl * LD2 + ia + R1 * qb] = hold[i2][qb];
                }
            }
            __syncthreads();
            // Pass 2B: R1-point DFTs, scale, sign and store (n fastest).
            float2* out = out_plane + (size_t)s * N * N;
#pragma unroll
            for (int task = tid; task < W * R2; task += THREADS) {
                const int pl = task % W, qb = task / W;
                const int p = c * W + pl;
                float2 v[R1];
#pragma unroll
                for (int ia = 0; ia < R1; ++ia) v[ia] = Wb[pl * LD2 + ia + R1 * qb];
                dft_reg<R1, 1, float>(v);
                const int ni = (p + N / 2) & (N - 1);
                // parity of mi = (qb + R2*qa + N/2) mod N equals the parity of qb
                float sc = ((ni + qb) & 1) ? -scale : scale;
                if (s) sc = -sc;
                const bool zero_col = (s == 0 && ni == 0);
#pragma unroll
                for (int qa = 0; qa < R1; ++qa) {
                    const int qq = qb + R2 * qa;
                    const int mi = (qq + N / 2) & (N - 1);
                    float2 val = make_float2(v[qa].x * sc, v[qa].y * sc);
                    if (zero_col || (s == 0 && mi == 0)) val = make_float2(0.f, 0.f);
                    out[(size_t)mi * N + ni] = val;
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Forward, persistent version with a bulk-copy exchange (N = 64, 128, 256;
// complex64).  Work items are (function, beta node, sector); one cluster of
// C = N/16 CTAs takes items q, q + nq, ...  CTA c holds the 16 columns
// j2 in [16c, 16c+16) of the item's N x N plane:
//   S[2]  column slabs [j1][16], filled one item ahead by TMA (one 3-D tensor
//         copy when the group's grids are regularly strided, else one bulk
//         copy per row);
//   1A    column DFT over j1, stride-R1 part, in place;
//   1B    R1-point DFTs; bin p is written to row p (natural order), so the 16
//         rows owned by CTA c' = p/16 form one contiguous 2 KB block;
//   push  one 2 KB bulk copy (shared -> shared) per destination CTA into its
//         receive buffer R[source][16 rows][16 columns], completion counted
//         on the destination's mbarrier;
//   2A/2B row DFTs over j2 (2A result written back XOR-swizzled so that 2B
//         reads one column across 16 rows without bank conflicts); 2B stores
//         16 consecutive n per half-warp.
// One cluster barrier per item, split: arrive after 2B (my R is free and I
// have received the item, so every sender's slab is free), wait before the
// next push and the next slab refill.
// ---------------------------------------------------------------------------
template <int N>
struct XCfg {
    static constexpr int W = 16;
    static constexpr int C = N / W;
    static constexpr int R1 = Radix<N>::R1, R2 = Radix<N>::R2;
    static constexpr int THREADS = 256;
    static constexpr int SLAB = N * W;                      // float2 per slab
    static constexpr int F2S = 2 * SLAB + W * N + N + 2 * N + N / 2;
    static constexpr size_t smem_bytes() { return (size_t)F2S * sizeof(float2) + 3 * sizeof(uint64_t); }
};

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)) : "memory");
}

template <int N>
__global__ void __launch_bounds__(256, 2)
fft_fwd_xchg(BandArgs a, const __grid_constant__ CUtensorMap gmap, const float2* __restrict__ grid,
             float2* __restrict__ ws) {
    using P = XCfg<N>;
    constexpr int C = P::C, W = P::W, R1 = P::R1, R2 = P::R2, THREADS = P::THREADS, SLAB = P::SLAB;
    static_assert(C >= 2 && C <= 16, "cluster size");
    static_assert(W * R2 <= THREADS && W * R1 <= THREADS, "one task per thread");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);       // [2][N][W]
    float2* R = S + 2 * SLAB;                               // [C][W][W] received, then [W][N] swizzled
    float2* om = R + W * N;                                 // exp(+2 pi i t/N)
    float2* tw2 = om + N;                                   // exp(i pi t/N), t < 2N
    float* wk = reinterpret_cast<float*>(tw2 + 2 * N);      // beta weights
    uint64_t* mbS = reinterpret_cast<uint64_t*>(tw2 + 2 * N + N / 2);   // [2]
    uint64_t* mbR = mbS + 2;

    const int c = (int)cluster_ctarank();
    const int q = blockIdx.x / C, nq = gridDim.x / C;
    const int nitems = a.nfunc * N * 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int t = tid; t < N; t += THREADS) {
        om[t] = a.om32[t];
        wk[t] = a.w32[t];
    }
    for (int t = tid; t < 2 * N; t += THREADS) {
        const float2 z = a.twist32[t & (N - 1)];
        tw2[t] = (t < N) ? z : make_float2(-z.x, -z.y);
    }
    if (tid == 0) {
        mbar_init(&mbS[0], 1);
        mbar_init(&mbS[1], 1);
        mbar_init(mbR, 1);
        mbar_fence_init();
    }
    __syncthreads();
    // every CTA's barriers are initialised before any remote copy can target them
    cluster_arrive_release();
    cluster_wait_acquire();

    auto load_slab = [&](int item, int buf) {      // warp 0
        const int plane = item >> 1;
        const int fb = plane / N, k = plane % N;
        float2* dst = S + buf * SLAB;
        if (a.grid_regular) {
            if (lane == 0) {
                mbar_arrive_expect_tx(&mbS[buf], (uint32_t)(SLAB * sizeof(float2)));
                tma_load_3d(dst, &gmap, c * W, k, fb * N, &mbS[buf]);
            }
        } else {
            const int f = a.fidx[fb];
            const float2* src = grid + a.grid_off[f] + (size_t)k * N + c * W;
            if (lane == 0) mbar_arrive_expect_tx(&mbS[buf], (uint32_t)(SLAB * sizeof(float2)));
            __syncwarp();
            for (int j1 = lane; j1 < N; j1 += 32)
                bulk_g2s(dst + j1 * W, src + (size_t)j1 * N * N, (uint32_t)(W * sizeof(float2)), &mbS[buf]);
        }
    };

    if (q < nitems && warp == 0) load_slab(q, 0);
    int it = 0;
    for (int item = q; item < nitems; item += nq, ++it) {
        const int buf = it & 1;
        const int s = item & 1, plane = item >> 1;
        const int fb = plane / N, k = plane % N;
        float2* Sb = S + buf * SLAB;
        mbar_wait_bounded(&mbS[buf], (uint32_t)((it >> 1) & 1), a.err);

        // Pass 1A: column DFT over j1, stride-R1 part, in place (sector 1 pre-twisted).
        if (tid < W * R1) {
            const int jc = tid % W, ia = tid / W;
            const int j2 = c * W + jc;
            float2 v[R2];
#pragma unroll
            for (int b = 0; b < R2; ++b) v[b] = Sb[(ia + R1 * b) * W + jc];
            if (s) {
#pragma unroll
                for (int b = 0; b < R2; ++b) v[b] = cmul(v[b], tw2[ia + R1 * b + j2]);
            }
            dft_reg<R2, 1, float>(v);
#pragma unroll
            for (int qb = 0; qb < R2; ++qb)
                Sb[(ia + R1 * qb) * W + jc] = (qb == 0) ? v[0] : cmul(v[qb], om[ia * qb]);
        }
        __syncthreads();
        // Pass 1B: R1-point DFTs; bin p = qb + R2*qa goes to row p.
        {
            float2 v[R1];
            const int jc = tid % W, qb = tid / W;
            if (tid < W * R2) {
#pragma unroll
                for (int ia = 0; ia < R1; ++ia) v[ia] = Sb[(ia + R1 * qb) * W + jc];
                dft_reg<R1, 1, float>(v);
            }
            __syncthreads();
            if (tid < W * R2) {
#pragma unroll
                for (int qa = 0; qa < R1; ++qa) Sb[(qb + R2 * qa) * W + jc] = v[qa];
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (it > 0) cluster_wait_acquire();
        if (warp == 0) {
            const int next = item + nq;
            if (next < nitems) {
                fence_proxy_async_smem();
                load_slab(next, buf ^ 1);
            }
        } else if (warp == 1) {
            if (lane == 0) mbar_arrive_expect_tx(mbR, (uint32_t)(W * N * sizeof(float2)));
            __syncwarp();
            if (lane < C)   // rows [16*lane, 16*lane + 16) to CTA `lane`, block `c` of its R
                bulk_s2s_remote(R + c * W * W, Sb + lane * W * W, (uint32_t)(W * W * sizeof(float2)), mbR,
                                (unsigned)lane);
        }
        mbar_wait_bounded(mbR, (uint32_t)(it & 1), a.err);

        // Pass 2A: row DFT over j2, stride-R1 part; lanes run along the row.
        {
            float2 v[R2];
            const int ia = tid % R1, pl = tid / R1;
            if (tid < W * R1) {
#pragma unroll
                for (int b = 0; b < R2; ++b) {
                    const int j2 = ia + R1 * b;
                    v[b] = R[(j2 / W) * W * W + pl * W + (j2 % W)];
                }
                dft_reg<R2, 1, float>(v);
#pragma unroll
                for (int qb = 1; qb < R2; ++qb) v[qb] = cmul(v[qb], om[ia * qb]);
            }
            __syncthreads();
            if (tid < W * R1) {
#pragma unroll
                for (int qb = 0; qb < R2; ++qb) R[pl * N + ((ia + R1 * qb) ^ (pl & 15))] = v[qb];
            }
        }
        __syncthreads();
        // Pass 2B: R1-point DFTs, scale, sign, store F2 (16 consecutive n per half-warp).
        if (tid < W * R2) {
            const float scale = wk[k] / (2.f * (float)N * (float)N);
            const size_t plane_off = a.grid_regular ? a.ws_group_off + (size_t)fb * 2 * N * N * N
                                                    : a.ws_off[a.fidx[fb]];
            float2* out = ws + plane_off + ((size_t)k * 2 + s) * N * N;
            const int pl = tid % W, qb = tid / W;
            const int p = c * W + pl;
            float2 v[R1];
#pragma unroll
            for (int ia = 0; ia < R1; ++ia) v[ia] = R[pl * N + ((ia + R1 * qb) ^ (pl & 15))];
            dft_reg<R1, 1, float>(v);
            const int ni = (p + N / 2) & (N - 1);
            float sc = ((ni + qb) & 1) ? -scale : scale;     // parity of mi = parity of qb
            if (s) sc = -sc;
            const bool zero_col = (s == 0 && ni == 0);
#pragma unroll
            for (int qa = 0; qa < R1; ++qa) {
                const int qq = qb + R2 * qa;
                const int mi = (qq + N / 2) & (N - 1);
                float2 val = make_float2(v[qa].x * sc, v[qa].y * sc);
                if (zero_col || (s == 0 && mi == 0)) val = make_float2(0.f, 0.f);
                out[(size_t)mi * N + ni] = val;
            }
        }
        fence_proxy_async_smem();
        cluster_arrive_release();
    }
    if (it > 0) cluster_wait_acquire();
}

// ---------------------------------------------------------------------------
// Inverse, cluster version.  CTA c owns the n-bins p in [32c, 32c+32) for pass 1
// and the output columns j2 in [32c, 32c+32) for pass 2; both sectors are
// accumulated in registers before the single store.
// ---------------------------------------------------------------------------
template <typename T, int N, int C, int THREADS>
__global__ void __launch_bounds__(THREADS)
fft_inv_cluster(BandArgs a, const cplx<T>* __restrict__ ws, cplx<T>* __restrict__ grid) {
    using Cx = cplx<T>;
    using S = FftShape<T, N, C>;
    constexpr int W = S::W, R1 = S::R1, R2 = S::R2, LD1 = S::LD1, LD2 = S::LD2;
    static_assert(W == 32, "one warp of columns per CTA");
    static_assert((W * R1) % THREADS == 0 && (W * R2) % THREADS == 0, "task split");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx* buf = reinterpret_cast<Cx*>(smem_raw);
    Cx* om = buf + S::BUF;

    const int c = (C > 1) ? (int)cluster_ctarank() : 0;
    const int k = blockIdx.y;
    const int f = a.fidx[blockIdx.z];
    const int tid = threadIdx.x;

    for (int t = tid; t < N; t += THREADS) om[t] = cconj(om_at<T>(a, t));   // exp(-2 pi i t/N)
    __syncthreads();

    constexpr int NTB = (W * R2) / THREADS;
    Cx acc[NTB][R1];

    for (int s = 0; s < 2; ++s) {
        const Cx* G = plane_base(ws, a, f, k, s, N);   // [mi][ni]
        // Pass 1A: DFT over q (rows of G) for the owned columns p.
#pragma unroll
        for (int it = 0; it < (W * R1) / THREADS; ++it) {
            const int task = tid + it * THREADS;
            const int pl = task % W, ia = task / W;
            const int p = c * W + pl;
            const int ni = (p + N / 2) & (N - 1);
            Cx v[R2];
#pragma unroll
            for (int b = 0; b < R2; ++b) {
                const int q = ia + R1 * b;
                const int mi = (q + N / 2) & (N - 1);
                T sg = ((ni + mi) & 1) ? T(-1) : T(1);
                if (s) sg = -sg;
                v[b] = (s == 0 && (ni == 0 || mi == 0)) ? mk<T>(T(0), T(0))
                                                        : cscale(G[plane_index(a, mi, ni, N)], sg);
            }
            dft_reg<R2, -1, T>(v);
#pragma unroll
            for (int qb = 0; qb < R2; ++qb)
                buf[(ia + R1 * qb) * LD1 + pl] = (qb == 0) ? v[0] : cmul(v[qb], om[ia * qb]);
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < (W * R2) / THREADS; ++it) {
            const int task = tid + it * THREADS;
            const int pl = task % W, qb = task / W;
            Cx v[R1];
#pragma unroll
            for (int ia = 0; ia < R1; ++ia) v[ia] = buf[(ia + R1 * qb) * LD1 + pl];
            dft_reg<R1, -1, T>(v);
#pragma unroll
            for (int qa = 0; qa < R1; ++qa) buf[(qa + R1 * qb) * LD1 + pl] = v[qa];
        }
        if constexpr (C > 1) cluster_sync_all(); else __syncthreads();

        // Pass 2A: gather, for the owned output columns j2, all p from every CTA.
        constexpr int NT2 = (W * R1) / THREADS;
        Cx hold[NT2][R2];
#pragma unroll
        for (int it = 0; it < NT2; ++it) {
            const int task = tid + it * THREADS;
            const int jl = task % W, ia = task / W;
            const int j2 = c * W + jl;
            const int rowj = j2 / R2 + R1 * (j2 % R2);
            Cx v[R2];
#pragma unroll
            for (int b = 0; b < R2; ++b) {
                const int p = ia + R1 * b;
                const Cx* src = &buf[rowj * LD1 + (p % W)];
                if constexpr (C > 1) v[b] = ld_dsmem(map_shared(src, (unsigned)(p / W)), Cx());
                else v[b] = *src;
            }
            dft_reg<R2, -1, T>(v);
#pragma unroll
            for (int qb = 0; qb < R2; ++qb) hold[it][qb] = (qb == 0) ? v[0] : cmul(v[qb], om[ia * qb]);
        }
        if constexpr (C > 1) cluster_sync_all(); else __syncthreads();
#pragma unroll
        for (int it = 0; it < NT2; ++it) {
            const int task = tid + it * THREADS;
            const int jl = task % W, ia = task / W;
#pragma unroll
            for (int qb = 0; qb < R2; ++qb) buf[jl * LD2 + ia + R1 * qb] = hold[it][qb];
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < NTB; ++it) {
            const int task = tid + it * THREADS;
            const int jl = task % W, qb = task / W;
            const int j2 = c * W + jl;
            Cx v[R1];
#pragma unroll
            for (int ia = 0; ia < R1; ++ia) v[ia] = buf[jl * LD2 + ia + R1 * qb];
            dft_reg<R1, -1, T>(v);
#pragma unroll
            for (int qa = 0; qa < R1; ++qa) {
                Cx val = v[qa];
                if (s) {
                    const int j1 = qb + R2 * qa;
                    val = cmul(val, cconj(cmul(twist_at<T>(a, j1), twist_at<T>(a, j2))));
                    acc[it][qa] = cadd(acc[it][qa], val);
                } else {
                    acc[it][qa] = val;
                }
            }
        }
        __syncthreads();
    }
    Cx* Y = grid + a.grid_off[f] + (size_t)k * N;
#pragma unroll
    for (int it = 0; it < NTB; ++it) {
        const int task = tid + it * THREADS;
        const int jl = task % W, qb = task / W;
        const int j2 = c * W + jl;
#pragma unroll
        for (int qa = 0; qa < R1; ++qa) {
            const int j1 = qb + R2 * qa;
            Y[(size_t)j1 * N * N + j2] = acc[it][qa];
        }
    }
}

// ---------------------------------------------------------------------------
// Small bandwidths (N <= 16): one CTA per plane, direct DFT sums in shared memory.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
fft_fwd_small(BandArgs a, const cplx<T>* __restrict__ grid, cplx<T>* __restrict__ ws) {
    using Cx = cplx<T>;
    __shared__ Cx x[16 * 16], y[16 * 16], om[16];
    const int N = a.N;
    const int s = blockIdx.x, k = blockIdx.y, f = a.fidx[blockIdx.z];
    const int tid = threadIdx.x;
    if (tid < N) om[tid] = om_at<T>(a, tid);
    const Cx* X = grid + a.grid_off[f] + (size_t)k * N;
    for (int e = tid; e < N * N; e += blockDim.x) {
        const int j1 = e / N, j2 = e % N;
        Cx v = X[(size_t)j1 * N * N + j2];
        if (s) v = cmul(v, cmul(twist_at<T>(a, j1), twist_at<T>(a, j2)));
        x[e] = v;
    }
    __syncthreads();
    for (int e = tid; e < N * N; e += blockDim.x) {        // y[j1][q] = sum_j2 x omega^{q j2}
        const int j1 = e / N, q = e % N;
        Cx acc = mk<T>(T(0), T(0));
        for (int j2 = 0; j2 < N; ++j2) acc = cadd(acc, cmul(x[j1 * N + j2], om[(q * j2) % N]));
        y[e] = acc;
    }
    __syncthreads();
    const T scale = weight_at<T>(a, k) / (T(2) * T(N) * T(N));
    Cx* out = ws + a.ws_off[f] + ((size_t)k * 2 + s) * N * N;
    for (int e = tid; e < N * N; e += blockDim.x) {        // z[p][q] = sum_j1 y omega^{p j1}
        const int q = e / N, p = e % N;
        Cx acc = mk<T>(T(0), T(0));
        for (int j1 = 0; j1 < N; ++j1) acc = cadd(acc, cmul(y[j1 * N + q], om[(p * j1) % N]));
        const int ni = (p + N / 2) % N, mi = (q + N / 2) % N;
        T sg = ((ni + mi) & 1) ? T(-1) : T(1);
        if (s) sg = -sg;
        Cx val = cscale(acc, sg * scale);
        if (s == 0 && (ni == 0 || mi == 0)) val = mk<T>(T(0), T(0));
        out[(size_t)mi * N + ni] = val;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
fft_inv_small(BandArgs a, const cplx<T>* __restrict__ ws, cplx<T>* __restrict__ grid) {
    using Cx = cplx<T>;
    __shared__ Cx x[16 * 16], y[16 * 16], om[16];
    const int N = a.N;
    const int k = blockIdx.y, f = a.fidx[blockIdx.z];
    const int tid = threadIdx.x;
    if (tid < N) om[tid] = cconj(om_at<T>(a, tid));
    Cx acc2[1];
    const int nE = N * N;
    // each thread owns output elements e = tid (N*N <= 256)
    acc2[0] = mk<T>(T(0), T(0));
    for (int s = 0; s < 2; ++s) {
        const Cx* G = plane_base(ws, a, f, k, s, N);
        __syncthreads();
        for (int e = tid; e < nE; e += blockDim.x) {      // x[q][p] = signed G
            const int q = e / N, p = e % N;
            const int ni = (p + N / 2) % N, mi = (q + N / 2) % N;
            T sg = ((ni + mi) & 1) ? T(-1) : T(1);
            if (s) sg = -sg;
            x[e] = (s == 0 && (ni == 0 || mi == 0)) ? mk<T>(T(0), T(0))
                                                    : cscale(G[plane_index(a, mi, ni, N)], sg);
        }
        __syncthreads();
        for (int e = tid; e < nE; e += blockDim.x) {      // y[j2][p] = sum_q x[q][p] om^{q j2}
            const int j2 = e / N, p = e % N;
            Cx acc = mk<T>(T(0), T(0));
            for (int q = 0; q < N; ++q) acc = cadd(acc, cmul(x[q * N + p], om[(q * j2) % N]));
            y[e] = acc;
        }
        __syncthreads();
        if (tid < nE) {
            const int j1 = tid / N, j2 = tid % N;
            Cx acc = mk<T>(T(0), T(0));
            for (int p = 0; p < N; ++p) acc = cadd(acc, cmul(y[j2 * N + p], om[(p * j1) % N]));
            if (s) acc = cmul(acc, cconj(cmul(twist_at<T>(a, j1), twist_at<T>(a, j2))));
            acc2[0] = cadd(acc2[0], acc);
        }
    }
    if (tid < nE) {
        const int j1 = tid / N, j2 = tid % N;
        grid[a.grid_off[f] + ((size_t)j1 * N + k) * N + j2] = acc2[0];
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T, int N, int C, int THREADS, bool FWD>
static cudaError_t launch_cluster(const BandArgs& a, const void* in, void* out, cudaStream_t st) {
    using S = FftShape<T, N, C>;
    auto kern = FWD ? (void (*)(BandArgs, const cplx<T>*, cplx<T>*))fft_fwd_cluster<T, N, C, THREADS>
                    : (void (*)(BandArgs, const cplx<T>*, cplx<T>*))fft_inv_cluster<T, N, C, THREADS>;
    const size_t smem = S::smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(FWD ? 2 * C : C, N, a.nfunc);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, (const cplx<T>*)in, (cplx<T>*)out);
}

template <int N>
static cudaError_t launch_pipe(const BandArgs& a, const void* in, void* out, cudaStream_t st) {
    using P = PipeCfg<N>;
    auto kern = fft_fwd_pipe<N>;
    const size_t smem = P::smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    static int max_clusters = 0;      // per N, per process (the device's cluster capacity)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(P::THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (max_clusters == 0) {
        cfg.gridDim = dim3(P::C * 1024, 1, 1);
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
        if (e != cudaSuccess) return e;
        max_clusters = n > 0 ? n : 1;
    }
    const int nplanes = a.nfunc * N;
    const int ncl = nplanes < max_clusters ? nplanes : max_clusters;
    cfg.gridDim = dim3(P::C * ncl, 1, 1);
    return cudaLaunchKernelEx(&cfg, kern, a, (const float2*)in, (float2*)out);
}

template <int N>
static cudaError_t launch_xchg(const BandArgs& a, const void* in, void* out, cudaStream_t st) {
    using P = XCfg<N>;
    auto kern = fft_fwd_xchg<N>;
    const size_t smem = P::smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (P::C > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    static int max_clusters = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(P::THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (max_clusters == 0) {
        cfg.gridDim = dim3(P::C * 512, 1, 1);
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
        if (e != cudaSuccess) return e;
        max_clusters = n > 0 ? n : 1;
    }
    const int nitems = a.nfunc * N * 2;
    const int ncl = nitems < max_clusters ? nitems : max_clusters;
    cfg.gridDim = dim3(P::C * ncl, 1, 1);
    CUtensorMap gmap;
    memset(&gmap, 0, sizeof(gmap));
    BandArgs b = a;
    if (b.grid_regular) {
        // rows (function, j1) x beta nodes k x gamma nodes j2 of the group's grids
        const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)a.nfunc * N};
        const cuuint64_t strides[2] = {(cuuint64_t)N * 8, (cuuint64_t)N * N * 8};
        const cuuint32_t box[3] = {(cuuint32_t)P::W, 1, (cuuint32_t)N};
        const void* base = (const float2*)in + a.grid_group_off;
        if (!encode_tensor_map_8b(&gmap, 3, base, dims, strides, box)) b.grid_regular = 0;
    }
    return cudaLaunchKernelEx(&cfg, kern, b, gmap, (const float2*)in, (float2*)out);
}

template <typename T, bool FWD>
static cudaError_t launch_any(const BandArgs& a, const void* in, void* out, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    switch (a.N) {
        case 4: case 8: case 16: {
            dim3 g(FWD ? 2 : 1, a.N, a.nfunc);
            if (FWD) fft_fwd_small<T><<<g, 256, 0, st>>>(a, (const cplx<T>*)in, (cplx<T>*)out);
            else fft_inv_small<T><<<g, 256, 0, st>>>(a, (const cplx<T>*)in, (cplx<T>*)out);
            return cudaGetLastError();
        }
        case 32: return launch_cluster<T, 32, 1, 128, FWD>(a, in, out, st);
        case 64:
            if constexpr (FWD && sizeof(T) == 4) return launch_xchg<64>(a, in, out, st);
            else return launch_cluster<T, 64, 2, 256, FWD>(a, in, out, st);
        case 128:
            if constexpr (FWD && sizeof(T) == 4) return launch_xchg<128>(a, in, out, st);
            else return launch_cluster<T, 128, 4, 256, FWD>(a, in, out, st);
        case 256:
            if constexpr (FWD && sizeof(T) == 4) return launch_xchg<256>(a, in, out, st);
            else return launch_cluster<T, 256, 8, 256, FWD>(a, in, out, st);
        case 512:
            if constexpr (sizeof(T) == 4) return launch_cluster<T, 512, 16, 512, FWD>(a, in, out, st);
            else return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fft_forward(const BandArgs& a, bool fp64, const void* grid, void* ws, cudaStream_t st) {
    if (a.literal) return fp64 ? cudaErrorInvalidValue : launch_fft_forward_literal(a, grid, ws, st);
    if (a.aux_ring > 0 && a.s1_two_phase && fft_forward_two_phase_supported(a.N, fp64))
        return launch_fft_forward_two_phase(a, grid, ws, st);
    return fp64 ? launch_any<double, true>(a, grid, ws, st) : launch_any<float, true>(a, grid, ws, st);
}

cudaError_t launch_fft_inverse(const BandArgs& a, bool fp64, const void* ws, void* grid, cudaStream_t st) {
    if (a.literal) return fp64 ? cudaErrorInvalidValue : launch_fft_inverse_literal(a, ws, grid, st);
    if (a.full_group)                   // two-phase only (N = 128, 256; the caller checks)
        return (a.aux_ring > 0 && !fp64) ? launch_fft_inverse_two_phase(a, ws, grid, st) : cudaErrorInvalidValue;
    if (a.aux_ring > 0 && a.ws_tile_major && fft_inverse_two_phase_supported(a.N, fp64))
        return launch_fft_inverse_two_phase(a, ws, grid, st);
    return fp64 ? launch_any<double, false>(a, ws, grid, st) : launch_any<float, false>(a, ws, grid, st);
}

}  // namespace su2

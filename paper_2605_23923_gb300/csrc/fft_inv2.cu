// Inverse of stage 1 for complex64 at N = 128, 256, 512 (synthesis, Sec. 3
// expansion, and the adjoint of the Sec. 4 quadrature): from the tile-major
// planes G_s[k][mi][ni] (element (k, s, mi, ni) at s N^3 + mi N^2 + (ni/4) 4N +
// 4k + ni%4 of the function's planes) to the grid
//
//   f[j1,k,j2] = sum_s e^{-i pi (j1+j2) s/N} sum_{p,q} sg_s(p,q) G_s[mi(q)][ni(p)] w^{-(p j1 + q j2)}
//
// with w = e^{2 pi i/N}, sg_s = (-1)^{ni+mi} (negated for s = 1), the integer
// sector's index-0 row and column left out, as two phases meeting in L2:
//
//   A item (plane, sector s, 16 rows mi): rows read straight from the planes
//       (four consecutive n share a 32-byte sector) -> inverse DFT over p for
//       each row -> untwist e^{-i pi j1 s/N} -> intermediate rows H_s[mi][j1].
//   B item (plane, 16 columns j1): both sectors' columns from L2 -> inverse DFT
//       over q -> untwist e^{-i pi j2 s/N} -> sector sum -> 16 grid rows of N
//       contiguous nodes j2.
//
// Full-group grid (template FULL, psi over [-2 pi, 2 pi) with 2N nodes,
// psi_j = gamma_{(j - N/2) mod N} - 2 pi [j < N/2] + 2 pi [j >= 3N/2]): a
// half-integer m changes sign over 2 pi, so the grid row is f_int + f_half at
// j in [N/2, 3N/2) and f_int - f_half at the other N nodes, from the same two
// sector sums.
//
// The intermediate ring, its counters and the in-order item queue are the
// forward two-phase DFT's scratch (the same workspace region; a plan's calls on
// one workspace are serialised).  Items: block t holds the A items of plane t
// then the B items of plane t - D; the CTAs take item numbers in order; a B
// item waits for all A items of its plane, an A item reusing a ring slot for
// the B items of the plane before it.  Every wait is bounded and for a smaller
// item number already held by a running CTA.  No TMA: loads go straight to
// registers; between the two DFT passes each row (column) is transposed
// through shared memory laid out [R1][R2 + 1] (odd pitch, no bank conflicts),
// one buffer per sector in B items.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "su2_internal.h"

namespace su2 {
namespace inv2 {

template <int N>
struct Cfg {
    static constexpr int R1 = Radix<N>::R1, R2 = Radix<N>::R2;
    static constexpr int W = 16;                        // rows per A item, columns per B item
    static constexpr int NH = N / W;
    static constexpr int NA = 2 * NH, NB = NH, IB = NA + NB;
    static constexpr int THREADS = W * (R1 > R2 ? R1 : R2);
    // padded transpose buffer of one row (R2 + 1 per R1 block), plus one so that
    // the B items' columns (one per lane) start in different banks
    static constexpr int RP = R1 * (R2 + 1) + 1;
    static constexpr size_t smem_bytes() { return (size_t)2 * W * RP * 8 + (size_t)2 * N * 8 + 16; }
    static constexpr int BLOCKS_PER_SM = (N <= 256) ? 2 : 1;
};

__device__ __forceinline__ void discard_line(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

template <int N, bool FULL = false>
__global__ void __launch_bounds__(Cfg<N>::THREADS, Cfg<N>::BLOCKS_PER_SM)
fft_inv_two_phase(BandArgs a, const float2* __restrict__ ws, float2* __restrict__ grid, int D, int RING,
                  int discard_ok) {
    using P = Cfg<N>;
    constexpr int R1 = P::R1, R2 = P::R2, W = P::W, RP = P::RP, T = P::THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* X = reinterpret_cast<float2*>(smem_raw);    // [2][W][RP] transpose buffers
    float2* om = X + 2 * W * RP;                        // e^{-2 pi i t/N}
    float2* ut = om + N;                                // e^{-i pi t/N}
    int* s_item = reinterpret_cast<int*>(ut + N);

    const int tid = threadIdx.x;
    const int nplanes = a.nfunc * N;
    const int nitems = (nplanes + D) * P::IB;
    float2* ring = const_cast<float2*>(ws) + a.ws_aux_off;       // [RING][2][N][N]
    unsigned* doneA = reinterpret_cast<unsigned*>(ring + (size_t)RING * 2 * N * N);
    unsigned* doneB = doneA + RING;
    unsigned* queue = doneB + RING;

    for (int t = tid; t < N; t += T) {
        om[t] = cconj(a.om32[t]);
        ut[t] = cconj(a.twist32[t]);
    }
    __syncthreads();

    for (;;) {
        if (tid == 0) {
            int i, t, j;
            bool ok;
            do {
                i = (int)atomicAdd(queue, 1u);
                t = i / P::IB;
                j = i % P::IB;
                ok = (j < P::NA) ? (t < nplanes) : (t - D >= 0 && t - D < nplanes);
            } while (i < nitems && !ok);
            if (i < nitems) {
                const int plane = (j < P::NA) ? t : t - D;
                const int r = plane % RING;
                const unsigned use = (unsigned)(plane / RING);
                if (j < P::NA) {
                    if (use > 0) wait_counter_bounded(&doneB[r], use * P::NB, a.err);
                } else {
                    wait_counter_bounded(&doneA[r], (use + 1) * P::NA, a.err);
                }
            }
            *s_item = i;
        }
        __syncthreads();
        const int i = *s_item;
        if (i >= nitems) break;
        const int t = i / P::IB, j = i % P::IB;
        const bool isA = j < P::NA;
        const int plane = isA ? t : t - D;
        const int r = plane % RING;
        const int fb = plane / N, k = plane % N;
        const int f = a.fidx[fb];

        if (isA) {
            // ------------------------------------------------- A: rows mi -> H_s[mi][j1]
            const int s = j / P::NH, mb = j % P::NH;
            const float2* Gs = ws + a.ws_off[f] + (size_t)s * N * N * N + (size_t)4 * k;
            {
                // pass a: R2-point inverse DFTs over p = ia + R1*q of row pl
                const int ia = tid % R1, pl = tid / R1;           // W * R1 == T
                const int mi = mb * W + pl;
                float2 v[R2];
#pragma unroll
                for (int q = 0; q < R2; ++q) {
                    const int p = ia + R1 * q;
                    const int ni = (p + N / 2) & (N - 1);
                    const float2 g = Gs[(size_t)mi * N * N + (size_t)(ni >> 2) * 4 * N + (ni & 3)];
                    float sg = ((ni + mi) & 1) ? -1.f : 1.f;
                    if (s) sg = -sg;
                    // the integer sector's row and column 0 (Nyquist) are not part of the
                    // transform; nothing writes them, so they are selected away, not scaled
                    // by zero (whatever bits the workspace holds there, NaN included)
                    v[q] = (s == 0 && (ni == 0 || mi == 0)) ? make_float2(0.f, 0.f) : make_float2(g.x * sg, g.y * sg);
                }
                dft_reg<R2, -1, float>(v);
#pragma unroll
                for (int q = 1; q < R2; ++q) v[q] = cmul(v[q], om[ia * q]);
#pragma unroll
                for (int q = 0; q < R2; ++q) X[pl * RP + ia * (R2 + 1) + q] = v[q];
            }
            __syncthreads();
            if (tid < W * R2) {
                // pass b: R1-point inverse DFTs; j1 = qb + R2*qa; lanes along qb
                const int qb = tid % R2, pl = tid / R2;
                float2 v[R1];
#pragma unroll
                for (int ia = 0; ia < R1; ++ia) v[ia] = X[pl * RP + ia * (R2 + 1) + qb];
                dft_reg<R1, -1, float>(v);
                float2* H = ring + ((size_t)(r * 2 + s) * N + mb * W + pl) * N + qb;
#pragma unroll
                for (int qa = 0; qa < R1; ++qa) {
                    float2 w = v[qa];
                    if (s) w = cmul(w, ut[qb + R2 * qa]);
                    H[R2 * qa] = w;
                }
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicAdd(&doneA[r], 1u);
        } else {
            // ------------------------------------------------- B: columns j1 -> grid rows
            const int jb = j - P::NA;
            for (int s = 0; s < 2; ++s) {
                // pass a: R2-point inverse DFTs over q = ia + R1*b of column c (sector s)
                const float2* Hs = ring + (size_t)(r * 2 + s) * N * N + jb * W;
                float2* Xs = X + s * W * RP;
                const int c = tid % W, ia = tid / W;          // lanes along the 16 columns
                float2 v[R2];
#pragma unroll
                for (int b = 0; b < R2; ++b) {
                    const int q = ia + R1 * b;
                    const int mi = (q + N / 2) & (N - 1);
                    v[b] = __ldcs(Hs + (size_t)mi * N + c);
                }
                dft_reg<R2, -1, float>(v);
#pragma unroll
                for (int b = 1; b < R2; ++b) v[b] = cmul(v[b], om[ia * b]);
#pragma unroll
                for (int b = 0; b < R2; ++b) Xs[c * RP + ia * (R2 + 1) + b] = v[b];
            }
            __syncthreads();
            // both sectors' columns have been consumed: drop them from L2, release the slot
            if (discard_ok) {
                for (int l = tid; l < 2 * N; l += T) {
                    const int s = l / N, row = l % N;
                    discard_line(ring + ((size_t)(r * 2 + s) * N + row) * N + jb * W);
                }
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicAdd(&doneB[r], 1u);
            if (tid < W * R2) {
                // pass b: R1-point inverse DFTs; j2 = qb + R2*qa; sector 0's result goes
                // back to this thread's own slots, sector 1 adds it on the way out
                const int qb = tid % R2, cb = tid / R2;
                float2 v[R1];
                float2* X0 = X + cb * RP + qb;
                float2* X1 = X + W * RP + cb * RP + qb;
#pragma unroll
                for (int ia = 0; ia < R1; ++ia) v[ia] = X0[ia * (R2 + 1)];
                dft_reg<R1, -1, float>(v);
#pragma unroll
                for (int qa = 0; qa < R1; ++qa) X0[qa * (R2 + 1)] = v[qa];
#pragma unroll
                for (int ia = 0; ia < R1; ++ia) v[ia] = X1[ia * (R2 + 1)];
                dft_reg<R1, -1, float>(v);
                const int j1 = jb * W + cb;
                if constexpr (FULL) {
                    float2* out = grid + a.grid_off[f] + (size_t)j1 * N * 2 * N + (size_t)k * 2 * N;
#pragma unroll
                    for (int qa = 0; qa < R1; ++qa) {
                        const int j2 = qb + R2 * qa;
                        const float2 w = cmul(v[qa], ut[j2]);
                        const float2 z = X0[qa * (R2 + 1)];
                        __stcs(out + j2 + N / 2, make_float2(z.x + w.x, z.y + w.y));
                        __stcs(out + ((j2 + 3 * N / 2) & (2 * N - 1)), make_float2(z.x - w.x, z.y - w.y));
                    }
                } else {
                    float2* out = grid + a.grid_off[f] + (size_t)j1 * N * N + (size_t)k * N + qb;
#pragma unroll
                    for (int qa = 0; qa < R1; ++qa) {
                        const float2 w = cmul(v[qa], ut[qb + R2 * qa]);
                        const float2 z = X0[qa * (R2 + 1)];
                        __stcs(out + R2 * qa, make_float2(w.x + z.x, w.y + z.y));
                    }
                }
            }
        }
    }
}

template <int N, bool FULL>
static cudaError_t geometry(int device, int* G, int* D) {
    using P = Cfg<N>;
    int sms = 0, per = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    auto kern = fft_inv_two_phase<N, FULL>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::smem_bytes());
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, P::THREADS, P::smem_bytes());
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    *G = sms * per;
    const int inflight = (2 * *G + P::IB - 1) / P::IB;
    *D = 2 * inflight + 2;
    return cudaSuccess;
}

template <int N, bool FULL = false>
static cudaError_t launch_n(const BandArgs& a, const void* ws, void* grid, cudaStream_t st) {
    using P = Cfg<N>;
    int dev = 0, G = 0, D = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = geometry<N, FULL>(dev, &G, &D)) != cudaSuccess) return e;
    // the forward's ring and counters (same scratch); any lag D < RING keeps the
    // slot-reuse waits pointing at smaller item numbers
    const int RING = a.aux_ring;
    if (D > RING - 2) D = RING - 2;
    if (D < 1) return cudaErrorInvalidValue;
    float2* ring = (float2*)ws + a.ws_aux_off;
    unsigned* ctr = reinterpret_cast<unsigned*>(ring + (size_t)RING * 2 * N * N);
    if ((e = cudaMemsetAsync(ctr, 0, sizeof(unsigned) * (2 * RING + 1), st)) != cudaSuccess) return e;
    const int nitems = (a.nfunc * N + D) * P::IB;
    const int g = G < nitems ? G : nitems;
    const int discard_ok = ((uintptr_t)ring % 128) == 0;
    fft_inv_two_phase<N, FULL><<<g, P::THREADS, P::smem_bytes(), st>>>(a, (const float2*)ws, (float2*)grid, D,
                                                                     RING, discard_ok);
    return cudaGetLastError();
}

}  // namespace inv2

bool fft_inverse_two_phase_supported(int N, bool fp64) { return !fp64 && (N == 128 || N == 256 || N == 512); }

cudaError_t launch_fft_inverse_two_phase(const BandArgs& a, const void* ws, void* grid, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    if (a.full_group) {
        switch (a.N) {
            case 128: return inv2::launch_n<128, true>(a, ws, grid, st);
            case 256: return inv2::launch_n<256, true>(a, ws, grid, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (a.N) {
        case 128: return inv2::launch_n<128>(a, ws, grid, st);
        case 256: return inv2::launch_n<256>(a, ws, grid, st);
        case 512: return inv2::launch_n<512>(a, ws, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace su2

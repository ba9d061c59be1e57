// Ragged batches in one persistent launch: the whole forward transform (stage 1
// and stage 2, Sec. 6 first- and second-stage Propositions) of every function of
// a complex64 plan whose bandwidths all lie in {8, 16, 32, 64, 128}, in a single
// kernel.
//
// Work list, built on the host once per plan, in this order:
//   S1 items   P consecutive beta planes of one function: the 2-D DFT over
//              (alpha, gamma) of those planes, both sectors, scaled by
//              w_k/(2N^2) (-1)^{n+m} and written in the layout the band's
//              contraction reads (tile-major for tensor-core bands);
//   F32 items  one tile of the FP32 fused recurrence + contraction (4
//              consecutive n at fixed (sector, m), a block of functions);
//   TC items   one tile of the split-BF16 tensor-core contraction (4
//              consecutive n at fixed (sector, m), 64 functions).
// One CTA per SM (512 threads) takes item numbers in order from a counter.  An
// S1 item adds 1 to the completion counter of its function block once its
// stores are visible; a contraction item first waits (bounded) until its
// block's counter reaches the number of S1 items of that block.  Every S1 item
// comes before every contraction item in the list and S1 items wait for
// nothing, so each wait is on items already handed to running CTAs: it ends
// whichever CTAs are resident.
//
// Phase A: a CTA runs S1 and F32 items with all its threads.  The first TC item
// it takes (TC items follow every other item) switches it to phase B, the
// warp-specialised pipeline of the tensor-core contraction (TMA, MMA issue,
// converters, generators, epilogue: the roles of the per-group tensor-core
// kernel), fed through a ring of item numbers in shared memory that the TMA
// warp fills from the same counter.
//
// Stage 1 per plane (N <= 128 fits in shared memory): the rows, then the
// columns, each by a four-step split N = R1 x R2 with the two register DFTs
// of a line in place (the second step writes its outputs over the block it
// read, so the index order of the result is digit-reversed and undone on the
// way out).  The half-integer sector's pre-twist e^{i pi (j1 + j2)/N} is applied
// as the samples are loaded; its grid is read a second time (from L2).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "contract_fwd.cuh"
#include "recurrence.cuh"
#include "su2_internal.h"
#include "tc_common.cuh"

namespace su2 {
namespace rg {

using namespace tc;

constexpr int IT_S1 = 0, IT_F32 = 1, IT_TC = 2;
constexpr int DR = 4;                       // item-number ring of phase B
constexpr int NMAXR = 128;                  // largest bandwidth
constexpr int RMAXR = NMAXR / 2;            // rows of l per pair
constexpr int TABN = 64 + 128;              // node-table entries of the tensor-core bands
constexpr int LF2N = 2 * NMAXR + 2;
constexpr int OFF_B_ = NSA * SA;
constexpr int OFF_COEF_ = OFF_B_ + 2 * B_BYTES;
constexpr int OFF_TAB_ = OFF_COEF_ + 2 * NP * RMAXR * (int)sizeof(StepCoef<float>);
constexpr int OFF_SEED = OFF_TAB_;
constexpr int OFF_XS = OFF_SEED + TABN * 16;
constexpr int OFF_LF2 = OFF_XS + TABN * 8;
constexpr int OFF_ROW = OFF_LF2 + LF2N * 8;
constexpr int OFF_GP = OFF_ROW + NMAXR * 4;
constexpr int OFF_BAR_ = (OFF_GP + 2 * NP * (int)sizeof(SeedPair) + 7) / 8 * 8;
constexpr int NBAR_ = 3 * NSA + 2 * 4 + 2 * DR;
constexpr int SMEM = OFF_BAR_ + NBAR_ * 8 + DR * 4 + 16;
static_assert(SMEM <= 232448, "shared memory budget");
constexpr int PHASE_A_BYTES = OFF_TAB_;     // phase A uses [0, OFF_TAB_)
constexpr uint32_t TMEM_COLS_ = 512;        // two halves of 4 pairs x 64 columns

// Stage-1 split and planes per item: P planes of N rows at pitch N + 1.
template <int N> struct S1Cfg;
template <> struct S1Cfg<8>   { static constexpr int R1 = 4,  R2 = 2, P = 8; };
template <> struct S1Cfg<16>  { static constexpr int R1 = 4,  R2 = 4, P = 16; };
template <> struct S1Cfg<32>  { static constexpr int R1 = 8,  R2 = 4, P = 16; };
template <> struct S1Cfg<64>  { static constexpr int R1 = 8,  R2 = 8, P = 4; };
template <> struct S1Cfg<128> { static constexpr int R1 = 16, R2 = 8, P = 1; };

// FP32 contraction tile shapes: 4 pairs x LW rows x BT functions on 512 threads.
template <int N> struct F32Cfg;
template <> struct F32Cfg<8>   { static constexpr int BT = 64, KC = 8,  LW = 4,  ML = 1, MB = 2; };
template <> struct F32Cfg<16>  { static constexpr int BT = 32, KC = 16, LW = 8,  ML = 1, MB = 2; };
template <> struct F32Cfg<32>  { static constexpr int BT = 32, KC = 32, LW = 16, ML = 2, MB = 2; };
template <> struct F32Cfg<64>  { static constexpr int BT = 64, KC = 32, LW = 32, ML = 4, MB = 4; };
template <> struct F32Cfg<128> { static constexpr int BT = 32, KC = 32, LW = 64, ML = 4, MB = 4; };

template <int N> struct Checks {
    using S = S1Cfg<N>;
    using F = F32Cfg<N>;
    using FC = FwdCfg<float, 4, F::BT, F::KC, F::LW, F::ML, F::MB>;
    static_assert(S::R1 * S::R2 == N && N % S::P == 0 && S::R1 >= 4, "stage-1 split");
    static_assert((size_t)S::P * N * (N + 1) * 8 <= (size_t)PHASE_A_BYTES, "stage-1 planes fit");
    static_assert(FC::THREADS == THREADS && F::LW >= N / 2, "FP32 tile on 512 threads, one row window");
    static constexpr bool ok = true;
};
static_assert(Checks<8>::ok && Checks<16>::ok && Checks<32>::ok && Checks<64>::ok && Checks<128>::ok, "");

struct Args {
    const RaggedBand* bands;
    const int4* items;           // (kind | band << 4, a, b, c): see ragged_items
    int nitems;
    unsigned* ctr;               // [0] next item, [1 + i] S1 items done of block i
    const float2* grid;
    float2* ws;
    float2* coeffs;
    int* err;
    const double* lf2;
    int lf2_len;
    int nbands;
};
struct Maps { CUtensorMap m[2]; };  // planes of the tensor-core bands

// Bounded mbarrier wait that also gives up at once when the launch has latched
// an error (a broken hand-off then costs one timeout, not one per wait).
__device__ __forceinline__ void wait_bar(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return;
    const long long t0 = clock64();
    unsigned spins = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++spins & 255u) == 0 && *(volatile int*)err != 0) return;
        if (clock64() - t0 > 2000000000LL) {
            atomicExch(err, 1);
            return;
        }
    }
}

// The samples of an S1 item into L2 (N rows of P N contiguous complex values),
// one bulk prefetch per row, so that the CTA that takes the item finds them there.
template <int N>
__device__ __forceinline__ void s1_prefetch(const BandArgs& a, const float2* grid, int fi, int k0) {
    constexpr int P = S1Cfg<N>::P;
    const int j1 = threadIdx.x;
    if (j1 >= N) return;
    const float2* src = grid + a.grid_off[a.fidx[fi]] + ((size_t)j1 * N + k0) * N;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"((uint32_t)(P * N * 8)) : "memory");
}

// ---------------------------------------------------------------------------
// Stage 1: planes k0 .. k0 + P - 1 of function fi of the band.
// ---------------------------------------------------------------------------
template <int N>
__device__ __noinline__ void s1_item(const BandArgs& a, const float2* __restrict__ grid, float2* __restrict__ ws,
                                     int fi, int k0, float2* sm) {
    using C = S1Cfg<N>;
    constexpr int R1 = C::R1, R2 = C::R2, P = C::P, PITCH = N + 1, PL = N * PITCH;
    const int tid = threadIdx.x;
    const int f = a.fidx[fi];
    const float2* X = grid + a.grid_off[f];            // sample (j1, k, j2) at (j1 N + k) N + j2
    float2* out = ws + a.ws_off[f];
    const bool tm = a.ws_tile_major != 0;
    const float inv = 1.f / (2.f * (float)N * (float)N);
    for (int s = 0; s < 2; ++s) {
        // rows, step 1: R1-point DFTs over j2 = jb + R2 ja, twiddle w^{pa jb}
        for (int t = tid; t < P * N * R2; t += THREADS) {
            const int jb = t % R2, j1 = (t / R2) % N, pl = t / (R2 * N);
            const float2* src = X + ((size_t)j1 * N + k0 + pl) * N + jb;
            float2 v[R1];
#pragma unroll
            for (int ja = 0; ja < R1; ++ja) v[ja] = __ldg(src + R2 * ja);
            if (s) {
                const float2 t1 = __ldg(a.twist32 + j1);
#pragma unroll
                for (int ja = 0; ja < R1; ++ja) v[ja] = cmul(v[ja], cmul(t1, __ldg(a.twist32 + jb + R2 * ja)));
            }
            dft_reg<R1, 1, float>(v);
            float2* dst = sm + pl * PL + j1 * PITCH + jb;
#pragma unroll
            for (int pa = 0; pa < R1; ++pa) dst[R2 * pa] = (pa == 0 || jb == 0) ? v[pa] : cmul(v[pa], __ldg(a.om32 + pa * jb));
        }
        __syncthreads();
        // rows, step 2: R2-point DFTs over jb; position R2 pa + pb <- q = pa + R1 pb
        for (int t = tid; t < P * N * R1; t += THREADS) {
            const int j1 = t % N, pa = (t / N) % R1, pl = t / (N * R1);
            float2* row = sm + pl * PL + j1 * PITCH + R2 * pa;
            float2 v[R2];
#pragma unroll
            for (int jb = 0; jb < R2; ++jb) v[jb] = row[jb];
            dft_reg<R2, 1, float>(v);
#pragma unroll
            for (int pb = 0; pb < R2; ++pb) row[pb] = v[pb];
        }
        __syncthreads();
        // columns, step 1: R1-point DFTs over j1 = jb + R2 ja
        for (int t = tid; t < P * N * R2; t += THREADS) {
            const int qp = t % N, jb = (t / N) % R2, pl = t / (N * R2);
            float2* col = sm + pl * PL + qp;
            float2 v[R1];
#pragma unroll
            for (int ja = 0; ja < R1; ++ja) v[ja] = col[(jb + R2 * ja) * PITCH];
            dft_reg<R1, 1, float>(v);
#pragma unroll
            for (int pa = 0; pa < R1; ++pa)
                col[(jb + R2 * pa) * PITCH] = (pa == 0 || jb == 0) ? v[pa] : cmul(v[pa], __ldg(a.om32 + pa * jb));
        }
        __syncthreads();
        // columns, step 2, and the store: lanes take 4 consecutive pa (4 consecutive n,
        // one 32-byte piece of either layout) for 8 columns
        for (int t = tid; t < P * N * R1; t += THREADS) {
            const int pal = t & 3, qp = (t >> 2) % N, rest = t / (4 * N);
            const int pa = (rest % (R1 / 4)) * 4 + pal, pl = rest / (R1 / 4);
            const float2* col = sm + pl * PL + qp;
            float2 v[R2];
#pragma unroll
            for (int jb = 0; jb < R2; ++jb) v[jb] = col[(R2 * pa + jb) * PITCH];
            dft_reg<R2, 1, float>(v);
            const int q = qp / R2 + R1 * (qp % R2);
            const int mi = (q + N / 2) & (N - 1);
            const int k = k0 + pl;
            const float sc = __ldg(a.w32 + k) * inv;
#pragma unroll
            for (int pb = 0; pb < R2; ++pb) {
                const int p = pa + R1 * pb, ni = (p + N / 2) & (N - 1);
                float sg = ((ni + mi) & 1) ? -sc : sc;
                if (s) sg = -sg;
                float2 val = make_float2(v[pb].x * sg, v[pb].y * sg);
                if (s == 0 && (ni == 0 || mi == 0)) val = make_float2(0.f, 0.f);
                const size_t idx = tm ? (size_t)s * N * N * N + (size_t)mi * N * N + (size_t)(ni >> 2) * 4 * N +
                                            (size_t)4 * k + (ni & 3)
                                      : ((size_t)k * 2 + s) * N * N + (size_t)mi * N + ni;
                out[idx] = val;
            }
        }
        __syncthreads();
    }
}

template <int N>
__device__ __noinline__ void f32_item(const BandArgs& a, const float2* F2, float2* coeffs, int tile, int bb,
                                      unsigned char* smem) {
    using C = F32Cfg<N>;
    contract_fwd_tile<float, 4, C::BT, C::KC, C::LW, C::ML, C::MB>(a, F2, coeffs, tile, bb, 0, true, smem);
}

__device__ __forceinline__ void s1_dispatch(const BandArgs& a, const float2* grid, float2* ws, int fi, int k0,
                                            float2* sm) {
    switch (a.N) {
        case 8: s1_item<8>(a, grid, ws, fi, k0, sm); break;
        case 16: s1_item<16>(a, grid, ws, fi, k0, sm); break;
        case 32: s1_item<32>(a, grid, ws, fi, k0, sm); break;
        case 64: s1_item<64>(a, grid, ws, fi, k0, sm); break;
        default: s1_item<128>(a, grid, ws, fi, k0, sm); break;
    }
}
__device__ __forceinline__ void s1_prefetch_dispatch(const BandArgs& a, const float2* grid, int fi, int k0) {
    switch (a.N) {
        case 8: s1_prefetch<8>(a, grid, fi, k0); break;
        case 16: s1_prefetch<16>(a, grid, fi, k0); break;
        case 32: s1_prefetch<32>(a, grid, fi, k0); break;
        case 64: s1_prefetch<64>(a, grid, fi, k0); break;
        default: s1_prefetch<128>(a, grid, fi, k0); break;
    }
}
__device__ __forceinline__ void f32_dispatch(const BandArgs& a, const float2* ws, float2* coeffs, int tile, int bb,
                                             unsigned char* smem) {
    switch (a.N) {
        case 8: f32_item<8>(a, ws, coeffs, tile, bb, smem); break;
        case 16: f32_item<16>(a, ws, coeffs, tile, bb, smem); break;
        case 32: f32_item<32>(a, ws, coeffs, tile, bb, smem); break;
        case 64: f32_item<64>(a, ws, coeffs, tile, bb, smem); break;
        default: f32_item<128>(a, ws, coeffs, tile, bb, smem); break;
    }
}

__global__ void __launch_bounds__(THREADS, 1) ragged_kernel(Args g, const __grid_constant__ Maps maps) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OFF_BAR_);
    uint64_t* bar_full = bars;                   // [NSA] F2 chunk landed        (1 + tx)
    uint64_t* bar_afull = bars + NSA;            // [NSA] A operands written     (N_CONV)
    uint64_t* bar_opa = bars + 2 * NSA;          // [NSA] MMAs of the stage done (commit)
    uint64_t* bar_bfull = bars + 3 * NSA;        // [2] B operands written       (2)
    uint64_t* bar_opb = bar_bfull + 2;           // [2] MMAs of the B stage done (commit)
    uint64_t* bar_accfull = bar_opb + 2;         // [2] accumulators of half h   (commit)
    uint64_t* bar_hfree = bar_accfull + 2;       // [2] half h drained           (4)
    uint64_t* bar_ifull = bar_hfree + 2;         // [DR] item number published   (1)
    uint64_t* bar_iempty = bar_ifull + DR;       // [DR] item number read        (15)
    int* iring = reinterpret_cast<int*>(bar_iempty + DR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(iring + DR);
    int* sh_item = reinterpret_cast<int*>(tslot + 1);
    float4* t_seed = reinterpret_cast<float4*>(smem + OFF_SEED);
    float2* t_xs = reinterpret_cast<float2*>(smem + OFF_XS);
    double* t_lf2 = reinterpret_cast<double*>(smem + OFF_LF2);
    uint32_t* t_rowoff = reinterpret_cast<uint32_t*>(smem + OFF_ROW);
    SeedPair* t_gp = reinterpret_cast<SeedPair*>(smem + OFF_GP);
    int* err = g.err;

    // node tables of the tensor-core bands, log2 k!, packed-row offsets
    for (int b = 0; b < g.nbands; ++b) {
        const RaggedBand& rb = g.bands[b];
        if (!rb.tc) continue;
        for (int k = tid; k < rb.a.N; k += THREADS) {
            t_seed[rb.tab + k] = rb.a.seed32[k];
            t_xs[rb.tab + k] = rb.a.xsplit[k];
        }
    }
    for (int t = tid; t < LF2N; t += THREADS) t_lf2[t] = t < g.lf2_len ? g.lf2[t] : 0.0;
    for (int t = tid; t < NMAXR; t += THREADS) t_rowoff[t] = (uint32_t)block_offset(t);
    if (warp == W_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tslot)), "r"(TMEM_COLS_) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < NSA; ++i) {
            mbar_init(&bar_full[i], 1);
            mbar_init(&bar_afull[i], N_CONV);
            mbar_init(&bar_opa[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_bfull[i], 2);
            mbar_init(&bar_opb[i], 1);
            mbar_init(&bar_accfull[i], 1);
            mbar_init(&bar_hfree[i], 4);
        }
        for (int i = 0; i < DR; ++i) {
            mbar_init(&bar_ifull[i], 1);
            mbar_init(&bar_iempty[i], 1 + N_CONV + 4 + 4);
        }
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;

    // ------------------------------------------------------------------ phase A
    int first_tc = -1;
    for (;;) {
        if (tid == 0) {
            const unsigned nx = atomicAdd(&g.ctr[0], 1u);
            *sh_item = nx < (unsigned)g.nitems ? (int)nx : -1;
        }
        __syncthreads();
        const int it = *sh_item;
        if (it < 0) break;
        const int4 d = g.items[it];
        const int kind = d.x & 15;
        if (kind == IT_TC) { first_tc = it; break; }
        const RaggedBand& rb = g.bands[d.x >> 4];
        if (kind == IT_S1) {
            // the item one grid further on is most likely taken about one item's
            // time later by another CTA: its samples into L2 now
            const int pf = it + (int)gridDim.x;
            if (pf < g.nitems) {
                const int4 dn = g.items[pf];
                if ((dn.x & 15) == IT_S1) s1_prefetch_dispatch(g.bands[dn.x >> 4].a, g.grid, dn.y, dn.z);
            }
            s1_dispatch(rb.a, g.grid, g.ws, d.y, d.z, reinterpret_cast<float2*>(smem));
            __threadfence();                    // this thread's plane stores, before the count
            __syncthreads();
            if (tid == 0) atomicAdd(&g.ctr[1 + d.w], 1u);
        } else {
            if (tid == 0) wait_counter_bounded(&g.ctr[1 + rb.cbase + d.z], (unsigned)rb.s1_per_block(d.z), err);
            __syncthreads();
            f32_dispatch(rb.a, g.ws, g.coeffs, d.y, d.z, smem);
            __syncthreads();
        }
    }
    fence_proxy_async_smem();       // phase A's generic shared-memory writes, before the TMA's
    __syncthreads();

    // ------------------------------------------------------------------ phase B
    if (warp == W_TMA) {
        if (lane == 0) {
            uint64_t pol;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
            uint32_t gc = 0, ip = 0;
            int it = first_tc;
            for (;;) {
                const int slot = (int)(ip % DR);
                const uint32_t u = ip / DR;
                if (u > 0) wait_bar(&bar_iempty[slot], (u - 1) & 1, err);
                int4 d = make_int4(0, 0, 0, 0);
                if (it >= 0) {
                    d = g.items[it];
                    if ((d.x & 15) != IT_TC) {          // the list puts every TC item last
                        atomicExch(err, 2);
                        it = -1;
                    }
                }
                iring[slot] = it;
                mbar_arrive(&bar_ifull[slot]);
                ++ip;
                if (it < 0) break;
                const RaggedBand& rb = g.bands[d.x >> 4];
                const int N = rb.a.N;
                Tile<NP> tl;
                tl.decode(N, d.y);
                const int bb = d.z;
                wait_counter_bounded(&g.ctr[1 + rb.cbase + bb], (unsigned)rb.s1_per_block(bb), err);
                fence_proxy_async_global();          // the acquire above orders the TMA reads
                const CUtensorMap* map = &maps.m[rb.tcmap];
                for (int c = 0; c < N / KC; ++c, ++gc) {
                    const int st = (int)(gc % NSA);
                    const uint32_t us = gc / NSA;
                    if (us > 0) wait_bar(&bar_opa[st], (us - 1) & 1, err);
                    mbar_arrive_expect_tx(&bar_full[st], (uint32_t)STAGE_BYTES);
                    tma_load_5d(smem + st * SA, map, c * KC * NP, tl.nb, tl.mi, tl.s, bb * BM, &bar_full[st], pol);
                }
                const unsigned nx = atomicAdd(&g.ctr[0], 1u);
                it = nx < (unsigned)g.nitems ? (int)nx : -1;
            }
        }
    } else if (warp == W_MMA) {
        if (lane == 0) {
            uint32_t gc = 0, ic = 0, uses[2] = {0, 0};
            int nexth = 0;
            for (;;) {
                const int slot = (int)(ic % DR);
                wait_bar(&bar_ifull[slot], (ic / DR) & 1, err);
                const int it = iring[slot];
                mbar_arrive(&bar_iempty[slot]);
                ++ic;
                if (it < 0) break;
                const int4 d = g.items[it];
                const int N = g.bands[d.x >> 4].a.N;
                Tile<NP> tl;
                tl.decode(N, d.y);
                const int nmma = (tl.L + 15) & ~15;           // <= 64 rows: one half of tensor memory
                const uint32_t idesc = instr_desc(nmma);
                const int h0 = nexth;
                nexth ^= 1;
                if (uses[h0] > 0) wait_bar(&bar_hfree[h0], (uses[h0] - 1) & 1, err);
                ++uses[h0];
                const uint32_t base = taddr + (uint32_t)(h0 * 256);
                tc_fence_after();
                for (int c = 0; c < N / KC; ++c, ++gc) {
                    const int sa = (int)(gc % NSA), sb = (int)(gc & 1);
                    wait_bar(&bar_afull[sa], (gc / NSA) & 1, err);
                    wait_bar(&bar_bfull[sb], (gc >> 1) & 1, err);
                    tc_fence_after();
                    unsigned char* Ab = smem + sa * SA;
                    unsigned char* Bb = smem + OFF_B_ + sb * B_BYTES;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        if (!tl.valid[p]) continue;
                        const uint32_t dt = base + (uint32_t)p * 64u;
                        const uint64_t ah = smem_desc(Ab + p * OPA, LBO_A, SBO_A);
                        const uint64_t al = smem_desc(Ab + (NP + p) * OPA, LBO_A, SBO_A);
                        const uint64_t bh = smem_desc(Bb + p * OPB, LBO_B, SBO_B);
                        const uint64_t bl = smem_desc(Bb + (NP + p) * OPB, LBO_B, SBO_B);
                        mma_bf16(dt, ah, bh, idesc, c > 0);
                        mma_bf16(dt, ah, bl, idesc, true);
                        mma_bf16(dt, al, bh, idesc, true);
                    }
                    mma_commit(&bar_opa[sa]);
                    mma_commit(&bar_opb[sb]);
                }
                mma_commit(&bar_accfull[h0]);
            }
        }
    } else if ((warp >= W_CONV && warp < W_CONV + 4) || warp == W_CONV2 || warp == W_CONV2 + 1) {
        // F2 chunk (fp32) -> BF16 hi/lo A operands in place (as in the per-group kernel)
        const int cw = (warp < W_CONV + 4) ? warp - W_CONV : 4 + (warp - W_CONV2);
        const int ct = cw * 32 + lane;
        constexpr int NIT = BM * (KC / 4) * NP;
        constexpr int MAXI = (NIT + 32 * N_CONV - 1) / (32 * N_CONV);
        uint32_t gc = 0, ic = 0;
        for (;;) {
            const int slot = (int)(ic % DR);
            wait_bar(&bar_ifull[slot], (ic / DR) & 1, err);
            const int it = iring[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_iempty[slot]);
            ++ic;
            if (it < 0) break;
            const int N = g.bands[g.items[it].x >> 4].a.N;
            for (int c = 0; c < N / KC; ++c, ++gc) {
                const int st = (int)(gc % NSA);
                wait_bar(&bar_full[st], (gc / NSA) & 1, err);
                const float2* stg = reinterpret_cast<const float2*>(smem + st * SA);
                unsigned char* Ab = smem + st * SA;
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
    } else if (warp >= W_GEN && warp < W_GEN + 4) {
        // d-values by the three-term recurrence -> BF16 hi/lo B operands (as in the
        // per-group kernel; every tile here has at most 64 rows of l)
        const int grp = (warp - W_GEN) >> 1;
        const int gt = tid - W_GEN * 32 - grp * 64;
        const int p = gt >> 4, kk = gt & 15;
        StepCoef<float>* coef = reinterpret_cast<StepCoef<float>*>(smem + OFF_COEF_) + grp * NP * RMAXR;
        SeedPair* gp = t_gp + grp * NP;
        uint32_t gc = 0, ic = 0;
        for (;;) {
            const int slot = (int)(ic % DR);
            wait_bar(&bar_ifull[slot], (ic / DR) & 1, err);
            const int it = iring[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_iempty[slot]);
            ++ic;
            if (it < 0) break;
            const int4 d = g.items[it];
            const RaggedBand& rb = g.bands[d.x >> 4];
            const int N = rb.a.N;
            const float4* tseed = t_seed + rb.tab;
            const float2* txs = t_xs + rb.tab;
            Tile<NP> tl;
            tl.decode(N, d.y);
            const int Lt = tl.L, nmma = (Lt + 15) & ~15;
            named_sync(1 + grp, 64);                       // previous tile's tables no longer read
            for (int idx = gt; idx < NP * (Lt - 1); idx += 64) {
                const int pp = idx % NP, r = idx / NP;
                const int J = tl.j0 + 2 * r;
                if (J >= tl.mu2[pp]) coef[pp * RMAXR + r] = step_coef<float>(J, tl.n2[pp], tl.m2);
            }
            if (gt < NP) gp[gt] = make_seed_pair(t_lf2, tl.n2[gt], tl.m2);
            named_sync(1 + grp, 64);
            const bool valid = tl.valid[p];
            const int rp = valid ? (tl.mu2[p] - tl.j0) / 2 : nmma;
            const SeedPair q = gp[p];
            const StepCoef<float>* cp = coef + p * RMAXR;
            for (int c = 0; c < N / KC; ++c, ++gc) {
                const int st = (int)(gc & 1);
                if (st != grp) continue;
                const uint32_t u = gc >> 1;
                if (u > 0) wait_bar(&bar_opb[st], (u - 1) & 1, err);
                unsigned char* Bh = smem + OFF_B_ + st * B_BYTES + p * OPB + (kk >> 3) * LBO_B + (kk & 7) * 16;
                unsigned char* Bl = Bh + NP * OPB;
                const int k = c * KC + ((kk >> 2) | ((kk & 3) << 2));
                int E;
                float cur = seed_value32(q, tseed[k], k, N, E);
                float prev = 0.f;
                const float2 xs = txs[k];
                const bool fast = __all_sync(0xffffffffu, E == 0);
                int rb8 = 0;
                for (; rb8 + 8 <= rp && rb8 < nmma; rb8 += 8) {
                    *reinterpret_cast<uint4*>(Bh + (rb8 >> 3) * SBO_B) = make_uint4(0, 0, 0, 0);
                    *reinterpret_cast<uint4*>(Bl + (rb8 >> 3) * SBO_B) = make_uint4(0, 0, 0, 0);
                }
                for (; rb8 < nmma; rb8 += 8) {
                    float v[8];
                    const bool full_blk = (rb8 >= rp) && (rb8 + 8 < Lt);
                    if (fast && full_blk) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const StepCoef<float> cf = cp[rb8 + i];
                            v[i] = cur;
                            const float xb = (xs.x - cf.bh) + (xs.y - cf.bl);
                            const float nxt = fmaf(cf.A * xb, cur, -cf.C * prev);
                            prev = cur;
                            cur = nxt;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int r = rb8 + i;
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
                    *reinterpret_cast<uint4*>(Bh + (rb8 >> 3) * SBO_B) = h;
                    *reinterpret_cast<uint4*>(Bl + (rb8 >> 3) * SBO_B) = l;
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_bfull[st]);
            }
        }
    } else if (warp >= W_EPI && warp < W_EPI + 4) {
        // tensor memory -> i^{n-m} * coefficients (tiles of at most 64 rows)
        const int q = warp - W_EPI;
        uint32_t commits[2] = {0, 0}, ic = 0;
        int nexth = 0;
        for (;;) {
            const int slot = (int)(ic % DR);
            wait_bar(&bar_ifull[slot], (ic / DR) & 1, err);
            const int it = iring[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_iempty[slot]);
            ++ic;
            if (it < 0) break;
            const int4 d = g.items[it];
            const RaggedBand& rb = g.bands[d.x >> 4];
            const int N = rb.a.N;
            Tile<NP> tl;
            tl.decode(N, d.y);
            const int bb = d.z;
            const int Lt = tl.L, nmma = (Lt + 15) & ~15;
            const int h0 = nexth;
            nexth ^= 1;
            wait_bar(&bar_accfull[h0], commits[h0] & 1, err);
            ++commits[h0];
            tc_fence_after();
            const uint32_t base = taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)(h0 * 256);
            const int pt = lane & 3;
            float2* cfh[2];
            bool okh[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int fb = bb * BM + 16 * q + 8 * h + (lane >> 2);
                okh[h] = fb < rb.a.nfunc;
                cfh[h] = g.coeffs + (okh[h] ? rb.a.coeff_off[rb.a.fidx[fb]] : 0);
            }
            const int n2t = tl.n2[pt], mu2t = tl.mu2[pt];
            const bool vt = tl.valid[pt];
            const int ipw = (n2t - tl.m2) / 2;
            for (int cc = 0; cc < nmma; cc += 16) {
                uint32_t rv[NP][16];
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) tmem_ld16(base + (uint32_t)pp * 64u + (uint32_t)cc, rv[pp]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int r = cc + j;
                    const int J = tl.j0 + 2 * r;
                    const size_t rowbase = (size_t)t_rowoff[J < N ? J : N - 1] + (size_t)((tl.m2 + J) / 2) * (J + 1);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int src = 16 * h + 2 * (lane >> 2);
                        float re = 0.f, im = 0.f;
#pragma unroll
                        for (int pp = 0; pp < NP; ++pp) {
                            const float vr = __shfl_sync(0xffffffffu, __uint_as_float(rv[pp][j]), src);
                            const float vi = __shfl_sync(0xffffffffu, __uint_as_float(rv[pp][j]), src + 1);
                            if (pp == pt) { re = vr; im = vi; }
                        }
                        if (r < Lt && okh[h] && vt && J >= mu2t)
                            __stcs(&cfh[h][rowbase + (n2t + J) / 2], cmul_ipow(make_float2(re, im), ipw));
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_hfree[h0]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == W_MMA)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS_) : "memory");
}

// Tile<4> validity on the host (a tile without a coefficient is left out of the list).
bool tile_any(int N, int t) {
    const int nbk = N / 4;
    const int nb = t % nbk, mi = (t / nbk) % N, s = t / (nbk * N);
    if (s == 0 && mi == 0) return false;
    for (int p = 0; p < 4; ++p)
        if (!(s == 0 && nb * 4 + p == 0)) return true;
    return false;
}

}  // namespace rg

bool ragged_supported(int N, bool tc) {
    if (tc) return N == 64 || N == 128;
    return N == 8 || N == 16 || N == 32 || N == 64 || N == 128;
}

int ragged_block(int N, bool tc) {
    if (tc) return tc::BM;
    switch (N) {
        case 8: return rg::F32Cfg<8>::BT;
        case 16: return rg::F32Cfg<16>::BT;
        case 32: return rg::F32Cfg<32>::BT;
        case 64: return rg::F32Cfg<64>::BT;
        default: return rg::F32Cfg<128>::BT;
    }
}

int ragged_planes(int N) {
    switch (N) {
        case 8: return rg::S1Cfg<8>::P;
        case 16: return rg::S1Cfg<16>::P;
        case 32: return rg::S1Cfg<32>::P;
        case 64: return rg::S1Cfg<64>::P;
        default: return rg::S1Cfg<128>::P;
    }
}

int ragged_min_block() { return 32; }

void ragged_items(std::vector<RaggedBand>& bands, std::vector<int4>& items, int* nctr) {
    // bands: a, tc filled in; cbase, fblk, nblk, s1pf, tcmap, tab set here
    std::vector<int> order(bands.size());
    for (size_t i = 0; i < bands.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return bands[x].a.N > bands[y].a.N; });
    int c = 0, tcmap = 0, tab = 0;
    for (int b : order) {
        RaggedBand& rb = bands[b];
        const int N = rb.a.N;
        rb.fblk = ragged_block(N, rb.tc != 0);
        rb.nblk = (rb.a.nfunc + rb.fblk - 1) / rb.fblk;
        rb.s1pf = N / ragged_planes(N);
        rb.cbase = c;
        c += rb.nblk;
        rb.tcmap = rb.tc ? tcmap++ : -1;
        rb.tab = rb.tc ? tab : 0;
        if (rb.tc) tab += N;
    }
    *nctr = 1 + c;
    items.clear();
    for (int b : order) {                       // stage 1, largest bandwidth first
        const RaggedBand& rb = bands[b];
        const int N = rb.a.N, P = ragged_planes(N);
        for (int fi = 0; fi < rb.a.nfunc; ++fi)
            for (int k0 = 0; k0 < N; k0 += P) items.push_back(make_int4(rg::IT_S1 | (b << 4), fi, k0, rb.cbase + fi / rb.fblk));
    }
    for (int pass = 0; pass < 2; ++pass)        // FP32 tiles, then tensor-core tiles
        for (int b : order) {
            const RaggedBand& rb = bands[b];
            if ((rb.tc != 0) != (pass == 1)) continue;
            const int N = rb.a.N;
            for (int t = 0; t < 2 * N * (N / 4); ++t) {
                if (!rg::tile_any(N, t)) continue;
                for (int bb = 0; bb < rb.nblk; ++bb)
                    items.push_back(make_int4((pass ? rg::IT_TC : rg::IT_F32) | (b << 4), t, bb, 0));
            }
        }
}

size_t ragged_smem_bytes() { return (size_t)rg::SMEM; }

cudaError_t launch_ragged(const std::vector<RaggedBand>& hb, const RaggedBand* d_bands, const int4* d_items,
                          int nitems, unsigned* ctr, int nctr, const double* lf2, int lf2_len, int* err,
                          const void* grid, void* ws, void* coeffs, cudaStream_t st) {
    rg::Maps maps;
    memset(&maps, 0, sizeof(maps));
    for (const RaggedBand& rb : hb) {
        if (!rb.tc) continue;
        if (rb.tcmap < 0 || rb.tcmap > 1) return cudaErrorInvalidValue;
        const cuuint64_t N = (cuuint64_t)rb.a.N;
        const cuuint64_t dims[5] = {N * tc::NP, N / tc::NP, N, 2, (cuuint64_t)rb.a.nfunc};
        const cuuint64_t strides[4] = {N * tc::NP * 8, N * N * 8, N * N * N * 8, 2 * N * N * N * 8};
        const cuuint32_t box[5] = {tc::KC * tc::NP, 1, 1, 1, tc::BM};
        const void* base = (const char*)ws + rb.a.ws_group_off * sizeof(float2);
        if (!encode_tensor_map_8b(&maps.m[rb.tcmap], 5, base, dims, strides, box)) return cudaErrorNotSupported;
    }
    cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(unsigned) * (size_t)nctr, st);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rg::ragged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, rg::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    rg::Args g;
    g.bands = d_bands;
    g.items = d_items;
    g.nitems = nitems;
    g.ctr = ctr;
    g.grid = (const float2*)grid;
    g.ws = (float2*)ws;
    g.coeffs = (float2*)coeffs;
    g.err = err;
    g.lf2 = lf2;
    g.lf2_len = lf2_len;
    g.nbands = (int)hb.size();
    const int grid_ctas = std::max(1, std::min(sms, nitems));
    rg::ragged_kernel<<<grid_ctas, tc::THREADS, rg::SMEM, st>>>(g, maps);
    return cudaGetLastError();
}

}  // namespace su2

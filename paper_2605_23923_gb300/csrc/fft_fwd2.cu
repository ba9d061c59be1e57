// Stage 1 (Sec. 4 factorised Riemann sum, Sec. 6 first-stage Proposition) for
// complex64 at N = 128, 256, 512: the 2-D DFT over (alpha, gamma) of every
// beta-node plane as two phases that meet in L2 instead of in a thread-block
// cluster.
//
//   phase A, item (plane, jb):   16 columns j2 in [16 jb, 16 jb + 16) of the
//       plane f[., k, .] (one 3-D TMA box, N x 128 B) -> column DFTs over j1,
//       once plain (sector 0) and once with the pre-twist exp(i pi j1/N)
//       (sector 1) -> intermediate rows I_s[p][j2] (128-byte segments).
//   phase B, item (plane, s, pb): the 16 rows p in [16 pb, 16 pb + 16) of I_s
//       (one 16 N x 8 B bulk copy) -> row DFTs over j2 with the pre-twist
//       exp(i pi j2/N) for s = 1 -> sign (-1)^{n+m}, weight w_k/(2N^2) -> a
//       block of N rows mi x 16 consecutive ni of F2_s, staged in the item's
//       slot and written to the planes by the producer warp with tensor stores
//       (plain layout: 128-byte rows; tile-major: 32-byte rows) before it
//       refills the slot.
//
// The intermediate lives in a ring of plane slots at the end of the workspace;
// a B item discards the L2 lines it has read (discard.global.L2), so a slot's
// data normally never reaches DRAM.  Items are numbered in blocks: block t
// holds the A items of plane t followed by the B items of plane t - D, and the
// CTAs take item numbers in order from a counter in the scratch.  Ordering is
// carried by two counters per ring slot: a B item waits until all A items of
// its plane are done, and an A item reusing a slot waits until the B items of
// the previous plane in that slot have read it.  Every wait is for an item with
// a smaller number, which some running CTA already holds, so the kernel makes
// progress whatever number of its CTAs is resident; every wait is also bounded
// (it latches the error word and gives up).
//
// Full-group grid (psi over [-2 pi, 2 pi), 2N nodes; template FULL): an A item
// loads both psi halves of its 16 columns and folds them, x + x' for integer m
// and (x - x') e^{i pi j2/N} for half-integer m (the 2N-point psi sum reduced to
// N points); weight w_k/(4N^2); origin phase (-1)^n and i (-1)^{n0}.
//
// CTA layout: warps 0 .. CT/32-1 compute, one producer warp issues the loads
// (after the dependency waits) into a two-slot ring (mbarriers full/empty) and
// the B items' tensor stores, and
// one signaller thread publishes the per-slot counters.  The compute warps hand
// each finished phase to the signaller through a small record ring (mbarriers
// sig_full/sig_empty); the signaller makes their global writes visible at GPU
// scope (fence, cumulative over what it observed through the mbarrier) and
// increments the counter, so no compute warp waits for its own stores to drain.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

#include "common.cuh"
#include "su2_internal.h"

namespace su2 {
namespace fwd2 {

template <int N, bool FULL = false>
struct Cfg {
    static constexpr int R1 = Radix<N>::R1, R2 = Radix<N>::R2;
    static_assert(R1 >= R2, "pass a of both item kinds uses every compute thread");
    static constexpr int W = 16;                        // columns per A item, rows per B item
    static constexpr int NH = N / W;                    // A items per plane; B items per sector
    static constexpr int NA = NH, NB = 2 * NH, IB = NA + NB;
    static constexpr int CT = W * (R1 > R2 ? R1 : R2);  // compute threads
    static constexpr int THREADS = CT + 64;             // + producer warp + signaller warp
    static constexpr int SLOT = W * N;                  // float2 of an A slab / B block
    static constexpr int PB = N + 1;                    // row pitch of a B block in the slot
    static constexpr int YP = SLOT + 16;                // B block with its pitch padding (128-B multiple)
    // full-group grid: an A slab holds both psi halves (columns j2 and j2 + N)
    static constexpr int SLOTP = (FULL ? 2 * SLOT : SLOT) + 16;   // slot stride
    static constexpr int NS = 2;                        // ring slots
    static constexpr int NR = 4;                        // signal records
    static constexpr int BOXR = N < 256 ? N : 256;      // rows per TMA box (at most 256)
    static constexpr size_t smem_bytes() {
        return (size_t)NS * SLOTP * 8 + (size_t)YP * 8 + (size_t)N * 8 * 4 + (size_t)N * 4 + 2 * NS * 8 + 2 * NR * 8 +
               NS * 4 + NR * 4;
    }
    static constexpr int BLOCKS_PER_SM =
        FULL ? (N <= 128 ? 2 : 1) : ((N <= 64) ? 4 : (N <= 128) ? 3 : (N <= 256 ? 2 : 1));
};

__device__ __forceinline__ void tma_load_3d_hint(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                                 uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1, {%2, %3, %4}], [%5], %6;"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
// Prefetch of a box into L2 (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];"
                 ::"l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2) : "memory");
}
// Tensor store of a box from this CTA's shared memory (bulk async-group) with an
// L2 eviction policy.  The planes take evict-first: with the default policy a
// line of the tile-major planes (four beta nodes, written by four B items) was
// often written back before it was complete, 18% more DRAM traffic.
__device__ __forceinline__ void tma_store_5d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3,
                                             int c4, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%1, %2, %3, %4, %5}], [%6], %7;"
        ::"l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(src)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void mbar_arrive_cta(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void discard_l2_line(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }


struct Item {
    bool valid, isA;
    int plane, jb, s, pb;
};

template <int N>
__device__ __forceinline__ Item decode(int i, int nplanes, int D) {
    using P = Cfg<N>;
    Item it;
    const int t = i / P::IB, j = i % P::IB;
    if (j < P::NA) {
        it.isA = true;
        it.plane = t;
        it.jb = j;
        it.s = 0;
        it.pb = 0;
        it.valid = t < nplanes;
    } else {
        it.isA = false;
        it.plane = t - D;
        const int jj = j - P::NA;
        it.s = jj / P::NH;
        it.pb = jj % P::NH;
        it.jb = 0;
        it.valid = it.plane >= 0 && it.plane < nplanes;
    }
    return it;
}

// SLAB: a launch over a slab of a.nk beta nodes (starting at a.k_base) writing
// the exchange layout; otherwise every node of every function (nk = N, a
// compile-time constant) writing the planes.
template <int N, bool FULL, bool SLAB = false>
__global__ void __launch_bounds__(Cfg<N, FULL>::THREADS, Cfg<N, FULL>::BLOCKS_PER_SM)
fft_fwd_two_phase(BandArgs a, const __grid_constant__ CUtensorMap gmap, const __grid_constant__ CUtensorMap omap,
                  const float2* __restrict__ grid, float2* __restrict__ ws, int D, int RING, int discard_ok, int ostore) {
    using P = Cfg<N, FULL>;
    constexpr int R1 = P::R1, R2 = P::R2, W = P::W, CT = P::CT, SLOT = P::SLOT, NS = P::NS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);          // [NS][SLOT] ring
    float2* Y = S + NS * P::SLOTP;                             // sector-1 columns of an A item
    float2* om = Y + P::YP;                                    // exp(+2 pi i t/N)
    float2* tw = om + N;                                       // exp(+i pi t/N)
    float2* omq = tw + N;                                      // [q][ia] = om[ia * q] (B items: lanes vary ia)
    float2* omq1 = omq + N;                                    // [q][ia] = e^{i pi ia (2q+1)/N} (B items, sector 1)
    float* wk = reinterpret_cast<float*>(omq1 + N);
    uint64_t* full = reinterpret_cast<uint64_t*>(wk + N);      // [NS]
    uint64_t* empty = full + NS;                               // [NS]
    uint64_t* sig_full = empty + NS;                           // [NR]
    uint64_t* sig_empty = sig_full + P::NR;                    // [NR]
    int* slot_item = reinterpret_cast<int*>(sig_empty + P::NR);   // [NS] item held by a slot (-1: end)
    int* sig_rec = slot_item + NS;                             // [NR] counter to increment (-1: end)

    const int tid = threadIdx.x;
    const int NK = SLAB ? a.nk : N;                            // planes per function in this launch
    const int nplanes = a.nfunc * NK;
    const int nitems = (nplanes + D) * P::IB;
    float2* ring = ws + a.ws_aux_off;                          // [RING][2][N][N]
    unsigned* doneA = reinterpret_cast<unsigned*>(ring + (size_t)RING * 2 * N * N);
    unsigned* doneB = doneA + RING;
    unsigned* queue = doneB + RING;                            // next item number to hand out

    for (int t = tid; t < N; t += blockDim.x) {
        om[t] = a.om32[t];
        omq[t] = a.om32[(t % R1) * (t / R1)];                  // t = q * R1 + ia, ia * q < N
        const int u = (t % R1) * (2 * (t / R1) + 1);           // ia (2q + 1) < 2N
        const float2 tu = a.twist32[u < N ? u : u - N];
        omq1[t] = u < N ? tu : make_float2(-tu.x, -tu.y);
        tw[t] = a.twist32[t];
        wk[t] = a.w32[t];
    }
    if (tid == 0) {
        for (int b = 0; b < NS; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], CT / 32);
        }
        for (int j = 0; j < P::NR; ++j) {
            mbar_init(&sig_full[j], 1);
            mbar_init(&sig_empty[j], 1);
        }
        mbar_fence_init();
    }
    __syncthreads();

    if (tid >= CT + 32) {
        // ------------------------------------------------------------ signaller
        // Record c: counter index (doneA: r, doneB: RING + r) of a phase whose
        // global effects every compute thread has issued before thread 0's arrive.
        if (tid != CT + 32) return;
        for (int c = 0;; ++c) {
            const int j = c % P::NR;
            if (!mbar_wait_bounded(&sig_full[j], (unsigned)(c / P::NR) & 1, a.err)) break;
            const int rec = sig_rec[j];
            mbar_arrive_cta(&sig_empty[j]);
            if (rec < 0) break;
            __threadfence();
            atomicAdd(&doneA[rec], 1u);            // doneB follows doneA in memory
        }
        return;
    }

    if (tid >= CT) {
        // ------------------------------------------------------------- producer
        const int lane = tid - CT;
        const uint64_t pol = policy_evict_first();
        // ostore: a B item leaves its output block (N rows mi x W columns ni, one
        // plane k, one sector) in its slot, and this warp writes it to the planes
        // with tensor stores before the slot is refilled.  pend(b): that B item.
        static_assert(NS == 2, "one pending block per slot, held in two registers");
        int pend0 = -1, pend1 = -1;
        auto pend = [&](int j) -> int& { return j ? pend1 : pend0; };
        auto store_block = [&](int item, const float2* src) {      // lane 0
            const Item ob = decode<N>(item, nplanes, D);
            const int fb = ob.plane / NK, k = ob.plane % NK;
            const int ni0 = (ob.pb * W + N / 2) & (N - 1);
#pragma unroll
            for (int h = 0; h < N / P::BOXR; ++h) {
                if (SLAB)                  // exchange layout [s N + mi][fb][ni/4][k][ni%4]
                    tma_store_5d(&omap, src + h * P::BOXR * W, 0, k, ni0 / 4, fb, ob.s * N + h * P::BOXR, pol);
                else if (a.ws_tile_major)  // [fb*2 + s][mi][ni/4][k][ni%4]
                    tma_store_5d(&omap, src + h * P::BOXR * W, 0, k, ni0 / 4, h * P::BOXR, fb * 2 + ob.s, pol);
                else                       // [fb][k][s][mi][ni]
                    tma_store_5d(&omap, src + h * P::BOXR * W, ni0, h * P::BOXR, ob.s, k, fb, pol);
            }
            bulk_commit();
        };
        int n = 0;
        for (;;) {
            // Items are handed out in number order, so every item this CTA waits
            // on below is already held by a running CTA (no residency assumption).
            // Per item: once the slot is released, the staged output block of the
            // B item it held goes out by tensor stores (not waited for here), then
            // the next item number is taken and its dependency waited on while the
            // stores read the slot; the read is waited for just before the refill.
            const int b = n % NS;
            const unsigned u = (unsigned)(n / NS);
            ++n;
            bool stop = u > 0 && !mbar_wait_bounded(&empty[b], (u - 1) & 1, a.err);
            if (lane == 0 && pend(b) >= 0) {
                store_block(pend(b), S + b * P::SLOTP);
                pend(b) = -1;
            }
            int i = 0;
            if (lane == 0) {
                do {
                    i = (int)atomicAdd(queue, 1u);
                } while (i < nitems && !decode<N>(i, nplanes, D).valid);
            }
            i = __shfl_sync(0xffffffffu, i, 0);
            if (stop) i = nitems;
            if (i >= nitems && lane == 0) bulk_wait_read_all();
            if (i >= nitems) {
                if (lane == 0) {
                    slot_item[b] = -1;
                    mbar_arrive_cta(&full[b]);
                    // the other slot's last item, once its block is staged
                    const int b2 = n % NS;
                    if (pend(b2) >= 0 && mbar_wait_bounded(&empty[b2], (unsigned)((n - 2) / NS) & 1, a.err))
                        store_block(pend(b2), S + b2 * P::SLOTP);
                    bulk_wait_all();
                }
                break;
            }
            const Item it = decode<N>(i, nplanes, D);
            if (lane == 0) {
                slot_item[b] = i;                     // published by the arrive on full[b]
                if (ostore && !it.isA) pend(b) = i;
            }
            __syncwarp();
            const int r = it.plane % RING;
            const unsigned use = (unsigned)(it.plane / RING);
            float2* dst = S + b * P::SLOTP;
            if (it.isA) {
                const int fb = it.plane / NK, k = it.plane % NK;
                if (lane == 0 && use > 0) wait_counter_bounded(&doneB[r], use * P::NB, a.err);
                constexpr int NSL = FULL ? 2 : 1;                 // slabs per A item
                constexpr int GN = FULL ? 2 * N : N;              // psi nodes of a grid row
                if (a.grid_regular) {
                    if (lane == 0) {
                        bulk_wait_read_all();          // the slot's staged block has been read
                        mbar_arrive_expect_tx(&full[b], (uint32_t)(NSL * SLOT * 8));
#pragma unroll
                        for (int sl = 0; sl < NSL; ++sl)
#pragma unroll
                            for (int h = 0; h < N / P::BOXR; ++h)
                                tma_load_3d_hint(dst + sl * SLOT + h * P::BOXR * W, &gmap, it.jb * W + sl * N, k,
                                                 fb * N + h * P::BOXR, &full[b], pol);
                        // the same column stripe of the plane PF planes ahead into L2: its A
                        // item, handed out about PF blocks later, then loads from L2
                        constexpr int PF = 8;
                        const int tp = it.plane + PF;
                        if (tp < nplanes) {
#pragma unroll
                            for (int sl = 0; sl < NSL; ++sl)
#pragma unroll
                                for (int h = 0; h < N / P::BOXR; ++h)
                                    tma_prefetch_3d(&gmap, it.jb * W + sl * N, tp % NK, (tp / NK) * N + h * P::BOXR);
                        }
                    }
                } else {
                    const float2* src = grid + a.grid_off[a.fidx[fb]] + (size_t)k * GN + it.jb * W;
                    if (lane == 0) bulk_wait_read_all();
                    if (lane == 0) mbar_arrive_expect_tx(&full[b], (uint32_t)(NSL * SLOT * 8));
                    __syncwarp();
                    for (int sl = 0; sl < NSL; ++sl)
                        for (int j1 = lane; j1 < N; j1 += 32)
                            bulk_g2s(dst + sl * SLOT + j1 * W, src + sl * N + (size_t)j1 * N * GN, (uint32_t)(W * 8),
                                     &full[b]);
                }
            } else if (lane == 0) {
                // B item: its W intermediate rows are contiguous in the ring (they stay in
                // L2); one bulk copy brings them into the slot once the plane's A items
                // are done, so the compute warps never wait on L2 latency themselves.
                wait_counter_bounded(&doneA[r], (use + 1) * P::NA, a.err);
                fence_proxy_async_global();          // the acquire above orders the copy's reads
                bulk_wait_read_all();                // the slot's staged block has been read
                mbar_arrive_expect_tx(&full[b], (uint32_t)(SLOT * 8));
                bulk_g2s(dst, ring + ((size_t)(r * 2 + it.s) * N + it.pb * W) * N, (uint32_t)(SLOT * 8), &full[b]);
            }
            __syncwarp();
        }
        return;
    }

    // ----------------------------------------------------------------- compute
    const int lane = tid & 31;
    int nrec = 0;                                  // records pushed (thread 0)
    auto push = [&](int rec) {                     // thread 0, after a barrier of all compute threads
        const int j = nrec % P::NR;
        const unsigned v = (unsigned)(nrec / P::NR);
        ++nrec;
        if (v > 0) mbar_wait_bounded(&sig_empty[j], (v - 1) & 1, a.err);
        sig_rec[j] = rec;
        mbar_arrive_cta(&sig_full[j]);
    };
    int n = 0;
    for (;;) {
        const int b = n % NS;
        const unsigned u = (unsigned)(n / NS);
        ++n;
        if (!mbar_wait_bounded(&full[b], u & 1, a.err)) break;
        const int i = slot_item[b];
        if (i < 0) break;
        const Item it = decode<N>(i, nplanes, D);
        float2* X = S + b * P::SLOTP;
        const int r = it.plane % RING;
        const int fb = it.plane / NK, k = it.plane % NK;       // k: node within this launch

        if (it.isA) {
            // Pass a: R2-point DFTs over j1 = ia + R1*b (stride R1), both sectors.
            if (tid < W * R1) {
                const int jc = tid % W, ia = tid / W;
                float2 v[R2], w[R2];
#pragma unroll
                for (int q = 0; q < R2; ++q) {
                    if constexpr (FULL) {
                        // fold the two psi halves: integer m sees x + x', half-integer m (x - x') e^{i pi j2/N}
                        const float2 x0 = X[(ia + R1 * q) * W + jc], x1 = X[SLOT + (ia + R1 * q) * W + jc];
                        v[q] = make_float2(x0.x + x1.x, x0.y + x1.y);
                        w[q] = cmul(make_float2(x0.x - x1.x, x0.y - x1.y), tw[ia + R1 * q]);
                    } else {
                        v[q] = X[(ia + R1 * q) * W + jc];
                        w[q] = cmul(v[q], tw[ia + R1 * q]);
                    }
                }
                dft_reg<R2, 1, float>(w);
                dft_reg<R2, 1, float>(v);
                // one twiddle load for both sectors; X written back to the positions
                // this thread read: no barrier needed before
                Y[ia * W + jc] = w[0];
                X[ia * W + jc] = v[0];
#pragma unroll
                for (int q = 1; q < R2; ++q) {
                    const float2 t = om[ia * q];
                    Y[(ia + R1 * q) * W + jc] = cmul(w[q], t);
                    X[(ia + R1 * q) * W + jc] = cmul(v[q], t);
                }
                fence_proxy_async_smem();   // before the slot is refilled by TMA
            }
            named_sync(1, CT);
            // Pass b: R1-point DFTs over ia; bin p = qb + R2*qa -> intermediate row p.
            if (tid < W * R2) {
                const int jc = tid % W, qb = tid / W;
                float2* I0 = ring + (size_t)(r * 2) * N * N + it.jb * W + jc;
                float2* I1 = I0 + (size_t)N * N;
                float2 v[R1];
#pragma unroll
                for (int ia = 0; ia < R1; ++ia) v[ia] = X[(ia + R1 * qb) * W + jc];
                dft_reg<R1, 1, float>(v);
#pragma unroll
                for (int qa = 0; qa < R1; ++qa) I0[(size_t)(qb + R2 * qa) * N] = v[qa];
#pragma unroll
                for (int ia = 0; ia < R1; ++ia) v[ia] = Y[(ia + R1 * qb) * W + jc];
                dft_reg<R1, 1, float>(v);
#pragma unroll
                for (int qa = 0; qa < R1; ++qa) I1[(size_t)(qb + R2 * qa) * N] = v[qa];
            }
            named_sync(1, CT);                   // slot and Y read; intermediate written
            if (lane == 0) mbar_arrive_cta(&empty[b]);
            if (tid == 0) push(r);               // doneA[r]
        } else {
            // Pass a: R2-point DFTs over j2 = ia + R1*q of row pl, from the rows the
            // producer copied into the slot (pitch N), into Y with the odd row pitch
            // N + 1 (Y is free during B items), so the slot is released after one
            // barrier.
            const float2* rows = ring + ((size_t)(r * 2 + it.s) * N + it.pb * W) * N;
            {
                const int ia = tid % R1, pl = tid / R1;            // W * R1 == CT
                float2 v[R2];
#pragma unroll
                for (int q = 0; q < R2; ++q) v[q] = X[pl * N + ia + R1 * q];
                if (it.s) {
                    // pre-twist e^{i pi (ia + R1 q)/N} = e^{i pi q/R2} e^{i pi ia/N}: the first
                    // factor is a constant per q, the second joins the inter-pass twiddle
#pragma unroll
                    for (int q = 1; q < R2; ++q) {
                        constexpr int S = 16 / R2;                 // e^{i pi q/R2} = omega_32^{S q}
                        v[q] = cmul(v[q], make_float2(tw32_cos<float>(S * q), tw32_sin<float>(S * q)));
                    }
                    dft_reg<R2, 1, float>(v);
#pragma unroll
                    for (int q = 0; q < R2; ++q) v[q] = cmul(v[q], omq1[q * R1 + ia]);
                } else {
                    dft_reg<R2, 1, float>(v);
#pragma unroll
                    for (int q = 1; q < R2; ++q) v[q] = cmul(v[q], omq[q * R1 + ia]);
                }
#pragma unroll
                for (int q = 0; q < R2; ++q) Y[pl * P::PB + ia + R1 * q] = v[q];   // odd pitch: no conflicts
            }
            // The rows are in shared memory: drop them from L2, release them.
            if (discard_ok) {             // ring rows on 128-byte lines: no line is shared
                const char* src = reinterpret_cast<const char*>(rows);
                for (int l = tid; l < SLOT * 8 / 128; l += CT) discard_l2_line(src + (size_t)l * 128);
            }
            named_sync(1, CT);            // slot read, Y written, discards issued
            if (!ostore && lane == 0) mbar_arrive_cta(&empty[b]);
            if (tid == 0) push(RING + r);        // doneB[r]
            // Pass b: R1-point DFTs; output bin q = qb + R2*qa; 16 consecutive ni per row.
            if (tid < W * R2) {
                const int pl = tid % W, qb = tid / W;
                float2 v[R1];
#pragma unroll
                for (int ia = 0; ia < R1; ++ia) v[ia] = Y[pl * P::PB + ia + R1 * qb];
                named_sync(2, CT);        // Y read before the next item rewrites it
                dft_reg<R1, 1, float>(v);
                const float scale = wk[SLAB ? a.k_base + k : k] / ((FULL ? 4.f : 2.f) * (float)N * (float)N);
                const size_t plane_off = a.grid_regular ? a.ws_group_off + (size_t)fb * 2 * N * N * N
                                                        : a.ws_off[a.fidx[fb]];
                const int p = it.pb * W + pl;
                const int ni = (p + N / 2) & (N - 1);
                // element (mi) of this thread's column ni: [k][s][mi][ni] or, tile-major,
                // [s][mi][ni/4][k][ni%4] (4 consecutive n of all nodes contiguous).  Bin
                // q = qb + R2*qa has mi = q + N/2 for qa < R1/2 and q - N/2 after, so
                // every store is a fixed offset from one of two bases.
                // phase of the grid origin: (-1)^{n+m} (sector 0) and -(-1)^{n0+m0}
                // (sector 1, n = n0 + 1/2) on the paper's domain; on the full-group grid
                // (psi from -2 pi) (-1)^n and i (-1)^{n0}
                float sc;
                if constexpr (FULL) {
                    sc = (ni & 1) ? -scale : scale;
                } else {
                    sc = ((ni + qb) & 1) ? -scale : scale;     // parity of mi = parity of qb
                    if (it.s) sc = -sc;
                }
                const bool rot = FULL && it.s;                   // times i
                const bool zero_col = (it.s == 0 && ni == 0);
                const bool zero_nyq = (it.s == 0 && qb == 0);    // mi = 0 at qa = R1/2
                auto store_all = [&](float2* out, auto ms_c) {
                    constexpr size_t MS = decltype(ms_c)::value;
                    float2* lo = out + (size_t)(qb + N / 2) * MS;
                    float2* hi = out + (size_t)qb * MS - (size_t)(N / 2) * MS;
#pragma unroll
                    for (int qa = 0; qa < R1; ++qa) {
                        float2 val = rot ? make_float2(-v[qa].y * sc, v[qa].x * sc)
                                         : make_float2(v[qa].x * sc, v[qa].y * sc);
                        if (zero_col || (zero_nyq && qa == R1 / 2)) val = make_float2(0.f, 0.f);
                        float2* dst = (qa < R1 / 2) ? lo + (size_t)R2 * qa * MS : hi + (size_t)R2 * qa * MS;
                        __stcs(dst, val);
                    }
                };
                if (ostore) {
                    // block [mi][pl] in the slot (rows of W consecutive ni); the producer
                    // writes it out with tensor stores
#pragma unroll
                    for (int qa = 0; qa < R1; ++qa) {
                        float2 val = rot ? make_float2(-v[qa].y * sc, v[qa].x * sc)
                                         : make_float2(v[qa].x * sc, v[qa].y * sc);
                        if (zero_col || (zero_nyq && qa == R1 / 2)) val = make_float2(0.f, 0.f);
                        const int mi = qb + R2 * qa + ((qa < R1 / 2) ? N / 2 : -N / 2);
                        X[mi * W + pl] = val;
                    }
                    fence_proxy_async_smem();
                } else if (a.ws_tile_major) {
                    store_all(ws + plane_off + (size_t)it.s * N * N * N + (size_t)(ni >> 2) * N * 4 + (size_t)k * 4 +
                                  (ni & 3),
                              std::integral_constant<size_t, (size_t)N * N>());
                } else {
                    store_all(ws + plane_off + ((size_t)k * 2 + it.s) * N * N + ni,
                              std::integral_constant<size_t, (size_t)N>());
                }
            } else {
                named_sync(2, CT);
            }
            if (ostore) {                 // block staged: hand the slot to the producer
                __syncwarp();
                if (lane == 0) mbar_arrive_cta(&empty[b]);
            }
        }
    }
    if (tid == 0) push(-1);                       // end of the signaller's records
}

// Work-distribution parameters shared by the plan (workspace size) and the launch.
template <int N, bool FULL>
static cudaError_t geometry(int device, int* G, int* D, int* RING) {
    using P = Cfg<N, FULL>;
    int sms = 0, per = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    auto kern = fft_fwd_two_phase<N, FULL>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::smem_bytes());
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, P::THREADS, P::smem_bytes());
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    *G = sms * per;
    const int inflight = (2 * *G + P::IB - 1) / P::IB;        // planes touched by two items per CTA
    *D = 2 * inflight + 2;
    *RING = *D + inflight + 4;
    return cudaSuccess;
}

template <int N, bool FULL, bool SLAB = false>
static cudaError_t launch_n(const BandArgs& a, const void* in, void* out, cudaStream_t st) {
    using P = Cfg<N, FULL>;
    int dev = 0, G = 0, D = 0, RING = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = geometry<N, FULL>(dev, &G, &D, &RING)) != cudaSuccess) return e;
    if (RING != a.aux_ring) return cudaErrorInvalidValue;          // plan built for another device shape
    float2* ring = (float2*)out + a.ws_aux_off;
    unsigned* ctr = reinterpret_cast<unsigned*>(ring + (size_t)RING * 2 * N * N);
    if ((e = cudaMemsetAsync(ctr, 0, sizeof(unsigned) * (2 * RING + 1), st)) != cudaSuccess) return e;
    CUtensorMap gmap;
    memset(&gmap, 0, sizeof(gmap));
    BandArgs b = a;
    if (b.grid_regular) {
        constexpr int GN = FULL ? 2 * N : N;                      // psi nodes per grid row
        // grids [fb][j1][k][j2] with a.nk beta nodes (all N, or a slab of them)
        const cuuint64_t dims[3] = {(cuuint64_t)GN, (cuuint64_t)a.nk, (cuuint64_t)a.nfunc * N};
        const cuuint64_t strides[2] = {(cuuint64_t)GN * 8, (cuuint64_t)a.nk * GN * 8};
        const cuuint32_t box[3] = {(cuuint32_t)P::W, 1, (cuuint32_t)P::BOXR};
        const void* base = (const float2*)in + a.grid_group_off;
        if (!encode_tensor_map_8b(&gmap, 3, base, dims, strides, box)) b.grid_regular = 0;
    }
    const int nitems = (a.nfunc * a.nk + D) * P::IB;
    int grid = G < nitems ? G : nitems;
    // SU2_STAGE1_MAX_CTAS caps the grid (robustness checks: the in-order queue
    // must finish with any number of resident CTAs, down to one)
    if (const char* cap = getenv("SU2_STAGE1_MAX_CTAS")) {
        const int c = atoi(cap);
        if (c >= 1 && c < grid) grid = c;
    }
    const int discard_ok = ((uintptr_t)ring % 128) == 0;
    // Output planes of the group (function i at ws_group_off + 2 N^3 i) as a 5-D
    // tensor for the B items' tensor stores; boxes of BOXR rows mi x W columns ni.
    CUtensorMap omap;
    memset(&omap, 0, sizeof(omap));
    int ostore = 0;
    if (b.grid_regular && a.xout) {   // exchange layout [s N + mi][fb][ni/4][k][ni%4], k < nk
        const cuuint64_t n = (cuuint64_t)N, e = 8, nk = (cuuint64_t)a.nk;
        const cuuint64_t dims[5] = {4, nk, n / 4, (cuuint64_t)a.nfunc, 2 * n};
        const cuuint64_t strides[4] = {4 * e, nk * 4 * e, n * nk * e, (cuuint64_t)a.nfunc * n * nk * e};
        const cuuint32_t box[5] = {4, 1, (cuuint32_t)P::W / 4, 1, (cuuint32_t)P::BOXR};
        ostore = encode_tensor_map_8b(&omap, 5, a.xout, dims, strides, box) ? 1 : 0;
    } else if (b.grid_regular) {
        const cuuint64_t n = (cuuint64_t)N, e = 8;
        const void* base = (const float2*)out + a.ws_group_off;
        if (a.ws_tile_major) {         // [fb*2 + s][mi][ni/4][k][ni%4]
            const cuuint64_t dims[5] = {4, n, n / 4, n, 2 * (cuuint64_t)a.nfunc};
            const cuuint64_t strides[4] = {4 * e, 4 * n * e, n * n * e, n * n * n * e};
            const cuuint32_t box[5] = {4, 1, (cuuint32_t)P::W / 4, (cuuint32_t)P::BOXR, 1};
            ostore = encode_tensor_map_8b(&omap, 5, base, dims, strides, box) ? 1 : 0;
        } else {                       // [fb][k][s][mi][ni]
            const cuuint64_t dims[5] = {n, n, 2, n, (cuuint64_t)a.nfunc};
            const cuuint64_t strides[4] = {n * e, n * n * e, 2 * n * n * e, 2 * n * n * n * e};
            const cuuint32_t box[5] = {(cuuint32_t)P::W, (cuuint32_t)P::BOXR, 1, 1, 1};
            ostore = encode_tensor_map_8b(&omap, 5, base, dims, strides, box) ? 1 : 0;
        }
    }
    // the exchange layout is written by tensor stores only
    if (a.xout && (!b.grid_regular || !ostore)) return cudaErrorNotSupported;
    if (SLAB != (a.xout != nullptr)) return cudaErrorInvalidValue;
    auto kern = fft_fwd_two_phase<N, FULL, SLAB>;
    if (SLAB && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::smem_bytes())) !=
                    cudaSuccess)
        return e;
    kern<<<grid, P::THREADS, P::smem_bytes(), st>>>(b, gmap, omap, (const float2*)in, (float2*)out, D, RING,
                                                    discard_ok, ostore);
    return cudaGetLastError();
}

}  // namespace fwd2

bool fft_forward_two_phase_supported(int N, bool fp64) { return !fp64 && (N == 64 || N == 128 || N == 256 || N == 512); }

cudaError_t fft_forward_aux(int N, int device, bool full_group, int* ring, size_t* elems) {
    int G = 0, D = 0, R = 0;
    cudaError_t e;
    if (full_group) {
        switch (N) {
            case 64: e = fwd2::geometry<64, true>(device, &G, &D, &R); break;
            case 128: e = fwd2::geometry<128, true>(device, &G, &D, &R); break;
            case 256: e = fwd2::geometry<256, true>(device, &G, &D, &R); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (N) {
            case 64: e = fwd2::geometry<64, false>(device, &G, &D, &R); break;
            case 128: e = fwd2::geometry<128, false>(device, &G, &D, &R); break;
            case 256: e = fwd2::geometry<256, false>(device, &G, &D, &R); break;
            case 512: e = fwd2::geometry<512, false>(device, &G, &D, &R); break;
            default: return cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return e;
    *ring = R;
    // ring planes (2 N^2 complex each) + 2 R counters + the item queue, rounded up to 256 bytes so
    // that the next bandwidth's ring starts on a 128-byte L2 line as well
    *elems = (size_t)R * 2 * N * N + ((size_t)(2 * R + 1) * sizeof(unsigned) + 255) / 256 * 32;
    return cudaSuccess;
}

cudaError_t launch_fft_forward_two_phase(const BandArgs& a, const void* grid, void* ws, cudaStream_t st) {
    if (a.nfunc <= 0) return cudaSuccess;
    if (a.xout) {                       // beta slab -> exchange layout (sharded transform)
        if (a.full_group) return cudaErrorInvalidValue;
        switch (a.N) {
            case 64: return fwd2::launch_n<64, false, true>(a, grid, ws, st);
            case 128: return fwd2::launch_n<128, false, true>(a, grid, ws, st);
            case 256: return fwd2::launch_n<256, false, true>(a, grid, ws, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (a.full_group) {
        switch (a.N) {
            case 64: return fwd2::launch_n<64, true>(a, grid, ws, st);
            case 128: return fwd2::launch_n<128, true>(a, grid, ws, st);
            case 256: return fwd2::launch_n<256, true>(a, grid, ws, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (a.N) {
        case 64: return fwd2::launch_n<64, false>(a, grid, ws, st);
        case 128: return fwd2::launch_n<128, false>(a, grid, ws, st);
        case 256: return fwd2::launch_n<256, false>(a, grid, ws, st);
        case 512: return fwd2::launch_n<512, false>(a, grid, ws, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace su2

// Device utilities shared by the SU(2) transform kernels: complex helpers,
// compile-time-unrolled register DFTs, cluster shared-memory access and the
// per-band argument structures.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace su2 {

// ---------------------------------------------------------------------------
// Complex numbers as (re, im) pairs of the working real type.
// ---------------------------------------------------------------------------
template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using cplx = typename cplx_t<T>::type;

template <typename T> __device__ __forceinline__ cplx<T> mk(T r, T i) { cplx<T> z; z.x = r; z.y = i; return z; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C z; z.x = a.x + b.x; z.y = a.y + b.y; return z; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C z; z.x = a.x - b.x; z.y = a.y - b.y; return z; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { C z; z.x = a.x; z.y = -a.y; return z; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { C z; z.x = a.x * s; z.y = a.y * s; return z; }
// multiply by i^e (e taken mod 4)
template <typename C> __device__ __forceinline__ C cmul_ipow(C a, int e) {
    C z;
    switch (e & 3) {
        case 0: z = a; break;
        case 1: z.x = -a.y; z.y = a.x; break;
        case 2: z.x = -a.x; z.y = -a.y; break;
        default: z.x = a.y; z.y = -a.x; break;
    }
    return z;
}

// cos and sin of 2*pi*t/32 for t = 0..31, constant-folded when t is known.
template <typename T> __device__ __forceinline__ T tw32_cos(int t) {
    switch (t & 31) {
    case 0: return T(1);
    case 1: return T(0.98078528040323043);
    case 2: return T(0.92387953251128674);
    case 3: return T(0.83146961230254524);
    case 4: return T(0.70710678118654757);
    case 5: return T(0.55557023301960229);
    case 6: return T(0.38268343236508984);
    case 7: return T(0.19509032201612833);
    case 8: return T(0);
    case 9: return T(-0.19509032201612819);
    case 10: return T(-0.38268343236508973);
    case 11: return T(-0.55557023301960196);
    case 12: return T(-0.70710678118654746);
    case 13: return T(-0.83146961230254535);
    case 14: return T(-0.92387953251128674);
    case 15: return T(-0.98078528040323043);
    case 16: return T(-1);
    case 17: return T(-0.98078528040323043);
    case 18: return T(-0.92387953251128685);
    case 19: return T(-0.83146961230254546);
    case 20: return T(-0.70710678118654768);
    case 21: return T(-0.55557023301960218);
    case 22: return T(-0.38268343236509034);
    case 23: return T(-0.19509032201612866);
    case 24: return T(0);
    case 25: return T(0.1950903220161283);
    case 26: return T(0.38268343236509);
    case 27: return T(0.55557023301960184);
    case 28: return T(0.70710678118654735);
    case 29: return T(0.83146961230254524);
    case 30: return T(0.92387953251128652);
    case 31: return T(0.98078528040323032);
    }
    return T(0);
}
template <typename T> __device__ __forceinline__ T tw32_sin(int t) {
    switch (t & 31) {
    case 0: return T(0);
    case 1: return T(0.19509032201612825);
    case 2: return T(0.38268343236508978);
    case 3: return T(0.55557023301960218);
    case 4: return T(0.70710678118654746);
    case 5: return T(0.83146961230254524);
    case 6: return T(0.92387953251128674);
    case 7: return T(0.98078528040323043);
    case 8: return T(1);
    case 9: return T(0.98078528040323043);
    case 10: return T(0.92387953251128674);
    case 11: return T(0.83146961230254546);
    case 12: return T(0.70710678118654757);
    case 13: return T(0.55557023301960218);
    case 14: return T(0.38268343236508989);
    case 15: return T(0.19509032201612861);
    case 16: return T(0);
    case 17: return T(-0.19509032201612836);
    case 18: return T(-0.38268343236508967);
    case 19: return T(-0.55557023301960196);
    case 20: return T(-0.70710678118654746);
    case 21: return T(-0.83146961230254524);
    case 22: return T(-0.92387953251128652);
    case 23: return T(-0.98078528040323032);
    case 24: return T(-1);
    case 25: return T(-0.98078528040323043);
    case 26: return T(-0.92387953251128663);
    case 27: return T(-0.83146961230254546);
    case 28: return T(-0.70710678118654768);
    case 29: return T(-0.55557023301960218);
    case 30: return T(-0.38268343236509039);
    case 31: return T(-0.19509032201612872);
    }
    return T(0);
}

// Ratio used by the tangent-form butterfly for t = 1..15, t != 8 (omega_32^t =
// cos + i sin): tan(2 pi t/32) where |cos| >= |sin| (t <= 4 or t >= 12), else
// cot(2 pi t/32); both in [-1, 1].
template <typename T> __device__ __forceinline__ T tw32_ratio(int t) {
    switch (t & 31) {
    case 1: return T(0.19891236737965800691);
    case 2: return T(0.41421356237309504880);
    case 3: return T(0.66817863791929892000);
    case 4: return T(1.0000000000000000000);
    case 5: return T(0.66817863791929892000);
    case 6: return T(0.41421356237309504880);
    case 7: return T(0.19891236737965800691);
    case 9: return T(-0.19891236737965800691);
    case 10: return T(-0.41421356237309504880);
    case 11: return T(-0.66817863791929892000);
    case 12: return T(-1.0000000000000000000);
    case 13: return T(-0.66817863791929892000);
    case 14: return T(-0.41421356237309504880);
    case 15: return T(-0.19891236737965800691);
    }
    return T(0);
}

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
__host__ __device__ __forceinline__ constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r = (r << 1) | ((i >> b) & 1);
    return r;
}

// In-register DFT of length R (power of two, R <= 32):
//   x[q] <- sum_j x[j] * exp(SIGN * 2 pi i q j / R).
// Radix-2 decimation in time on a bit-reversed copy; the butterfly stages are
// unrolled at compile time (template recursion over the stage length), so all
// indices are constants and trivial twiddles (1, +-i) cost nothing.
template <int R, int SIGN, typename T, int LEN>
__device__ __forceinline__ void dft_stage(cplx<T> (&y)[R]) {
    if constexpr (LEN <= R) {
        constexpr int half = LEN / 2;
        constexpr int step = 32 / LEN;           // omega_LEN^k = omega_32^(k * step)
#pragma unroll
        for (int i = 0; i < R; i += LEN) {
#pragma unroll
            for (int k = 0; k < half; ++k) {
                const int t = k * step;
                const cplx<T> b = y[i + k + half];
                const cplx<T> a = y[i + k];
                if (t == 0 || t == 8) {
                    // omega = 1 or SIGN * i: additions only
                    const cplx<T> tb = (t == 0) ? b : ((SIGN > 0) ? mk<T>(-b.y, b.x) : mk<T>(b.y, -b.x));
                    y[i + k] = cadd(a, tb);
                    y[i + k + half] = csub(a, tb);
                } else {
                    // a +- omega b with omega = c + i sn in the tangent form: omega b = g u with
                    // u = b + i (sn/c) b, g = c when |c| >= |sn|, else u = i b + (c/sn) b,
                    // g = sn (ratio in [-1, 1]); then 2 + 4 fused multiply-adds instead of 8
                    const T c = tw32_cos<T>(t);
                    const T sn = (SIGN > 0) ? tw32_sin<T>(t) : -tw32_sin<T>(t);
                    const bool cdom = (t <= 4 || t >= 12);      // |cos| >= |sin| (t < 16)
                    const T r = (SIGN > 0) ? tw32_ratio<T>(t) : -tw32_ratio<T>(t);
                    const T g = cdom ? c : sn;
                    const cplx<T> u = cdom ? mk<T>(b.x - r * b.y, b.y + r * b.x) : mk<T>(r * b.x - b.y, b.x + r * b.y);
                    y[i + k] = mk<T>(a.x + g * u.x, a.y + g * u.y);
                    y[i + k + half] = mk<T>(a.x - g * u.x, a.y - g * u.y);
                }
            }
        }
        dft_stage<R, SIGN, T, LEN * 2>(y);
    }
}

template <int R, int SIGN, typename T>
__device__ __forceinline__ void dft_reg(cplx<T> (&x)[R]) {
    if constexpr (R > 1) {
        constexpr int B = ilog2c(R);
        cplx<T> y[R];
#pragma unroll
        for (int i = 0; i < R; ++i) y[i] = x[bitrev(i, B)];
        dft_stage<R, SIGN, T, 2>(y);
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = y[i];
    }
}

// Four-step split of a length-N DFT used by every transform kernel:
// N = R1 * R2, pass A: R2-point DFTs over the stride-R1 subsequences,
// pass B: R1-point DFTs over contiguous blocks.
template <int N> struct Radix;
template <> struct Radix<32>  { static constexpr int R1 = 8,  R2 = 4; };
template <> struct Radix<64>  { static constexpr int R1 = 8,  R2 = 8; };
template <> struct Radix<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct Radix<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct Radix<512> { static constexpr int R1 = 32, R2 = 16; };
template <> struct Radix<1024> { static constexpr int R1 = 32, R2 = 32; };

// ---------------------------------------------------------------------------
// Thread-block cluster helpers (distributed shared memory).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory location in CTA `rank` of this cluster.
__device__ __forceinline__ uint32_t map_shared(const void* p, unsigned rank) {
    uint32_t local = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    return remote;
}
__device__ __forceinline__ float2 ld_dsmem(uint32_t addr, float2) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}
__device__ __forceinline__ double2 ld_dsmem(uint32_t addr, double2) {
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(addr));
    return v;
}

// ---------------------------------------------------------------------------
// mbarrier + bulk-copy (TMA) helpers.  Every wait is bounded: after ~1 s of
// SM clock it latches an error in *err and gives up (the caller then keeps
// going on stale data, so that all cluster barriers are still met and the
// kernel ends; the host reports SU2_ERR_TIMEOUT).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > 2000000000LL) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}
// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Acquire load of a counter that other CTAs increment (each after a
// __threadfence and an atomicAdd).
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Spin until *ctr >= target (wrap-safe comparison), bounded like the mbarrier
// waits: after 2e9 SM cycles (about a second) latch the error word and return.
// Once any wait of the launch has timed out (error word set) the others return
// at once, so a broken dependency costs one timeout, not one per item.
__device__ __forceinline__ void wait_counter_bounded(const unsigned* ctr, unsigned target, int* err) {
    if ((int)(ld_acquire_gpu(ctr) - target) >= 0) return;
    const long long t0 = clock64();
    while ((int)(ld_acquire_gpu(ctr) - target) < 0) {
        if (*(volatile int*)err != 0) return;
        __nanosleep(64);
        if (clock64() - t0 > 2000000000LL) {
            atomicExch(err, 1);
            return;
        }
    }
}
// 1-D bulk copy global -> shared (this CTA), completion counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// 1-D bulk copy from this CTA's shared memory to shared memory of CTA `rank`
// of the cluster; completion is counted on the mbarrier at the same offset
// (`bar_local`) in the destination CTA.
__device__ __forceinline__ void bulk_s2s_remote(const void* dst_local, const void* src, uint32_t bytes,
                                                const uint64_t* bar_local, unsigned rank) {
    const uint32_t dst = map_shared(dst_local, rank);
    const uint32_t bar = map_shared(bar_local, rank);
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "r"(smem_u32(src)), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Arguments of one launch over a group of functions sharing the bandwidth N.
// Element offsets are in complex elements.
// ---------------------------------------------------------------------------
struct BandArgs {
    int N;
    int nfunc;                    // functions in this launch group
    const int* fidx;              // [nfunc] function ids
    const size_t* grid_off;       // [num_functions] grid offsets
    const size_t* coeff_off;      // [num_functions] coefficient offsets
    const size_t* ws_off;         // [num_functions] stage-1 plane offsets
    // per-band tables (device)
    const double* cosb;           // cos(beta_k)
    const double* log2c;          // log2 cos(beta_k/2)
    const double* log2s;          // log2 sin(beta_k/2)
    const float4* seed32;         // (c_hi, c_lo, s_hi, s_lo): log2 cos(beta_k/2) = c_hi + c_lo,
                                  // log2 sin(beta_k/2) = s_hi + s_lo, hi parts on a 2^-11 grid
                                  // (so pc * hi is exact in FP32 for pc < 2^8); 0 at the poles
    const double* w64;            // beta weights w_k
    const float* w32;
    const float2* xsplit;         // (hi, lo) float split of cos(beta_k)
    const double* lf2;            // log2(k!) for k = 0..2N
    const float2* om32;           // exp(+2 pi i t/N), t = 0..N-1
    const double2* om64;
    const float2* twist32;        // exp(+i pi t/N), t = 0..N-1
    const double2* twist64;
    int* err;                     // device error word
    size_t ws_group_off;          // stage-1 plane offset of the group's first function
                                  // (a group's planes are contiguous: function i of
                                  // the group at ws_group_off + i * 2 N^3)
    size_t grid_group_off;        // grid offset of the group's first function
    int grid_regular;             // 1: function i of the group at grid_group_off + i * N^3
    size_t ws_aux_off;            // stage-1 scratch of the group (two-phase DFT ring), in
                                  // complex elements from the workspace start
    int aux_ring;                 // plane slots of that ring (0: none)
    int ws_tile_major;            // 1: stage-1 planes of a function stored [s][mi][ni/4][k][ni%4]
                                  // (tensor-core plans), 0: [k][s][mi][ni]
    int s1_two_phase;             // forward 2-D DFT: 1 two-phase kernel (needs aux_ring > 0), 0 cluster
    int s2_bt;                    // FP32 forward contraction: functions per block (8 or 16; 0: by batch)
    int s2_rc;                    // FP32 forward contraction in row classes: -1 when >= 48 functions, 0 no, 1 yes
    int full_group;               // grids on the full-group grid (psi over [-2 pi, 2 pi), 2N nodes)
    int literal;                  // grids on the printed grid (spacing 2 pi/(N-1), endpoint repeated);
                                  // aux_ring then counts the literal kernel's CTAs (one N^2 slab each)
    const float2* lit_w;          // [N][N] e^{2 pi i (r - N/2) t/(N-1)}, column N-1 zero (literal grid)
    const float2* lit_twist;      // [2N] e^{i pi u/(N-1)} (literal grid)
    const float2* lit_bs;         // literal grid, N >= 64: Bluestein tables (chirps, filter, twiddles;
                                  // layout in fft_literal.cu); aux_ring then counts planes per chunk
    // Sharded transform (a function's beta nodes split over several GPUs for stage 1,
    // its (s, m) rows for stage 2; defaults describe the whole transform):
    int nk;                       // beta nodes per function in this stage-1 launch (N: all)
    int k_base;                   // global index of the first of them
    float2* xout;                 // stage 1 output in the exchange layout [2N][nfunc][N/4][nk][4]
                                  // (row s N + mi, then function, then n/4, node, n%4); null: planes
    int tc_t0, tc_ntiles;         // tensor-core stage 2: tiles [t0, t0 + ntiles) (ntiles 0: all)
    const float2* xrecv;          // tensor-core stage 2 input in the received exchange layout
                                  // [N/nk][x_nrows][nfunc][N/4][nk][4] (null: the planes)
    int x_row0, x_nrows;          // the rows s N + mi that xrecv holds
    const int* s2_tiles;          // FP32 contraction tiles by rows of l: L <= 32, then 32 < L <= 64,
                                  // then L > 64, concatenated (tile numbers as Tile<4>::decode takes)
    int s2_ntiles[3];             // tiles in each of those classes
};

}  // namespace su2

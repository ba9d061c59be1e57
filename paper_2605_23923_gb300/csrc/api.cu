// C ABI of the SU(2) transform library (declared in include/su2fft.h).
//
// A plan groups the functions of a batch by bandwidth N and uploads, per
// distinct N, the FP64 tables the kernels read: beta_k = k pi/(N-1) (Sec. 4
// sampling grid), cos(beta_k) and its float hi/lo split, log2 cos(beta_k/2),
// log2 sin(beta_k/2), the beta weights (Clenshaw-Curtis on cos(beta_k), or the
// paper-literal sin(beta_k) pi/(N-1)), the DFT twiddles exp(2 pi i t/N) and
// the half-bin twists exp(i pi t/N); plus log2(k!) for the recurrence seeds.
// Execution calls launch, per group, stage 1 (2-D DFT per beta node) and
// stage 2 (beta contraction with the recurrence fused in), asynchronously on
// the caller's stream, allocating nothing.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/su2fft.h"
#include "su2_internal.h"

namespace {

struct Band {
    int N = 0;
    std::vector<int> fids;
    int* d_fidx = nullptr;
    double* d_cosb = nullptr;
    double* d_log2c = nullptr;
    double* d_log2s = nullptr;
    float4* d_seed32 = nullptr;
    double* d_w64 = nullptr;
    float* d_w32 = nullptr;
    float2* d_xsplit = nullptr;
    float2* d_om32 = nullptr;
    double2* d_om64 = nullptr;
    float2* d_twist32 = nullptr;
    double2* d_twist64 = nullptr;
    size_t aux_off = 0;           // stage-1 scratch (two-phase DFT ring) in the workspace
    int aux_ring = 0;
    bool tc = false;              // contraction on tensor cores (tile-major planes)
    bool full_group = false;      // grids on the full-group grid (forward only)
    bool literal = false;         // grids on the printed grid (forward only)
    float2* d_lit_w = nullptr;
    float2* d_lit_twist = nullptr;
    float2* d_lit_bs = nullptr;
    int s1_two_phase = 0;         // kernel choices (defaults, or the autotuner's)
    int s2_bt = 0;
    int s2_rc = -1;               // FP32 row classes: -1 by batch size, 0 off, 1 on
    int* d_s2_tiles = nullptr;    // FP32 contraction tiles grouped by rows of l (see BandArgs)
    int s2_ntiles[3] = {0, 0, 0};
};

// Tiles of 4 consecutive n at fixed (sector, m) for the FP32 contraction, grouped
// by their number of rows of l (L <= 32, 32 < L <= 64, L > 64), so that each
// group runs with a row window that fits it; tiles without a coefficient are left
// out.  The numbering and L follow the device-side tile decode.
void fp32_tile_classes(int N, std::vector<int>& tiles, int counts[3]) {
    std::vector<int> cls[3];
    const int nbk = N / 4;
    for (int t = 0; t < 2 * N * nbk; ++t) {
        const int nb = t % nbk, mi = (t / nbk) % N, s = t / (nbk * N);
        const int m2 = 2 * (mi - N / 2) + s, jtop = N - 2 + s;
        int j0 = 1 << 30;
        for (int p = 0; p < 4; ++p) {
            const int ni = nb * 4 + p, n2 = 2 * (ni - N / 2) + s;
            const bool valid = !(s == 0 && mi == 0) && !(s == 0 && ni == 0);
            if (valid) j0 = std::min(j0, std::max(std::abs(n2), std::abs(m2)));
        }
        if (j0 == (1 << 30)) continue;
        const int L = (jtop - j0) / 2 + 1;
        cls[L <= 32 ? 0 : (L <= 64 ? 1 : 2)].push_back(t);
    }
    tiles.clear();
    for (int c = 0; c < 3; ++c) {
        counts[c] = (int)cls[c].size();
        tiles.insert(tiles.end(), cls[c].begin(), cls[c].end());
    }
}

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return;
        ok = true;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

size_t ncoef(int N) { return N < 1 ? 0 : (size_t)N * (N + 1) * (2 * N + 1) / 6; }

// Clenshaw-Curtis weights on x_k = cos(k pi/n), n = N-1: interpolate at the
// nodes with sum'' a_j T_j (a_j = (2/n) sum''_k g_k cos(j k pi/n)) and
// integrate termwise (int T_j = 2/(1-j^2), j even).
void cc_weights(int N, std::vector<double>& w) {
    const int n = N - 1;
    w.assign(N, 0.0);
    for (int k = 0; k < N; ++k) {
        double s = 0.0;
        for (int j = 0; j <= n; j += 2) {
            const double hj = (j == 0 || j == n) ? 0.5 : 1.0;
            s += hj * (2.0 / (1.0 - (double)j * j)) * cos((double)j * k * M_PI / n);
        }
        const double hk = (k == 0 || k == n) ? 0.5 : 1.0;
        w[k] = (2.0 / n) * hk * s;
    }
}

}  // namespace

struct su2_plan_s {
    int device = 0;
    int B = 0;
    su2_dtype dtype = SU2_C64;
    su2_algo algo = SU2_ALGO_FP32;
    su2_weights weights = SU2_WEIGHTS_CC;
    std::vector<int> Ns;
    std::vector<size_t> grid_off, coeff_off, ws_off;
    size_t grid_total = 0, coeff_total = 0, ws_total = 0;
    std::map<int, Band> bands;
    std::vector<void*> allocs;
    size_t* d_grid_off = nullptr;
    size_t* d_coeff_off = nullptr;
    size_t* d_ws_off = nullptr;
    double* d_lf2 = nullptr;
    int* d_err = nullptr;
    unsigned flags = 0;
    // concurrent bandwidth groups: one stream per group, fork/join events
    std::vector<cudaStream_t> band_streams;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    cudaStream_t cap_stream = nullptr;
    // host-resident batches (su2_forward_pipelined): upload / download streams and hand-off events
    cudaStream_t pipe_up = nullptr, pipe_down = nullptr;
    cudaEvent_t ev_up = nullptr, ev_s1done = nullptr, ev_s2 = nullptr, ev_down = nullptr;
    struct GraphEntry {
        const void* grid;
        void* coeffs;
        void* ws;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;   // most recent last
    // the whole forward as one persistent launch (ragged.cu): every group fits it
    // (rg_ok), su2_forward runs it (rg_use); its counters sit in the workspace
    bool rg_ok = false, rg_use = false;
    std::vector<su2::RaggedBand> rg_bands;
    su2::RaggedBand* d_rg_bands = nullptr;
    int4* d_rg_items = nullptr;
    int rg_nitems = 0, rg_nctr = 0;
    size_t rg_ctr_off = 0;            // in complex elements from the workspace start
    int lf2_len = 0;

    template <typename T>
    cudaError_t upload(T** dst, const T* src, size_t count) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) return e;
        allocs.push_back(p);
        *dst = (T*)p;
        return cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice);
    }
    void release() {
        for (auto& ge : graphs) cudaGraphExecDestroy(ge.exec);
        graphs.clear();
        for (cudaStream_t s : band_streams) cudaStreamDestroy(s);
        band_streams.clear();
        for (cudaEvent_t ev : ev_join) cudaEventDestroy(ev);
        ev_join.clear();
        if (ev_fork) cudaEventDestroy(ev_fork);
        ev_fork = nullptr;
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (cudaStream_t* s : {&pipe_up, &pipe_down})
            if (*s) { cudaStreamDestroy(*s); *s = nullptr; }
        for (cudaEvent_t* ev : {&ev_up, &ev_s1done, &ev_s2, &ev_down})
            if (*ev) { cudaEventDestroy(*ev); *ev = nullptr; }
        cap_stream = nullptr;
        for (void* p : allocs) cudaFree(p);
        allocs.clear();
    }
};

namespace {

su2_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return SU2_OK;
    if (e == cudaErrorMemoryAllocation) return SU2_ERR_OOM;
    return SU2_ERR_CUDA;
}

cudaError_t build_band(su2_plan_s* P, Band& b) {
    const int N = b.N;
    std::vector<double> cosb(N), l2c(N), l2s(N), w;
    std::vector<float> w32(N);
    std::vector<float2> xs(N), om32(N), tw32(N);
    std::vector<double2> om64(N), tw64(N);
    for (int k = 0; k < N; ++k) {
        const double beta = M_PI * k / (N - 1);
        cosb[k] = cos(beta);
        const double ch = cos(beta / 2), sh = sin(beta / 2);
        l2c[k] = (k == N - 1) ? -INFINITY : log2(ch);
        l2s[k] = (k == 0) ? -INFINITY : log2(sh);
        const float hi = (float)cosb[k];
        xs[k] = make_float2(hi, (float)(cosb[k] - (double)hi));
    }
    if (P->weights == SU2_WEIGHTS_CC) {
        cc_weights(N, w);
    } else {
        w.resize(N);
        for (int k = 0; k < N; ++k) w[k] = sin(M_PI * k / (N - 1)) * (M_PI / (N - 1));
    }
    for (int k = 0; k < N; ++k) w32[k] = (float)w[k];
    for (int t = 0; t < N; ++t) {
        const double a = 2.0 * M_PI * t / N, h = M_PI * t / N;
        om64[t] = make_double2(cos(a), sin(a));
        om32[t] = make_float2((float)cos(a), (float)sin(a));
        tw64[t] = make_double2(cos(h), sin(h));
        tw32[t] = make_float2((float)cos(h), (float)sin(h));
    }
    cudaError_t e;
    if ((e = P->upload(&b.d_fidx, b.fids.data(), b.fids.size())) != cudaSuccess) return e;
    if (P->dtype == SU2_C64 && !b.tc && !b.literal) {
        std::vector<int> tiles;
        fp32_tile_classes(N, tiles, b.s2_ntiles);
        if ((e = P->upload(&b.d_s2_tiles, tiles.data(), tiles.size())) != cudaSuccess) return e;
    }
    if ((e = P->upload(&b.d_cosb, cosb.data(), N)) != cudaSuccess) return e;
    if ((e = P->upload(&b.d_log2c, l2c.data(), N)) != cudaSuccess) return e;
    if ((e = P->upload(&b.d_log2s, l2s.data(), N)) != cudaSuccess) return e;
    {
        // split logarithms for the FP32 seed evaluation (exact products with pc, ps < 256)
        std::vector<float4> s32(N);
        auto split = [](double v, float* hi, float* lo) {
            if (!std::isfinite(v)) { *hi = 0.f; *lo = 0.f; return; }   // pole: the seed is 0 there
            const double h = std::rint(v * 2048.0) / 2048.0;
            *hi = (float)h;
            *lo = (float)(v - h);
        };
        for (int k = 0; k < N; ++k) {
            float ch, cl, sh, sl;
            split(l2c[k], &ch, &cl);
            split(l2s[k], &sh, &sl);
            s32[k] = make_float4(ch, cl, sh, sl);
        }
        if ((e = P->upload(&b.d_seed32, s32.data(), N)) != cudaSuccess) return e;
    }
    if ((e = P->upload(&b.d_w64, w.data(), N)) != cudaSuccess) return e;
    if ((e = P->upload(&b.d_w32, w32.data(), N)) != cudaSuccess) return e;
    if ((e = P->upload(&b.d_xsplit, xs.data(), N)) != cudaSuccess) return e;
    if ((e = P->upload(&b.d_om32, om32.data(), N)) != cudaSuccess) return e;
    if ((e = P->upload(&b.d_om64, om64.data(), N)) != cudaSuccess) return e;
    if ((e = P->upload(&b.d_twist32, tw32.data(), N)) != cudaSuccess) return e;
    if ((e = P->upload(&b.d_twist64, tw64.data(), N)) != cudaSuccess) return e;
    if (b.literal && su2::fft_literal_bluestein(N)) {
        // chirps, chirp filter spectrum and twiddles of the Bluestein DFTs
        std::vector<float2> bs;
        su2::fft_literal_bluestein_tables(N, bs);
        if ((e = P->upload(&b.d_lit_bs, bs.data(), bs.size())) != cudaSuccess) return e;
    } else if (b.literal) {
        // (N-1)-point DFT matrix at the output frequencies r - N/2 and the half-bin twist
        const int M = N - 1;
        std::vector<float2> W((size_t)N * N), lt(2 * N);
        for (int r = 0; r < N; ++r)
            for (int t = 0; t < N; ++t) {
                const long q = ((long)(r - N / 2) * t) % M;          // exact phase reduction
                const double a = 2.0 * M_PI * (double)q / M;
                W[(size_t)r * N + t] = t < M ? make_float2((float)cos(a), (float)sin(a)) : make_float2(0.f, 0.f);
            }
        for (int u = 0; u < 2 * N; ++u) {
            const double a = M_PI * u / M;
            lt[u] = make_float2((float)cos(a), (float)sin(a));
        }
        if ((e = P->upload(&b.d_lit_w, W.data(), W.size())) != cudaSuccess) return e;
        if ((e = P->upload(&b.d_lit_twist, lt.data(), lt.size())) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

su2::BandArgs band_args(const su2_plan_s* P, const Band& b) {
    su2::BandArgs a;
    a.N = b.N;
    a.nfunc = (int)b.fids.size();
    a.fidx = b.d_fidx;
    a.grid_off = P->d_grid_off;
    a.coeff_off = P->d_coeff_off;
    a.ws_off = P->d_ws_off;
    a.cosb = b.d_cosb;
    a.log2c = b.d_log2c;
    a.log2s = b.d_log2s;
    a.seed32 = b.d_seed32;
    a.w64 = b.d_w64;
    a.w32 = b.d_w32;
    a.xsplit = b.d_xsplit;
    a.lf2 = P->d_lf2;
    a.om32 = b.d_om32;
    a.om64 = b.d_om64;
    a.twist32 = b.d_twist32;
    a.twist64 = b.d_twist64;
    a.err = P->d_err;
    a.ws_group_off = b.fids.empty() ? 0 : P->ws_off[b.fids[0]];
    a.grid_group_off = b.fids.empty() ? 0 : P->grid_off[b.fids[0]];
    a.grid_regular = 1;
    a.ws_aux_off = b.aux_off;
    a.aux_ring = b.aux_ring;
    a.ws_tile_major = b.tc ? 1 : 0;
    a.s1_two_phase = b.s1_two_phase;
    a.s2_bt = b.s2_bt;
    a.s2_rc = b.s2_rc;
    a.full_group = b.full_group ? 1 : 0;
    a.literal = b.literal ? 1 : 0;
    a.lit_w = b.d_lit_w;
    a.lit_twist = b.d_lit_twist;
    a.lit_bs = b.d_lit_bs;
    a.s2_tiles = b.d_s2_tiles;
    a.nk = b.N;
    a.k_base = 0;
    a.xout = nullptr;
    a.tc_t0 = 0;
    a.tc_ntiles = 0;
    a.xrecv = nullptr;
    a.x_row0 = 0;
    a.x_nrows = 0;
    for (int c = 0; c < 3; ++c) a.s2_ntiles[c] = b.s2_ntiles[c];
    const size_t n3 = (b.full_group ? 2 : 1) * (size_t)b.N * b.N * b.N;   // elements of one grid
    for (size_t i = 0; i < b.fids.size(); ++i)
        if (P->grid_off[b.fids[i]] != a.grid_group_off + i * n3) a.grid_regular = 0;
    return a;
}

// Forward transform of one bandwidth group on one stream.
cudaError_t launch_band_forward(const su2_plan_s* P, const Band& b, const void* grid, void* coeffs, void* ws,
                                cudaStream_t st) {
    const su2::BandArgs a = band_args(P, b);
    const bool fp64 = P->dtype == SU2_C128;
    cudaError_t e = su2::launch_fft_forward(a, fp64, grid, ws, st);
    if (e != cudaSuccess) return e;
    if (b.tc) return su2::launch_contract_forward_tc(a, ws, coeffs, st);
    return su2::launch_contract_forward(a, fp64, ws, coeffs, st);
}

// Every group's forward transform; with several groups they run concurrently
// on the plan's streams, forked from and joined back into `st`.
// The forward transform as one persistent launch over every group (ragged.cu).
cudaError_t launch_ragged_plan(const su2_plan_s* P, const void* grid, void* coeffs, void* ws, cudaStream_t st) {
    const size_t esz = sizeof(float2);
    unsigned* ctr = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + P->rg_ctr_off * esz);
    return su2::launch_ragged(P->rg_bands, P->d_rg_bands, P->d_rg_items, P->rg_nitems, ctr, P->rg_nctr, P->d_lf2,
                              P->lf2_len, P->d_err, grid, ws, coeffs, st);
}

cudaError_t enqueue_forward(su2_plan_s* P, const void* grid, void* coeffs, void* ws, cudaStream_t st) {
    if (P->rg_use) return launch_ragged_plan(P, grid, coeffs, ws, st);
    if (P->band_streams.empty()) {
        for (auto& kv : P->bands) {
            const cudaError_t e = launch_band_forward(P, kv.second, grid, coeffs, ws, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    cudaError_t e = cudaEventRecord(P->ev_fork, st);
    if (e != cudaSuccess) return e;
    size_t i = 0;
    for (auto& kv : P->bands) {
        cudaStream_t bs = P->band_streams[i];
        if ((e = cudaStreamWaitEvent(bs, P->ev_fork, 0)) != cudaSuccess) return e;
        const cudaError_t el = launch_band_forward(P, kv.second, grid, coeffs, ws, bs);
        if ((e = cudaEventRecord(P->ev_join[i], bs)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, P->ev_join[i], 0)) != cudaSuccess) return e;
        if (el != cudaSuccess) return el;
        ++i;
    }
    return cudaSuccess;
}

// Band arguments restricted to functions [f0, f0 + cnt) of the band (contiguous
// grids and planes, so the group offsets are those of function f0).
su2::BandArgs sub_band_args(const su2_plan_s* P, const Band& b, int f0, int cnt) {
    su2::BandArgs a = band_args(P, b);
    a.nfunc = cnt;
    a.fidx = b.d_fidx + f0;
    a.grid_group_off = P->grid_off[b.fids[f0]];
    a.ws_group_off = P->ws_off[b.fids[f0]];
    return a;
}

// Host-resident batch: uploads in chunks of about 1 GiB of grids on pipe_up,
// stage 1 of each chunk on `st` as soon as it has landed, then stage 2 per
// group and the download of its coefficients on pipe_down; `st` finally waits
// for the downloads.  The next call's uploads wait only for this call's
// stage 1 (the last reader of dev_grid), so they overlap this call's stage 2
// and downloads.
cudaError_t forward_pipelined(su2_plan_s* P, const void* hgrid, void* hcoeffs, void* dgrid, void* dcoeffs,
                              void* ws, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (!P->pipe_up) {
        if ((e = cudaStreamCreateWithFlags(&P->pipe_up, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithFlags(&P->pipe_down, cudaStreamNonBlocking)) != cudaSuccess) return e;
        for (cudaEvent_t* ev : {&P->ev_up, &P->ev_s1done, &P->ev_s2, &P->ev_down})
            if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    const bool fp64 = P->dtype == SU2_C128;
    const size_t esz = fp64 ? 16 : 8;
    const char* hg = static_cast<const char*>(hgrid);
    char* dg = static_cast<char*>(dgrid);
    if ((e = cudaStreamWaitEvent(P->pipe_up, P->ev_s1done, 0)) != cudaSuccess) return e;
    for (auto& kv : P->bands) {
        const Band& b = kv.second;
        const size_t N = (size_t)b.N;
        const size_t gbytes = (b.full_group ? 2 : 1) * N * N * N * esz;     // one grid
        const int nf = (int)b.fids.size();
        const int per = (int)std::max<size_t>(1, ((size_t)1 << 30) / gbytes);
        for (int f0 = 0; f0 < nf; f0 += per) {
            const int cnt = std::min(per, nf - f0);
            const size_t off = P->grid_off[b.fids[f0]] * esz;                // grids of a group are contiguous
            if ((e = cudaMemcpyAsync(dg + off, hg + off, (size_t)cnt * gbytes, cudaMemcpyHostToDevice,
                                     P->pipe_up)) != cudaSuccess)
                return e;
            if ((e = cudaEventRecord(P->ev_up, P->pipe_up)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(st, P->ev_up, 0)) != cudaSuccess) return e;
            if ((e = su2::launch_fft_forward(sub_band_args(P, b, f0, cnt), fp64, dgrid, ws, st)) != cudaSuccess)
                return e;
        }
    }
    if ((e = cudaEventRecord(P->ev_s1done, st)) != cudaSuccess) return e;
    const char* dc = static_cast<const char*>(dcoeffs);
    char* hc = static_cast<char*>(hcoeffs);
    for (auto& kv : P->bands) {
        const Band& b = kv.second;
        const su2::BandArgs a = band_args(P, b);
        e = b.tc ? su2::launch_contract_forward_tc(a, ws, dcoeffs, st)
                 : su2::launch_contract_forward(a, fp64, ws, dcoeffs, st);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventRecord(P->ev_s2, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(P->pipe_down, P->ev_s2, 0)) != cudaSuccess) return e;
        const size_t csz = ncoef(b.N) * esz;
        for (size_t i = 0; i < b.fids.size();) {           // runs of adjacent coefficient blocks
            size_t j = i + 1;
            while (j < b.fids.size() && P->coeff_off[b.fids[j]] == P->coeff_off[b.fids[j - 1]] + ncoef(b.N)) ++j;
            const size_t off = P->coeff_off[b.fids[i]] * esz;
            if ((e = cudaMemcpyAsync(hc + off, dc + off, (j - i) * csz, cudaMemcpyDeviceToHost, P->pipe_down)) !=
                cudaSuccess)
                return e;
            i = j;
        }
    }
    if ((e = cudaEventRecord(P->ev_down, P->pipe_down)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(st, P->ev_down, 0);
}

// The forward transform as a CUDA graph recorded once per pointer triple.
cudaError_t forward_graph(su2_plan_s* P, const void* grid, void* coeffs, void* ws, cudaStream_t st) {
    for (size_t i = 0; i < P->graphs.size(); ++i) {
        const auto ge = P->graphs[i];
        if (ge.grid == grid && ge.coeffs == coeffs && ge.ws == ws) {
            P->graphs.erase(P->graphs.begin() + (long)i);
            P->graphs.push_back(ge);
            return cudaGraphLaunch(ge.exec, st);
        }
    }
    cudaError_t e = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t eq = enqueue_forward(P, grid, coeffs, ws, P->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(P->cap_stream, &graph);
    if (eq != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return eq != cudaSuccess ? eq : e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    if (P->graphs.size() >= 8) {
        cudaGraphExecDestroy(P->graphs.front().exec);
        P->graphs.erase(P->graphs.begin());
    }
    P->graphs.push_back({grid, coeffs, ws, exec});
    return cudaGraphLaunch(exec, st);
}

// Autotuner: for each complex64 group, time the candidate kernels on scratch
// buffers holding up to 32 of its functions and keep the fastest.
cudaError_t time_ms(cudaStream_t st, float* ms, const std::function<cudaError_t()>& fn) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
    e = fn();                                            // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

// One group's kernel choice: contraction on tensor cores (tile-major planes) or
// FP32 (plain planes), stage-1 variant, FP32 contraction form.
struct TuneChoice {
    int tc = 0;      // 1: tensor-core contraction
    int s1 = 1;      // 1: two-phase stage 1, 0: DSMEM cluster stage 1
    int rc = 1;      // FP32: 1 row classes, 0 one launch with bt functions per block
    int bt = 16;     // FP32 without row classes: 8 or 16 functions per block
};

// Autotuner cache (SU2_TUNE_CACHE = path of a JSON file): one object per group
// key, {"tc": 0|1, "s1": 0|1, "rc": 0|1, "bt": 8|16}.  Read before tuning, merged
// and rewritten (temporary file + rename) after.
std::map<std::string, TuneChoice> read_tune_cache(const char* path) {
    std::map<std::string, TuneChoice> out;
    FILE* f = path ? fopen(path, "rb") : nullptr;
    if (!f) return out;
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
    fclose(f);
    size_t pos = 0;
    auto read_str = [&](std::string& str) -> bool {
        const size_t a = text.find('"', pos);
        if (a == std::string::npos) return false;
        const size_t b = text.find('"', a + 1);
        if (b == std::string::npos) return false;
        str = text.substr(a + 1, b - a - 1);
        pos = b + 1;
        return true;
    };
    for (;;) {
        std::string key;
        if (!read_str(key)) break;
        const size_t open = text.find('{', pos), close = text.find('}', pos);
        if (open == std::string::npos || close == std::string::npos || open > close) break;
        TuneChoice c;
        const std::string body = text.substr(open + 1, close - open - 1);
        auto field = [&](const char* name, int* v) {
            const size_t q = body.find(std::string("\"") + name + "\"");
            if (q == std::string::npos) return;
            const size_t colon = body.find(':', q);
            if (colon != std::string::npos) *v = atoi(body.c_str() + colon + 1);
        };
        field("tc", &c.tc);
        field("s1", &c.s1);
        field("rc", &c.rc);
        field("bt", &c.bt);
        if (c.bt != 8) c.bt = 16;
        out[key] = c;
        pos = close + 1;
    }
    return out;
}

void write_tune_cache(const char* path, const std::map<std::string, TuneChoice>& m) {
    if (!path) return;
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (const auto& kv : m) {
        fprintf(f, "  \"%s\": {\"tc\": %d, \"s1\": %d, \"rc\": %d, \"bt\": %d}%s\n", kv.first.c_str(), kv.second.tc,
                kv.second.s1, kv.second.rc, kv.second.bt, ++i < m.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

std::string tune_key(const su2_plan_s* P, int N, int nfunc) {
    cudaDeviceProp prop;
    std::string name = "device";
    int sms = 0;
    if (cudaGetDeviceProperties(&prop, P->device) == cudaSuccess) {
        name = prop.name;
        sms = prop.multiProcessorCount;
    }
    for (char& ch : name)
        if (ch == '"' || ch == '\\') ch = '_';
    char k[256];
    snprintf(k, sizeof(k), "%s|sm%d|N%d|nf%d|algo%d|w%d|g%u|v1", name.c_str(), sms, N, nfunc, (int)P->algo,
             (int)P->weights, P->flags & (SU2_FLAG_FULL_GROUP | SU2_FLAG_LITERAL_GRID));
    return k;
}

void apply_choice(Band& b, const TuneChoice& c) {
    b.tc = c.tc != 0;
    b.s1_two_phase = c.s1;
    b.s2_rc = c.rc;
    b.s2_bt = c.bt;
}

// For each complex64 group on the paper's grid: time, on scratch buffers with
// min(group size, 64) functions, stage 1 + stage 2 for every candidate -- the
// tensor-core contraction (tensor-core plans, N = 64..256) and the FP32
// contraction with each stage-1 variant (two-phase; the DSMEM cluster one at
// N = 64, 128) and each FP32 form (row classes; 8 or 16 functions per block) --
// and keep the fastest.  Results do not depend on the choice.
cudaError_t build_ragged(su2_plan_s* P);
cudaError_t autotune_ragged(su2_plan_s* P, std::map<std::string, TuneChoice>& cache, bool* dirty);

cudaError_t autotune(su2_plan_s* P) {
    if (P->dtype != SU2_C64) return cudaSuccess;
    const char* cache_path = getenv("SU2_TUNE_CACHE");
    std::map<std::string, TuneChoice> cache = read_tune_cache(cache_path);
    bool cache_dirty = false;
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    for (auto& kv : P->bands) {
        Band& b = kv.second;
        const int N = kv.first;
        if (b.full_group || b.literal) continue;
        const bool can_tc = b.tc;                       // tensor-core plan and a supported N
        const bool can_s1 = b.aux_ring > 0 && (N == 64 || N == 128);
        const int nb = std::min((int)b.fids.size(), 64);
        const std::string key = tune_key(P, N, (int)b.fids.size());
        auto hit = cache.find(key);
        if (hit != cache.end() && (hit->second.tc == 0 || can_tc) && (hit->second.s1 == 1 ? b.aux_ring > 0 : true)) {
            apply_choice(b, hit->second);
            continue;
        }
        const size_t n3 = (size_t)N * N * N;
        std::vector<int> fidx(nb);
        std::vector<size_t> goff(nb), coff(nb), woff(nb);
        for (int i = 0; i < nb; ++i) {
            fidx[i] = i;
            goff[i] = (size_t)i * n3;
            coff[i] = (size_t)i * ncoef(N);
            woff[i] = (size_t)i * 2 * n3;
        }
        const size_t aux = b.aux_ring > 0 ? (b.aux_ring * 2 * (size_t)N * N + 64 * 32) : 0;
        void *dg = nullptr, *dw = nullptr, *dc = nullptr, *dt = nullptr;
        const size_t tbytes = nb * sizeof(int) + 3 * nb * sizeof(size_t);
        e = cudaMalloc(&dg, nb * n3 * 8);
        if (e == cudaSuccess) e = cudaMalloc(&dw, (nb * 2 * n3 + aux) * 8);
        if (e == cudaSuccess) e = cudaMalloc(&dc, nb * ncoef(N) * 8);
        if (e == cudaSuccess) e = cudaMalloc(&dt, tbytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(dg, 0, nb * n3 * 8, st);
        size_t* dgo = reinterpret_cast<size_t*>(dt);
        size_t* dco = dgo + nb;
        size_t* dwo = dco + nb;
        int* dfi = reinterpret_cast<int*>(dwo + nb);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dgo, goff.data(), nb * sizeof(size_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dco, coff.data(), nb * sizeof(size_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dwo, woff.data(), nb * sizeof(size_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dfi, fidx.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        // the FP32 contraction's row-class tile list, also for tensor-core groups
        if (e == cudaSuccess && !b.d_s2_tiles) {
            std::vector<int> tiles;
            fp32_tile_classes(N, tiles, b.s2_ntiles);
            e = P->upload(&b.d_s2_tiles, tiles.data(), tiles.size());
        }
        su2::BandArgs t = band_args(P, b);
        t.nfunc = nb;
        t.fidx = dfi;
        t.grid_off = dgo;
        t.coeff_off = dco;
        t.ws_off = dwo;
        t.ws_group_off = 0;
        t.grid_group_off = 0;
        t.grid_regular = 1;
        t.ws_aux_off = (size_t)nb * 2 * n3;
        t.s2_tiles = b.d_s2_tiles;
        for (int c = 0; c < 3; ++c) t.s2_ntiles[c] = b.s2_ntiles[c];
        std::vector<TuneChoice> cands;
        if (can_tc) cands.push_back(TuneChoice{1, 1, 1, 16});
        for (int s1 : {1, 0}) {
            if (s1 == 1 && b.aux_ring <= 0) continue;
            if (s1 == 0 && !(can_s1 || b.aux_ring <= 0)) continue;
            if (nb >= 48) cands.push_back(TuneChoice{0, s1, 1, 16});
            cands.push_back(TuneChoice{0, s1, 0, 8});
            cands.push_back(TuneChoice{0, s1, 0, 16});
        }
        TuneChoice best_c;
        float best = 1e30f;
        for (const TuneChoice& c : cands) {
            if (e != cudaSuccess) break;
            su2::BandArgs u = t;
            u.ws_tile_major = c.tc;
            u.s1_two_phase = c.s1;
            u.s2_rc = c.rc;
            u.s2_bt = c.bt;
            float ms = 0.f;
            e = time_ms(st, &ms, [&]() {
                cudaError_t ee = su2::launch_fft_forward(u, false, dg, dw, st);
                if (ee != cudaSuccess) return ee;
                return c.tc ? su2::launch_contract_forward_tc(u, dw, dc, st)
                            : su2::launch_contract_forward(u, false, dw, dc, st);
            });
            if (e == cudaSuccess && ms < best) {
                best = ms;
                best_c = c;
            }
        }
        cudaStreamSynchronize(st);
        if (dg) cudaFree(dg);
        if (dw) cudaFree(dw);
        if (dc) cudaFree(dc);
        if (dt) cudaFree(dt);
        if (e != cudaSuccess) break;
        if (!cands.empty()) {
            apply_choice(b, best_c);
            cache[key] = best_c;
            cache_dirty = true;
        }
    }
    cudaStreamDestroy(st);
    if (e == cudaSuccess && P->rg_ok) e = build_ragged(P);
    if (e == cudaSuccess && P->rg_ok && !(P->flags & SU2_FLAG_PERSISTENT) && P->bands.size() > 1)
        e = autotune_ragged(P, cache, &cache_dirty);
    if (e == cudaSuccess && cache_dirty) write_tune_cache(cache_path, cache);
    return e;
}

// Work list and group table of the persistent launch, from the groups' final
// contraction choices; leaves rg_ok false when a group does not fit it.
cudaError_t build_ragged(su2_plan_s* P) {
    P->rg_bands.clear();
    for (auto& kv : P->bands) {
        su2::RaggedBand rb;
        memset(&rb, 0, sizeof(rb));
        rb.a = band_args(P, kv.second);
        rb.tc = kv.second.tc ? 1 : 0;
        if (!su2::ragged_supported(kv.first, rb.tc != 0)) {
            P->rg_ok = false;
            return cudaSuccess;
        }
        P->rg_bands.push_back(rb);
    }
    std::vector<int4> items;
    su2::ragged_items(P->rg_bands, items, &P->rg_nctr);
    P->rg_nitems = (int)items.size();
    cudaError_t e = P->upload(&P->d_rg_bands, P->rg_bands.data(), P->rg_bands.size());
    if (e == cudaSuccess) e = P->upload(&P->d_rg_items, items.data(), items.size());
    return e;
}

// Persistent launch or one launch pair per group on forked streams: time the
// whole forward both ways on scratch buffers of the plan's size (when they fit
// in half the free memory) and keep the faster.  The cache key is the plan's
// bandwidth multiset.
cudaError_t autotune_ragged(su2_plan_s* P, std::map<std::string, TuneChoice>& cache, bool* dirty) {
    std::string key = tune_key(P, 0, P->B) + "|ragged";
    for (auto& kv : P->bands) key += "|" + std::to_string(kv.first) + "x" + std::to_string(kv.second.fids.size()) +
                                     (kv.second.tc ? "t" : "f");
    auto hit = cache.find(key);
    if (hit != cache.end()) {
        P->rg_use = hit->second.tc != 0;
        return cudaSuccess;
    }
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return e;
    const size_t need = (P->grid_total + P->coeff_total + P->ws_total) * sizeof(float2);
    if (need > free_b / 2) return cudaSuccess;          // keep the default
    void *dg = nullptr, *dc = nullptr, *dw = nullptr;
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&dg, P->grid_total * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&dc, P->coeff_total * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&dw, P->ws_total * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemsetAsync(dg, 0, P->grid_total * sizeof(float2), st);
    float ms[2] = {1e30f, 1e30f};
    for (int use = 0; use < 2 && e == cudaSuccess; ++use) {
        P->rg_use = use != 0;
        e = time_ms(st, &ms[use], [&]() { return enqueue_forward(P, dg, dc, dw, st); });
    }
    if (st) cudaStreamSynchronize(st);
    if (dg) cudaFree(dg);
    if (dc) cudaFree(dc);
    if (dw) cudaFree(dw);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return e;
    P->rg_use = ms[1] < ms[0];
    TuneChoice c;
    c.tc = P->rg_use ? 1 : 0;
    cache[key] = c;
    *dirty = true;
    return cudaSuccess;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

su2_status check_exec(su2_plan_t plan, const void* in, const void* out, const void* ws) {
    if (!plan || !in || !out) return SU2_ERR_INVALID_ARG;
    if (plan->ws_total > 0 && !ws) return SU2_ERR_WORKSPACE;
    if (!aligned16(in) || !aligned16(out) || (ws && !aligned16(ws))) return SU2_ERR_ALIGNMENT;
    return SU2_OK;
}

}  // namespace

namespace su2 {
int forward_direct(su2_plan_s* plan, const void* grid, void* coeffs, void* ws, void* stream) {
    su2_status s = check_exec(plan, grid, coeffs, ws);
    if (s != SU2_OK) return s;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    return from_cuda(enqueue_forward(plan, grid, coeffs, ws, (cudaStream_t)stream));
}
}  // namespace su2

namespace su2 {
int plan_device(const su2_plan_s* plan) { return plan ? plan->device : -1; }
}  // namespace su2

extern "C" {

size_t su2_num_coeffs(int N) { return ncoef(N); }

const char* su2_status_string(su2_status s) {
    switch (s) {
        case SU2_OK: return "ok";
        case SU2_ERR_INVALID_ARG: return "invalid argument";
        case SU2_ERR_UNSUPPORTED: return "unsupported bandwidth or dtype/algo combination";
        case SU2_ERR_OOM: return "device allocation failed";
        case SU2_ERR_CUDA: return "CUDA runtime error";
        case SU2_ERR_TIMEOUT: return "device-side bounded wait expired";
        case SU2_ERR_WORKSPACE: return "workspace missing";
        case SU2_ERR_ALIGNMENT: return "device pointer not 16-byte aligned";
    }
    return "unknown status";
}

su2_status su2_plan(su2_plan_t* out, const su2_plan_desc* desc) {
    if (!out || !desc) return SU2_ERR_INVALID_ARG;
    if (desc->num_functions < 1 ||
        (desc->flags & ~(SU2_FLAG_CUDA_GRAPH | SU2_FLAG_AUTOTUNE | SU2_FLAG_FULL_GROUP | SU2_FLAG_LITERAL_GRID |
                         SU2_FLAG_PERSISTENT)) != 0)
        return SU2_ERR_INVALID_ARG;
    const bool full_group = (desc->flags & SU2_FLAG_FULL_GROUP) != 0;
    const bool literal = (desc->flags & SU2_FLAG_LITERAL_GRID) != 0;
    if (full_group && literal) return SU2_ERR_INVALID_ARG;             // two different grids
    if ((full_group || literal) && desc->dtype != SU2_C64) return SU2_ERR_UNSUPPORTED;
    if (desc->dtype != SU2_C64 && desc->dtype != SU2_C128) return SU2_ERR_INVALID_ARG;
    if (desc->weights != SU2_WEIGHTS_CC && desc->weights != SU2_WEIGHTS_RIEMANN) return SU2_ERR_INVALID_ARG;
    su2_algo algo = desc->algo;
    if (algo == SU2_ALGO_AUTO) algo = (desc->dtype == SU2_C128) ? SU2_ALGO_FP64 : SU2_ALGO_FP32;
    if (algo != SU2_ALGO_FP64 && algo != SU2_ALGO_FP32 && algo != SU2_ALGO_TC_BF16X3) return SU2_ERR_INVALID_ARG;
    if ((algo == SU2_ALGO_FP64) != (desc->dtype == SU2_C128)) return SU2_ERR_UNSUPPORTED;
    const int Nmax_allowed = (desc->dtype == SU2_C128) ? 256 : 512;
    std::vector<int> Ns(desc->num_functions);
    for (int f = 0; f < desc->num_functions; ++f) {
        const int N = desc->N ? desc->N[f] : desc->N_uniform;
        if (!is_pow2(N) || N < 4 || N > Nmax_allowed) return SU2_ERR_UNSUPPORTED;
        if (full_group && (N < 64 || N > 256)) return SU2_ERR_UNSUPPORTED;
        Ns[f] = N;
    }
    // the persistent launch: complex64 on the periodic grid, N = 8..128 (decided
    // here on the host, before any device call; the plan repeats the check below)
    if (desc->flags & SU2_FLAG_PERSISTENT) {
        if (desc->dtype != SU2_C64 || full_group || literal) return SU2_ERR_UNSUPPORTED;
        for (int N : Ns)
            if (!su2::ragged_supported(N, false)) return SU2_ERR_UNSUPPORTED;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SU2_ERR_CUDA;
    if (desc->device < 0 || desc->device >= ndev) return SU2_ERR_INVALID_ARG;
    DeviceGuard g(desc->device);
    if (!g.ok) return SU2_ERR_CUDA;

    // address of the allocation-free entry point's scratch array on this device
    if (su2::noalloc_prepare(desc->device) != cudaSuccess) return SU2_ERR_CUDA;
    su2_plan_s* P = new (std::nothrow) su2_plan_s();
    if (!P) return SU2_ERR_OOM;
    P->device = desc->device;
    P->B = desc->num_functions;
    P->dtype = desc->dtype;
    P->algo = algo;
    P->weights = desc->weights;
    P->flags = desc->flags;
    P->Ns = Ns;
    P->grid_off.resize(P->B);
    P->coeff_off.resize(P->B);
    P->ws_off.resize(P->B);
    int Nmax = 0;
    for (int f = 0; f < P->B; ++f) {
        const size_t N = (size_t)Ns[f];
        P->coeff_off[f] = P->coeff_total;
        P->coeff_total += ncoef((int)N);
        P->bands[(int)N].fids.push_back(f);
        Nmax = std::max(Nmax, (int)N);
    }
    // grids: contiguous per bandwidth group (bands in increasing N, batch order inside)
    for (auto& kv : P->bands) {
        const size_t N = (size_t)kv.first;
        for (int f : kv.second.fids) {
            P->grid_off[f] = P->grid_total;
            P->grid_total += (full_group ? 2 : 1) * N * N * N;
        }
    }
    // stage-1 planes: contiguous per bandwidth group, functions in batch order,
    // so that a group's planes form one regularly strided array
    for (auto& kv : P->bands) {
        const size_t N = (size_t)kv.first;
        for (int f : kv.second.fids) {
            P->ws_off[f] = P->ws_total;
            P->ws_total += 2 * N * N * N;
        }
    }
    // scratch of the two-phase stage-1 DFT (or of the literal-grid DFT), after all planes
    for (auto& kv : P->bands) {
        kv.second.tc = algo == SU2_ALGO_TC_BF16X3 && su2::tc_supported(kv.first);
        if (literal) {
            size_t elems = 0;
            int ctas = 0;
            const cudaError_t ea = su2::fft_forward_literal_aux(kv.first, desc->device, &ctas, &elems);
            if (ea != cudaSuccess) {
                delete P;
                return from_cuda(ea);
            }
            kv.second.literal = true;
            kv.second.aux_off = P->ws_total;
            kv.second.aux_ring = ctas;
            P->ws_total += elems;
            continue;
        }
        // complex64 at N >= 128; the tensor-core path also at N = 64 (its planes are tile-major)
        if (!su2::fft_forward_two_phase_supported(kv.first, desc->dtype == SU2_C128)) continue;
        if (kv.first < 128 && !kv.second.tc && !(desc->flags & SU2_FLAG_AUTOTUNE) && !full_group) continue;
        size_t elems = 0;
        int ring = 0;
        const cudaError_t ea = su2::fft_forward_aux(kv.first, desc->device, full_group, &ring, &elems);
        if (ea != cudaSuccess) {
            delete P;
            return from_cuda(ea);
        }
        kv.second.aux_off = P->ws_total;
        kv.second.aux_ring = ring;
        kv.second.s1_two_phase = (kv.first >= 128 || kv.second.tc || full_group) ? 1 : 0;
        kv.second.full_group = full_group;
        P->ws_total += elems;
    }
    // completion counters of the persistent launch (ragged.cu), sized for the
    // smallest function block any contraction choice uses; only plans that ask
    // for it or may choose it (autotuner) carry them
    P->rg_ok = desc->dtype == SU2_C64 && !full_group && !literal &&
               (desc->flags & (SU2_FLAG_PERSISTENT | SU2_FLAG_AUTOTUNE)) != 0;
    for (auto& kv : P->bands)
        if (!su2::ragged_supported(kv.first, false)) P->rg_ok = false;
    if (P->rg_ok) {
        size_t blocks = 0;
        for (auto& kv : P->bands)
            blocks += (kv.second.fids.size() + su2::ragged_min_block() - 1) / su2::ragged_min_block();
        P->rg_ctr_off = P->ws_total;
        P->ws_total += ((1 + blocks) * sizeof(unsigned) + sizeof(float2) - 1) / sizeof(float2);
    }
    if ((desc->flags & SU2_FLAG_PERSISTENT) && !P->rg_ok) {
        delete P;
        return SU2_ERR_UNSUPPORTED;
    }
    std::vector<double> lf2(2 * Nmax + 2);
    P->lf2_len = (int)lf2.size();
    for (size_t k = 0; k < lf2.size(); ++k) lf2[k] = lgamma((double)k + 1.0) / log(2.0);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = P->upload(&P->d_grid_off, P->grid_off.data(), P->B);
    if (e == cudaSuccess) e = P->upload(&P->d_coeff_off, P->coeff_off.data(), P->B);
    if (e == cudaSuccess) e = P->upload(&P->d_ws_off, P->ws_off.data(), P->B);
    if (e == cudaSuccess) e = P->upload(&P->d_lf2, lf2.data(), lf2.size());
    if (e == cudaSuccess) {
        const int zero[2] = {0, 0};      // error word; a word nothing ever writes (self-test)
        e = P->upload(&P->d_err, zero, 2);
    }
    for (auto& kv : P->bands) {
        if (e != cudaSuccess) break;
        kv.second.N = kv.first;
        e = build_band(P, kv.second);
        if (kv.second.s2_bt == 0) kv.second.s2_bt = kv.second.fids.size() <= 8 ? 8 : 16;
    }
    if (e == cudaSuccess && P->bands.size() > 1) {
        e = cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming);
        for (size_t i = 0; i < P->bands.size() && e == cudaSuccess; ++i) {
            cudaStream_t bs = nullptr;
            cudaEvent_t ev = nullptr;
            e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
            if (e == cudaSuccess) P->band_streams.push_back(bs);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) P->ev_join.push_back(ev);
        }
    }
    if (e == cudaSuccess && (P->flags & SU2_FLAG_CUDA_GRAPH))
        e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && (P->flags & SU2_FLAG_AUTOTUNE)) e = autotune(P);
    else if (e == cudaSuccess && P->rg_ok) e = build_ragged(P);
    if (e == cudaSuccess && (P->flags & SU2_FLAG_PERSISTENT)) {
        if (!P->rg_ok) {
            P->release();
            delete P;
            return SU2_ERR_UNSUPPORTED;
        }
        P->rg_use = true;
    }
    if (e != cudaSuccess) {
        P->release();
        delete P;
        return from_cuda(e);
    }
    *out = P;
    return SU2_OK;
}

su2_status su2_plan_persistent(su2_plan_t plan, int* used) {
    if (!plan || !used) return SU2_ERR_INVALID_ARG;
    *used = plan->rg_use ? 1 : 0;
    return SU2_OK;
}

su2_status su2_workspace_size(su2_plan_t plan, size_t* bytes) {
    if (!plan || !bytes) return SU2_ERR_INVALID_ARG;
    *bytes = plan->ws_total * (plan->dtype == SU2_C128 ? 16 : 8);
    return SU2_OK;
}

su2_status su2_grid_offset(su2_plan_t plan, int f, size_t* elems) {
    if (!plan || !elems || f < 0 || f >= plan->B) return SU2_ERR_INVALID_ARG;
    *elems = plan->grid_off[f];
    return SU2_OK;
}

su2_status su2_coeff_offset(su2_plan_t plan, int f, size_t* elems) {
    if (!plan || !elems || f < 0 || f >= plan->B) return SU2_ERR_INVALID_ARG;
    *elems = plan->coeff_off[f];
    return SU2_OK;
}

su2_status su2_plane_offset(su2_plan_t plan, int f, size_t* elems) {
    if (!plan || !elems || f < 0 || f >= plan->B) return SU2_ERR_INVALID_ARG;
    *elems = plan->ws_off[f];
    return SU2_OK;
}

su2_status su2_grid_elems(su2_plan_t plan, size_t* elems) {
    if (!plan || !elems) return SU2_ERR_INVALID_ARG;
    *elems = plan->grid_total;
    return SU2_OK;
}

su2_status su2_coeff_elems(su2_plan_t plan, size_t* elems) {
    if (!plan || !elems) return SU2_ERR_INVALID_ARG;
    *elems = plan->coeff_total;
    return SU2_OK;
}

su2_status su2_forward(su2_plan_t plan, const void* grid, void* coeffs, void* ws, void* stream) {
    su2_status s = check_exec(plan, grid, coeffs, ws);
    if (s != SU2_OK) return s;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t e = (plan->flags & SU2_FLAG_CUDA_GRAPH) ? forward_graph(plan, grid, coeffs, ws, st)
                                                             : enqueue_forward(plan, grid, coeffs, ws, st);
    return from_cuda(e);
}

su2_status su2_forward_pipelined(su2_plan_t plan, const void* host_grid, void* host_coeffs, void* dev_grid,
                                 void* dev_coeffs, void* ws, void* stream) {
    su2_status s = check_exec(plan, dev_grid, dev_coeffs, ws);
    if (s != SU2_OK) return s;
    if (!host_grid || !host_coeffs) return SU2_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    return from_cuda(forward_pipelined(plan, host_grid, host_coeffs, dev_grid, dev_coeffs, ws, (cudaStream_t)stream));
}

su2_status su2_forward_stage1(su2_plan_t plan, const void* grid, void* ws, void* stream) {
    su2_status s = check_exec(plan, grid, ws ? ws : grid, ws);
    if (s != SU2_OK) return s;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    const bool fp64 = plan->dtype == SU2_C128;
    for (auto& kv : plan->bands) {
        cudaError_t e = su2::launch_fft_forward(band_args(plan, kv.second), fp64, grid, ws, (cudaStream_t)stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return SU2_OK;
}

su2_status su2_forward_stage2(su2_plan_t plan, const void* ws, void* coeffs, void* stream) {
    su2_status s = check_exec(plan, ws ? ws : coeffs, coeffs, ws);
    if (s != SU2_OK) return s;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    const bool fp64 = plan->dtype == SU2_C128;
    for (auto& kv : plan->bands) {
        const su2::BandArgs a = band_args(plan, kv.second);
        cudaError_t e = kv.second.tc
                            ? su2::launch_contract_forward_tc(a, ws, coeffs, (cudaStream_t)stream)
                            : su2::launch_contract_forward(a, fp64, ws, coeffs, (cudaStream_t)stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return SU2_OK;
}

// Sharded transform: the plan must hold one bandwidth group on the tensor-core
// path (complex64, N = 64, 128, 256) on the paper's grid.
static const Band* sharded_band(su2_plan_t plan) {
    if (plan->bands.size() != 1 || plan->dtype != SU2_C64 ||
        (plan->flags & (SU2_FLAG_FULL_GROUP | SU2_FLAG_LITERAL_GRID)))
        return nullptr;
    const Band& b = plan->bands.begin()->second;
    if (!b.tc || b.aux_ring <= 0 || !b.s1_two_phase) return nullptr;
    return &b;
}

su2_status su2_forward_stage1_slab(su2_plan_t plan, int k_base, int nk, const void* grid_slab, void* xplanes,
                                   void* ws, void* stream) {
    su2_status s = check_exec(plan, grid_slab, xplanes, ws);
    if (s != SU2_OK) return s;
    const Band* b = sharded_band(plan);
    if (!b) return SU2_ERR_UNSUPPORTED;
    if (nk < 1 || k_base < 0 || k_base + nk > b->N) return SU2_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    su2::BandArgs a = band_args(plan, *b);
    a.nk = nk;
    a.k_base = k_base;
    a.xout = static_cast<float2*>(xplanes);
    a.grid_group_off = 0;               // the slab is its own buffer: [fb][j1][k][j2], k < nk
    a.grid_regular = 1;
    return from_cuda(su2::launch_fft_forward_two_phase(a, grid_slab, ws, (cudaStream_t)stream));
}

su2_status su2_forward_stage2_rows(su2_plan_t plan, int row0, int nrows, int nk, const void* xrecv, void* coeffs,
                                   void* stream) {
    if (!plan || !xrecv || !coeffs) return SU2_ERR_INVALID_ARG;
    if (!aligned16(xrecv) || !aligned16(coeffs)) return SU2_ERR_ALIGNMENT;    // no workspace is used
    const Band* b = sharded_band(plan);
    if (!b) return SU2_ERR_UNSUPPORTED;
    const int N = b->N;
    if (nk < 16 || nk % 16 || N % nk || row0 < 0 || nrows < 1 || row0 + nrows > 2 * N) return SU2_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    su2::BandArgs a = band_args(plan, *b);
    a.xrecv = static_cast<const float2*>(xrecv);
    a.nk = nk;
    a.x_row0 = row0;
    a.x_nrows = nrows;
    a.tc_t0 = row0 * (N / 4);           // the tiles of those rows (4 consecutive n each)
    a.tc_ntiles = nrows * (N / 4);
    return from_cuda(su2::launch_contract_forward_tc(a, nullptr, coeffs, (cudaStream_t)stream));
}

su2_status su2_forward_stage2_depth(su2_plan_t plan, int depth, const void* ws, void* coeffs, void* stream) {
    su2_status s = check_exec(plan, ws ? ws : coeffs, coeffs, ws);
    if (s != SU2_OK) return s;
    if (depth < 1 || depth > 5) return SU2_ERR_INVALID_ARG;
    if (plan->dtype != SU2_C128 || (plan->flags & (SU2_FLAG_FULL_GROUP | SU2_FLAG_LITERAL_GRID)))
        return SU2_ERR_UNSUPPORTED;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    for (auto& kv : plan->bands) {
        const su2::BandArgs a = band_args(plan, kv.second);
        const cudaError_t e = su2::launch_contract_forward_depth(a, depth, ws, coeffs, (cudaStream_t)stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return SU2_OK;
}

static su2_status run_transpose(su2_plan_t plan, su2::TransposeMode mode, const void* coeffs, void* grid,
                                void* ws, void* stream) {
    su2_status s = check_exec(plan, coeffs, grid, ws);
    if (s != SU2_OK) return s;
    if (plan->flags & SU2_FLAG_LITERAL_GRID)                               // printed grid: N >= 64
        for (const auto& kv : plan->bands)
            if (!su2::fft_literal_bluestein(kv.first)) return SU2_ERR_UNSUPPORTED;
    if (plan->flags & SU2_FLAG_FULL_GROUP)                                 // full group: N = 128, 256
        for (const auto& kv : plan->bands)
            if ((kv.first != 128 && kv.first != 256) || kv.second.aux_ring <= 0) return SU2_ERR_UNSUPPORTED;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const bool fp64 = plan->dtype == SU2_C128;
    for (auto& kv : plan->bands) {
        su2::BandArgs a = band_args(plan, kv.second);
        a.ws_tile_major = fp64 ? 0 : 1;      // complex64 synthesis planes are tile-major
        cudaError_t e = su2::launch_contract_transpose(a, fp64, mode, coeffs, ws, st);
        if (e == cudaSuccess) e = su2::launch_fft_inverse(a, fp64, ws, grid, st);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return SU2_OK;
}

su2_status su2_inverse(su2_plan_t plan, const void* coeffs, void* grid, void* ws, void* stream) {
    return run_transpose(plan, su2::TransposeMode::Synthesis, coeffs, grid, ws, stream);
}

su2_status su2_backward(su2_plan_t plan, const void* grad_coeffs, void* grad_grid, void* ws, void* stream) {
    return run_transpose(plan, su2::TransposeMode::Adjoint, grad_coeffs, grad_grid, ws, stream);
}

su2_status su2_sync_status(su2_plan_t plan, void* stream) {
    if (!plan) return SU2_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return SU2_ERR_CUDA;
    int err = 0;
    e = cudaMemcpy(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return SU2_ERR_CUDA;
    if (err != 0) {
        const int zero = 0;
        cudaMemcpy(plan->d_err, &zero, sizeof(int), cudaMemcpyHostToDevice);
        return SU2_ERR_TIMEOUT;
    }
    return SU2_OK;
}

su2_status su2_selftest_bounded_wait(su2_plan_t plan, int kind, void* stream) {
    if (!plan || (kind != 0 && kind != 1)) return SU2_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return SU2_ERR_CUDA;
    const unsigned* never = reinterpret_cast<const unsigned*>(plan->d_err + 1);
    return from_cuda(su2::launch_bounded_wait_selftest(never, plan->d_err, kind, (cudaStream_t)stream));
}

su2_status su2_destroy(su2_plan_t plan) {
    if (!plan) return SU2_ERR_INVALID_ARG;
    {
        DeviceGuard g(plan->device);
        plan->release();
    }
    delete plan;
    return SU2_OK;
}

}  // extern "C"

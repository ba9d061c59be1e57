// Internal declarations shared by the C-ABI implementation and the kernel files.
#pragma once

#include <cuda_runtime.h>

#include <cuda.h>

#include <vector>

#include "common.cuh"

struct su2_plan_s;

namespace su2 {

// Stage 1: 2-D DFT over (alpha, gamma) for every beta node (forward), and the
// inverse torus synthesis.  `fp64` selects complex128 data.
cudaError_t launch_fft_forward(const BandArgs& a, bool fp64, const void* grid, void* ws, cudaStream_t st);
// Two-phase complex64 forward DFT (N = 64, 128, 256, 512): its scratch ring
// (plane slots and size in complex elements, for the plan's workspace) and launch.
bool fft_forward_two_phase_supported(int N, bool fp64);
cudaError_t fft_forward_aux(int N, int device, bool full_group, int* ring, size_t* elems);
cudaError_t launch_fft_forward_two_phase(const BandArgs& a, const void* grid, void* ws, cudaStream_t st);
// Complex64 forward DFT on the printed grid (endpoint folded, (N-1)-point DFTs as
// dense products): CTAs and per-CTA scratch (complex elements), and launch.
cudaError_t fft_forward_literal_aux(int N, int device, int* ctas, size_t* elems);
// N >= 64 on the printed grid: Bluestein (chirp-z) DFTs; their host-made tables.
bool fft_literal_bluestein(int N);
void fft_literal_bluestein_tables(int N, std::vector<float2>& out);
cudaError_t launch_fft_forward_literal(const BandArgs& a, const void* grid, void* ws, cudaStream_t st);
// Synthesis / adjoint grid from the tile-major planes on the printed grid (N >= 64).
cudaError_t launch_fft_inverse_literal(const BandArgs& a, const void* ws, void* grid, cudaStream_t st);
// Two-phase complex64 inverse DFT (N = 128, 256, 512) over the tile-major
// planes, using the forward's scratch ring.
bool fft_inverse_two_phase_supported(int N, bool fp64);
cudaError_t launch_fft_inverse_two_phase(const BandArgs& a, const void* ws, void* grid, cudaStream_t st);
cudaError_t launch_fft_inverse(const BandArgs& a, bool fp64, const void* ws, void* grid, cudaStream_t st);

// One-block kernel whose bounded wait (kind 0: counter, 1: mbarrier) never
// completes: it latches *err after about a second and returns.
cudaError_t launch_bounded_wait_selftest(const unsigned* never, int* err, int kind, cudaStream_t st);

// Stage 2: beta contraction with the recurrence fused in (forward), and the
// transposed contraction (synthesis with weight 2l+1, or adjoint with weight
// w_k/(2N^2)).
cudaError_t launch_contract_forward(const BandArgs& a, bool fp64, const void* ws, void* coeffs, cudaStream_t st);
// The same contraction by the depth-k divide-and-conquer projection (complex128
// planes, N <= 256, depth 1..5).
cudaError_t launch_contract_forward_depth(const BandArgs& a, int depth, const void* ws, void* coeffs,
                                          cudaStream_t st);
enum class TransposeMode { Synthesis = 0, Adjoint = 1 };
cudaError_t launch_contract_transpose(const BandArgs& a, bool fp64, TransposeMode mode, const void* coeffs,
                                      void* ws, cudaStream_t st);

// Stage 2 on tensor cores (split-BF16 operands, FP32 accumulation).
cudaError_t launch_contract_forward_tc(const BandArgs& a, const void* ws, void* coeffs, cudaStream_t st);
bool tc_supported(int N);

// Encodes a tiled TMA descriptor over 8-byte elements (no swizzle, zero fill);
// false if the driver entry point is unavailable or the arguments are rejected.
bool encode_tensor_map_8b(CUtensorMap* map, int rank, const void* base, const cuuint64_t* dims,
                          const cuuint64_t* strides_bytes, const cuuint32_t* box);

// One bandwidth group of the ragged-batch kernel (one persistent launch over
// every group; ragged.cu).
struct RaggedBand {
    BandArgs a;          // the group's arguments (tables, offsets, plane layout)
    int tc;              // 1: contraction on tensor cores (tile-major planes)
    int fblk;            // functions per block (completion counters, contraction items)
    int nblk;            // blocks of the group
    int s1pf;            // stage-1 items per function
    int cbase;           // first completion counter of the group's blocks
    int tcmap;           // tensor map of the group's planes (tensor-core groups), else -1
    int tab;             // first entry of the group's node tables in shared memory
    // stage-1 items of block bb (functions bb*fblk .. min(nfunc, (bb+1)*fblk) - 1)
    __host__ __device__ int s1_per_block(int bb) const {
        const int rest = a.nfunc - bb * fblk;
        return (rest < fblk ? rest : fblk) * s1pf;
    }
};
// Bandwidths the ragged kernel takes (tensor-core groups: 64 and 128).
bool ragged_supported(int N, bool tc);
// Functions per block of a group, and the smallest over all groups (for sizing
// the completion counters before the contraction choice is final).
int ragged_block(int N, bool tc);
int ragged_min_block();
// Fills cbase, fblk, nblk, s1pf, tcmap, tab of the groups and builds the work
// list; *nctr = counters the launch uses (item counter + one per block).
void ragged_items(std::vector<RaggedBand>& bands, std::vector<int4>& items, int* nctr);
// The launch: zeroes the nctr counters at ctr (in the workspace), encodes the
// tensor maps of the tensor-core groups' planes, and runs the kernel on `st`.
cudaError_t launch_ragged(const std::vector<RaggedBand>& hb, const RaggedBand* d_bands, const int4* d_items,
                          int nitems, unsigned* ctr, int nctr, const double* lf2, int lf2_len, int* err,
                          const void* grid, void* ws, void* coeffs, cudaStream_t st);

// Device ordinal a plan's tables live on.
int plan_device(const su2_plan_s* plan);
// su2_forward's checks and launches, always enqueued launch by launch (never
// recorded into a CUDA graph, whatever the plan's flags); returns an su2_status.
int forward_direct(su2_plan_s* plan, const void* grid, void* coeffs, void* ws, void* stream);
// Looks up, with `device` current, the device address of the allocation-free
// entry point's scratch array and caches it for that device (the lookup loads
// the module holding the array under lazy module loading, so it is done at
// plan creation, which allocates anyway).  Idempotent.
cudaError_t noalloc_prepare(int device);

}  // namespace su2

/*
 * su2fft.h -- C ABI of the GB300 (sm_103a) Fourier transform on SU(2).
 *
 * The transform follows Delgado & Umana, "On The Fast Fourier Transform on
 * SU(2)":
 *
 *   analysis (Sec. 3, Definition of the Fourier transform; Sec. 4, Euler-angle
 *   integral with the normalised Haar measure 1/(8 pi^2)):
 *       f^(l)_{mn} = <f, t^l_{nm}>,   t^l_{nm} = e^{-i(n alpha + m gamma)} P^l_{nm}(cos beta)
 *   on the sampling grid of Sec. 4 (Definition of the sampling grid),
 *       alpha_j = gamma_j = -pi + 2 pi j / N,  beta_k = k pi / (N - 1),  j, k = 0..N-1,
 *   evaluated by the two-stage split of Sec. 4 (Proposition on the factorised
 *   Riemann sum) and Sec. 6 (first- and second-stage Propositions, depth k = 1):
 *     stage 1: for every beta_k a 2-D DFT over (alpha, gamma) -> f_2(beta_k; m, n);
 *     stage 2: per (m, n) the beta contraction <s, P^l_{nm}> with the Wigner-d
 *              values regenerated by their three-term recurrence in l (Sec. 4
 *              Lemma for m = n = 0; Jacobi analogue for general m, n).
 *   Discrete form computed (exactly, up to rounding):
 *       f^(l)_{mn} = 1/(2N^2) sum_{j1,k,j2} w_k f[j1,k,j2] conj(t^l_{nm}(alpha_j1, beta_k, gamma_j2))
 *   with w_k the Clenshaw-Curtis weights on x_k = cos(beta_k) (default) or the
 *   paper-literal Riemann weights sin(beta_k) pi/(N-1).
 *
 *   synthesis (Sec. 3, Peter-Weyl expansion):
 *       f = sum_l (2l+1) sum_{m,n} f^(l)_{mn} t^l_{nm}
 *   backward (adjoint of the analysis map, used for gradients):
 *       g_grid[j1,k,j2] = w_k/(2N^2) sum_{l,m,n} t^l_{nm}(j1,k,j2) g^(l)_{mn}
 *
 * Index domain (Sec. 3, Definition of t^l): l in {0, 1/2, 1, ...}, -l <= m, n <= l,
 * l - m and l - n integers.  For bandwidth N the coefficients cover 2l = 0..N-1.
 *
 * Layouts (all complex numbers interleaved (re, im); c64 = 2 x float32,
 * c128 = 2 x float64):
 *   grid   : per function f[j1][k][j2], N^3 elements, j2 fastest;
 *            function f starts at element su2_grid_offset(plan, f).
 *   coeffs : per function, blocks j = 2l = 0..N-1; block j is the (j+1)x(j+1)
 *            matrix f^(l) stored row-major with row m+l and column n+l, starting
 *            at element j(j+1)(2j+1)/6; N(N+1)(2N+1)/6 elements per function;
 *            function f starts at su2_coeff_offset(plan, f).
 *
 * Ownership: every pointer passed to su2_forward / su2_inverse / su2_backward
 * is caller-owned DEVICE memory (the grid, the coefficients and the
 * workspace), 16-byte aligned.  A plan owns only small device tables it
 * allocates in su2_plan and frees in su2_destroy.  Execution calls allocate
 * nothing, never modify their inputs, and are asynchronous on the given CUDA
 * stream (NULL = legacy default stream).
 *
 * Errors: every call returns a su2_status; nothing throws across the ABI.
 * Argument errors are detected on the host before any launch.  Device-side
 * errors (a bounded wait that expired) are latched in a per-plan error word
 * and reported by su2_sync_status.
 */
#ifndef SU2FFT_H
#define SU2FFT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct su2_plan_s* su2_plan_t;

typedef enum {
    SU2_OK = 0,
    SU2_ERR_INVALID_ARG = 1,   /* null pointer, bad enum, bad batch size    */
    SU2_ERR_UNSUPPORTED = 2,   /* bandwidth or dtype/algo combination       */
    SU2_ERR_OOM = 3,           /* plan-table allocation failed              */
    SU2_ERR_CUDA = 4,          /* a CUDA runtime call failed                */
    SU2_ERR_TIMEOUT = 5,       /* a device-side bounded wait expired        */
    SU2_ERR_WORKSPACE = 6,     /* workspace pointer null while size > 0     */
    SU2_ERR_ALIGNMENT = 7      /* a device pointer is not 16-byte aligned   */
} su2_status;

typedef enum { SU2_C64 = 0, SU2_C128 = 1 } su2_dtype;

typedef enum {
    SU2_ALGO_AUTO = 0,         /* FP64 for c128; FP32 for c64                     */
    SU2_ALGO_FP64 = 1,         /* c128 only: FP64 DFT, FP64 recurrence/contraction */
    SU2_ALGO_FP32 = 2,         /* c64: FP32 DFT, FP32 recurrence, FP32 FMA contraction */
    SU2_ALGO_TC_BF16X3 = 3     /* c64: FP32 DFT, contraction on tensor cores with
                                  split-BF16 operands (3 products), FP32 accumulate,
                                  for N = 64, 128, 256; functions of other
                                  bandwidths in the plan take the FP32 path */
} su2_algo;

typedef enum {
    SU2_WEIGHTS_CC = 0,        /* Clenshaw-Curtis on cos(beta_k): exact per sector */
    SU2_WEIGHTS_RIEMANN = 1    /* paper-literal sin(beta_k) * pi/(N-1)            */
} su2_weights;

typedef struct {
    int num_functions;   /* batch size, >= 1                                     */
    const int* N;        /* host array [num_functions] of bandwidths, or NULL    */
    int N_uniform;       /* bandwidth of every function when N == NULL           */
    su2_dtype dtype;
    su2_algo algo;
    su2_weights weights;
    unsigned flags;      /* SU2_FLAG_* bits below, others must be 0               */
    int device;          /* CUDA device ordinal the plan's tables live on        */
} su2_plan_desc;

/* Plan flags (library services; the paper has no counterpart).
 * SU2_FLAG_CUDA_GRAPH: su2_forward records the whole forward transform (every
 *   bandwidth group, groups running concurrently) once per (grid, coeffs, ws)
 *   pointer triple into a CUDA graph owned by the plan and afterwards replays
 *   it with one graph launch on the caller's stream.  The plan keeps the 8
 *   most recent graphs.  The first call with new pointers must not itself be
 *   made during a stream capture.
 * SU2_FLAG_AUTOTUNE: su2_plan times, for every complex64 bandwidth group on
 *   the periodic grid, stage 1 + stage 2 of each candidate on scratch buffers
 *   it allocates and frees (min(group size, 64) functions) and keeps the
 *   fastest: the tensor-core contraction (SU2_ALGO_TC_BF16X3 plans, N = 64..256)
 *   or the FP32 one, the stage-1 variant (two-phase, or the DSMEM cluster one
 *   at N = 64, 128), and the FP32 contraction's form (row classes, or 8 or 16
 *   functions per block).  A group that ends on the FP32 contraction keeps its
 *   stage-1 planes in the plain layout (su2_plane_offset).  With the
 *   environment variable SU2_TUNE_CACHE set to a file path, choices are read
 *   from that JSON file (keyed by device name, SM count, N, group size,
 *   algorithm, weights, grid) and new ones are added to it.  Results do not
 *   depend on the choice beyond rounding of the contraction arithmetic. */
#define SU2_FLAG_CUDA_GRAPH 0x1u
#define SU2_FLAG_AUTOTUNE 0x2u
/* SU2_FLAG_FULL_GROUP: grids are sampled on the full group, psi (gamma) over
 * [-2 pi, 2 pi) with 2N nodes psi_j = -2 pi + 2 pi j/N, so a grid is
 * f[j1][k][j2] with j2 < 2N (2 N^3 elements per function), and the forward
 * transform uses the normalised Haar measure of all of SU(2), prefactor
 * 1/(4N^2).  On the paper's domain (Sec. 4, psi over [-pi, pi]) the integer-l
 * and half-integer-l sectors are not orthogonal; on the full group they are,
 * and a band-limited function mixing both sectors is recovered exactly.
 * complex64, N = 64, 128, 256; su2_inverse and su2_backward (adjoint prefactor
 * 1/(4N^2)) for plans whose bandwidths are all 128 or 256, else
 * SU2_ERR_UNSUPPORTED. */
#define SU2_FLAG_FULL_GROUP 0x4u
/* SU2_FLAG_LITERAL_GRID: grids are sampled on the grid as Sec. 4 prints it,
 * alpha_j = gamma_j = -pi + 2 pi j/(N-1), j = 0..N-1 (the last node, +pi,
 * repeats the first), beta_k unchanged; the forward transform carries the cell
 * (2 pi/(N-1))^2, prefactor 1/(2(N-1)^2).  Grids keep the N^3 layout.  The
 * repeated node is folded onto the first; for N >= 64 the (N-1)-point DFTs are
 * taken by Bluestein's chirp-z convolution (O(N^3 log N) per function), below
 * as dense products.  complex64, any supported N for the forward transform;
 * su2_inverse and su2_backward (synthesis and adjoint at every printed node,
 * the repeated ones included; adjoint prefactor 1/(2(N-1)^2)) for plans whose
 * bandwidths are all >= 64, else SU2_ERR_UNSUPPORTED; combined with
 * SU2_FLAG_FULL_GROUP it is SU2_ERR_INVALID_ARG. */
#define SU2_FLAG_LITERAL_GRID 0x8u
/* SU2_FLAG_PERSISTENT: su2_forward runs the whole forward transform of every
 * function (stage 1 and stage 2 of Sec. 6, every bandwidth group) as one
 * persistent kernel launch (after a memset of its counters in the workspace):
 * one thread block per SM takes items in order from a work list (stage-1 DFTs
 * of a few beta planes of one function, then FP32 contraction tiles, then
 * tensor-core contraction tiles); a contraction item waits, with a bounded
 * spin that latches SU2_ERR_TIMEOUT, until the stage-1 items of its block of
 * functions are done.  Only for complex64 plans on the periodic grid whose
 * bandwidths are all in {8, 16, 32, 64, 128} (tensor-core groups: 64, 128),
 * else su2_plan returns SU2_ERR_UNSUPPORTED.  Without this flag, a plan that
 * qualifies and is created with SU2_FLAG_AUTOTUNE times the whole forward
 * both ways (on scratch buffers of its size, when they fit in half the free
 * device memory) and keeps the faster; other plans launch each group's two
 * stages separately.  su2_forward_stage1 / su2_forward_stage2 and
 * su2_forward_pipelined always run per group. */
#define SU2_FLAG_PERSISTENT 0x10u

/* Supported bandwidths: N a power of two with 4 <= N <= 512 (c64) and
 * 4 <= N <= 256 (c128).  Anything else returns SU2_ERR_UNSUPPORTED. */

/* Creates a plan: validates the descriptor, uploads the beta nodes, weights,
 * half-angle logarithms, log-factorials and DFT twiddles for every distinct
 * bandwidth.  *out is set only on SU2_OK. */
su2_status su2_plan(su2_plan_t* out, const su2_plan_desc* desc);

/* Bytes of device workspace that su2_forward / su2_inverse / su2_backward
 * need: the stage-1 planes of every function (2 N^3 complex each), followed,
 * for complex64 bandwidths N = 128, 256, 512, by scratch of the forward 2-D DFT
 * (a ring of intermediate planes and its counters; tens of MB per bandwidth),
 * and, for plans created with SU2_FLAG_PERSISTENT or SU2_FLAG_AUTOTUNE whose
 * bandwidths qualify for the persistent launch, that launch's counters (a few
 * bytes per 32 functions).
 * The content is undefined between calls and needs no initialisation. */
su2_status su2_workspace_size(su2_plan_t plan, size_t* bytes);
/* *used = 1 when su2_forward runs the persistent launch of SU2_FLAG_PERSISTENT
 * (set by that flag or chosen by SU2_FLAG_AUTOTUNE), else 0. */
su2_status su2_plan_persistent(su2_plan_t plan, int* used);
/* (The environment variable SU2_STAGE1_MAX_CTAS, if set to n >= 1, caps the
 * grid of that forward 2-D DFT at n thread blocks; it exists to check that the
 * kernel completes with any number of resident blocks.  Results do not change.) */

/* Element offset of function f's stage-1 planes in the workspace.  Plane
 * (k, s) of f (beta node k; s = 0: integer l, s = 1: half-integer l) starts at
 * that offset + (2k + s) N^2 and is stored row-major [mi][ni] (ni fastest):
 *   F2_s[k][m][n] = w_k/(2N^2) sum_{j1,j2} f[j1,k,j2] e^{i(n alpha_j1 + m gamma_j2)}
 * with mi = m + N/2, ni = n + N/2 for s = 0 (row and column 0 unused, zero)
 * and mi = m - 1/2 + N/2, ni = n - 1/2 + N/2 for s = 1 (Sec. 6 first-stage
 * Proposition; Sec. 4 grid).  Plans of algorithm SU2_ALGO_TC_BF16X3 store the
 * same values tile-major instead (except groups the autotuner moved to the
 * FP32 contraction): element (k, s, mi, ni) at that offset +
 * s N^3 + mi N^2 + (ni / 4) 4N + 4k + ni % 4 (four consecutive n of all beta
 * nodes contiguous, the operand tiles of the tensor-core contraction). */
su2_status su2_plane_offset(su2_plan_t plan, int f, size_t* elems);

/* Element offsets of function f inside the grid and coefficient buffers.
 * Grids are grouped by bandwidth (increasing N; batch order inside a group), so
 * each group is one regularly strided array; coefficients follow batch order.
 * For a uniform batch both are simply f * N^3 and f * su2_num_coeffs(N). */
su2_status su2_grid_offset(su2_plan_t plan, int f, size_t* elems);
su2_status su2_coeff_offset(su2_plan_t plan, int f, size_t* elems);
/* Total elements of the grid and coefficient buffers for the whole batch. */
su2_status su2_grid_elems(su2_plan_t plan, size_t* elems);
su2_status su2_coeff_elems(su2_plan_t plan, size_t* elems);

/* N(N+1)(2N+1)/6: coefficients of one function of bandwidth N (0 if N < 1). */
size_t su2_num_coeffs(int N);

/* Analysis: grid -> coeffs (Sec. 4 two-stage split).  ws: >= su2_workspace_size. */
su2_status su2_forward(su2_plan_t plan, const void* grid, void* coeffs, void* ws,
                       void* cuda_stream);

/* The two stages of su2_forward, for callers that time or reuse them
 * separately.  Stage 1 (Sec. 6 first-stage Proposition): grid -> stage-1 planes
 * in ws (2-D DFT over alpha, gamma for every beta node, weights folded in).
 * Stage 2 (Sec. 6 second-stage Proposition, depth 1): planes in ws -> coeffs
 * (beta contraction with the Wigner-d recurrence fused in).  Running stage 1
 * then stage 2 on the same stream is exactly su2_forward. */
su2_status su2_forward_stage1(su2_plan_t plan, const void* grid, void* ws, void* cuda_stream);
su2_status su2_forward_stage2(su2_plan_t plan, const void* ws, void* coeffs, void* cuda_stream);

/* Stage 2 by the divide-and-conquer projection of Sec. 4 (Theorem
 * "Divide-and-conquer" with the composition Proposition) at recursion depth
 * k = depth, 1 <= depth <= 5.  Per pair (n, m): l = mu, mu + 1 directly; from
 * the base L = mu + 1, every l = L + r is the sum of the Theorem's 2^k inner
 * products <s^L or s^{L-1}, V>, V a Hadamard product of k shifted polynomials
 * (for m, n != 0 those of the Wigner recurrence, the analogue the end of
 * Sec. 4 states), the shift r split into its digits in base b, b the smallest
 * base with b^k > R.  The result equals su2_forward_stage2's up to rounding;
 * the cost grows as 2^k inner products per coefficient (Sec. 6, Proposition
 * "Second Stage Complexity"; Theorem "optimal k" picks k = 1, which
 * su2_forward_stage2 computes with one inner product per coefficient), so
 * this entry point is for measuring that cost, not for speed.
 *   ws:     workspace holding the stage-1 planes (su2_forward_stage1);
 *   coeffs: output, layout as su2_forward.
 * complex128 plans on the periodic grid only (FP64 arithmetic: the shifted
 * polynomials and the seeds span more range than FP32 holds); other plans
 * return SU2_ERR_UNSUPPORTED, depth outside 1..5 SU2_ERR_INVALID_ARG. */
su2_status su2_forward_stage2_depth(su2_plan_t plan, int depth, const void* ws, void* coeffs,
                                    void* cuda_stream);

/* Sharded forward transform (a service of this library; the paper's Sec. 6
 * Propositions make stage 1 independent per beta node and stage 2 independent
 * per (m, n) pair, so a transform can be split over R GPUs with one exchange of
 * the stage-1 planes between the two stages).  Rank r computes stage 1 for its
 * beta nodes k in [k_base, k_base + nk), sends each rank the rows (s, m) that
 * rank owns, and computes stage 2 for its own rows from what it received; the
 * coefficients of all ranks together are su2_forward's (bit for bit: every
 * plane value and every contraction is computed exactly as there).
 *
 * Both calls need a plan with one bandwidth N in {64, 128, 256}, complex64,
 * algorithm SU2_ALGO_TC_BF16X3, on the periodic grid (else SU2_ERR_UNSUPPORTED).
 * Row index: row = s N + mi, s the sector (0: integer l, 1: half-integer l) and
 * mi = m + N/2 (s = 0) or m - 1/2 + N/2 (s = 1), 0 <= row < 2N.
 *
 * su2_forward_stage1_slab: stage 1 for beta nodes [k_base, k_base + nk) of every
 * function of the plan.
 *   grid_slab: device, [nfunc][N (alpha)][nk (beta)][N (gamma)] complex64, the
 *              grids restricted to those nodes;
 *   xplanes:   device, output, the exchange layout [2N (row)][nfunc][N/4][nk][4]:
 *              element (row, f, n/4, k - k_base, n % 4) is F2_s[k][m][n] of
 *              function f (same values as su2_plane_offset describes), so the rows
 *              owned by one rank are one contiguous range;
 *   ws:        the plan's workspace (its stage-1 scratch is used).
 *   0 <= k_base, 1 <= nk, k_base + nk <= N, else SU2_ERR_INVALID_ARG.
 *
 * su2_forward_stage2_rows: stage 2 for rows [row0, row0 + nrows).
 *   xrecv:  device, [N/nk (source)][nrows][nfunc][N/4][nk][4] complex64: block q
 *           is the part of source q's xplanes (beta nodes [q nk, q nk + nk)) for
 *           these rows;
 *   coeffs: device, su2_coeff_elems elements; exactly the coefficients f^(l)_{mn}
 *           of the rows' (s, m) are written (the rest is left as it is).
 *   16 <= nk, nk % 16 == 0, N % nk == 0, 0 <= row0, 1 <= nrows,
 *   row0 + nrows <= 2N, else SU2_ERR_INVALID_ARG.  No workspace. */
su2_status su2_forward_stage1_slab(su2_plan_t plan, int k_base, int nk, const void* grid_slab, void* xplanes,
                                   void* ws, void* cuda_stream);
su2_status su2_forward_stage2_rows(su2_plan_t plan, int row0, int nrows, int nk, const void* xrecv, void* coeffs,
                                   void* cuda_stream);

/* Synthesis: coeffs -> grid (Sec. 3 expansion with the (2l+1) factor). */
su2_status su2_inverse(su2_plan_t plan, const void* coeffs, void* grid, void* ws,
                       void* cuda_stream);

/* Adjoint of su2_forward: grad_coeffs -> grad_grid (conjugate transpose of the
 * analysis map; for a real loss this is the PyTorch gradient convention). */
su2_status su2_backward(su2_plan_t plan, const void* grad_coeffs, void* grad_grid,
                        void* ws, void* cuda_stream);

/* Allocation-free forward transform (no counterpart in the paper; a service of
 * this library).  Same result as su2_forward, but the stage-1 planes go to a
 * scratch array of SU2_NOALLOC_SCRATCH_BYTES (4 MiB) that this library keeps on
 * every GPU that loads it, for the whole process lifetime, so callers that
 * cannot allocate device memory at transform time need no workspace.
 *  - Plans whose su2_workspace_size exceeds SU2_NOALLOC_SCRATCH_BYTES are
 *    rejected with SU2_ERR_WORKSPACE (e.g. c64: one function up to N = 64).
 *  - No cudaMalloc / cudaFree or other allocation happens in this call; a plan
 *    created with SU2_FLAG_CUDA_GRAPH runs its kernels launch by launch here,
 *    since recording and instantiating a graph would allocate.
 *  - su2_plan (which allocates anyway) looks up the array's device address on
 *    the plan's device (cudaGetSymbolAddress, which under CUDA's lazy module
 *    loading loads the array onto the device) and caches it; this call only
 *    reads that cache.
 *  - Under lazy module loading (CUDA's default) the first launch of each
 *    kernel in the process also loads that kernel's code onto the device.
 *    Callers that may not allocate at all at transform time make one call with
 *    the plan beforehand (this entry point or su2_forward), or run with
 *    CUDA_MODULE_LOADING=EAGER, which loads everything when the context is
 *    created.
 *  - All calls on a device share the one array and every call rewrites the
 *    part it reads (nothing needs to start at zero): calls whose kernels
 *    overlap on the GPU (other streams, or other host threads) race on it;
 *    serialise them on one stream.
 *  - grid, coeffs: caller-owned device memory as for su2_forward. */
#define SU2_NOALLOC_SCRATCH_BYTES (4u << 20)
su2_status su2_forward_noalloc(su2_plan_t plan, const void* grid, void* coeffs, void* cuda_stream);

/* Synchronises the stream and reports any latched device-side error; clears it. */
su2_status su2_sync_status(su2_plan_t plan, void* cuda_stream);

/* Self-test of the device-side bounded waits (a library service, no
 * counterpart in the paper).  Enqueues on cuda_stream one small kernel that
 * waits, with the same bounded helpers the transform kernels use, for an event
 * that never happens: kind 0 a counter in the plan's memory that nothing
 * increments, kind 1 an mbarrier phase that nothing arrives on.  After about a
 * second (2e9 SM cycles) the wait gives up, latches the plan's error word and
 * the kernel returns, so the next su2_sync_status on that stream returns
 * SU2_ERR_TIMEOUT (and clears the word) and the context stays usable.
 * kind outside {0, 1}: SU2_ERR_INVALID_ARG. */
su2_status su2_selftest_bounded_wait(su2_plan_t plan, int kind, void* cuda_stream);

/* Forward transform of a batch held in host memory (a library service; the
 * transform is su2_forward's).  The grids are uploaded in chunks of about
 * 1 GiB on a plan-owned copy stream while stage 1 runs on the chunks already
 * resident; stage 2 then runs per bandwidth group over all its functions and
 * each group's coefficients are downloaded on a second copy stream; finally
 * `cuda_stream` waits for the downloads, so host_coeffs is complete once that
 * stream has passed this call (e.g. after cudaStreamSynchronize).
 *   host_grid:   host memory, su2_grid_elems elements (page-locked memory is
 *                needed for the copies to overlap the kernels); it must stay
 *                unchanged until the stream has passed this call.
 *   host_coeffs: host memory, su2_coeff_elems elements (page-locked likewise).
 *   dev_grid:    device memory, su2_grid_elems elements, used as the staging
 *                buffer of this call: the uploads start as soon as this plan's
 *                previous su2_forward_pipelined call has finished its stage 1,
 *                without waiting for other work queued on cuda_stream, so it
 *                must not be in use by such work.
 *   dev_coeffs:  device memory, su2_coeff_elems elements (device copy of the
 *                result, left in place).
 *   ws:          workspace as for su2_forward.
 * Consecutive calls on one plan must use the same stream (they then overlap:
 * the next call's uploads run during this call's stage 2 and downloads).
 * The first call creates the plan's two copy streams and four events.  Not
 * recorded into the plan's CUDA graph.  Errors as su2_forward; a null host
 * pointer is SU2_ERR_INVALID_ARG. */
su2_status su2_forward_pipelined(su2_plan_t plan, const void* host_grid, void* host_coeffs, void* dev_grid,
                                 void* dev_coeffs, void* ws, void* cuda_stream);

su2_status su2_destroy(su2_plan_t plan);

const char* su2_status_string(su2_status s);

#ifdef __cplusplus
}
#endif

#endif /* SU2FFT_H */

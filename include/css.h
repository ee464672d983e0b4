/*
 * libcss -- greedy column subset selection on one GB300 (sm_103a).
 *
 * C ABI of the CUDA library.  It follows Farahat, Elgohary, Ghodsi, Kamel,
 * "Greedy Column Subset Selection for Large-scale Data Sets" (arXiv:1312.6838):
 *
 *   css_select          Problem 1 by the greedy heuristic of Algorithm 1
 *                       (Sec. 4.2; score recursion of Theorem 2, error
 *                       recursion of Theorem 1).
 *   gcss_select         Problem 4 / Problem 5: columns of A chosen to
 *                       reconstruct a target B, Algorithm 3 (Sec. 5.2;
 *                       Theorems 3 and 4).
 *   gcss_distributed    Algorithm 4 (Sec. 5.2): GCSS inside every column block,
 *                       then GCSS on the union of the blocks' selections.
 *   css_project         B = A Omega, the random projection of Sec. 5.1
 *                       (Algorithm 2: per-block partial sums, then row sums).
 *   css_select_batched  many independent Algorithm 1 instances in one launch;
 *                       css_select_batched_prepare / _run split it so that
 *                       the device work can be captured in a CUDA graph.
 *   css_residual_backward
 *                       loss ||A - P^(S) A||_F^2 (Problem 1's criterion,
 *                       Eq. Projection of Sec. 3.1) and its gradient with
 *                       respect to A at a fixed selected set S.
 *   css_embed           Q = orth(A_:S) and the embedding W = Q^T A of all
 *                       columns into the span of a selection (Sec. 3.2,
 *                       Eq. CSS_LowDim).
 *   css_lowrank         the column-based rank-k approximation
 *                       A~_{S,k} = Q W~_k and the approximate SVD of
 *                       Eq. (ApproxSVD) from Q and W (Sec. 3.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout     Matrices are column-major with a leading dimension (the paper's
 *            column view <i, A_:i>, Sec. 5.1): element (i, j) of A sits at
 *            A[i + j * lda], lda >= m.  Column indices are 0-based int32
 *            (the paper counts from 1).  Selections are returned in selection
 *            order.
 * Pointers   Every data pointer is a DEVICE pointer (cudaMalloc'd or a
 *            device tensor's storage) unless its comment says HOST.  The
 *            caller owns all memory.  No entry point allocates device
 *            memory: scratch space is a caller-provided workspace whose size
 *            comes from css_workspace_size() (ws may be NULL only when that
 *            size is 0).
 * Streams    Work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 *            default stream).  With opts->sync = 1 (the default) the call
 *            synchronises the stream before returning so it can report
 *            device-side status (rank exhaustion, non-finite input, timeout);
 *            with sync = 0 it returns CSS_OK after enqueueing and device
 *            status is read later with css_read_status().
 * Errors     Argument errors are found on the host before anything is
 *            enqueued (CSS_ERR_INVALID_ARG / CSS_ERR_WORKSPACE).  The library
 *            never exits, traps or asserts on the device; every device-side
 *            wait is bounded and reports CSS_ERR_TIMEOUT when it runs out.
 * Precision  A may be FP64, FP32 or BF16.  FP64 input is processed entirely
 *            in FP64.  FP32/BF16 input is streamed as stored with FP32
 *            accumulation of the per-column dot products; the score state
 *            (f, g), the orthonormal basis of the selected columns, the pivot
 *            norm and the error trace are FP64.
 */
#ifndef LIBCSS_CSS_H
#define LIBCSS_CSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* css_stream_t;

typedef enum {
    CSS_OK = 0,
    /* Warning: every remaining candidate column has a residual norm at or
       below tau_rel times its initial norm (A has numerical rank < k).
       *n_sel < k; sel and the error trace are valid up to *n_sel. */
    CSS_RANK_EXHAUSTED = 1,
    CSS_ERR_INVALID_ARG = -1,
    CSS_ERR_CUDA = -2,
    CSS_ERR_NO_MEMORY = -3,
    CSS_ERR_WORKSPACE = -4,   /* ws NULL, misaligned or smaller than required */
    CSS_ERR_TIMEOUT = -5,     /* a bounded device-side wait ran out */
    CSS_ERR_NONFINITE = -6,   /* A (or B) holds a NaN or an infinity */
    CSS_ERR_UNSUPPORTED = -7, /* no sm_103a device, or a dtype combination
                                 the entry point does not take */
    CSS_ERR_NOT_CONVERGED = -8 /* css_lowrank: the eigenvalue iteration did
                                  not converge within its sweep limit */
} css_status;

typedef enum { CSS_F64 = 0, CSS_F32 = 1, CSS_BF16 = 2 } css_dtype;

typedef enum {
    CSS_OP_SELECT = 0,
    CSS_OP_GCSS = 1,
    CSS_OP_DISTRIBUTED = 2,
    CSS_OP_PROJECT = 3,
    CSS_OP_BACKWARD = 4,
    CSS_OP_HOST_SELECT = 5,
    CSS_OP_PROJECT_RANDOM = 6,
    CSS_OP_RANDOMIZED = 7,
    CSS_OP_EMBED = 8,
    CSS_OP_LOWRANK = 9
} css_op;

/* Options.  Fill with css_opts_default() and change fields as needed;
   passing NULL means the defaults. */
typedef struct {
    /* Candidate threshold: column i stays a candidate while its residual
       norm g_i exceeds tau_rel * g_i^(0).  < 0 selects the default
       (1e-12 for FP64 input, 1e-6 for FP32/BF16). */
    double tau_rel;
    /* DEVICE int32[n_forced] or NULL: column indices taken at the first
       n_forced iterations instead of the argmax (resume / teacher forcing).
       n_forced <= k; the indices are copied to the host and checked to be
       distinct and in range before anything is enqueued (a synchronous
       copy).  css_select and gcss_select only. */
    const int32_t* forced;
    int32_t n_forced;
    /* 0: the paper's criterion f_i / g_i.  1: g_i alone (QR with column
       pivoting; a test hook). */
    int32_t score_mode;
    /* 1 (default): synchronise at the end and report device status. */
    int32_t sync;
    /* Upper bound for any single device-side wait, in nanoseconds.
       0 selects the default (2 s). */
    uint64_t spin_budget_ns;
    /* Number of CTAs of the persistent greedy kernel (0 = all SMs times the
       occupancy).  Tuning knob.  gcss_distributed's blocks' launch counts
       CTAs of 256 threads (two per SM); every other launch, and its union
       launch, CTAs of 512 threads (one per SM). */
    int32_t grid_ctas;
    /* Columns per warp tile of the fused step: 2, 4 or 8 (0 = default, 8).
       The last tiles of each step are further cut into row chunks. */
    int32_t tile_cols;
    /* Optional DEVICE diagnostics, NULL to skip (css_select, gcss_select):
       diag_argmax  int32[k]: the kernel's own argmax at each iteration (also
                    when a forced index is taken instead);
       diag_f, diag_g double[n]: the score state f, g after the last
                    iteration (Theorem 2's numerator and denominator). */
    int32_t* diag_argmax;
    /* HOST double[2] or NULL (sync mode only): milliseconds of the
       initial-score phase and of the greedy iterations, from CUDA events on
       `stream` (gcss_distributed: the initial scores and the blocks'
       persistent launch; css_lowrank: double[4], see there). */
    double* timing_ms;
    double* diag_f;
    double* diag_g;
    /* Dense-GEMM path: 0 = automatic, 1 = CUDA-core (SIMT) kernels only.
       Automatic means tcgen05 tensor cores: for css_project and the initial
       scores of gcss_select / gcss_distributed when A is BF16 and its layout
       allows TMA (16-byte aligned base, leading dimension a multiple of 8,
       r <= 512; B split into three BF16 parts, all 24 bits); for the initial
       scores of css_select and css_select_batched when A is BF16 (a layout
       TMA refuses is copied to an aligned buffer first) or FP32 (split into
       three BF16 parts, the six products of parts down to 2^-16 summed):
       C = A A^T, then C split into three BF16 parts. */
    int32_t init_path;
    /* Test hook for the bounded device waits (0 = off, the default).
       1: one team barrier of the persistent greedy kernel (the first of
       the first iteration) waits for an arrival that no CTA makes; 2: the
       tensor-core initial-score kernels wait on an mbarrier phase that
       nothing completes.  The wait runs out after spin_budget_ns, the call
       reports CSS_ERR_TIMEOUT, nothing faults and the context stays usable
       for the next call.  css_select and gcss_select. */
    int32_t test_unmet_wait;
    /* Plan knobs (0 = the value the tuning table holds for this device and
       shape, else the default).  split_share: the fused step splits the
       last tiles of each step for 1 / split_share of the team's warps (1,
       2, 4 or 8; default 2).  pivot_cost: gcss_distributed's planner
       charges each block iteration's pivot as this many streamed columns
       when it sizes the blocks' teams (default 1500). */
    int32_t split_share;
    int32_t pivot_cost;
    int32_t reserved[4];
    /* DEVICE uint64[k * 16] or NULL (css_select, gcss_select): per-iteration
       trace of the persistent kernel; entry [t * 16 + j] is the GPU global
       timer (ns) when the team's first CTA reached point j of iteration t:
       0 start, 1 argmax done, 2/3 before/after the first team barrier,
       4/5 around the second, 6 target vectors staged, 7 C e or B B^T e
       done, 8 Z^T e done, 9 after the third barrier, 10/11 around the
       fourth, 12 fused step starts, 13 fused step done (the first warp),
       15 the CTA's argmax candidate published, 14 after the last barrier.
       Unused entries are 0. */
    uint64_t* trace_ns;
    /* DEVICE double[m * k] or NULL (css_select, gcss_select): the orthonormal
       basis Q of the selected columns, column t (basis[t * m + i]) = q_t,
       the normalised part of the t-th selected column outside the span of
       the earlier ones (Gram-Schmidt in selection order; W = Q^T A).
       FP32/BF16 input: the basis is held as double-float pairs and returned
       as their FP64 sum.  Columns t >= *n_sel are set to zero. */
    double* basis;
} css_opts;

/* Fill *opts with the defaults. */
void css_opts_default(css_opts* opts);

/* Human-readable name of a status code (static storage). */
const char* css_status_string(css_status s);

/* Library version string (static storage). */
const char* css_version(void);

/* Bytes of device workspace the entry point `op` needs for the given sizes
   (m rows, n columns, r target columns for GCSS/projection, k columns to
   select; unused sizes may be 0).  For CSS_OP_DISTRIBUTED, n is the total
   column count and r the target width; the per-block limit l_block must be
   passed in k_block.  For CSS_OP_BACKWARD and CSS_OP_EMBED, k is |S|.  For
   CSS_OP_LOWRANK, r is the embedding dimension l and k the rank.  Returns 0
   when the sizes are invalid. */
size_t css_workspace_size(css_op op, css_dtype dtype, int64_t m, int64_t n,
                          int64_t r, int32_t k, int32_t k_block,
                          const css_opts* opts);

/*
 * Greedy CSS, Algorithm 1 (Sec. 4.2).
 *
 *   A        DEVICE m x n, column-major, leading dimension lda >= m.
 *   dtype    element type of A.
 *   k        number of columns to select, 1 <= k <= min(m, n, 1024).
 *            m is limited by shared memory: up to about 17000 rows for
 *            FP32/BF16 input and 13000 for FP64 (CSS_ERR_UNSUPPORTED above).
 *   sel      DEVICE int32[k]: selected columns in selection order.
 *   trace    DEVICE double[k+1]: F^(0) = ||A||_F^2 and F^(t) after each
 *            iteration by Theorem 1 (F^(t) = F^(t-1) - f_p / g_p).
 *   n_sel    DEVICE int32[1]: number of columns selected (k unless the rank
 *            ran out).
 *   W        DEVICE double[k * n] or NULL: row t (W[t * n + i]) is
 *            omega^(t) of Eq. (delta_omega), the embedding row of all columns
 *            (Sec. 3.1, W = Q^T A; W Pi is upper triangular, Sec. 6).
 *   ws       DEVICE workspace of at least css_workspace_size(CSS_OP_SELECT,
 *            ...) bytes, 256-byte aligned.
 * Returns CSS_OK, CSS_RANK_EXHAUSTED or an error code.
 */
css_status css_select(const void* A, css_dtype dtype, int64_t m, int64_t n,
                      int64_t lda, int32_t k, int32_t* sel, double* trace,
                      int32_t* n_sel, double* W, void* ws, size_t ws_bytes,
                      const css_opts* opts, css_stream_t stream);

/*
 * Greedy generalized CSS, Algorithm 3 (Sec. 5.2): columns of A that best
 * reconstruct the target B (Problem 4's criterion ||B - P^(S) B||_F^2).
 *
 *   A      DEVICE m x n (lda), dtype dtype.
 *   B      DEVICE m x r (ldb >= m).  FP64 when dtype is CSS_F64, FP32 otherwise.
 *   trace  DEVICE double[k+1]: Fbar^(0) = ||B||_F^2 and Fbar^(t) (Theorem 3).
 *   Other arguments as css_select.
 */
css_status gcss_select(const void* A, css_dtype dtype, int64_t m, int64_t n,
                       int64_t lda, const void* B, int64_t r, int64_t ldb,
                       int32_t k, int32_t* sel, double* trace, int32_t* n_sel,
                       double* W, void* ws, size_t ws_bytes,
                       const css_opts* opts, css_stream_t stream);

/*
 * Distributed CSS, Algorithm 4 (Sec. 5.2), on one GPU: every column block b
 * (columns block_offsets[b] .. block_offsets[b+1]-1) selects
 * l_b = min(l_block, width_b) columns by GCSS against B (the map phase, all
 * blocks in one persistent launch); the union of those columns, in block
 * order and each block's selection order, is A_(0); GCSS(A_(0), B, k) picks
 * the final k columns (the reduce phase).
 *
 *   block_offsets  HOST int64[nblocks + 1], strictly increasing, from 0 to n.
 *   block_sel      DEVICE int32[nblocks * l_block] or NULL: per-block global
 *                  column ids in selection order, -1 where a block selected
 *                  fewer than l_block.
 *   sel, trace, n_sel
 *                  the final selection as global column ids of A, with the
 *                  error trace of the union step.
 */
/* Exact workspace bytes of gcss_distributed for a given block partition
   (css_workspace_size(CSS_OP_DISTRIBUTED, ...) returns a bound that holds
   for every partition with blocks of at least k_block columns). */
size_t gcss_distributed_workspace_size(css_dtype dtype, int64_t m, int64_t n,
                                       int64_t r, const int64_t* block_offsets,
                                       int32_t nblocks, int32_t l_block,
                                       int32_t k);

css_status gcss_distributed(const void* A, css_dtype dtype, int64_t m,
                            int64_t n, int64_t lda, const void* B, int64_t r,
                            int64_t ldb, const int64_t* block_offsets,
                            int32_t nblocks, int32_t l_block, int32_t k,
                            int32_t* sel, double* trace, int32_t* n_sel,
                            int32_t* block_sel, void* ws, size_t ws_bytes,
                            const css_opts* opts, css_stream_t stream);

/*
 * Algorithm 4 in two steps, so that the whole pipeline can be repeated or
 * captured in a CUDA graph (no implementation detail of the paper; the
 * reduce step's union of the blocks' picks is built on the device):
 *
 *   gcss_distributed_prepare  validates (arguments as gcss_distributed),
 *       plans both persistent launches (the blocks', and the union's for its
 *       largest size, sum_b min(l_block, width_b)) and writes every
 *       descriptor and the block offsets into the workspace; returns after
 *       the copies finished (it synchronises `stream`).  Not capturable.
 *   gcss_distributed_run      enqueues on `stream` the initial scores
 *       ||B^T a_i||^2, the block launch, the union (prefix sums of the
 *       blocks' pick counts, global ids, gathered columns and initial
 *       scores, the union size written into the union launch's descriptor),
 *       the union launch and the mapping of its picks to global ids: device
 *       work only, with no host copy and no synchronisation.  It reads A and
 *       B and writes sel, trace, n_sel and block_sel through the DEVICE
 *       pointers given to prepare, which must stay valid; the status (the
 *       first error of either launch, or CSS_RANK_EXHAUSTED when the union
 *       step ran out of candidates) is read with css_read_status(ws).
 *
 * `plan` is HOST memory owned by the caller, filled by prepare and read by
 * run; it belongs to `ws` (run rejects another workspace with
 * CSS_ERR_INVALID_ARG).  Runs on the same workspace must not overlap on the
 * GPU.  The workspace size is gcss_distributed_workspace_size().
 */
typedef struct {
    uint64_t opaque[128];
} css_distributed_plan;

css_status gcss_distributed_prepare(const void* A, css_dtype dtype, int64_t m,
                                    int64_t n, int64_t lda, const void* B,
                                    int64_t r, int64_t ldb,
                                    const int64_t* block_offsets,
                                    int32_t nblocks, int32_t l_block, int32_t k,
                                    int32_t* sel, double* trace, int32_t* n_sel,
                                    int32_t* block_sel, void* ws,
                                    size_t ws_bytes, const css_opts* opts,
                                    css_distributed_plan* plan,
                                    css_stream_t stream);
css_status gcss_distributed_run(const css_distributed_plan* plan, void* ws,
                                css_stream_t stream);

/*
 * Random projection B = A Omega (Sec. 5.1, Algorithm 2).
 *
 *   A       DEVICE m x n (lda), CSS_BF16 or CSS_F32 or CSS_F64.
 *   Omega   DEVICE n x r (ldo >= n), same dtype as A.  Entries drawn i.i.d.
 *           from the caller's distribution Psi (Gaussian, +-1, sparse sign).
 *   Bout    DEVICE m x r (ldb >= m): FP32 for BF16/FP32 input, FP64 for FP64.
 *   BF16 x BF16 products accumulate in FP32 (tensor cores); column-block
 *   partial sums are added in FP32 in a fixed order, so results are
 *   reproducible run to run.
 */
css_status css_project(const void* A, css_dtype dtype, int64_t m, int64_t n,
                       int64_t lda, const void* Omega, int64_t r, int64_t ldo,
                       void* Bout, int64_t ldb, void* ws, size_t ws_bytes,
                       const css_opts* opts, css_stream_t stream);

/*
 * Omega drawn on the device from the counter-based generator Philox4x32-10
 * (Salmon, Moraes, Dror and Shaw, SC 2011): entry (i, j) is a function of
 * (i, j, seed) alone -- the Philox block at counter (i, j, 0, 0) under key
 * (seed mod 2^32, seed >> 32) -- so the same seed gives the same matrix at
 * any size, on any device.
 *   CSS_OMEGA_GAUSSIAN     N(0, 1/r) by Box-Muller on the first two words
 *                          (u1 = (w0 + 1) / 2^32, u2 = w1 / 2^32); FP32
 *                          arithmetic for BF16/FP32 output, FP64 for FP64.
 *   CSS_OMEGA_SPARSE_SIGN  the sparse random sign matrix of Sec. 5.1: +1 or
 *                          -1 (lowest bit of w1) where w0 < floor(2^32/sqrt n),
 *                          i.e. with probability 1/sqrt(n); 0 elsewhere.
 *                          Unscaled (the selection does not depend on B's
 *                          scale).
 */
typedef enum {
    CSS_OMEGA_GAUSSIAN = 0,
    CSS_OMEGA_SPARSE_SIGN = 1
} css_omega;

/*
 * css_random_omega: write Omega (n x r, DEVICE, leading dimension ldo >= n,
 * dtype BF16/FP32/FP64) on `stream`.
 *
 * css_project_random: B = A Omega (Algorithm 2) with Omega drawn as above.
 *   Gaussian: Omega is written into the workspace in A's dtype and multiplied
 *   as in css_project (tensor cores for BF16).  Sparse sign: Omega is never
 *   formed; each column of B adds the +-columns of A its column of Omega
 *   selects, in increasing row order (FP32 sums for BF16/FP32 A, FP64 for
 *   FP64), and the workspace is unused (ws may be NULL).  The workspace size
 *   is css_workspace_size(CSS_OP_PROJECT_RANDOM, dtype, m, n, r, 0, 0, opts).
 *   Other arguments as css_project.
 */
css_status css_random_omega(int64_t n, int64_t r, uint64_t seed, css_omega dist,
                            css_dtype dtype, void* Omega, int64_t ldo,
                            css_stream_t stream);
css_status css_project_random(const void* A, css_dtype dtype, int64_t m, int64_t n,
                              int64_t lda, int64_t r, uint64_t seed, css_omega dist,
                              void* Bout, int64_t ldb, void* ws, size_t ws_bytes,
                              const css_opts* opts, css_stream_t stream);

/*
 * RndGreedyCSS (Sec. 7): the greedy generalized CSS of Algorithm 3 for the
 * random target B = A Omega, Omega n x l drawn on the device as in
 * css_project_random (r = l).  Selects l columns; outputs as css_select
 * (sel int32[l], trace double[l+1] with trace[0] = ||B||_F^2).  Workspace:
 * css_workspace_size(CSS_OP_RANDOMIZED, dtype, m, n, 0, l, 0, opts).
 */
css_status css_select_randomized(const void* A, css_dtype dtype, int64_t m, int64_t n,
                                 int64_t lda, int32_t l, uint64_t seed, css_omega dist,
                                 int32_t* sel, double* trace, int32_t* n_sel, void* ws,
                                 size_t ws_bytes, const css_opts* opts, css_stream_t stream);

/* One independent greedy CSS problem of a batch (HOST struct; the pointers
   inside are DEVICE pointers with the meaning they have in css_select). */
typedef struct {
    const void* A;
    int64_t m, n, lda;
    int32_t k;
    int32_t pad_;
    int32_t* sel;
    double* trace;
    int32_t* n_sel;
    double* W; /* may be NULL */
} css_problem;

/*
 * Many independent Algorithm 1 instances of uneven sizes in one persistent
 * launch (all instances share dtype).  probs is a HOST array of `count`
 * descriptors; the workspace size is css_batched_workspace_size().
 * Returns CSS_OK when every instance selected its k columns,
 * CSS_RANK_EXHAUSTED when some ran out of rank (their n_sel says how many).
 */
size_t css_batched_workspace_size(const css_problem* probs, int32_t count,
                                  css_dtype dtype, const css_opts* opts);
css_status css_select_batched(const css_problem* probs, int32_t count,
                              css_dtype dtype, void* ws, size_t ws_bytes,
                              const css_opts* opts, css_stream_t stream);

/*
 * The same batch in two steps, so that the device work can be repeated or
 * captured in a CUDA graph (no implementation detail of the paper; this is
 * how a batch is replayed without host work):
 *
 *   css_select_batched_prepare  validates, plans the teams and writes every
 *       descriptor into the workspace; returns after the copies finished
 *       (it synchronises `stream`).  Not capturable.
 *   css_select_batched_run      resets the status, barriers and counters
 *       from device-side values and enqueues the initial scores (three
 *       launches) and the persistent launch on `stream`: device work only,
 *       with no host copy and no synchronisation, so it may be captured and
 *       replayed.  It reads the problems' A and writes sel, trace, n_sel
 *       (and W) through the DEVICE pointers given to prepare, which must stay
 *       valid; the status is read afterwards with css_read_status(ws).
 *
 * `plan` is HOST memory owned by the caller, filled by prepare and read by
 * run; it belongs to `ws` (run rejects another workspace with
 * CSS_ERR_INVALID_ARG).  Runs on the same workspace must not overlap on the
 * GPU.  opts as for css_select_batched except timing_ms and sync, which
 * only css_select_batched uses.
 */
typedef struct {
    uint64_t opaque[64];
} css_batched_plan;

css_status css_select_batched_prepare(const css_problem* probs, int32_t count,
                                      css_dtype dtype, void* ws, size_t ws_bytes,
                                      const css_opts* opts, css_batched_plan* plan,
                                      css_stream_t stream);
css_status css_select_batched_run(const css_batched_plan* plan, void* ws,
                                  css_stream_t stream);

/*
 * Tile-width autotuner of the fused streaming step (no counterpart in the
 * paper; a tuning aid).  The fused step hands out tiles of 2, 4 or 8 columns;
 * css_select, gcss_select, gcss_distributed and css_select_batched with
 * opts->tile_cols == 0 use the width recorded for the current device, the
 * dtype and the shape's bucket (floor(log2 m), floor(log2 n)), else 8.
 *
 *   css_autotune_select  runs css_select on the caller's problem (arguments
 *       as css_select; the outputs hold the last run's selection) once per
 *       width untimed and once timed, records the fastest and returns it in
 *       *best_tile (HOST int32); times_ms is a HOST double[3] or NULL (greedy
 *       iterations in ms for widths 2, 4, 8).  Synchronises `stream`.
 *   css_tile_record / css_tile_lookup  set / read an entry for a device
 *       name (HOST string, as cudaDeviceProp::name); lookup returns 0 when
 *       there is none.  Host only.
 *   css_tile_cache_save / css_tile_cache_load  write / merge the table as a
 *       flat JSON object {"<device>|<dtype>|m<b>|n<b>": <width>, ...};
 *       CSS_ERR_INVALID_ARG on an unreadable file or a malformed entry (the
 *       table is then unchanged).  Host only.
 * The table is process-wide and guarded by a mutex.
 */
css_status css_autotune_select(const void* A, css_dtype dtype, int64_t m, int64_t n,
                               int64_t lda, int32_t k, int32_t* sel, double* trace,
                               int32_t* n_sel, void* ws, size_t ws_bytes,
                               int32_t* best_tile, double* times_ms, css_stream_t stream);
css_status css_tile_record(const char* device_name, css_dtype dtype, int64_t m, int64_t n,
                           int32_t tile_cols);
int32_t css_tile_lookup(const char* device_name, css_dtype dtype, int64_t m, int64_t n);
css_status css_tile_cache_save(const char* path);
css_status css_tile_cache_load(const char* path);

/*
 * The same table holds the other plan knobs (css_opts.split_share and
 * pivot_cost), under the keys "<device>|<dtype>|m<b>|n<b>|split" and
 * "...|pivot" in the JSON cache:
 *   css_tune_record / css_tune_lookup  set / read one knob (tile widths 2,
 *       4, 8; split shares 1, 2, 4, 8; pivot costs 0 .. 1000000 columns);
 *       lookup returns -1 when there is no entry.  Host only.
 *   css_autotune_select (above) also times split shares 1, 2 and 4 at the
 *       fastest width and records the fastest share.
 *   css_autotune_distributed  runs gcss_distributed on the caller's problem
 *       (arguments as gcss_distributed) with pivot costs 300, 700, 1500
 *       and 3000 columns, each once untimed and once timed (the blocks'
 *       launch), records the fastest for the device, dtype and (m, n)
 *       bucket and returns it in *best_cost (HOST int32); times_ms is a HOST
 *       double[4] or NULL.  Synchronises `stream`.
 */
typedef enum {
    CSS_KNOB_TILE_COLS = 0,
    CSS_KNOB_SPLIT_SHARE = 1,
    CSS_KNOB_PIVOT_COST = 2
} css_knob;
css_status css_tune_record(const char* device_name, css_dtype dtype, int64_t m, int64_t n,
                           css_knob knob, int32_t value);
int32_t css_tune_lookup(const char* device_name, css_dtype dtype, int64_t m, int64_t n,
                        css_knob knob);
css_status css_autotune_distributed(const void* A, css_dtype dtype, int64_t m, int64_t n,
                                    int64_t lda, const void* B, int64_t r, int64_t ldb,
                                    const int64_t* block_offsets, int32_t nblocks,
                                    int32_t l_block, int32_t k, int32_t* sel, double* trace,
                                    int32_t* n_sel, void* ws, size_t ws_bytes,
                                    int32_t* best_cost, double* times_ms, css_stream_t stream);

/*
 * Loss and gradient of the reconstruction error at a fixed selected set S
 * (Problem 1's criterion; P^(S) = A_S (A_S^T A_S)^-1 A_S^T, Eq. Projection).
 *
 *   loss = ||R||_F^2,  R = A - A_S T,  T = (A_S^T A_S)^-1 A_S^T A
 *   dA   = grad_out * 2 R            for columns outside S
 *   dA_S = grad_out * (-2 R T^T)     for the columns in S
 *
 *   sel       DEVICE int32[k], distinct column indices.
 *   dA        DEVICE, same dtype as A, m x n with leading dimension ldda, or
 *             NULL to compute the loss only.
 *   loss      DEVICE double[1] or NULL.
 * The k x k factor of A_S^T A_S is recomputed here (FP64 Cholesky), not
 * carried over from a forward pass; a pivot at or below 1e-12 of its
 * column's squared norm (dependent columns in S) gives CSS_ERR_INVALID_ARG
 * (reported in sync mode), as do out-of-range or repeated indices.
 * FP32/BF16 input: the two products that cancel (Q^T A and A - Q W, with
 * Q = A_S L^-T) run in double-float arithmetic (FP32 pairs, error-free
 * products and sums), R W^T accumulates in FP32, the factorisation and the
 * loss are FP64; dA is rounded once to the dtype of A.  k <= 1024.
 */
css_status css_residual_backward(const void* A, css_dtype dtype, int64_t m,
                                 int64_t n, int64_t lda, const int32_t* sel,
                                 int32_t k, double grad_out, void* dA,
                                 int64_t ldda, double* loss, void* ws,
                                 size_t ws_bytes, const css_opts* opts,
                                 css_stream_t stream);

/*
 * Embedding into the span of a selection (Sec. 3.2, Eq. CSS_LowDim):
 *
 *   Q = orth(A_:S)   m x l: the thin QR factor of A_:S whose R has a positive
 *                    diagonal, i.e. the Gram-Schmidt basis of the selected
 *                    columns in the order of `sel` (the basis css_select
 *                    builds, opts->basis)
 *   W = Q^T A        l x n: row t at W[t * ldw + j] (the layout of
 *                    css_select's omega rows), W[:, sel] = R
 *
 *   sel       DEVICE int32[l], distinct column indices (checked on the host
 *             through a small synchronous copy).
 *   Q         DEVICE double, m x l, leading dimension ldq >= m, or NULL.
 *   W         DEVICE double, l rows of stride ldw >= n, or NULL (not both).
 * Q comes from CholeskyQR2 in FP64 (Fukaya, Nakatsukasa, Yanagisawa and
 * Yamamoto, 2014: Q1 = A_S L1^-T from A_S^T A_S = L1 L1^T, then the same once
 * more on Q1), orthonormal to working precision while the condition number of
 * A_S stays below about 1e7.  A pivot at or below 1e-12 of its column's
 * squared norm (dependent columns) gives CSS_ERR_INVALID_ARG (sync mode).
 * W: FP64 products for FP64 input; FP32/BF16 input runs in double-float
 * arithmetic (FP32 pairs with error-free products and sums).  l <= 1024,
 * l <= min(m, n).  Workspace: css_workspace_size(CSS_OP_EMBED, dtype, m, n,
 * 0, l, 0, opts).
 */
css_status css_embed(const void* A, css_dtype dtype, int64_t m, int64_t n,
                     int64_t lda, const int32_t* sel, int32_t l, double* Q,
                     int64_t ldq, double* W, int64_t ldw, void* ws,
                     size_t ws_bytes, const css_opts* opts,
                     css_stream_t stream);

/*
 * Rank-k approximation and approximate SVD from an embedding (Sec. 3.2):
 *
 *   W = U^(W) Sigma^(W) V^(W)^T          SVD of the l x n embedding
 *   W~_k = U^(W)_k Sigma^(W)_k V^(W)_k^T  its best rank-k approximation
 *   A~_{S,k} = Q W~_k = U~ Sigma~ V~^T    the column-based rank-k
 *                                        approximation of A
 *   U~ = Q U^(W)_k,  Sigma~ = Sigma^(W)_k,  V~ = V^(W)_k   (Eq. ApproxSVD)
 *
 * Inputs (DEVICE, FP64):
 *   W         l rows of stride ldw >= n (W[t * ldw + j]), e.g. css_select's
 *             omega rows or css_embed's output.
 *   Q         m x l, leading dimension ldq >= m, orthonormal columns, or
 *             NULL when U is not requested.
 * Outputs (DEVICE, FP64; every one but sigma may be NULL):
 *   sigma     double[k]: sigma_1 >= ... >= sigma_k >= 0.
 *   U         m x k, leading dimension ldu >= m: U~ (needs Q).
 *   V         n x k, leading dimension ldv >= n: V~ = W^T U^(W)_k
 *             Sigma_k^-1.  A column whose sigma_i^2 is at or below
 *             (n + l) * 2^-52 * ||W||_F^2 -- below what the method resolves,
 *             e.g. W of rank < k -- is returned as zeros.
 *   Uw        l x k, leading dimension l: U^(W)_k.
 *   tail      double[1]: sum_{i >= k} sigma_i^2 = ||W - W~_k||_F^2.  With
 *             W = Q^T A, ||A - A~_{S,k}||_F^2 = ||A - P^(S) A||_F^2 + tail,
 *             the first term being css_select's final error trace entry.
 * Each singular vector is signed so that the entry of largest magnitude of
 * its U^(W) column (lowest index on ties) is positive.
 * Method: G = W W^T (FP64), its eigendecomposition by cyclic Jacobi
 * rotations in FP64 (parallel round-robin ordering, one cooperative
 * kernel), sigma_i^2 = lambda_i, then U~ and V~ as products of FP64
 * operands accumulated in double-float (48 significant bits; Q's entries,
 * at most 1 for an orthonormal basis, must lie in FP32's range).  The
 * eigenvalues carry an absolute error of about (n + l) 2^-53 ||W||_F^2 (the
 * Gram matrix's rounding): sigma_i is accurate relative to sigma_1^2 /
 * sigma_i, not to sigma_i.  CSS_ERR_NOT_CONVERGED if the rotations have not
 * converged after 40 sweeps; CSS_ERR_NONFINITE for NaN/Inf in W.
 * 1 <= k <= l <= 1024.  Workspace: css_workspace_size(CSS_OP_LOWRANK,
 * CSS_F64, m, n, l, k, 0, opts).  opts->timing_ms (sync mode) is HOST
 * double[4] here: milliseconds of the Gram matrix, of the eigendecomposition
 * and of the ordering and products, then the number of Jacobi sweeps.
 */
css_status css_lowrank(const double* W, int64_t ldw, const double* Q,
                       int64_t ldq, int64_t m, int64_t n, int32_t l, int32_t k,
                       double* sigma, double* U, int64_t ldu, double* V,
                       int64_t ldv, double* Uw, double* tail, void* ws,
                       size_t ws_bytes, const css_opts* opts,
                       css_stream_t stream);

/*
 * css_select from HOST buffers: copies A (HOST, m x n, lda; pinned memory
 * for full speed) into the caller's DEVICE staging buffer `A_dev` (at least
 * lda * n elements), runs css_select, and copies sel (HOST int32[k]), trace
 * (HOST double[k+1]) and n_sel (HOST int32[1]) back.  Always synchronous.
 * The workspace is css_workspace_size(CSS_OP_SELECT, ...) plus 256 bytes.
 * For BF16 and FP32, A goes over in column chunks on a copy stream of the
 * library's own (one per device, with its events, made on first use and
 * kept until the process exits), ordered after the work already on
 * `stream`; the initial scores start on the chunks already in.  The result
 * is that of css_select on the copied matrix, bit for bit.
 */
css_status css_select_host(const void* A_host, css_dtype dtype, int64_t m,
                           int64_t n, int64_t lda, int32_t k, int32_t* sel,
                           double* trace, int32_t* n_sel, void* A_dev,
                           void* ws, size_t ws_bytes, const css_opts* opts,
                           css_stream_t stream);

/*
 * css_select without a caller workspace.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (a
 * service whose device memory is fully pre-reserved by its host application,
 * a plugin whose framework forbids allocation calls, or latency-sensitive
 * code that must avoid cudaMalloc/cudaFree because they can synchronise the
 * device).
 *
 * Its scratch memory is a fixed array of CSS_NOALLOC_SCRATCH_BYTES inside the
 * library, one copy per device that loads it, held until the process exits.
 * Arguments are those of css_select (inputs and outputs are still the
 * caller's); problems whose css_select workspace
 * (css_workspace_size(CSS_OP_SELECT, ...)) exceeds the array are rejected
 * with CSS_ERR_WORKSPACE before anything is enqueued -- for example FP32
 * m = 1024, n = 16384, k = 64 fits, m = 4096, n = 65536 does not.
 * opts->timing_ms must be NULL, and opts->sync must be 1 (the default):
 * the device status of the call lives in the library's array, which the
 * caller cannot hand to css_read_status, so the call always waits for its
 * stream and returns that status (CSS_ERR_INVALID_ARG for sync = 0).
 * Nothing is allocated: no cudaMalloc, cudaFree or allocating library
 * routine is called.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the
 * life of the process; make that first call before any stream capture.  A
 * device reset (cudaDeviceReset) after that first call is not supported:
 * the kept address would no longer be valid.  All calls on a device share
 * the one array: calls whose work overlaps on the GPU (calls on other
 * streams or host threads) race on it and corrupt each other's results.
 * Each call initialises every scratch word it reads, so stale contents
 * from an earlier call are harmless.
 */
#define CSS_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
css_status css_select_noalloc(const void* A, css_dtype dtype, int64_t m,
                              int64_t n, int64_t lda, int32_t k,
                              int32_t* sel, double* trace, int32_t* n_sel,
                              double* W, const css_opts* opts,
                              css_stream_t stream);

/* Device status left by the last call that used `ws` (for opts->sync = 0)
   of css_select, gcss_select, gcss_distributed, css_select_randomized or
   css_select_batched(_run): synchronises `stream`, then returns CSS_OK,
   CSS_RANK_EXHAUSTED or the device error -- that of the greedy kernel, or
   that of the tensor-core initial-score kernel that ran before it (a
   bounded wait there that ran out reads as CSS_ERR_TIMEOUT). */
css_status css_read_status(const void* ws, css_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LIBCSS_CSS_H */

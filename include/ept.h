/*
 * ept.h -- C ABI of libept, GB300 (sm_103a) efficient permutation two-sample tests
 * for the energy distance (ED) and the Gaussian-kernel maximum mean discrepancy
 * (MMD), after Chaibub Neto, arXiv 2406.06488.
 *
 * The problem (Section 3.1): samples x (nx x p) and y (ny x p) from F_X and F_Y;
 * test H0: F_X = F_Y with the permutation test of Algorithm 1.  The library
 *   (1) builds the three blocks D_XX, D_YY, D_XY of Euclidean distances (or
 *       Gaussian kernel values) once (Algorithm 1, block construction;
 *       Algorithm 3; Appendix A.1), D_YX never stored (the memory-saving
 *       variant described after Algorithm 1);
 *   (2) assembles every permuted statistic from those blocks (Algorithm 1,
 *       permutation loop; Section 4.1 "swapping"), as batched quadratic forms
 *       s' C s over 0/1 relabeling vectors s on the tensor cores;
 *   (3) returns the observed statistic (Eq. 1 or Eq. 2), the permuted statistics
 *       and the permutation p-value (1 + #{stat* >= stat_o}) / (1 + B)
 *       (Section 3.1; Algorithm 1, last line).
 *
 * Conventions for every entry point:
 *   - Every function returns an ept_status; no exception or abort crosses the ABI.
 *     On an error the outputs are left unwritten and ept_last_error() describes it.
 *   - Array arguments are plain pointers.  When `on_device` is non-zero, every
 *     array argument of that call (inputs and outputs, except the host-side
 *     ept_result) is a device pointer on the context's device; otherwise every
 *     one is a host pointer and the library copies through pinned staging memory.
 *   - Inputs are borrowed for the duration of the call; the caller owns all
 *     memory it passes.  Device scratch is owned by the context and reused.
 *   - Calls on one context are serialised by a mutex; the library is safe to
 *     call from several threads.  `stream` (a cudaStream_t, may be NULL) orders
 *     the work after the caller's prior work on that stream; synchronous calls
 *     return when their results are ready.
 *   - X and Y are FP32, row-major, one sample per row (x_i in row i, Section 3).
 */
#ifndef EPT_H
#define EPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EPT_ABI_VERSION 6

typedef enum {
    EPT_OK = 0,
    EPT_EINVAL = 1,       /* bad argument: sizes, NaN/Inf data, malformed relabeling */
    EPT_ENOMEM = 2,       /* device memory or the context's budget exhausted */
    EPT_EBUSY = 3,        /* serving: no slot or memory for this request now */
    EPT_ECUDA = 4,        /* a CUDA call failed (message in ept_last_error) */
    EPT_ETIMEOUT = 5,     /* a device-side bounded wait gave up, or ept_wait timed out */
    EPT_ECANCELLED = 6,   /* serving: the request was cancelled */
    EPT_ENOTFOUND = 7,    /* serving: unknown ticket */
    EPT_EUNSUPPORTED = 8, /* the device is not an sm_103 GPU, or a mode is unavailable */
    EPT_EINTERNAL = 9     /* debug checks found a broken invariant (EPT_OPT_DEBUG_CHECKS) */
} ept_status;

typedef enum {
    EPT_STAT_ED = 0,           /* energy distance V-statistic, Eq. 1 */
    EPT_STAT_MMD_GAUSS = 1,    /* biased MMD^2, Eq. 2, k(x,y) = exp(-||x-y||^2 / (2 sigma^2)) */
    EPT_STAT_MMD_LAPLACE = 2   /* biased MMD^2, Eq. 2, k(x,y) = exp(-||x-y|| / sigma): the other
                                  reading of Appendix A.1's "exponential of the negative scaled
                                  Euclidean distance" */
} ept_stat;

/* sigma value selecting the median heuristic (MMD statistics): the bandwidth is the
   lower median (element floor((N-1)/2) in sorted order) of the N = n(n-1)/2
   distances between distinct pooled rows, found on the device by an exact radix
   selection; it does not depend on the split into x and y, so every relabeling
   sees the same kernel.  Returned in ept_result.sigma. */
#define EPT_SIGMA_MEDIAN (-1.0)

typedef enum {
    /* plain path: FP32 SIMT block build and FP32 SIMT permutation contraction,
       one launch per phase, no CUDA graph: the comparison baseline */
    EPT_PREC_PLAIN_FP32 = 0,
    /* tuned path: blocks built on tcgen05 tensor cores (split-FP16 Gram) and stored
       FP32; the contraction s' C s on tcgen05 with C scaled by a power of two and
       split into FP16 hi + lo parts accumulated in FP32 in tensor memory (the name
       is kept from the first version, which split into BF16) */
    EPT_PREC_SPLIT_BF16 = 1,
    /* the pre-computation strategy of Algorithm 5, the comparison the paper times
       the efficient test against (Section 5.1): the full n x n FP32 matrix of the
       pooled data computed once, each relabeling's three sub-matrices extracted by
       index and summed (TwoSum-compensated FP32 pairs, FP64 combination).  Single
       tests only (ept_test, ept_test_range, ept_test_masks; a given sigma); it needs
       4 n^2 bytes for the matrix.  Elsewhere EPT_EUNSUPPORTED. */
    EPT_PREC_POOLED_FP32 = 2
} ept_precision;

typedef struct ept_ctx ept_ctx;

typedef struct {
    double observed;      /* statistic of the original labels, Eq. 1 / Eq. 2 */
    double p_value;       /* (1 + n_ge) / (1 + B); 1 when B = 0 */
    int64_t n_ge;         /* #{b : stat*_b >= observed}, compared in FP64 */
    int64_t n_near_tie;   /* #{b : |stat*_b - observed| <= 1e-5 * |observed|} */
    int64_t n_fixup;      /* near-duplicate pairs whose distance was recomputed in FP64 */
    double ms_build;      /* device time of the block phase (norms .. packing) */
    double ms_perm;       /* device time of relabeling draws + contraction + combine */
    double ms_total;      /* device time of the whole call, copies included */
    double ms_masks;      /* device time of the relabeling draws alone */
    double ms_contract;   /* device time of the contraction kernel alone (CUDA events
                             recorded on the stream it is launched on) */
    double sigma;         /* kernel bandwidth used (the median heuristic's value when
                             EPT_SIGMA_MEDIAN was given); 0 for ED */
    int64_t n_windows;    /* 0: the packed blocks were resident; k > 0: the test ran in
                             the streaming mode, in k windows of row panels
                             (EPT_OPT_STREAM_BLOCKS); there ms_build covers the row split,
                             the first pass and the centring, ms_perm the second pass and
                             the combination, ms_contract the contraction launches summed
                             (0 beyond 64 windows) */
    int64_t n_refined;    /* statistics (the observed one included) whose a-posteriori
                             error estimate exceeded 1e-5 of their value and that were
                             recomputed in FP64 from the raw rows (EPT_OPT_REFINE); with
                             EPT_OPT_REFINE = 0, the number that would have been */
    int64_t tuning;       /* parameters of the tensor-core run: 10000 x contraction kernel
                             (0 the context's, 1..3 as EPT_OPT_CONTRACTION) + 100 x unit
                             length in K-blocks + 10 x relabeling-draw kernel (0 automatic,
                             1..3 as EPT_OPT_DRAW_MODE) + unit order (0
                             automatic, 1 by length, 2 by first K-block); 0 for other paths */
    int64_t tune_candidates; /* parameter sets the autotuner timed in this call (its first
                             call of a batch shape); 0 when the parameters came from its
                             cache or were not tuned */
    int64_t refine_launches; /* kernel launches of the call's recomputation of flagged
                             statistics (all tests of a batched call together; 0 when
                             nothing was recomputed) */
} ept_result;

/* Library ABI version (EPT_ABI_VERSION of the build). */
int ept_abi_version(void);

/* How this copy of the library was built: ABI version, host architecture
   (aarch64 / x86_64), the GPU architecture its kernels were compiled for, the nvcc
   version and the compile date and time.  A static string owned by the library;
   never NULL.  Needs no GPU. */
const char *ept_build_info(void);

/* Message describing the last error on the calling thread (owned by the library;
   valid until the next call on this thread).  Never NULL. */
const char *ept_last_error(void);

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the device
   scratch the context may hold (0 = no cap).  Fails with EPT_EUNSUPPORTED if the
   device is not compute capability 10.3.  *out receives the context. */
ept_status ept_create(ept_ctx **out, int device, size_t mem_budget_bytes);

/* Caller-supplied device memory for a context's scratch (ept_create_ex).
   alloc(bytes, stream, user): device memory of at least `bytes` bytes on the
   context's device, aligned to 256 bytes, usable by work enqueued on `stream` (a
   cudaStream_t) from now on; NULL if it cannot be had (the call then fails with
   EPT_ENOMEM).  free(ptr, stream, user): gives back memory from alloc; the
   memory's last use is the work already enqueued on `stream`, so a stream-ordered
   allocator (like cudaFreeAsync) may reuse it once that work is done, and any
   other allocator must synchronise `stream` before reusing it.  The callbacks may
   be called from the calling thread and from the serving scheduler's thread (one at
   a time per context), never from inside a CUDA callback.  The pinned host staging
   memory stays the library's own. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, void *stream, void *user);
    void *user;
} ept_allocator;

/* ept_create with a caller-supplied allocator for all device scratch of the
   context (the run arena, streaming windows, serving batches); alloc = NULL
   behaves as ept_create (cudaMalloc for runs, a stream-ordered memory pool for
   serving).  The struct is copied. */
ept_status ept_create_ex(ept_ctx **out, int device, size_t mem_budget_bytes, const ept_allocator *alloc);

/* Destroy a context and free its device and pinned memory.  NULL is accepted. */
ept_status ept_destroy(ept_ctx *ctx);

/* Device scratch bytes a test of this shape needs (0 on invalid sizes). */
size_t ept_estimate_bytes(int64_t nx, int64_t ny, int64_t p, int64_t B, int prec);

/* Totals of a run's plan (ept_plan_check). */
typedef struct {
    int64_t units;            /* contraction work units: chunk x 256 relabelings x row half */
    int64_t chunks;           /* chunks: a row panel's range of K-blocks */
    int64_t stored_blocks;    /* 256 x 64 blocks of the packed upper storage */
    int64_t partials;         /* partial-sum rows (two per chunk, one per row half), each one
                                 FP32 per relabeling column, over all tests */
    int64_t cta_kblocks_max;  /* contraction schedule: K-blocks of MMA work of the busiest CTA */
    int64_t cta_kblocks_min;  /*   and of the least busy one */
    int64_t windows;          /* streaming windows (0: resident) */
    size_t scratch_bytes;     /* device scratch of the run, with the 256-byte guard bands of
                                 EPT_OPT_DEBUG_CHECKS (whose placement is checked too) */
} ept_plan_info;

/* The run planner on the host alone (no context, no device work), for checking it:
   plans n_tests tests of sizes nx[t], ny[t], p[t] with B[t] relabelings each as a
   tensor-core run does (Algorithm 1's permutation loop as quadratic forms over row
   panels, K-block chunks and tiles of 256 relabelings), with contraction units of
   at most unit_kb K-blocks dealt over num_sms CTAs, or, when stream_blocks > 0 (one
   test), in streaming windows of at most stream_blocks stored blocks; then checks the
   plan's invariants (row and column padding, prefix sums, chunk ranges, the
   schedule covering every unit once, the windows covering the panels once and in
   order within their capacity, guard bands).  out (may be NULL) receives the totals.
   EPT_OK; EPT_EINVAL for bad arguments (the size limits of ept_test, unit_kb outside
   1..1024, num_sms outside 1..4096, stream_blocks with more than one test);
   EPT_EINTERNAL, with ept_last_error naming it, for a broken invariant. */
ept_status ept_plan_check(const int64_t *nx, const int64_t *ny, const int64_t *p, const int64_t *B,
                          int n_tests, int unit_kb, int num_sms, int64_t stream_blocks, ept_plan_info *out);

/* One permutation test (Algorithm 1).
   X: nx*p floats, Y: ny*p floats (row-major).  stat: ept_stat.  sigma: kernel
   bandwidth for the MMD statistics, > 0 or EPT_SIGMA_MEDIAN; ignored for ED.
   B >= 0 permutations; draw b (1..B) of the
   permutation stream of `seed` (ept_perm_masks) is relabeling b.
   perm_stats: B doubles (may be NULL), perm_stats[b-1] = statistic of draw b.
   out: host struct, required.  Errors: EPT_EINVAL for nx < 1, ny < 1, p < 1, B < 0,
   nx + ny > 2^22, p > 2^30, B > 2^31, any other sigma <= 0 with MMD, non-finite data, a median bandwidth of 0 (more than
   half of the pooled pairs coincide); EPT_ENOMEM over budget.
   A repeated call with the same shapes replays the CUDA graph captured by the
   first (EPT_OPT_GRAPHS); then only out->ms_total is timed (the per-phase times
   are filled in when graphs are off). */
ept_status ept_test(ept_ctx *ctx, const float *X, int64_t nx, const float *Y, int64_t ny,
                    int64_t p, int on_device, int stat, double sigma, int64_t B, uint64_t seed,
                    int prec, double *perm_stats, ept_result *out, void *stream);

/* A range of the permutation stream: the observed statistic and draws b_first ..
   b_first + count - 1 of the stream of `seed` (b_first >= 1), everything else as in
   ept_test; out->n_ge counts the range's draws and out->p_value is
   (1 + n_ge) / (1 + count).  Because the stream is counter-based, a test with B
   permutations can be split into ranges (checkpoint and resume, or one range per
   GPU): the ranges' statistics are those of ept_test for the same draws, and the
   test's p-value is (1 + the sum of the ranges' n_ge) / (1 + B).  The paper has no
   counterpart (its permutations come from an unspecified R generator). */
ept_status ept_test_range(ept_ctx *ctx, const float *X, int64_t nx, const float *Y, int64_t ny,
                          int64_t p, int on_device, int stat, double sigma, int64_t b_first,
                          int64_t count, uint64_t seed, int prec, double *perm_stats,
                          ept_result *out, void *stream);

/* The same test on caller-given relabelings (testing, exhaustive enumeration).
   masks: n_masks * ceil((nx+ny)/32) uint32 words, row-major by relabeling; pooled
   row t (x rows first, then y rows) is bit t%32 of word t/32; a set bit sends the
   row to x*.  Each relabeling must have exactly nx bits set and none at t >= nx+ny
   (EPT_EINVAL otherwise).  The observed statistic is the identity relabeling,
   evaluated by the same kernels.  perm_stats: n_masks doubles (may be NULL). */
ept_status ept_test_masks(ept_ctx *ctx, const float *X, int64_t nx, const float *Y, int64_t ny,
                          int64_t p, int on_device, int stat, double sigma,
                          const uint32_t *masks, int64_t n_masks, int prec,
                          double *perm_stats, ept_result *out, void *stream);

/* One test of a batch (ept_test_batch): the arguments of ept_test. */
typedef struct {
    const float *X;        /* nx * p floats, row-major */
    const float *Y;        /* ny * p floats, row-major */
    int64_t nx, ny, p;
    int stat;              /* ept_stat */
    double sigma;          /* kernel bandwidth (MMD): > 0 or EPT_SIGMA_MEDIAN */
    int64_t B;             /* permutations */
    uint64_t seed;         /* permutation-stream seed */
    double *perm_stats;    /* B doubles or NULL */
} ept_test_desc;

/* Many independent tests of different sizes in one batched run (Algorithm 1 for
   each): every phase is one launch over all tests (the tests' work units share the
   GPU), and a repeated call with the same shapes on the context's own stream
   (stream = NULL) replays the captured CUDA graph of the whole run.  Per-test
   results go to results[0 .. n_tests-1]; each test's draws come from its own
   seed exactly as in ept_test, and the statistics equal ept_test's within
   rounding.  on_device applies to every X, Y and perm_stats of the batch.
   With a caller stream, the run starts after that stream's prior work (a graph
   replays on the context's stream, ordered after it) and the call returns when
   the results are ready.
   The contraction's chunk length is autotuned on the first call for a batch shape
   (environment: EPT_AUTOTUNE=0 disables it; EPT_AUTOTUNE_CACHE=<file> keeps the
   choices across processes). */
ept_status ept_test_batch(ept_ctx *ctx, const ept_test_desc *tests, int64_t n_tests, int on_device,
                          int prec, ept_result *results, void *stream);

/* Context options (ept_set_option).  EPT_OPT_GRAPHS (default 1): capture and
   replay CUDA graphs of repeated batches; with 0 every run is launched directly
   and the per-phase times of ept_result are filled in.  EPT_OPT_AUTOTUNE (default
   1 unless the environment sets EPT_AUTOTUNE=0): the autotuner of tensor-core runs.
   On the first call of a batch shape (several tests, or one test with (nx+ny)^2 B of
   at least 2.5e10) it times whole device runs of the batch with each candidate
   parameter set -- the defaults, the other relabeling-draw kernel, the other order
   of the contraction's units (by length, or by first K-block then length), units of
   4 K-blocks, longer units where EPT_OPT_MAX_CHUNK allows them, and (unless
   EPT_OPT_CONTRACTION fixes it) the other two contraction kernels, i.e. the MMA
   shapes M = 256 across a pair of SMs and N = 128 -- each with its recomputation of
   flagged statistics, keeps the fastest for the shape (ept_result.tuning,
   .tune_candidates) and uses it from then on; every candidate computes the same
   statistics except for the accumulation order.
   EPT_OPT_DRAW_MODE (default 0): relabeling-draw kernel, 0 = automatic (a thread
   per column when the batch has at least 1024 columns per SM, else a warp per
   column), 1 = a warp per column, 2 = a thread per column, 3 = groups of 32
   columns, eight warps computing the slots' ranks and one warp the sequential
   decisions; the draws are identical in every mode (caller relabelings always
   take 1).
   EPT_OPT_FAULT_INJECT_ALLOC (test hook, default 0): the next `value` acquisitions
   of device scratch (a run's arena, a serving batch's pool allocation) fail with
   EPT_ENOMEM on the host, without touching the GPU, to exercise error paths.
   EPT_OPT_FAULT_INJECT_STALL (test hook, default 0): in the next run (tensor-core
   path, launched directly) the contraction's MMA issuer waits on a device flag that
   nothing sets; its bounded wait expires after 2 s, every role of the kernel takes
   the abort path (drain copies, free tensor memory, return) and the call returns
   EPT_ETIMEOUT; the context stays usable.  One-shot.
   EPT_OPT_DEBUG_CHECKS (default 0): a stand-in for a memory checker -- every scratch
   region of a run is followed by a 256-byte guard band filled with a pattern before
   the run and checked after it, and the host checks the plan's invariants (tables,
   chunk ranges, the contraction schedule covering every unit once); a violation
   returns EPT_EINTERNAL.
   EPT_OPT_STREAM_BLOCKS (default 0): the streaming mode for tests whose packed
   blocks do not fit in device memory (single tests: ept_test, ept_test_range,
   ept_test_masks; split precision; a given sigma).  The row panels are taken in
   windows, in two passes: the first builds each window's blocks for the exact row
   sums of the pooled matrix (the centring needs them before any block is packed);
   the second builds each window again, packs it and contracts it against every
   relabeling, and the next window reuses the memory.  The blocks then need one
   window of memory instead of about 2 n^2 bytes, at the price of a second build.
   0 = automatic: a test streams when its resident scratch would not fit (the
   context budget, else the device's free memory), with the largest window that
   fits; k > 0 = every single test streams, with windows of at most k stored
   blocks of 256 x 64 entries (at least one panel); -1 = never (a test that does
   not fit fails with EPT_ENOMEM).  Streaming with the plain precision or the
   median bandwidth gives EPT_EUNSUPPORTED.  The arithmetic is the resident path's;
   only the order in which the windows' FP64 partial sums are added differs.
   EPT_OPT_WAIT_LIMIT_MS (default 2000, 10..600000): the limit of every bounded wait
   inside the tensor-core kernels (a pipeline barrier or flag that does not arrive
   within it makes the kernel record an error, drain and return; the call returns
   EPT_ETIMEOUT).
   EPT_OPT_MAX_CHUNK (default 32; 4, 8, 16 or 32): the longest contraction work unit,
   in K-blocks of 64 pooled columns, that the autotuner may pick (untuned runs use 8).
   The tensor cores accumulate each unit in FP32, and the error grows faster than the
   unit's length (measured: the accumulation coefficient of the error estimate below
   has to be 6.8, 15.4 and 51.4 for units of 8, 16 and 32 K-blocks on one sweep of 200
   problems, 23.6 for one statistic with units of 16 on 400 more); the estimate takes
   8, 32 and 96, so every length keeps the returned statistics within 1e-5 of the FP64
   oracle through the recomputation of the flagged ones, and the autotuner, which
   times whole runs with their recomputation, picks a longer unit only where it is
   faster all included.  With EPT_OPT_REFINE = 0 the fast values of longer units can
   be off by up to a few 1e-3 relative on strongly ill-conditioned inputs.
   EPT_OPT_REFINE (default 1; 0 or 1): FP64 recomputation of flagged statistics
   (Section 3.1's statistics, Eq. 1 / Eq. 2, evaluated from the raw rows).  Every
   statistic of the split and plain precisions carries an a-posteriori estimate of
   its error, E_b = k_b u cT A_b + 4 u Wbar / m: u = 2^-24, cT = (n/(nx ny))^2, A_b
   the sum of the absolute values of its contraction partial sums (the magnitudes its
   FP32 accumulations carried), Wbar the mean entry of the pooled matrix, m =
   min(nx, ny), k_b = 8 for a relabeling (32 with units of 16 K-blocks, 96 with units
   of 32) and 8 times that for the observed statistic and every statistic within
   1e-5 |observed| + 2 E_0 of it.  A statistic with
   E_b > 1e-5 |stat_b| is recomputed: when its representation term (the second) is
   above 1/20 of the tolerance, from W built in FP64 by direct differences of the
   widened inputs (Algorithm 3) and its three block sums in FP64; otherwise by summing
   the packed operand the contraction read with compensated arithmetic (which
   removes the FP32 accumulation error and keeps the entries).  The counts are then
   taken again.  The run needs extra device memory for it (8 bytes per row panel and
   re-summed statistic; for the FP64 rebuild 8 n bytes per row of a window of at most
   2 GiB and 16 bytes per 64 rows and statistic).  Flagged
   statistics arise on ill-conditioned inputs, such as a wide-kernel MMD of a few
   features whose permuted statistics are far below the FP32 resolution of the
   kernel values; ept_result.n_refined counts them.  Not applied in the streaming
   mode, by the pre-computation baseline or by ept_test_static.
   EPT_OPT_UNIT_KB (default 0; 0, 4, 8, 16 or 32): the contraction unit length of
   every run, in K-blocks (0: 8, or the autotuner's choice); the autotuner then tries
   no other length.
   EPT_OPT_CONTRACTION (default 0; 0..3): the tensor-core contraction kernel.  1:
   relabelings as the MMA's shared-memory operand (N = 256 relabelings, M = 128 rows
   of C; producer warps expand the mask bits into shared memory).  2: the same on
   pairs of SMs (clusters of two CTAs, tcgen05 cta_group::2; a work unit covers a
   whole 256-row panel, each CTA loads its 128 rows of the operand and expands its
   half of the relabelings, one CTA issues the MMAs for both).  3: relabelings as the
   tensor-memory operand (M = 128 relabelings stored from registers with tcgen05.st,
   N = 128 rows of C from shared memory; each epilogue thread sums its own
   relabeling's row values, no transposes).  0: the library's choice (1).  Measured
   on a GB300 (n = 5000, B = 10^4 contraction): 1 303 us, 2 311 us, 3 451 us (the
   MMA pipe alone, with N = 128, needs 366 us for the work that N = 256 does in 254
   us).  The statistics agree to the accumulation order.
   EPT_OPT_SERVE_LANES (default 3, 1..16): serving batches in flight at once;
   EPT_OPT_SERVE_SLOTS (default 256): serving requests in flight at once; both
   before the first ept_submit.  EPT_EINVAL for an unknown option or value.
   Environment: EPT_GRAPHS, EPT_AUTOTUNE, EPT_DRAW_MODE, EPT_DEBUG_CHECKS,
   EPT_STREAM_BLOCKS, EPT_WAIT_LIMIT_MS, EPT_MAX_CHUNK, EPT_REFINE, EPT_CONTRACTION, EPT_UNIT_KB,
   EPT_SERVE_LANES and EPT_SERVE_SLOTS set the
   starting value of the option of that name in every new context (an invalid value
   makes ept_create fail with EPT_EINVAL); EPT_AUTOTUNE_CACHE names a file in which
   the autotuner keeps its choices across processes. */
enum {
    EPT_OPT_GRAPHS = 1,
    EPT_OPT_AUTOTUNE = 2,
    EPT_OPT_SERVE_LANES = 3,
    EPT_OPT_SERVE_SLOTS = 4,
    EPT_OPT_DRAW_MODE = 5,
    EPT_OPT_FAULT_INJECT_ALLOC = 6,
    EPT_OPT_FAULT_INJECT_STALL = 7,
    EPT_OPT_DEBUG_CHECKS = 8,
    EPT_OPT_STREAM_BLOCKS = 9,
    EPT_OPT_WAIT_LIMIT_MS = 10,
    EPT_OPT_MAX_CHUNK = 11,
    EPT_OPT_REFINE = 12,
    EPT_OPT_CONTRACTION = 13,
    EPT_OPT_UNIT_KB = 14
};
ept_status ept_set_option(ept_ctx *ctx, int option, int64_t value);

/* Serving.  ept_submit queues one test (inputs are HOST pointers, copied before it
   returns, so the caller may free them) and returns a ticket.  A scheduler thread
   of the context admits queued requests in arrival order while request slots and
   the device-memory budget (the context's mem_budget_bytes, or 80% of the free
   device memory when 0) allow, runs everything admitted as one batch, and keeps
   several batches in flight at once, so requests that arrive while others run are
   started beside them (continuous batching).  Errors: EPT_ENOMEM if the request
   can never fit the budget, EPT_EBUSY if the queue is full.  Results equal
   ept_test's on the same inputs within rounding.  A request whose data is
   rejected on the device (NaN/Inf) fails alone; the rest of its batch is kept. */
ept_status ept_submit(ept_ctx *ctx, const ept_test_desc *request, int prec, uint64_t *ticket);

/* *done = 1 when the request has finished (or was cancelled), else 0. */
ept_status ept_poll(ept_ctx *ctx, uint64_t ticket, int *done);

/* Waits for the request (timeout_ms < 0: no limit) and releases the ticket: its
   B permuted statistics go to perm_stats (host, may be NULL), the result to out;
   for a served request out->ms_total is its latency from ept_submit to the
   scheduler seeing it finished (host clock), and the other times are 0.
   EPT_ETIMEOUT when not finished in time (the ticket stays valid),
   EPT_ECANCELLED for a cancelled request, EPT_ENOTFOUND for an unknown ticket. */
ept_status ept_wait(ept_ctx *ctx, uint64_t ticket, double *perm_stats, ept_result *out, int64_t timeout_ms);

/* Cancels a request: removed if still queued; if already running, its result is
   discarded when its batch finishes.  The ticket must still be waited on. */
ept_status ept_cancel(ept_ctx *ctx, uint64_t ticket);

/* Serving state (any pointer may be NULL): device scratch held by running batches,
   requests running, requests queued, finished requests not yet waited on.  All
   zero before the first ept_submit. */
ept_status ept_serving_stats(ept_ctx *ctx, size_t *bytes_in_use, int64_t *running, int64_t *queued,
                             int64_t *finished);

/* Serving lanes (any pointer may be NULL): lanes holding a running batch now, the
   most lanes that held one at the same time since the context's first ept_submit,
   and the number of requests submitted while at least one lane held a running batch
   (requests that arrived while others were on the GPU).  All zero before the first
   ept_submit. */
ept_status ept_serving_lanes(ept_ctx *ctx, int64_t *busy, int64_t *peak_busy, int64_t *submits_while_busy);

/* Draws b0 .. b0+count-1 of the permutation stream of `seed` (Algorithm 2's
   SampleWithoutReplacement, fixed as Philox4x32-10 + Knuth's selection sampling;
   draw 0 is the identity), generated on the GPU, written row-major as in
   ept_test_masks: count * ceil((nx+ny)/32) words. */
ept_status ept_perm_masks(ept_ctx *ctx, uint64_t seed, int64_t nx, int64_t ny, int64_t b0,
                          int64_t count, uint32_t *out, int on_device, void *stream);

/* Phase 1 alone (Algorithm 1, block construction; Algorithm 3): writes the pooled
   (nx+ny) x (nx+ny) matrix [[D_XX, D_XY], [D_XY', D_YY]] (or kernel values) as the
   library built it, expanded from its packed upper storage into a row-major FP32
   array D_out of (nx+ny)^2 floats.  For checking the blocks; not on the hot path. */
ept_status ept_build_blocks(ept_ctx *ctx, const float *X, int64_t nx, const float *Y,
                            int64_t ny, int64_t p, int on_device, int stat, double sigma,
                            int prec, float *D_out, void *stream);

/* Size of the device array that ept_test_static uses as its only scratch memory
   (16 MiB; it is part of the library image, so every GPU that loads libept holds it
   until the process exits). */
#define EPT_STATIC_SCRATCH_BYTES (16u << 20)

/* ept_test_static -- the split-BF16 test of ept_test that allocates nothing.  The
   paper has no counterpart: this is a service for callers that cannot call
   cudaMalloc, such as a host application whose own memory pool already owns all
   of the GPU's memory, or a latency-critical loop in which an allocation (which
   can synchronise the whole device) is not acceptable.
   All scratch lives in one file-scope device array of EPT_STATIC_SCRATCH_BYTES; a
   test whose scratch does not fit (roughly nx + ny above ~2300 at B = 10^4, or more
   permutations for smaller n) is rejected with EPT_EINVAL and a message giving the
   bytes it needs.  The call runs on the calling thread's current device and on
   `stream` (NULL = the legacy default stream); its first call on a device looks up
   the array's device address (cudaGetSymbolAddress) and caches it.  The call is
   synchronous: it reads its counters back to the host and waits for `stream`
   before returning.  X, Y and perm_stats (B doubles, may be NULL) are DEVICE
   pointers; out is a host struct (ms_total is host wall time, the other timing
   fields are 0); on any error perm_stats is left unwritten.  The test is planned
   by ept_test's planner (same descriptor and contraction chunks, units of 8
   K-blocks); its blocks are built by the plain FP32 SIMT kernel (the tensor-core
   build needs FP16 copies of the rows that the array has no room for), its
   relabelings are contracted on the tensor cores as in ept_test.  Every call
   reuses the same array: each call clears what must start at zero, calls from one
   process are serialised, and calls that overlap on the GPU (e.g. from several
   processes) race on the array.  It calls no cudaMalloc, cudaFree or other
   allocating routine. */
ept_status ept_test_static(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p,
                           int stat, double sigma, int64_t B, uint64_t seed, double *perm_stats,
                           ept_result *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* EPT_H */

// ept_internal.cuh -- layouts, batch descriptors and launchers shared by libept's
// translation units.
//
// Packed block storage.  The pooled matrix W = [[D_XX, D_XY], [D_XY', D_YY]] of the
// n = nx + ny pooled rows (x rows first) is symmetric, so only its upper part is
// built and stored (Algorithm 1 builds D_XX, D_YY, D_XY once; the memory-saving
// variant after Algorithm 1 never stores D_YX).  Rows are grouped in panels of
// PANEL = 256, columns in K-blocks of KB = 64.  Panel I stores the K-blocks
// kb = 4I .. NKB-1, i.e. every column from the start of its own diagonal 256x256
// square to the end.  Each stored block is 256 rows x 64 columns, row-major and
// contiguous; blocks are numbered panel by panel:
//     blk(I, kb) = I*NKB - 2*I*(I-1) + (kb - 4I).
// n is padded to n_pad = multiple of 256; padded rows/columns hold zeros.
//
// Relabeling masks are stored transposed, maskT[w][c] (word w of column c), so
// that the 32 lanes of a warp read 32 consecutive relabelings of one word.
// Column 0 is always the identity relabeling (the observed statistic); columns
// 1..B are the permuted ones (draws b0 .. b0+B-1 of the stream, b0 = 1 unless a
// range of the stream is asked for); padding columns are all-zero.
//
// Contracted group.  Eq. 1 and Eq. 2 are symmetric in x and y, so a relabeling can
// be described by either of its two groups.  The quadratic form is taken over the
// SMALLER group (x* when nx <= ny, otherwise y*): the sums over the larger group are
// then differences S - 2L + T of sums over the smaller one, and using the smaller
// group keeps the rounding errors of T small relative to the statistic when the
// sample sizes are very unequal.  When ny < nx the stored masks mark y* (`comp`).
//
// Batches.  Every kernel works on a batch of independent tests (a single test is a
// batch of one).  Each test's arrays live at its own offsets in the batch's
// concatenated buffers (TestDesc); a kernel maps its global work index to a test
// by binary search in a prefix-sum array over the tests (BatchPrefix).
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace ept {

constexpr int PANEL = 256;       // rows per panel (MMA N of the contraction)
constexpr int KB = 64;           // columns per K-block (one 128-byte swizzle row of 16-bit values)
constexpr int KB_PER_PANEL = PANEL / KB;
// K-blocks per contraction work unit (512 columns).  The tensor cores accumulate in FP32 with
// an error that grows faster than linearly with the number of accumulation steps, so the
// unit length bounds the contraction's error: measured on a wide-kernel MMD test whose
// permuted statistics are 1/70 of the observed one, 9.3e-6 relative at 8 K-blocks, 3.1e-5
// at 16 or 32 (the plain FP32 path: 3.5e-6).  Longer units are faster (fewer epilogues).
constexpr int CHUNK_KB_DEFAULT = 8;
constexpr int COL_PAD = 256;     // relabeling columns padded to this multiple
constexpr int BUILD_KB = 64;     // p is padded to a multiple of this for the tensor-core build
constexpr int TC_TILE_N = 256;   // relabelings per contraction work unit (the MMA's N)
// cap on the relabeling-draw blocks per SM (0: none, one warp per column).  Capping
// lets the draws share SMs with the tensor-core build, but the draws are
// latency-bound and run fastest at full occupancy, which measured best overall.
constexpr int MASK_CTAS_PER_SM = 0;

__host__ __device__ inline int64_t blk_off(int64_t I, int64_t NKB) { return I * NKB - 2 * I * (I - 1); }
__host__ __device__ inline int64_t blk_index(int64_t I, int64_t kb, int64_t NKB) {
    return blk_off(I, NKB) + (kb - KB_PER_PANEL * I);
}

struct Counters {
    unsigned long long n_ge;
    unsigned long long n_near;
    unsigned long long n_fixup;
    unsigned long long bad_mask;
    unsigned long long nonfinite;
    unsigned long long err_code;     // device-side bounded waits that gave up (kept in test 0)
    unsigned int max_d_bits;         // max |D_ij| over the stored blocks (FP32 bits; non-negative values
    unsigned int max_u_bits;         //   order like their bit patterns), max |u_i|,
    unsigned int max_dc_bits;        //   max |dcorr_i|: they bound |C| for the FP16 scale of the packing
    unsigned int sel_prefix;         // median heuristic: radix-selection prefix, then the median's bits
    unsigned int never_set;          // stays 0: the failure-path test hook waits for it
    unsigned long long sel_k;        //   rank still to find within the prefix
    unsigned long long guard_bad;    // debug checks: words of the guard bands found overwritten
    unsigned long long batch_failed; // (test 0) some test of a batched call has an error: device outputs
                                     //   of the call are then left unwritten
    unsigned long long n_flag;       // statistics whose error estimate exceeds the tolerance (refined in FP64)
};

// A-posteriori error estimate of a statistic computed by the contraction, and the
// statistics that are recomputed in FP64 (ept_refine.cu).  For relabeling column b:
//     E_b = k_b u cT A_b + REFINE_KR u Wbar / m,
// u = 2^-24 (the FP32 unit roundoff), cT the statistic's factor on s'Cs, A_b the sum
// over the contraction's work units of |partial sum| (the magnitudes the FP32
// accumulations of column b carried), Wbar = 1'W1 / n^2 the mean entry of the
// pooled matrix and m the contracted group's size (the FP32 representation errors
// of the m^2 entries a relabeling sums average out; the kernel values come from
// exp_cw, whose rounding errors carry no smooth bias).  k_b = refine_ka(L) for a
// relabeling (L the run's unit length in K-blocks: the accumulation error of a unit
// grows faster than its length) and REFINE_KC_RATIO times that for the observed
// statistic and every statistic within 1e-5 |stat_0| + 2 E_0 of it: relabelings
// aligned with the samples sum entries of one sign and similar size in the same
// order on the tensor cores, so their accumulation errors add coherently.
// Statistics with E_b > REFINE_TOL |stat_b| are flagged: when the representation term
// exceeds REFINE_L2 of the tolerance, for entries rebuilt in FP64 from the raw rows
// (level 2); otherwise for an exact re-summation of the packed operand the
// contraction read (level 1), which removes the accumulation part and leaves the
// FP32 representation of the entries.  The constants were fitted to measured GPU
// errors (a sweep of 200 ill-conditioned problems against the FP64 oracle, both
// precisions, units of 8, 16 and 32 K-blocks) so that every statistic off by more
// than half the tolerance is flagged: the relabelings needed k = 6.8, 15.4 and 51.4
// (tensor cores; 2.2, 2.5 and 6.8 on the plain path) with REFINE_KR = 4; the largest
// accumulation errors of observed statistics were 40 (tensor cores) and 53 (plain
// FP32) u cT A_0 with units of 8.  On 400 further problems one statistic with units
// of 16 needed k = 23.6, hence the wider margins of the longer units (32 and 96).
__host__ __device__ constexpr double refine_ka(int unit_kb) { return unit_kb <= 8 ? 8.0 : unit_kb <= 16 ? 32.0 : 96.0; }
constexpr double REFINE_KC_RATIO = 8.0;
constexpr double REFINE_KR = 4.0;
constexpr double REFINE_TOL = 1e-5;
constexpr double REFINE_L2 = 0.05;
constexpr double REFINE_U = 5.9604644775390625e-08;   // 2^-24

// Debug checks: guard bands of GUARD_BYTES after every scratch region, filled with a
// per-band pattern before a run and checked after it.
constexpr int GUARD_BYTES = 256;
constexpr int MAX_GUARDS = 48;
struct GuardList {
    int n;
    uint64_t off[MAX_GUARDS];
};
void launch_guards(uint8_t *arena, const GuardList &g, bool check, Counters *ctr, cudaStream_t s);

// Power-of-two scale c of a test's packed contraction operand, from the bound
// |C_ij| <= 2 (max|D| + 2 max|u|) + max|dcorr|: c |C| < 2^14, inside FP16's range.
// The exponent is clamped to [-60, 60] (c and 1/c stay normal FP32 numbers).
__device__ __forceinline__ float packed_scale(const Counters &k) {
    const float bound = 2.f * (__uint_as_float(k.max_d_bits) + 2.f * __uint_as_float(k.max_u_bits)) +
                        __uint_as_float(k.max_dc_bits);
    if (!(bound > 0.f) || !(bound < 3.0e38f)) return 1.f;
    int e;
    frexpf(bound, &e);   // bound = f 2^e, 0.5 <= f < 1
    int k2 = 14 - e;
    k2 = k2 < -60 ? -60 : (k2 > 60 ? 60 : k2);
    return ldexpf(1.f, k2);
}

// chunk q of a test's contraction: panel I, K-blocks [kb0, kb1)
struct Chunk { int I, kb0, kb1, pad; };
// A tensor-core contraction work unit as its kernels need it, built on the host for
// every position of the schedule (so that a CTA reads its next unit with one 64-byte
// load instead of walking the test, chunk and schedule tables): chunk (panel I,
// K-blocks [kb0, kb1), the two all-zero K-blocks below the diagonal skipped for the
// second row half), row half h, the relabeling columns of its 256-column tile that
// exist (at most 256), the test's K-blocks per panel row (NKB) and column stride (Bp),
// its first stored block, the maskT offset of the tile's first column and the
// partials offset of the unit's row (part0 + (2q + h) Bp + 256 m).
struct alignas(16) UnitRec {
    int32_t I, kb0, kb1, h, left, NKB;
    int64_t Bp, blk0, mask_col, out_off;
    int32_t pad[2];
};
static_assert(sizeof(UnitRec) == 64, "unit record");
// a stored block of the batch: test t, panel I, K-block kb
struct BlkInfo { int t, I, kb, pad; };
// a build tile of the batch: test t, rows of panel I (half h), columns of panel J >= I
struct Tile { int t, I, J, h; };

// One test of a batch as the kernels see it.  Offsets are element offsets into the
// batch's concatenated buffers.
struct TestDesc {
    const float *X, *Y;              // device rows (nx x p, ny x p)
    const uint32_t *user_masks;      // caller relabelings (row-major, nwu words each) or null
    double *out_stats;               // device destination of the B permuted statistics, or null
    int64_t nx, ny, n, p, B;
    int64_t n_pad, NP, NKB, nblk, nw, ncols, Bp, MT, nchunks, nparts, m, other, p_pad;
    int64_t row0;     // rows: norms, inverse scales, r, u, dcorr, FP16 rows (n_pad)
    int64_t blk0;     // blocks: D, C hi/lo, row parts (x256), column parts (x64) (nblk)
    int64_t pan0;     // panels: Upart, Stpart (NP)
    int64_t sp0;      // row groups of 32: Spart (n_pad / 32)
    int64_t mask0;    // mask words (nw * Bp)
    int64_t chunk0;   // chunk table (nchunks)
    int64_t part0;    // partials (nparts * Bp)
    int64_t col0;     // statistics (ncols)
    uint64_t seed;
    int64_t b0;                      // relabeling column c >= 1 is draw b0 + c - 1 of the stream
    int32_t stat, comp, kblocks, nwu;
    int32_t scaled, pad_;            // scaled: the partials carry the packing scale (tensor-core path)
    float neg_inv_2s2, tau;
    float inv_sigma;                 // Laplacian kernel: 1 / sigma
    int32_t kern;                    // entries the build writes: 0 distance, 1 Gaussian, 2 Laplacian kernel
    int32_t median;                  // bandwidth from the median heuristic (build distances, select, transform)
    int32_t pad2_;
    double cT, inv_o2, sign, kappa, inv_n, inv_2n2;
    double sigma64;                  // the given bandwidth in FP64 (FP64 refinement; 0 for ED and median)
    double ka;                       // accumulation coefficient of the error estimate (refine_ka of the unit length)
};

// Prefix sums over the tests (n_tests + 1 entries each) of the work dimensions.
struct BatchPrefix {
    const int64_t *rows;    // n_pad
    const int64_t *panels;  // NP
    const int64_t *cols;    // Bp
    const int64_t *units;   // tc_units (tensor-core contraction work units)
    const int64_t *simt;    // nchunks * 2 * (Bp / 64) (plain contraction work items)
};

// Device view of one batched run.
struct Batch {
    int n_tests;
    const TestDesc *desc;
    BatchPrefix pre;
    const BlkInfo *blk;
    const Tile *tiles;
    const Chunk *chunks;
    const int64_t *sched, *sched_off;    // contraction schedule per CTA (null: units strided over the grid)
    const UnitRec *urec;                 // the scheduled units' records, in schedule order (null: none)
    const UnitRec *urec_pair;            // pair contraction: the record of unit 2 pu for pair unit pu (null: none)
    int tc_grid;                         // contraction CTAs when scheduled
    int64_t nblk_total, ntiles, nrows_total, npan_total, ncols_total, nunits_total, nsimt_total;
    int64_t p_stride;                    // row stride of the FP16 rows (max p_pad)
    float *norms, *iscale, *u;
    uint16_t *Zh, *Zl, *Chi, *Clo;       // Chi / Clo: the split parts of block b start at b * c_stride
    int64_t c_stride;
    float *D, *partial;
    double *rowpart, *colpart, *r, *Spart, *dcorr, *Upart, *Stpart, *stats, *observed;
    double *errest;                      // per relabeling column: the accumulation part of E_b
    uint8_t *flags;                      // per relabeling column: 1 = recompute in FP64
    uint32_t *maskT;
    Counters *ctr;
    uint32_t *sel_hist;                  // median heuristic: 2048 bins per test (null if no test needs it)
    double *sacc;                        // streaming mode: FP64 sums of the windows' partials (Bp)
    int inject_stall;                    // failure-path test hook: the contraction's MMA issuer waits on a
                                         //   flag that nothing sets until its bounded wait expires
    unsigned long long wait_ns;          // limit of the tensor-core kernels' bounded waits (0: 2 s)
};

// tensor-core contraction work units of a test: chunk x relabeling tile x row half
__host__ __device__ inline int64_t tc_units(const TestDesc &d) { return d.nchunks * d.MT * 2; }

// the record of local unit lu of test d (units of a test are ordered (q, m, h)), its chunk ch
__host__ __device__ inline UnitRec unit_record(const TestDesc &d, int64_t lu, Chunk ch) {
    UnitRec r;
    const int64_t h = lu & 1, q = (lu >> 1) / d.MT, m = (lu >> 1) % d.MT;
    if (h == 1 && ch.kb0 == KB_PER_PANEL * ch.I && ch.kb1 - ch.kb0 > 2) ch.kb0 += 2;
    r.I = ch.I;
    r.kb0 = ch.kb0;
    r.kb1 = ch.kb1;
    r.h = (int32_t)h;
    const int64_t left = d.ncols - m * TC_TILE_N;
    r.left = left > TC_TILE_N ? TC_TILE_N : (int32_t)left;
    r.NKB = (int32_t)d.NKB;
    r.Bp = d.Bp;
    r.blk0 = d.blk0;
    r.mask_col = d.mask0 + m * TC_TILE_N;
    r.out_off = d.part0 + (2 * q + h) * d.Bp + m * TC_TILE_N;
    r.pad[0] = r.pad[1] = 0;
    return r;
}


// Contraction chunks of a test: panel I covers the L = NKBc - 4I K-blocks from its
// diagonal to NKBc = ceil(n / KB), the last K-block holding real columns (the padding
// columns of C are zero, so the contraction stops there), in ceil(L / chunk_kb)
// chunks of as equal a length as possible (each at most chunk_kb): a short last
// chunk would leave the tensor cores idle while its epilogue runs.
__host__ __device__ inline int64_t contract_nkb(const TestDesc &d) { return (d.n + KB - 1) / KB; }
__host__ __device__ inline int64_t panel_chunks(const TestDesc &d, int64_t I, int chunk_kb) {
    const int64_t len = contract_nkb(d) - KB_PER_PANEL * I;
    return len > 0 ? (len + chunk_kb - 1) / chunk_kb : 0;
}
__host__ __device__ inline Chunk panel_chunk(const TestDesc &d, int64_t I, int64_t q, int chunk_kb) {
    const int64_t len = contract_nkb(d) - KB_PER_PANEL * I, nq = panel_chunks(d, I, chunk_kb);
    const int64_t kb0 = KB_PER_PANEL * I + q * len / nq, kb1 = KB_PER_PANEL * I + (q + 1) * len / nq;
    return Chunk{(int)I, (int)kb0, (int)kb1, 0};
}

// The planner's description of one test (ept_api.cu; every entry point plans its
// tests with it): padding, panels, K-blocks, relabeling columns, the contracted
// group, the statistic's parameters and the combination constants.  The batch
// offsets (row0, blk0, ...) and the chunk count are left at zero.  sigma is a
// bandwidth > 0 or EPT_SIGMA_MEDIAN (MMD); split selects the tensor-core path.
void describe_test(TestDesc &d, int64_t nx, int64_t ny, int64_t p, int64_t B, int stat, double sigma,
                   uint64_t seed, bool split);

// Raises a kernel's dynamic shared-memory limit on the calling thread's current
// device, once per device (the attribute is per device; `done` holds one bit per
// device and concurrent first calls both set the same value).
cudaError_t smem_limit_once(const void *func, int bytes, unsigned long long *done);

// Entry of the pooled matrix from a squared distance d2 (FP32 or, for the fix-up of
// cancellation-prone pairs, FP64): the distance (Algorithm 3), the Gaussian kernel
// exp(-d2 / (2 sigma^2)) or the Laplacian kernel exp(-sqrt(d2) / sigma) (Appendix A.1).
__device__ __forceinline__ double entry_from_d2(double d2, int kern, float neg_inv_2s2, float inv_sigma) {
    if (kern == 0) return sqrt(d2);
    if (kern == 1) return exp(d2 * (double)neg_inv_2s2);
    return exp(-sqrt(d2) * (double)inv_sigma);
}

// exp(x) for x <= 0 in FP32, for the kernel values of Eq. 2 (Appendix A.1): Cody and
// Waite's range reduction (x = k ln 2 + r, |r| <= ln 2 / 2, ln 2 split in a 9-bit head
// whose products with k are exact and a tail) and the Taylor polynomial of degree 8
// of e^r, whose truncation error (|r|^9 / 9! < 2.1e-10) is far below FP32's unit
// roundoff; what is left is the rounding of the few FMAs, which varies from argument
// to argument instead of following the argument smoothly.  That matters here: a
// smooth error in the kernel values differs between the XX, YY and XY blocks and
// does not average out of the observed statistic.  Arguments below -87 give 0 and
// arguments above 0 are taken as 0 (the kernels' arguments are never positive); the
// scaling by 2^k (-126 < k <= 0) is a multiplication by a normal power of two.
__host__ __device__ __forceinline__ float exp_cw(float x) {
    if (!(x > -87.f)) return 0.f;
    x = x < 0.f ? x : 0.f;
    // k = x log2(e) rounded to an integer by adding 1.5 2^23 (the sum's unit is 1, so the
    // addition rounds to the nearest integer, which then sits in the low mantissa bits):
    // two additions instead of a rounding and a float-to-integer conversion, which run at
    // a quarter of the FP32 rate
    const float t = fmaf(x, 1.44269504f, 12582912.f);
    const float k = t - 12582912.f;
    float r = fmaf(-k, 0.693359375f, x);     // head of ln 2: exact products with |k| <= 126
    r = fmaf(-k, -2.12194440e-4f, r);        // tail of ln 2
    float q = 2.48015873e-5f;                // 1/8!
    q = fmaf(q, r, 1.98412698e-4f);          // 1/7!
    q = fmaf(q, r, 1.38888889e-3f);          // 1/6!
    q = fmaf(q, r, 8.33333333e-3f);          // 1/5!
    q = fmaf(q, r, 4.16666667e-2f);          // 1/4!
    q = fmaf(q, r, 1.66666667e-1f);          // 1/3!
    q = fmaf(q, r, 0.5f);
    q = fmaf(q, r, 1.f);
    q = fmaf(q, r, 1.f);
#ifdef __CUDA_ARCH__
    const uint32_t tb = __float_as_uint(t);
#else
    uint32_t tb;
    memcpy(&tb, &t, sizeof(tb));
#endif
    const uint32_t bits = (tb - 0x4B400000u + 127u) << 23;   // (k + 127) << 23, k = low bits of t
#ifdef __CUDA_ARCH__
    return q * __uint_as_float(bits);
#else
    float scale;
    memcpy(&scale, &bits, sizeof(scale));
    return q * scale;
#endif
}

// Knuth's TwoSum: s = fl(a + b) and the exact rounding error e, a + b = s + e.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ int find_test(const int64_t *pre, int nt, int64_t g) {
    int lo = 0, hi = nt - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the record of schedule position k of a batch: the precomputed one, or built from
// the unit's test and chunk (unscheduled runs: position k is unit k)
__device__ __forceinline__ UnitRec unit_at_position(const Batch &bt, int64_t k) {
    if (bt.urec) return bt.urec[k];
    const int64_t u = bt.sched ? bt.sched[k] : k;
    const int t = find_test(bt.pre.units, bt.n_tests, u);
    const TestDesc &d = bt.desc[t];
    const int64_t lu = u - bt.pre.units[t];
    return unit_record(d, lu, bt.chunks[d.chunk0 + (lu >> 1) / d.MT]);
}

// ---- launchers (ept_kernels.cu) ----
void launch_norms(const Batch &b, cudaStream_t s);                       // plain path: norms + finite check
void launch_build_simt(const Batch &b, cudaStream_t s);
void launch_blocksums(const Batch &b, cudaStream_t s);   // median-heuristic tests: kernel transform first
void launch_median_select(const Batch &b, cudaStream_t s);   // exact radix selection of the median distance
void launch_rowsum_reduce(const Batch &b, cudaStream_t s);
void launch_center(const Batch &b, cudaStream_t s);
void launch_pack(const Batch &b, bool split, cudaStream_t s);   // split: FP16 hi/lo (tensor-core path)
// draw kernels: a warp per relabeling column (caller relabelings, or few columns),
// a thread per column (many columns: 32 warps per SM or more), or (an option) groups
// of 32 columns whose ranks eight producer warps compute and one scanner warp turns
// into decisions
enum { DRAW_WARPS = 1, DRAW_LANES = 2, DRAW_SCAN = 3 };
constexpr int64_t DRAW_LANES_MIN_COLS_PER_SM = 32 * 32;
void launch_masks(const Batch &b, int num_sms, int mode, cudaStream_t s);   // draws or caller masks
void launch_contract_simt(const Batch &b, cudaStream_t s);
void launch_combine(const Batch &b, cudaStream_t s);                     // statistics, flags, counts, outputs
void launch_combine_count(const Batch &b, cudaStream_t s);               // counts and outputs alone (recount)

// ---- FP64 refinement of flagged statistics (ept_refine.cu): one test ----
// W64 rows [r0, r1) of test t (n pooled rows; all n columns, FP64, row stride n) from
// the raw rows; r0 is a multiple of 64
void launch_refine_w(const Batch &b, int t, int64_t n, double sigma, int64_t r0, int64_t r1, double *W64,
                     cudaStream_t s);
// for the nflag listed columns (test-local indexes): per 64-row tile of [r0, r1)
// the sums T = s'W s and L = s'W 1 over those rows (part[tile][k][2]) and
// spart[tile] = the rows' total
void launch_refine_rows(const Batch &b, int t, int64_t r0, int64_t r1, const double *W64, const int32_t *list,
                        int64_t nflag, double *part, double *spart, cudaStream_t s);
// the statistics of the listed columns from the partial sums of all ntiles row tiles
void launch_refine_finish(const Batch &b, int t, const int32_t *list, int64_t nflag, const double *part,
                          const double *spart, int64_t ntiles, cudaStream_t s);
void launch_reset_counts(const Batch &b, cudaStream_t s);   // n_ge = n_near = 0 before a recount
// The statistics of flagged columns from the packed operand the contraction read,
// summed exactly: one job per group of up to REFINE_JOB_COLS columns of one test
// (list[list0 ..] test-local column indexes; part[part0 + g * ncol + k] for the
// test's np x nkc (panel, chunk) pairs g, nkc = refine_packed_chunks(NKB)); every job
// of a run in one launch (max_ctas = the largest np x nkc).
constexpr int REFINE_JOB_COLS = 16;
struct RefineJob {
    int32_t t, ncol;
    int32_t np, nkc;
    int64_t list0, part0;
};
int64_t refine_packed_chunks(int64_t NKB);
void launch_refine_packed(const Batch &b, const RefineJob *jobs, int64_t njobs, int64_t max_ctas,
                          const int32_t *list, double *part, cudaStream_t s);

// single-draw-stream export (ept_perm_masks): columns 0..count-1 = draws b0..b0+count-1
void launch_perm_masks_plain(uint64_t seed, int nx, int ny, int64_t b0, int64_t count, int nw, uint32_t *maskT,
                             cudaStream_t s);
void launch_masks_to_rows(const uint32_t *maskT, int64_t ncols, int nw, int64_t count, int nwu, uint32_t *rows,
                          cudaStream_t s);
void launch_expand_blocks(const float *D, int64_t n, int64_t NKB, float *out, cudaStream_t s);

// ---- tensor-core kernels (ept_build_tc.cu, ept_contract_tc.cu) ----
void launch_split_rows(const Batch &b, cudaStream_t s);                  // FP16 hi/lo rows, norms, checks
cudaError_t launch_build_tc(const Batch &b, const void *tmaps4, int num_sms, cudaStream_t s);
cudaError_t launch_contract_tc(const Batch &b, const void *tmap_hi, const void *tmap_lo, int num_sms,
                               cudaStream_t s);
// the same contraction on pairs of SMs (clusters of two CTAs, tcgen05 cta_group::2;
// ept_contract_tc2.cu): units of whole 256-row panels, strided over the pairs
cudaError_t launch_contract_tc2(const Batch &b, const void *tmap_hi, const void *tmap_lo, int num_sms,
                                cudaStream_t s);
// the same contraction with the relabeling tile as the tensor-memory operand
// (ept_contract_tm.cu): M = 128 relabelings, N = 128 rows of C; the same units and
// partial sums as launch_contract_tc
cudaError_t launch_contract_tm(const Batch &b, const void *tmap_hi, const void *tmap_lo, int num_sms,
                               cudaStream_t s);
// TMA descriptors: the packed hi/lo blocks [nblk_total x 256 x 64], block stride
// c_stride halves, and the FP16
// rows [nrows x p_stride] (hi, lo with 64 x 128 boxes, then hi, lo with 64 x 256 boxes)
bool encode_block_tmaps(void *tmap_hi, void *tmap_lo, const uint16_t *Chi, const uint16_t *Clo, int64_t nblk,
                        int64_t c_stride, char *err, size_t errlen);
bool encode_rows_tmaps(void *tmaps4, const uint16_t *Zh, const uint16_t *Zl, int64_t nrows, int64_t p_stride,
                       char *err, size_t errlen);

// ---- streaming mode (ept_stream.cu): one test, windows of row panels ----
// r += the row and column sums of the window [I0, I1) (its stored blocks' parts)
void launch_stream_rowsums(const Batch &g, int64_t I0, int64_t I1, int64_t n_pad, cudaStream_t s);
// Spart from the complete r (then the resident path's launch_center)
void launch_stream_spart(const Batch &b, cudaStream_t s);
// sacc += the window's contraction partials
void launch_stream_accum(const Batch &g, cudaStream_t s);
// the statistics from sacc (after the last window)
void launch_stream_stats(const Batch &b, cudaStream_t s);

// ---- pre-computation baseline (ept_pooled.cu): one test, Algorithm 5 ----
// row chunks of the per-relabeling sums (about four CTAs per SM in all)
int64_t pooled_row_chunks(int64_t n, int64_t ncols, int num_sms);
// W (into b.D, row stride ld), the per-chunk sums (part: nchunks x 3 x ncols doubles)
// and the statistics (b.stats); the relabelings must be in b.maskT (marking x*)
cudaError_t launch_pooled(const Batch &b, int64_t n, int64_t ld, int64_t ncols, double *part, int64_t nchunks,
                          int64_t nw, cudaStream_t s);

void set_last_error(const char *msg);   // ept_api.cu

}  // namespace ept

// ept_internal.cuh -- layouts and launchers shared by libept's translation units.
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
// 1..B are the permuted ones; padding columns are all-zero.
//
// Contracted group.  Eq. 1 and Eq. 2 are symmetric in x and y, so a relabeling can
// be described by either of its two groups.  The quadratic form is taken over the
// SMALLER group (x* when nx <= ny, otherwise y*): the sums over the larger group are
// then differences S - 2L + T of sums over the smaller one, and using the smaller
// group keeps the rounding errors of T small relative to the statistic when the
// sample sizes are very unequal.  When ny < nx the stored masks mark y* (`comp`).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ept {

constexpr int PANEL = 256;   // rows per panel (MMA N of the contraction)
constexpr int KB = 64;       // columns per K-block (one 128-byte swizzle row of BF16)
constexpr int KB_PER_PANEL = PANEL / KB;
constexpr int CHUNK_KB = 16; // K-blocks per contraction work unit (1024 columns)
constexpr int COL_PAD = 256; // relabeling columns padded to this multiple

struct Geom {
    int64_t nx, ny, n, p;
    int64_t n_pad, NP, NKB, nblk, nw;
    int64_t ncols;   // relabeling columns actually used (identity + permuted)
    int64_t Bp;      // ncols padded to COL_PAD
    int64_t nchunks; // contraction work chunks (panel, K-block range)
    bool comp;       // masks mark y* (ny < nx) instead of x*
    int64_t m;       // size of the contracted group: min(nx, ny)
    int64_t other;   // size of the other group: max(nx, ny)
};

__host__ __device__ inline int64_t blk_off(int64_t I, int64_t NKB) { return I * NKB - 2 * I * (I - 1); }
__host__ __device__ inline int64_t blk_index(int64_t I, int64_t kb, int64_t NKB) {
    return blk_off(I, NKB) + (kb - KB_PER_PANEL * I);
}

Geom make_geom(int64_t nx, int64_t ny, int64_t p, int64_t ncols);

// chunk q of the contraction: panel I, K-blocks [kb0, kb1)
struct Chunk { int I, kb0, kb1, pad; };

// device parameters of the statistic's final combination
struct StatConst {
    double cT;        // (n / (nx ny))^2
    double S_tilde;   // unused: S~ is summed from the per-panel parts by the combination
    double inv_o2;    // 1 / other^2 (the larger group's size)
    double sign;      // -1 for ED, +1 for MMD
};

struct Counters {
    unsigned long long n_ge;
    unsigned long long n_near;
    unsigned long long n_fixup;
    unsigned long long bad_mask;
    unsigned long long nonfinite;
    unsigned long long err_code;   // device-side bounded waits that gave up, etc.
    unsigned long long maxabs_bits;  // bit pattern of max |x| over the finite inputs (FP32, as an integer)
};

// ---- launchers (ept_kernels.cu) ----
void launch_perm_masks(uint64_t seed, int nx, int ny, int64_t b_first, int64_t count, int64_t ncols,
                       int nw, bool comp, uint32_t *maskT, cudaStream_t s);
void launch_user_masks(const uint32_t *user, int64_t n_masks, int nwu, int nx, int n, int64_t ncols,
                       int nw, bool comp, uint32_t *maskT, Counters *ctr, cudaStream_t s);
void launch_masks_to_rows(const uint32_t *maskT, int64_t ncols, int nw, int64_t count, int nwu,
                          uint32_t *rows, cudaStream_t s);
void launch_check_finite(const float *a, int64_t count, Counters *ctr, cudaStream_t s);
void launch_norms(const float *X, const float *Y, const Geom &g, float *norms, cudaStream_t s);
void launch_build_simt(const float *X, const float *Y, const float *norms, const Geom &g, int stat,
                       double sigma, double tau, const int2 *blk_info, float *D, Counters *ctr,
                       cudaStream_t s);
void launch_blocksums(const float *D, const Geom &g, double *rowpart, double *colpart, cudaStream_t s);
// r: n_pad doubles; Spart: n_pad / 32 doubles; Upart, Stpart: one double per panel (NP)
void launch_rowsum_reduce(const double *rowpart, const double *colpart, const Geom &g, double *r, double *Spart,
                          cudaStream_t s);
void launch_center(const double *r, const double *Spart, const Geom &g, float *u, double *dcorr, double *Upart,
                   double *Stpart, StatConst *sc, int stat, cudaStream_t s);
void launch_pack_fp32(const float *D, const float *u, const double *dcorr, const Geom &g,
                      const int2 *blk_info, float *C, cudaStream_t s);
void launch_pack_bf16(const float *D, const float *u, const double *dcorr, const Geom &g,
                      const int2 *blk_info, uint16_t *Chi, uint16_t *Clo, cudaStream_t s);
void launch_contract_simt(const float *C, const uint32_t *maskT, const Chunk *chunks, const Geom &g,
                          float *partial, cudaStream_t s);
void launch_combine(const float *partial, int64_t nparts, const Geom &g, const StatConst *sc,
                    const double *Stpart, double *stats, Counters *ctr, cudaStream_t s);
void launch_expand_blocks(const float *D, const Geom &g, float *out, cudaStream_t s);

// ---- tcgen05 contraction (ept_contract_tc.cu) ----
// Returns cudaSuccess or the launch error.  Chi/Clo: packed BF16 hi/lo parts.
cudaError_t launch_contract_tc(const void *tmap_hi, const void *tmap_lo, const uint32_t *maskT,
                               const Chunk *chunks, const Geom &g, float *partial, Counters *ctr,
                               int num_sms, cudaStream_t s);
// Encodes the two TMA tensor maps over the packed hi/lo blocks (host side).
bool encode_block_tmaps(void *tmap_hi, void *tmap_lo, const uint16_t *Chi, const uint16_t *Clo,
                        int64_t nblk, char *err, size_t errlen);
// Encodes four TMA tensor maps over the FP16 hi/lo pooled rows [n_pad x p_pad]:
// (hi, lo) with 64 x 128 boxes, then (hi, lo) with 64 x 256 boxes.
bool encode_rows_tmaps(void *tmaps4, const uint16_t *Zh, const uint16_t *Zl, int64_t n_pad, int64_t p_pad,
                       char *err, size_t errlen);

// ---- tcgen05 block build (ept_build_tc.cu) ----
constexpr int BUILD_KB = 64;   // p is padded to a multiple of this
// Zh, Zl: FP16 hi / lo parts of the rows scaled by per-row powers of two; inv_scale[i]
// is the inverse scale of row i; non-finite inputs are counted in ctr->nonfinite.
void launch_split_rows(const float *X, const float *Y, const Geom &g, int64_t p_pad, uint16_t *Zh, uint16_t *Zl,
                       float *norms, float *inv_scale, Counters *ctr, cudaStream_t s);
// tiles: (panel I, half h, column panel J >= I); tmaps: the four maps of encode_rows_tmaps
cudaError_t launch_build_tc(const void *tmaps, const int4 *tiles, int ntiles, int64_t p_pad, const float *norms,
                            const float *inv_scale, const float *X, const float *Y, const Geom &g, int stat,
                            double sigma, double tau, float *D, Counters *ctr, int num_sms, cudaStream_t s);

}  // namespace ept

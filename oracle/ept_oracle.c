/*
 * ept_oracle.c -- plain FP64 CPU oracle for the efficient permutation two-sample
 * test of Chaibub Neto, "Computationally efficient permutation tests for the
 * multivariate two-sample problem based on energy distance or maximum mean
 * discrepancy statistics" (arXiv 2406.06488).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
 * Python binding) may call, link or load this file; only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark use it.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes, each function citing the passage it follows:
 *   - the energy-distance V-statistic of Eq. 1 and the biased MMD^2 of Eq. 2,
 *     with Euclidean distances computed pair by pair as in Algorithm 3
 *     (Appendix A.1) and the Gaussian kernel exp(-||x-y||^2 / (2 sigma^2)), or the
 *     Laplacian kernel exp(-||x-y|| / sigma) (the other reading of Appendix A.1's
 *     "exponential of the negative scaled Euclidean distance");
 *   - the median heuristic for the bandwidth: the lower median of the distances
 *     between the distinct pairs of the pooled sample;
 *   - the standard permutation test (Algorithm 4, Appendix A.2): every permuted
 *     statistic recomputed from the permuted raw rows;
 *   - the pre-computation test (Algorithm 5, Appendix A.2): one pooled matrix,
 *     sliced per permutation;
 *   - the efficient test (Algorithm 1 with Algorithm 2, Section 4.1): three blocks
 *     built once, permuted matrices filled by the twelve block assignments;
 *   - the permutation p-value (1 + #{stat* >= stat_o}) / (1 + b) (Section 3.1);
 *   - the permutation stream: Philox4x32-10 (Salmon, Moraes, Dror and Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11) driving Knuth's
 *     selection sampling (Algorithm S, TAOCP vol. 2, Section 3.4.2), the library's
 *     fixed reading of "SampleWithoutReplacement" (Algorithm 2);
 *   - exhaustive enumeration of all C(n, nx) relabelings (exact p-value).
 *
 * All arithmetic is IEEE double; inputs are FP32 samples widened exactly.
 * Nothing here is blocked, fused or reordered beyond what the cited definition
 * states, except that independent permutations run on separate OpenMP threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EO_STAT_ED 0
#define EO_STAT_MMD 1          /* Gaussian kernel */
#define EO_STAT_MMD_LAPLACE 2  /* Laplacian kernel */

/* Test-only mutation switch.  The default build (EO_MUTANT undefined or 0) is the
 * oracle.  The pin tests compile copies with EO_MUTANT = 1..12, each planting one
 * plausible mistake, and check that at least one pin fails for every mutant. */
#ifndef EO_MUTANT
#define EO_MUTANT 0
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, written from Salmon et al. (SC'11): a 4x32-bit counter and a
 * 2x32-bit key; each round multiplies counter words 0 and 2 by the two Philox
 * multipliers, and mixes the high halves with words 1 and 3 and the round key;
 * the key is bumped by the two Weyl constants between rounds. */
void eo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0 && EO_MUTANT != 1) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------- */
/* One draw of the permutation stream: which of the n = nx + ny pooled rows go to
 * the permuted first sample x*.  Algorithm 2 samples nx of the n pooled indexes
 * without replacement (SampleWithoutReplacement); the paper leaves the generator
 * open, so the library fixes it as follows.
 *   b = 0 is the identity relabeling (rows 0..nx-1 form x*).
 *   b >= 1: Knuth's selection sampling visits slots t = 0 .. n-1 in order and keeps
 *   slot t with probability need/remaining, where need = nx - (slots kept so far)
 *   and remaining = n - t.  The uniform variate of slot t is the 64-bit word
 *   u_t = (w[2h+1] << 32) | w[2h] of Philox4x32-10 with key (seed lo, seed hi) and
 *   counter (t / 2, 0, b lo, b hi), where h = t mod 2.  Slot t is kept iff
 *   floor(u_t * remaining / 2^64) < need.
 * sel[t] = 1 marks slot t as a member of x*. */
void eo_perm_select(uint64_t seed, int64_t nx, int64_t ny, int64_t b, uint8_t *sel)
{
    const int64_t n = nx + ny;
    if (b == 0) {
        for (int64_t t = 0; t < n; ++t) sel[t] = (uint8_t)(t < nx);
        return;
    }
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t words[4] = {0, 0, 0, 0};
    int64_t kept = 0;
    for (int64_t t = 0; t < n; ++t) {
        if ((t & 1) == 0) {
            const uint32_t ctr[4] = {(uint32_t)(t >> 1), 0u, (uint32_t)(uint64_t)b,
                                     (uint32_t)((uint64_t)b >> 32)};
            eo_philox4x32_10(ctr, key, words);
        }
        const int h = (int)(t & 1);
        const uint64_t u = ((uint64_t)words[2 * h + 1] << 32) | (uint64_t)words[2 * h];
        const uint64_t remaining = (uint64_t)(n - t);
        const uint64_t need = (uint64_t)(nx - kept);
        const uint64_t r = (uint64_t)(((unsigned __int128)u * remaining) >> 64);
        if (EO_MUTANT == 2 ? (r <= need) : (r < need)) {
            sel[t] = 1;
            ++kept;
        } else {
            sel[t] = 0;
        }
    }
}

/* count draws of the stream, b = b0 .. b0+count-1, row-major [count][n]. */
void eo_perm_select_many(uint64_t seed, int64_t nx, int64_t ny, int64_t b0, int64_t count,
                         uint8_t *sel)
{
    const int64_t n = nx + ny;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < count; ++c) eo_perm_select(seed, nx, ny, b0 + c, sel + c * n);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2 (PermutationIndexesTwoSampleTest), given the sampled pooled indexes
 * idx_p1 (1-based, length nx, in the order they were drawn).  idx_p2 is the set
 * difference in increasing order.  Outputs (1-based, as in the paper), packed one
 * after another into out: i1, i2, i1*, i2*, j1, j2, j1*, j2*; lens[8] receives the
 * eight lengths.  Returns 0, or -1 if idx_p1 is not a set of nx distinct indexes
 * in 1..n. */
int eo_alg2_indices(int64_t nx, int64_t ny, const int64_t *idx_p1, int64_t *out, int64_t *lens)
{
    const int64_t n = nx + ny;
    /* idx_w = (1..n); idx_g = (1..nx, 1..ny) */
    int64_t *idx_g = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    uint8_t *in_p1 = (uint8_t *)calloc((size_t)(n + 1), 1);
    int64_t *idx_p2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!idx_g || !in_p1 || !idx_p2) {
        free(idx_g); free(in_p1); free(idx_p2);
        return -1;
    }
    for (int64_t w = 1; w <= n; ++w) idx_g[w] = (w <= nx) ? w : w - nx;
    for (int64_t k = 0; k < nx; ++k) {
        const int64_t w = idx_p1[k];
        if (w < 1 || w > n || in_p1[w]) {
            free(idx_g); free(in_p1); free(idx_p2);
            return -1;
        }
        in_p1[w] = 1;
    }
    int64_t np2 = 0;
    for (int64_t w = 1; w <= n; ++w)
        if (!in_p1[w]) idx_p2[np2++] = w;

    int64_t *o = out;
    /* i1 = idx_g[idx_p1[Which(idx_p1 <= nx)]] */
    int64_t l_i1 = 0;
    for (int64_t k = 0; k < nx; ++k)
        if (idx_p1[k] <= nx) o[l_i1++] = idx_g[idx_p1[k]];
    o += l_i1;
    /* i2 = idx_g[idx_p1[Which(idx_p1 > nx)]] */
    int64_t l_i2 = 0;
    for (int64_t k = 0; k < nx; ++k)
        if (idx_p1[k] > nx) o[l_i2++] = idx_g[idx_p1[k]];
    o += l_i2;
    /* i1* = (1..|i1|); i2* = (|i1|+1 .. nx) */
    for (int64_t k = 0; k < l_i1; ++k) *o++ = k + 1;
    for (int64_t k = l_i1; k < nx; ++k) *o++ = k + 1;
    /* j1 = idx_g[idx_p2[Which(idx_p2 <= nx)]]; j2 likewise with > nx */
    int64_t l_j1 = 0;
    for (int64_t k = 0; k < np2; ++k)
        if (idx_p2[k] <= nx) o[l_j1++] = idx_g[idx_p2[k]];
    o += l_j1;
    int64_t l_j2 = 0;
    for (int64_t k = 0; k < np2; ++k)
        if (idx_p2[k] > nx) o[l_j2++] = idx_g[idx_p2[k]];
    o += l_j2;
    /* j1* = (1..|j1|); j2* = (|j1|+1 .. ny) */
    for (int64_t k = 0; k < l_j1; ++k) *o++ = k + 1;
    for (int64_t k = l_j1; k < ny; ++k) *o++ = k + 1;

    lens[0] = l_i1; lens[1] = l_i2; lens[2] = l_i1; lens[3] = nx - l_i1;
    lens[4] = l_j1; lens[5] = l_j2; lens[6] = l_j1; lens[7] = ny - l_j1;
    free(idx_g); free(in_p1); free(idx_p2);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 3 (Appendix A.1): D = (sum_k (a_k - b_k)^2)^(1/2).  The Gaussian
 * kernel of Appendix A.1 (and Eq. 2) is exp(-(sum_k (a_k - b_k)^2) / (2 sigma^2));
 * the Laplacian kernel is exp(-D / sigma). */
static double eo_sqdist(const double *a, const double *b, int64_t p)
{
    double s = 0.0;
    for (int64_t k = 0; k < p; ++k) {
        const double d = a[k] - b[k];
        s += d * d;
    }
    return s;
}

static double eo_entry(const double *a, const double *b, int64_t p, int stat, double sigma)
{
    const double s = eo_sqdist(a, b, p);
    if (stat == EO_STAT_ED) return sqrt(s);
    if (stat == EO_STAT_MMD_LAPLACE) return exp(-(EO_MUTANT == 8 ? s : sqrt(s)) / sigma);
    return exp(-s / ((EO_MUTANT == 3 ? 1.0 : 2.0) * sigma * sigma));
}

/* The matrix of Algorithm 3 between the rows of a (na x p) and b (nb x p):
 * out[i * nb + j] = D(a_i, b_j) (or the kernel value). */
void eo_block_matrix(const double *a, int64_t na, const double *b, int64_t nb, int64_t p,
                     int stat, double sigma, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < na; ++i)
        for (int64_t j = 0; j < nb; ++j)
            out[i * nb + j] = eo_entry(a + i * p, b + j * p, p, stat, sigma);
}

/* Sum of all entries of a matrix, row by row. */
static double eo_matrix_sum(const double *m, int64_t rows, int64_t cols)
{
    double s = 0.0;
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) s += m[i * cols + j];
    return s;
}

/* Eq. 1 (ED) or Eq. 2 (biased MMD^2) from the three matrix sums:
 * ED    = 2/(nx ny) Sxy - 1/nx^2 Sxx - 1/ny^2 Syy
 * MMD^2 = 1/nx^2 Kxx + 1/ny^2 Kyy - 2/(nx ny) Kxy.
 * (Algorithms 4 and 5 print 2/(nx nx) for the cross term; Eq. 1, Algorithm 1 and
 * the text use 2/(nx ny), which is the reading taken here.) */
static double eo_combine(double sxx, double syy, double sxy, int64_t nx, int64_t ny, int stat)
{
    const double fx = (double)nx, fy = (double)ny;
    if (stat == EO_STAT_ED)
        return 2.0 / (fx * (EO_MUTANT == 4 ? fx : fy)) * sxy - sxx / (fx * fx) - syy / (fy * fy);
    return sxx / (fx * fx) + syy / (fy * fy) - 2.0 / (fx * fy) * sxy;
}

/* Eq. 1 / Eq. 2 computed directly from raw rows (the statistic line of
 * Algorithm 4): every pairwise distance recomputed, all k, l included (the
 * V-statistic: D_kk = 0, K_kk = 1 on the diagonal). */
double eo_stat_direct(const double *x, int64_t nx, const double *y, int64_t ny, int64_t p,
                      int stat, double sigma)
{
    double sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (int64_t k = 0; k < nx; ++k)
        for (int64_t l = 0; l < ny; ++l) sxy += eo_entry(x + k * p, y + l * p, p, stat, sigma);
    for (int64_t k = 0; k < nx; ++k)
        for (int64_t l = 0; l < nx; ++l)
            if (EO_MUTANT != 5 || k != l) sxx += eo_entry(x + k * p, x + l * p, p, stat, sigma);
    for (int64_t k = 0; k < ny; ++k)
        for (int64_t l = 0; l < ny; ++l)
            if (EO_MUTANT != 5 || k != l) syy += eo_entry(y + k * p, y + l * p, p, stat, sigma);
    return eo_combine(sxx, syy, sxy, nx, ny, stat);
}

/* Widen FP32 samples to the pooled FP64 matrix w = (x, y)^T. */
static double *eo_pool(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p)
{
    const int64_t n = nx + ny;
    double *w = (double *)malloc(sizeof(double) * (size_t)(n * p));
    if (!w) return NULL;
    for (int64_t i = 0; i < nx * p; ++i) w[i] = (double)X[i];
    for (int64_t i = 0; i < ny * p; ++i) w[nx * p + i] = (double)Y[i];
    return w;
}

/* ------------------------------------------------------------------------- */
/* Standard test (Algorithm 4): for each relabeling, x* = rows with sel = 1 and
 * y* = rows with sel = 0 of the pooled data (row order within x* and y* does not
 * change the statistic, Appendix A.4), and the statistic is recomputed from those
 * raw rows.  sel is [nperm][n]; stats[nperm] receives the statistics.  Returns 0,
 * or -1 on a malformed relabeling (wrong count of ones) or allocation failure. */
int eo_test_direct(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p, int stat,
                   double sigma, const uint8_t *sel, int64_t nperm, double *stats)
{
    const int64_t n = nx + ny;
    double *w = eo_pool(X, nx, Y, ny, p);
    if (!w) return -1;
    int bad = 0;
#pragma omp parallel
    {
        double *xs = (double *)malloc(sizeof(double) * (size_t)(nx * p));
        double *ys = (double *)malloc(sizeof(double) * (size_t)(ny * p));
        if (!xs || !ys) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < nperm; ++b) {
            if (!xs || !ys) continue;
            const uint8_t *s = sel + b * n;
            int64_t a = 0, c = 0;
            for (int64_t t = 0; t < n; ++t) {
                if (s[t]) {
                    if (a < nx) memcpy(xs + a * p, w + t * p, sizeof(double) * (size_t)p);
                    ++a;
                } else {
                    if (c < ny) memcpy(ys + c * p, w + t * p, sizeof(double) * (size_t)p);
                    ++c;
                }
            }
            if (a != nx) {
#pragma omp atomic write
                bad = 1;
                stats[b] = NAN;
                continue;
            }
            stats[b] = eo_stat_direct(xs, nx, ys, ny, p, stat, sigma);
        }
        free(xs);
        free(ys);
    }
    free(w);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Pre-computation test (Algorithm 5): D_WW of the pooled data computed once;
 * for each relabeling, the permuted matrices are slices of D_WW and the
 * statistic is Eq. 1 / Eq. 2 of their sums. */
int eo_test_pooled(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p, int stat,
                   double sigma, const uint8_t *sel, int64_t nperm, double *stats)
{
    const int64_t n = nx + ny;
    double *w = eo_pool(X, nx, Y, ny, p);
    double *dww = (double *)malloc(sizeof(double) * (size_t)(n * n));
    if (!w || !dww) {
        free(w); free(dww);
        return -1;
    }
    eo_block_matrix(w, n, w, n, p, stat, sigma, dww);
    int bad = 0;
#pragma omp parallel
    {
        int64_t *ix = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        int64_t *iy = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
#pragma omp for schedule(dynamic, 4)
        for (int64_t b = 0; b < nperm; ++b) {
            if (!ix || !iy) continue;
            const uint8_t *s = sel + b * n;
            int64_t a = 0, c = 0;
            for (int64_t t = 0; t < n; ++t) {
                if (s[t]) ix[a++] = t;
                else iy[c++] = t;
            }
            if (a != nx) {
#pragma omp atomic write
                bad = 1;
                stats[b] = NAN;
                continue;
            }
            double sxy = 0.0, sxx = 0.0, syy = 0.0;
            for (int64_t k = 0; k < nx; ++k)
                for (int64_t l = 0; l < ny; ++l) sxy += dww[ix[k] * n + iy[l]];
            for (int64_t k = 0; k < nx; ++k)
                for (int64_t l = 0; l < nx; ++l) sxx += dww[ix[k] * n + ix[l]];
            for (int64_t k = 0; k < ny; ++k)
                for (int64_t l = 0; l < ny; ++l) syy += dww[iy[k] * n + iy[l]];
            stats[b] = eo_combine(sxx, syy, sxy, nx, ny, stat);
        }
        if (!ix || !iy) {
#pragma omp atomic write
            bad = 1;
        }
        free(ix);
        free(iy);
    }
    free(w);
    free(dww);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Efficient test (Algorithm 1): D_XX, D_YY, D_XY built once (D_YX = D_XY^T);
 * per relabeling, Algorithm 2 maps the sampled pooled indexes to the index lists
 * i1, i2, j1, j2 (and their destination slots), the permuted matrices D_X*X*,
 * D_Y*Y*, D_X*Y* are filled by the twelve block assignments, and the statistic
 * is Eq. 1 / Eq. 2 of their sums.  The sampled indexes are taken in increasing
 * pooled order (the statistic does not depend on the row order, Appendix A.4). */
int eo_test_blocks(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p, int stat,
                   double sigma, const uint8_t *sel, int64_t nperm, double *stats)
{
    const int64_t n = nx + ny;
    double *w = eo_pool(X, nx, Y, ny, p);
    double *dxx = (double *)malloc(sizeof(double) * (size_t)(nx * nx));
    double *dyy = (double *)malloc(sizeof(double) * (size_t)(ny * ny));
    double *dxy = (double *)malloc(sizeof(double) * (size_t)(nx * ny));
    double *dyx = (double *)malloc(sizeof(double) * (size_t)(nx * ny));
    if (!w || !dxx || !dyy || !dxy || !dyx) {
        free(w); free(dxx); free(dyy); free(dxy); free(dyx);
        return -1;
    }
    const double *xw = w, *yw = w + nx * p;
    /* Algorithm 1, block construction and D_YX = D_XY^T */
    eo_block_matrix(xw, nx, xw, nx, p, stat, sigma, dxx);
    eo_block_matrix(yw, ny, yw, ny, p, stat, sigma, dyy);
    eo_block_matrix(xw, nx, yw, ny, p, stat, sigma, dxy);
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < ny; ++j) dyx[j * nx + i] = dxy[i * ny + j];

    int bad = 0;
#pragma omp parallel
    {
        int64_t *idx_p1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)nx);
        int64_t *lists = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * n));
        double *pxx = (double *)malloc(sizeof(double) * (size_t)(nx * nx));
        double *pyy = (double *)malloc(sizeof(double) * (size_t)(ny * ny));
        double *pxy = (double *)malloc(sizeof(double) * (size_t)(nx * ny));
        const int ok = idx_p1 && lists && pxx && pyy && pxy;
        if (!ok) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t b = 0; b < nperm; ++b) {
            if (!ok) continue;
            const uint8_t *s = sel + b * n;
            int64_t a = 0;
            for (int64_t t = 0; t < n; ++t)
                if (s[t]) {
                    if (a < nx) idx_p1[a] = t + 1;
                    ++a;
                }
            int64_t lens[8];
            if (a != nx || eo_alg2_indices(nx, ny, idx_p1, lists, lens) != 0) {
#pragma omp atomic write
                bad = 1;
                stats[b] = NAN;
                continue;
            }
            const int64_t *i1 = lists, *i2 = i1 + lens[0], *i1s = i2 + lens[1];
            const int64_t *i2s = i1s + lens[2], *j1 = i2s + lens[3], *j2 = j1 + lens[4];
            const int64_t *j1s = j2 + lens[5], *j2s = j1s + lens[6];
            const int64_t L1 = lens[0], L2 = lens[1], M1 = lens[4], M2 = lens[5];
            /* 1-based index lists; D(r, c) below uses them with -1 */
#define AT(m, ld, r, c) (m)[((r) - 1) * (ld) + ((c) - 1)]
            /* D_X*X*: [i1*, i1*] <- D_XX[i1, i1]; [i1*, i2*] <- D_XY[i1, i2];
             *         [i2*, i1*] <- D_YX[i2, i1]; [i2*, i2*] <- D_YY[i2, i2] */
            for (int64_t r = 0; r < L1; ++r)
                for (int64_t c = 0; c < L1; ++c) AT(pxx, nx, i1s[r], i1s[c]) = AT(dxx, nx, i1[r], i1[c]);
            for (int64_t r = 0; r < L1; ++r)
                for (int64_t c = 0; c < L2; ++c) AT(pxx, nx, i1s[r], i2s[c]) = AT(dxy, ny, i1[r], i2[c]);
            for (int64_t r = 0; r < L2; ++r)
                for (int64_t c = 0; c < L1; ++c)
                    AT(pxx, nx, i2s[r], i1s[c]) = (EO_MUTANT == 6) ? AT(dxy, ny, i1[c], (i2[r] % ny) + 1)
                                                                   : AT(dyx, nx, i2[r], i1[c]);
            for (int64_t r = 0; r < L2; ++r)
                for (int64_t c = 0; c < L2; ++c) AT(pxx, nx, i2s[r], i2s[c]) = AT(dyy, ny, i2[r], i2[c]);
            /* D_Y*Y*: [j1*, j1*] <- D_XX[j1, j1]; [j1*, j2*] <- D_XY[j1, j2];
             *         [j2*, j1*] <- D_YX[j2, j1]; [j2*, j2*] <- D_YY[j2, j2] */
            for (int64_t r = 0; r < M1; ++r)
                for (int64_t c = 0; c < M1; ++c) AT(pyy, ny, j1s[r], j1s[c]) = AT(dxx, nx, j1[r], j1[c]);
            for (int64_t r = 0; r < M1; ++r)
                for (int64_t c = 0; c < M2; ++c) AT(pyy, ny, j1s[r], j2s[c]) = AT(dxy, ny, j1[r], j2[c]);
            for (int64_t r = 0; r < M2; ++r)
                for (int64_t c = 0; c < M1; ++c) AT(pyy, ny, j2s[r], j1s[c]) = AT(dyx, nx, j2[r], j1[c]);
            for (int64_t r = 0; r < M2; ++r)
                for (int64_t c = 0; c < M2; ++c) AT(pyy, ny, j2s[r], j2s[c]) = AT(dyy, ny, j2[r], j2[c]);
            /* D_X*Y*: [i1*, j1*] <- D_XX[i1, j1]; [i1*, j2*] <- D_XY[i1, j2];
             *         [i2*, j1*] <- D_YX[i2, j1]; [i2*, j2*] <- D_YY[i2, j2] */
            for (int64_t r = 0; r < L1; ++r)
                for (int64_t c = 0; c < M1; ++c) AT(pxy, ny, i1s[r], j1s[c]) = AT(dxx, nx, i1[r], j1[c]);
            for (int64_t r = 0; r < L1; ++r)
                for (int64_t c = 0; c < M2; ++c) AT(pxy, ny, i1s[r], j2s[c]) = AT(dxy, ny, i1[r], j2[c]);
            for (int64_t r = 0; r < L2; ++r)
                for (int64_t c = 0; c < M1; ++c) AT(pxy, ny, i2s[r], j1s[c]) = AT(dyx, nx, i2[r], j1[c]);
            for (int64_t r = 0; r < L2; ++r)
                for (int64_t c = 0; c < M2; ++c) AT(pxy, ny, i2s[r], j2s[c]) = AT(dyy, ny, i2[r], j2[c]);
#undef AT
            stats[b] = eo_combine(eo_matrix_sum(pxx, nx, nx), eo_matrix_sum(pyy, ny, ny),
                                  eo_matrix_sum(pxy, nx, ny), nx, ny, stat);
        }
        free(idx_p1); free(lists); free(pxx); free(pyy); free(pxy);
    }
    free(w); free(dxx); free(dyy); free(dxy); free(dyx);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Permutation p-value of Section 3.1 (Phipson and Smyth):
 * (1 + #{b : stats[b] >= observed}) / (1 + B).  *n_ge receives the count. */
double eo_pvalue(const double *stats, int64_t B, double observed, int64_t *n_ge)
{
    int64_t c = 0;
    for (int64_t b = 0; b < B; ++b)
        if (stats[b] >= observed) ++c;
    if (n_ge) *n_ge = c;
    if (EO_MUTANT == 7) return B > 0 ? (double)c / (double)B : 1.0;
    return (1.0 + (double)c) / (1.0 + (double)B);
}

/* ------------------------------------------------------------------------- */
/* Exhaustive enumeration of all C(n, nx) relabelings in lexicographic order of
 * the kept index sets.  sel_out (if not NULL) receives [count][n]; stats[count]
 * the statistic of each, computed directly from raw rows.  When nx == ny a
 * relabeling and its complement give the same statistic in exact arithmetic
 * (Eq. 1 and Eq. 2 are symmetric in x and y); each pair is then evaluated once,
 * on the member that keeps pooled row 0, so that the two are bitwise equal.
 * Returns the number of relabelings, or -1 if more than max_count. */
int64_t eo_exhaustive(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p,
                      int stat, double sigma, int64_t max_count, uint8_t *sel_out,
                      double *stats)
{
    const int64_t n = nx + ny;
    /* count C(n, nx) */
    double cnt = 1.0;
    for (int64_t k = 1; k <= nx; ++k) cnt = cnt * (double)(n - nx + k) / (double)k;
    const int64_t count = (int64_t)(cnt + 0.5);
    if (count > max_count) return -1;

    uint8_t *all = (uint8_t *)calloc((size_t)(count * n), 1);
    uint8_t *canon = (uint8_t *)calloc((size_t)(count * n), 1);
    int64_t *comb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nx > 0 ? nx : 1));
    if (!all || !canon || !comb) {
        free(all); free(canon); free(comb);
        return -1;
    }
    for (int64_t k = 0; k < nx; ++k) comb[k] = k;
    for (int64_t c = 0; c < count; ++c) {
        uint8_t *s = all + c * n;
        for (int64_t k = 0; k < nx; ++k) s[EO_MUTANT == 11 ? n - 1 - comb[k] : comb[k]] = 1;
        uint8_t *q = canon + c * n;
        const int flip = (nx == ny) && !s[0];
        for (int64_t t = 0; t < n; ++t) q[t] = flip ? (uint8_t)!s[t] : s[t];
        /* next combination */
        int64_t k = nx - 1;
        while (k >= 0 && comb[k] == n - nx + k) --k;
        if (k < 0) break;
        ++comb[k];
        for (int64_t m = k + 1; m < nx; ++m) comb[m] = comb[m - 1] + 1;
    }
    const int rc = eo_test_direct(X, nx, Y, ny, p, stat, sigma, canon, count, stats);
    if (sel_out) memcpy(sel_out, all, (size_t)(count * n));
    free(all); free(canon); free(comb);
    return rc == 0 ? count : -1;
}

/* ------------------------------------------------------------------------- */
/* The statistic of ONE relabeling sel[n] (Eq. 1 / Eq. 2 recomputed from the
 * permuted raw rows, as in Algorithm 4), with the pairwise sums split over OpenMP
 * threads by rows and the per-row sums added in row order.  For checking sampled
 * outputs at sizes where one relabeling already costs O(n^2 p). */
double eo_stat_select_mt(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p, int stat,
                         double sigma, const uint8_t *sel)
{
    const int64_t n = nx + ny;
    double *w = eo_pool(X, nx, Y, ny, p);
    int64_t *ix = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *iy = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *rxx = (double *)calloc((size_t)n, sizeof(double));
    double *ryy = (double *)calloc((size_t)n, sizeof(double));
    double *rxy = (double *)calloc((size_t)n, sizeof(double));
    if (!w || !ix || !iy || !rxx || !ryy || !rxy) {
        free(w); free(ix); free(iy); free(rxx); free(ryy); free(rxy);
        return NAN;
    }
    int64_t a = 0, c = 0;
    for (int64_t t = 0; t < n; ++t) {
        if (sel[t]) ix[a++] = t;
        else iy[c++] = t;
    }
    double res = NAN;
    if (a == nx) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t k = 0; k < nx; ++k) {
            double s1 = 0.0, s2 = 0.0;
            for (int64_t l = (EO_MUTANT == 9); l < ny; ++l) s1 += eo_entry(w + ix[k] * p, w + iy[l] * p, p, stat, sigma);
            for (int64_t l = 0; l < nx; ++l) s2 += eo_entry(w + ix[k] * p, w + ix[l] * p, p, stat, sigma);
            rxy[k] = s1;
            rxx[k] = s2;
        }
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t k = 0; k < ny; ++k) {
            double s3 = 0.0;
            for (int64_t l = 0; l < ny; ++l) s3 += eo_entry(w + iy[k] * p, w + iy[l] * p, p, stat, sigma);
            ryy[k] = s3;
        }
        double sxx = 0.0, syy = 0.0, sxy = 0.0;
        for (int64_t k = 0; k < nx; ++k) { sxx += rxx[k]; sxy += rxy[k]; }
        for (int64_t k = 0; k < ny; ++k) syy += ryy[k];
        res = eo_combine(sxx, syy, sxy, nx, ny, stat);
    }
    free(w); free(ix); free(iy); free(rxx); free(ryy); free(rxy);
    return res;
}

/* Sum of all entries S = 1'W1 and trace of the pooled matrix W (distances or kernel
 * values of Algorithm 3 over all pooled pairs), for the closed-form mean of the
 * permutation distribution. */
void eo_pooled_moments(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p, int stat,
                       double sigma, double *S_out, double *trace_out)
{
    const int64_t n = nx + ny;
    double *w = eo_pool(X, nx, Y, ny, p);
    double *rs = (double *)calloc((size_t)n, sizeof(double));
    double *dg = (double *)calloc((size_t)n, sizeof(double));
    if (!w || !rs || !dg) {
        free(w); free(rs); free(dg);
        *S_out = NAN; *trace_out = NAN;
        return;
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += eo_entry(w + i * p, w + j * p, p, stat, sigma);
        rs[i] = s;
        dg[i] = eo_entry(w + i * p, w + (EO_MUTANT == 10 ? (i + 1) % n : i) * p, p, stat, sigma);
    }
    double S = 0.0, tr = 0.0;
    for (int64_t i = 0; i < n; ++i) { S += rs[i]; tr += dg[i]; }
    *S_out = S;
    *trace_out = tr;
    free(w); free(rs); free(dg);
}

/* Closed-form mean of the permutation distribution of Eq. 1 / Eq. 2 when the
 * relabeling s is a uniform random nx-subset of the n pooled rows (Section 3.1's
 * null distribution).  Inclusion probabilities: E[s_i] = nx/n and, for i != j,
 * E[s_i s_j] = nx(nx-1)/(n(n-1)).  With T = s'Ws, L = s'W1 and S = 1'W1 the three
 * block sums of the relabeled data are T (x*x*), L - T (x*y*) and S - 2L + T
 * (y*y*), so E[T] = nx/n tr W + nx(nx-1)/(n(n-1)) (S - tr W), E[L] = nx/n S and,
 * the statistic being linear in (T, L),
 *   E[ED*] = 2(E[L] - E[T])/(nx ny) - E[T]/nx^2 - (S - 2E[L] + E[T])/ny^2;
 * E[MMD*] is the same expression with the opposite sign. */
double eo_permutation_mean(double S, double trace, int64_t nx, int64_t ny, int stat)
{
    const double fx = (double)nx, fy = (double)ny, fn = (double)(nx + ny);
    const double pair = (EO_MUTANT == 12) ? (fx / fn) * (fx / fn) : fx * (fx - 1.0) / (fn * (fn - 1.0));
    const double ET = fx / fn * trace + pair * (S - trace);
    const double EL = fx / fn * S;
    const double ed = 2.0 * (EL - ET) / (fx * fy) - ET / (fx * fx) - (S - 2.0 * EL + ET) / (fy * fy);
    return stat == EO_STAT_ED ? ed : -ed;
}

int eo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Median heuristic for the kernel bandwidth (a reading: the paper leaves sigma to
 * the user): the lower median -- element floor((N - 1) / 2) of the sorted list --
 * of the N = n (n - 1) / 2 Euclidean distances between distinct pooled rows
 * (Algorithm 3 entries).  Taken over the pooled sample it does not depend on the
 * split into x and y, so every relabeling sees the same bandwidth.  Returns -1 when
 * n < 2 or on allocation failure. */
static int eo_cmp_double(const void *a, const void *b)
{
    const double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

double eo_median_pairs(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p)
{
    const int64_t n = nx + ny;
    if (n < 2) return -1.0;
    double *w = eo_pool(X, nx, Y, ny, p);
    const int64_t N = n * (n - 1) / 2;
    double *d = (double *)malloc(sizeof(double) * (size_t)N);
    if (!w || !d) {
        free(w);
        free(d);
        return -1.0;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) d[k++] = sqrt(eo_sqdist(w + i * p, w + j * p, p));
    qsort(d, (size_t)N, sizeof(double), eo_cmp_double);
    const double med = d[(N - 1) / 2];
    free(w);
    free(d);
    return med;
}

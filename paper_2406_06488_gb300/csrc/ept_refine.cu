// ept_refine.cu -- FP64 recomputation of the statistics whose error estimate
// exceeds the tolerance (the criterion is in ept_internal.cuh, REFINE_KA/KR/TOL;
// k_combine_count sets the flags).
//
// What it computes: for a flagged relabeling column with indicator s of the
// contracted group G (x* unless the test contracts y*, see ept_internal.cuh), the
// three block sums of Eq. 1 / Eq. 2 from the pooled matrix W built in FP64 from the
// raw rows (Algorithm 3, direct differences of the exactly widened FP32 inputs):
//     T = s'Ws = sum over G x G,   L = s'W1,   S = 1'W1,
//     sum over G x H = L - T,      sum over H x H = S - 2L + T   (H = the other group),
// which is Algorithm 1's block swapping written as sums over one pooled matrix.
// The statistic is then Eq. 1 (ED) or Eq. 2 (MMD^2) evaluated in FP64, with no
// centring and no FP32 anywhere after the inputs.
//
// Work: W64 rows [r0, r1) (a window sized to the scratch) are computed once by
// k_refine_w (64 x 64 tiles, FP64 differences staged through shared memory); then
// k_refine_rows gives every 64-row tile and every group of 64 flagged columns a
// CTA, which reads its rows of W64 once per column tile and keeps, per row and
// column, sum_j s_j W_ij in registers; the tile's sums over its rows are added in a
// fixed order (deterministic), and k_refine_finish adds the tiles in order.
#include <cstdint>

#include "../../include/ept.h"
#include "ept_internal.cuh"

namespace ept {

namespace {

constexpr int RT = 64;    // rows per tile
constexpr int CT = 64;    // columns per tile (of W64), and flagged columns per CTA
constexpr int FCH = 32;   // features staged per step

__device__ __forceinline__ const float *pooled_row(const TestDesc &d, int64_t i) {
    return i < d.nx ? d.X + i * d.p : d.Y + (i - d.nx) * d.p;
}

// the entry of W from a squared distance (FP64): the distance (Algorithm 3) or the
// Gaussian / Laplacian kernel value (Appendix A.1)
__device__ __forceinline__ double refine_entry(double d2, int stat, double sigma) {
    if (stat == EPT_STAT_ED) return sqrt(d2);
    if (stat == EPT_STAT_MMD_GAUSS) return exp(-d2 / (2.0 * sigma * sigma));
    return exp(-sqrt(d2) / sigma);
}

// one 64 x 64 tile of W64: rows r0 + 64 blockIdx.y .., columns 64 blockIdx.x ..
// (r0 is a multiple of 64)
__global__ void __launch_bounds__(256) k_refine_w(const Batch bt, int t, double sigma, int64_t r0, int64_t r1,
                                                  double *__restrict__ W64) {
    __shared__ float ra[RT][FCH + 1], rb[CT][FCH + 1];
    const TestDesc d = bt.desc[t];
    const int64_t i0 = r0 + (int64_t)blockIdx.y * RT, j0 = (int64_t)blockIdx.x * CT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 4 x 4 entries each
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int64_t f0 = 0; f0 < d.p; f0 += FCH) {
        for (int e = threadIdx.x; e < RT * FCH; e += 256) {
            const int r = e / FCH, f = e % FCH;
            const int64_t i = i0 + r, j = j0 + r;
            ra[r][f] = (i < r1 && f0 + f < d.p) ? pooled_row(d, i)[f0 + f] : 0.f;
            rb[r][f] = (j < d.n && f0 + f < d.p) ? pooled_row(d, j)[f0 + f] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int f = 0; f < FCH; ++f) {
            double x[4], y[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) x[a] = (double)ra[ty * 4 + a][f];
#pragma unroll
            for (int b = 0; b < 4; ++b) y[b] = (double)rb[tx * 4 + b][f];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const double df = x[a] - y[b];
                    acc[a][b] = fma(df, df, acc[a][b]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + ty * 4 + a;
        if (i >= r1) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t j = j0 + tx * 4 + b;
            if (j < d.n) W64[(i - r0) * d.n + j] = refine_entry(acc[a][b], d.stat, sigma);
        }
    }
}

// bit t of relabeling column c of test d (the contracted group's indicator)
__device__ __forceinline__ uint32_t mask_word(const Batch &bt, const TestDesc &d, int64_t w, int64_t c) {
    return bt.maskT[d.mask0 + w * d.Bp + c];
}

// per (64-row tile, group of 64 flagged columns): T and L over the tile's rows
__global__ void __launch_bounds__(256) k_refine_rows(const Batch bt, int t, int64_t r0, int64_t r1,
                                                     const double *__restrict__ W64, const int32_t *__restrict__ list,
                                                     int64_t nflag, double *__restrict__ part,
                                                     double *__restrict__ spart) {
    __shared__ double w[RT][CT + 1];    // the W64 tile; then the masked row sums
    __shared__ uint32_t jbits[CT][2];   // mask words of the column tile, per flagged column
    __shared__ double rsh[RT];          // the rows' totals
    const TestDesc d = bt.desc[t];
    const int64_t tile = (r0 / RT) + blockIdx.x;   // global row-tile index of the test
    const int64_t i0 = tile * RT;
    const int64_t k0 = (int64_t)blockIdx.y * CT;
    const int ti = threadIdx.x & 63, kq = threadIdx.x >> 6;   // row ti, columns k0 + kq + 4 q
    const int64_t i = i0 + ti;
    double P[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) P[q] = 0.0;
    double rs = 0.0;
    for (int64_t j0 = 0; j0 < d.n; j0 += CT) {
        for (int e = threadIdx.x; e < RT * CT; e += 256) {
            const int r = e / CT, cc = e % CT;
            const int64_t gi = i0 + r, gj = j0 + cc;
            w[r][cc] = (gi < r1 && gj < d.n) ? W64[(gi - r0) * d.n + gj] : 0.0;
        }
        if (threadIdx.x < CT) {
            const int64_t k = k0 + threadIdx.x;
            uint32_t lo = 0, hi = 0;
            if (k < nflag) {
                const int64_t c = list[k];
                lo = mask_word(bt, d, j0 / 32, c);
                hi = (j0 / 32 + 1 < d.nw) ? mask_word(bt, d, j0 / 32 + 1, c) : 0u;
            }
            jbits[threadIdx.x][0] = lo;
            jbits[threadIdx.x][1] = hi;
        }
        __syncthreads();
        if (kq == 0) {
            double s = 0.0;
            for (int cc = 0; cc < CT; ++cc) s += w[ti][cc];
            rs += s;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int kk = kq + 4 * q;
            const uint32_t lo = jbits[kk][0], hi = jbits[kk][1];
            double s = 0.0;
            for (int cc = 0; cc < 32; ++cc) s += ((lo >> cc) & 1u) ? w[ti][cc] : 0.0;
            for (int cc = 0; cc < 32; ++cc) s += ((hi >> cc) & 1u) ? w[ti][32 + cc] : 0.0;
            P[q] += s;
        }
        __syncthreads();
    }
    // T part: sum_i s_k(i) P[i][k]; L part: sum_i s_k(i) rs_i -- rows added in order
    // (the W64 tile's storage is free after the loop's last barrier)
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int kk = kq + 4 * q;
        const int64_t k = k0 + kk;
        uint32_t bit = 0;
        if (k < nflag && i < r1) bit = (mask_word(bt, d, i / 32, list[k]) >> (i & 31)) & 1u;
        w[ti][kk] = bit ? P[q] : 0.0;
    }
    if (kq == 0) rsh[ti] = (i < r1) ? rs : 0.0;
    __syncthreads();
    if (threadIdx.x < CT) {
        const int kk = threadIdx.x;
        const int64_t k = k0 + kk;
        if (k < nflag) {
            double T = 0.0, L = 0.0;
            for (int r = 0; r < RT; ++r) {
                T += w[r][kk];
                const int64_t gi = i0 + r;
                if (gi < r1 && ((mask_word(bt, d, gi / 32, list[k]) >> (gi & 31)) & 1u)) L += rsh[r];
            }
            part[(tile * nflag + k) * 2] = T;
            part[(tile * nflag + k) * 2 + 1] = L;
        }
    }
    if (blockIdx.y == 0 && threadIdx.x == 0) {
        double S = 0.0;
        for (int r = 0; r < RT; ++r) S += rsh[r];
        spart[tile] = S;
    }
}

// per flagged column: the tiles' sums in order, then Eq. 1 / Eq. 2 in FP64
__global__ void __launch_bounds__(256) k_refine_finish(const Batch bt, int t, const int32_t *__restrict__ list,
                                                       int64_t nflag, const double *__restrict__ part,
                                                       const double *__restrict__ spart, int64_t ntiles) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nflag) return;
    const TestDesc d = bt.desc[t];
    double T = 0.0, L = 0.0, S = 0.0;
    for (int64_t tl = 0; tl < ntiles; ++tl) {
        T += part[(tl * nflag + k) * 2];
        L += part[(tl * nflag + k) * 2 + 1];
        S += spart[tl];
    }
    // sums over the contracted group G (size m) and the other group H (size o)
    const double sGG = T, sGH = L - T, sHH = S - 2.0 * L + T;
    const double sxx = d.comp ? sHH : sGG, syy = d.comp ? sGG : sHH;
    const double fx = (double)d.nx, fy = (double)d.ny;
    const double ed = 2.0 * sGH / (fx * fy) - sxx / (fx * fx) - syy / (fy * fy);
    bt.stats[d.col0 + list[k]] = d.stat == EPT_STAT_ED ? ed : -ed;
}

}  // namespace

void launch_refine_w(const Batch &b, int t, int64_t n, double sigma, int64_t r0, int64_t r1, double *W64,
                     cudaStream_t s) {
    if (r1 <= r0) return;
    const dim3 grid((unsigned)((n + CT - 1) / CT), (unsigned)((r1 - r0 + RT - 1) / RT));
    k_refine_w<<<grid, 256, 0, s>>>(b, t, sigma, r0, r1, W64);
}

void launch_refine_rows(const Batch &b, int t, int64_t r0, int64_t r1, const double *W64, const int32_t *list,
                        int64_t nflag, double *part, double *spart, cudaStream_t s) {
    if (r1 <= r0 || nflag <= 0) return;
    const dim3 grid((unsigned)((r1 - r0 + RT - 1) / RT), (unsigned)((nflag + CT - 1) / CT));
    k_refine_rows<<<grid, 256, 0, s>>>(b, t, r0, r1, W64, list, nflag, part, spart);
}

void launch_refine_finish(const Batch &b, int t, const int32_t *list, int64_t nflag, const double *part,
                          const double *spart, int64_t ntiles, cudaStream_t s) {
    if (nflag <= 0) return;
    k_refine_finish<<<(unsigned)((nflag + 255) / 256), 256, 0, s>>>(b, t, list, nflag, part, spart, ntiles);
}

}  // namespace ept

// ept_pooled.cu -- the pre-computation strategy of Algorithm 5 on the GPU, kept as
// the measured comparison the paper makes (Section 5.1: the efficient test against
// the pre-computed one).  The distance (or kernel) matrix of the concatenated data
// W = D_WW is computed once, in full (n x n, both triangles, as Algorithm 5 does);
// each relabeling then extracts its three sub-matrices by index and sums them:
//     S_XX = sum_{i, j in x*} W_ij,  S_YY = sum_{i, j in y*} W_ij,  S_XY = sum_{i in x*, j in y*} W_ij,
// and Eq. 1 / Eq. 2 combine the sums.  Nothing is shared between relabelings but W.
//
// Precision: W in FP32 from direct differences (Algorithm 3's form); the sums are
// unevaluated FP32 pairs (Knuth's TwoSum, every rounding error kept) widened to
// FP64, and the combination is FP64.
#include "ept_internal.cuh"

namespace ept {
namespace {

constexpr int PW_TILE = 64;   // rows and columns of W per CTA of the build
constexpr int PW_P = 32;      // features per staged slice

__device__ __forceinline__ const float *pooled_row(const TestDesc &d, int64_t i) {
    return (i < d.nx) ? d.X + i * d.p : d.Y + (i - d.nx) * d.p;
}

__device__ __forceinline__ float pooled_entry(float d2, const TestDesc &d) {
    if (d.kern == 0) return sqrtf(d2);
    if (d.kern == 1) return exp_cw(d2 * d.neg_inv_2s2);
    return exp_cw(-sqrtf(d2) * d.inv_sigma);
}

// W[i][j] for i, j < n (row stride ld): a CTA computes a 64 x 64 tile, thread (ty,
// tx) rows 4ty..4ty+3 x columns 4tx..4tx+3, from slices of 32 features staged in
// shared memory (sum of squared differences in FP32, in feature order).
__global__ void __launch_bounds__(256) k_pooled_build(const Batch bt, int64_t ld) {
    __shared__ float As[PW_P][PW_TILE + 1];
    __shared__ float Bs[PW_P][PW_TILE + 1];
    const TestDesc &d = bt.desc[0];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.y * PW_TILE, j0 = (int64_t)blockIdx.x * PW_TILE;
    const int64_t n = d.n, p = d.p;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int64_t k0 = 0; k0 < p; k0 += PW_P) {
#pragma unroll
        for (int e = 0; e < (PW_TILE * PW_P) / 256; ++e) {
            const int idx = e * 256 + tid, r = idx >> 5, k = idx & 31;
            const int64_t kk = k0 + k, i = i0 + r, j = j0 + r;
            As[k][r] = (i < n && kk < p) ? pooled_row(d, i)[kk] : 0.f;
            Bs[k][r] = (j < n && kk < p) ? pooled_row(d, j)[kk] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < PW_P; ++k) {
            float av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[k][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float df = av[a] - bv[b];
                    acc[a][b] = fmaf(df, df, acc[a][b]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + ty * 4 + a;
        if (i >= n) continue;
        float *out = bt.D + i * ld + j0 + tx * 4;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (j0 + tx * 4 + b < n) out[b] = pooled_entry(acc[a][b], d);
    }
}

__device__ __forceinline__ void acc_two_sum(float &h, float &l, float v) {
    float s, e;
    two_sum(h, v, s, e);
    h = s;
    l += e;
}

// Sums of relabeling c over the rows [r0, r1) of W (grid: columns x row chunks): the
// CTA loads the relabeling's mask words into shared memory; warp w takes every
// eighth row, its lanes every 32nd column.  A row of x* adds its x* columns to
// S_XX and its y* columns to S_XY; a row of y* adds its y* columns to S_YY.
// part[(chunk * 3 + s) * ncols + c], s = XX, XY, YY, FP64.
__global__ void __launch_bounds__(256) k_pooled_sums(const Batch bt, const float *__restrict__ W, int64_t ld,
                                                     int64_t rows_per_chunk, double *part) {
    extern __shared__ uint32_t smask[];
    __shared__ double red[3][8];
    const TestDesc &d = bt.desc[0];
    const int64_t c = blockIdx.x, nw = d.nw, Bp = d.Bp, n = d.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t w = threadIdx.x; w < nw; w += 256) smask[w] = bt.maskT[d.mask0 + w * Bp + c];
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t r1 = r0 + rows_per_chunk < n ? r0 + rows_per_chunk : n;
    float xxh = 0.f, xxl = 0.f, xyh = 0.f, xyl = 0.f, yyh = 0.f, yyl = 0.f;
    for (int64_t i = r0 + warp; i < r1; i += 8) {
        const bool in_x = (smask[i >> 5] >> (i & 31)) & 1u;
        const float *row = W + i * ld;
        for (int64_t j0 = 0; j0 < n; j0 += 32) {
            const int64_t j = j0 + lane;
            if (j >= n) break;
            const float v = row[j];
            const bool bx = (smask[j0 >> 5] >> lane) & 1u;
            if (in_x) {
                if (bx) acc_two_sum(xxh, xxl, v);
                else acc_two_sum(xyh, xyl, v);
            } else if (!bx) {
                acc_two_sum(yyh, yyl, v);
            }
        }
    }
    double s[3] = {(double)xxh + (double)xxl, (double)xyh + (double)xyl, (double)yyh + (double)yyl};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int off = 16; off; off >>= 1) s[k] += __shfl_xor_sync(0xFFFFFFFFu, s[k], off);
        if (lane == 0) red[k][warp] = s[k];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
        part[((int64_t)blockIdx.y * 3 + threadIdx.x) * gridDim.x + c] = t;
    }
}

// Eq. 1 (ED = 2 S_XY / (nx ny) - S_XX / nx^2 - S_YY / ny^2) or Eq. 2 (the opposite
// sign) of each relabeling from its row chunks' sums (fixed order).
__global__ void __launch_bounds__(256) k_pooled_stats(const Batch bt, const double *part, int nchunks) {
    const TestDesc &d = bt.desc[0];
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x, nc = d.ncols;
    if (c >= nc) return;
    double xx = 0.0, xy = 0.0, yy = 0.0;
    for (int k = 0; k < nchunks; ++k) {
        xx += part[((int64_t)k * 3 + 0) * nc + c];
        xy += part[((int64_t)k * 3 + 1) * nc + c];
        yy += part[((int64_t)k * 3 + 2) * nc + c];
    }
    const double fx = (double)d.nx, fy = (double)d.ny;
    const double ed = 2.0 * xy / (fx * fy) - xx / (fx * fx) - yy / (fy * fy);
    bt.stats[d.col0 + c] = d.stat == 0 ? ed : -ed;
}

}  // namespace

int64_t pooled_row_chunks(int64_t n, int64_t ncols, int num_sms) {
    // enough CTAs for about four per SM, each with at least 256 rows
    int64_t want = (4 * (int64_t)num_sms + ncols - 1) / ncols;
    const int64_t most = (n + 255) / 256;
    if (want > most) want = most;
    return want < 1 ? 1 : want;
}

cudaError_t launch_pooled(const Batch &b, int64_t n, int64_t ld, int64_t ncols, double *part, int64_t nchunks,
                          int64_t nw, cudaStream_t s) {
    const unsigned tiles = (unsigned)((n + PW_TILE - 1) / PW_TILE);
    k_pooled_build<<<dim3(tiles, tiles), 256, 0, s>>>(b, ld);
    const int64_t rows = (n + nchunks - 1) / nchunks;
    const size_t smem = (size_t)nw * 4;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_pooled_sums, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_pooled_sums<<<dim3((unsigned)ncols, (unsigned)nchunks), 256, smem, s>>>(b, b.D, ld, rows, part);
    k_pooled_stats<<<(unsigned)((ncols + 255) / 256), 256, 0, s>>>(b, part, (int)nchunks);
    return cudaGetLastError();
}

}  // namespace ept

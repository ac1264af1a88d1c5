// ept_stream.cu -- the kernels that are particular to the streaming mode: a test
// whose packed blocks do not fit in device memory is run one window of row panels
// at a time.
//
// The permuted statistics are sums over the pooled matrix W (Algorithm 1: the
// three blocks are built once; Section 4.1: every permuted statistic is a sum of
// their entries), and the part of s'Cs that the rows of one panel contribute only
// needs that panel's stored blocks.  So the panels are taken in windows, and the
// next window reuses the memory of the last.  The double centring needs the exact
// row sums r = W 1 before any block is packed (with a cruder centring vector the
// packed entries keep a per-row mean, and the FP32 accumulation of the contraction
// is then no longer small against the cancellation that follows), so there are two
// passes over the windows:
//  1. build the window's blocks and add their row and column sums into r;
//  2. (after the centring constants, the resident path's kernels) build the window
//     again -- the build is deterministic, so the blocks are the same bit for bit --
//     pack it, contract it against every relabeling and fold its partial sums into
//     FP64 per-relabeling accumulators.
// The blocks need one window of memory instead of about 2 n^2 bytes; the price is a
// second build of every block.
#include "ept_internal.cuh"

namespace ept {
namespace {

// Row sums r += the window's share: row i (panel P >= I0) gets the row segments of
// its own panel's blocks when P is in the window, and column i's segments of the
// window's panels J < P (the transposed lower part).  Eight threads per row, fixed
// shuffle tree; windows are added in order (deterministic).  CTA = 32 rows.
__global__ void __launch_bounds__(256) k_stream_rowsums(const Batch bt, int64_t I0, int64_t I1) {
    const int sub = threadIdx.x & 7, rl = threadIdx.x >> 3;
    const TestDesc &d = bt.desc[0];
    const int64_t i = I0 * PANEL + (int64_t)blockIdx.x * 32 + rl;
    const int64_t P = i / PANEL, rr = i % PANEL, NKB = d.NKB;
    double acc = 0.0;
    if (i < d.n) {
        if (P < I1) {
            const int64_t nkb = NKB - KB_PER_PANEL * P;
            const int64_t base = d.blk0 + blk_off(P, NKB);
            for (int64_t k = sub; k < nkb; k += 8) acc += bt.rowpart[(base + k) * PANEL + rr];
        }
        const int64_t kbi = i / KB, ci = i % KB, Jend = P < I1 ? P : I1;
        for (int64_t J = I0 + sub; J < Jend; J += 8) acc += bt.colpart[(d.blk0 + blk_index(J, kbi, NKB)) * KB + ci];
    }
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
    if (sub == 0 && i < d.n) bt.r[d.row0 + i] += acc;
}

// sacc[b] += the window's partials of relabeling b (FP64, fixed order).  CTA = 32
// columns, warp w takes every eighth partial row.
__global__ void __launch_bounds__(256) k_stream_accum(const Batch bt) {
    __shared__ double ws[8][32];
    const TestDesc &d = bt.desc[0];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * 32 + lane, Bp = d.Bp;
    const float *part = bt.partial + d.part0 + c;
    double acc = 0.0;
    for (int64_t k = warp; k < d.nparts; k += 8) acc += (double)part[k * Bp];
    ws[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        double q = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) q += ws[w][lane];
        bt.sacc[c] += q;
    }
}

// Spart[k] = r_{32k} + ... + r_{32k+31} (fixed order), the input of the resident
// path's centring kernels.  One warp per 32 rows.
__global__ void __launch_bounds__(256) k_stream_spart(const Batch bt) {
    const TestDesc &d = bt.desc[0];
    const int lane = threadIdx.x & 31;
    const int64_t k = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (k >= d.n_pad / 32) return;
    double v = bt.r[d.row0 + k * 32 + lane];
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    if (lane == 0) bt.Spart[d.sp0 + k] = v;
}

// stat_b = sign (cT sacc_b / c + S~ / o^2), S~ = sum of the panels' Stpart: the
// resident path's combination with the windows' FP64 sums in place of the partials.
// CTA = 256 relabeling columns.
__global__ void __launch_bounds__(256) k_stream_stats(const Batch bt) {
    __shared__ double bSt;
    const TestDesc &d = bt.desc[0];
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int64_t k = threadIdx.x; k < d.NP; k += 32) s += bt.Stpart[d.pan0 + k];
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
        if (threadIdx.x == 0) bSt = s;
    }
    __syncthreads();
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const double inv_c = 1.0 / (double)packed_scale(bt.ctr[0]);
    if (c < d.ncols) bt.stats[d.col0 + c] = d.sign * (d.cT * (bt.sacc[c] * inv_c) + bSt * d.inv_o2);
}

}  // namespace

void launch_stream_spart(const Batch &b, cudaStream_t s) {
    if (b.nrows_total <= 0) return;
    k_stream_spart<<<(unsigned)((b.nrows_total / 32 + 7) / 8), 256, 0, s>>>(b);
}

void launch_stream_rowsums(const Batch &g, int64_t I0, int64_t I1, int64_t n_pad, cudaStream_t s) {
    const int64_t rows = n_pad - I0 * PANEL;
    if (rows <= 0 || I1 <= I0) return;
    k_stream_rowsums<<<(unsigned)(rows / 32), 256, 0, s>>>(g, I0, I1);
}

void launch_stream_accum(const Batch &g, cudaStream_t s) {
    if (g.ncols_total <= 0) return;
    k_stream_accum<<<(unsigned)(g.ncols_total / 32), 256, 0, s>>>(g);
}

void launch_stream_stats(const Batch &b, cudaStream_t s) {
    if (b.ncols_total <= 0) return;
    k_stream_stats<<<(unsigned)(b.ncols_total / 256), 256, 0, s>>>(b);
}

}  // namespace ept

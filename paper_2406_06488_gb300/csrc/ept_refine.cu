// ept_refine.cu -- FP64 recomputation of the statistics whose error estimate
// exceeds the tolerance (the criterion is in ept_internal.cuh, refine_ka, REFINE_KR, REFINE_TOL;
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
// k_refine_w (64 x 64 tiles; the squared distances as FP32 pairs with error-free
// transformations -- about 48 significant bits on the FP32 pipes, which run many
// times faster than FP64 on this GPU -- then the entry in FP64); then
// k_refine_rows gives every 64-row tile and every group of 64 flagged columns a
// CTA, which reads its rows of W64 once per column tile and keeps, per row and
// column, sum_j s_j W_ij in registers; the tile's sums over its rows are added in a
// fixed order (deterministic), and k_refine_finish adds the tiles (lanes over tiles,
// then a butterfly: the same order on every run).
#include <cuda_fp16.h>

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
    // d^2 as an unevaluated FP32 pair (hi, lo): each difference is split exactly
    // (TwoSum), its square's leading part exactly (FMA), and the pair accumulates with
    // TwoSum -- about 48 significant bits, on the FP32 pipes
    float ahi[4][4], alo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ahi[a][b] = alo[a][b] = 0.f;
    for (int64_t f0 = 0; f0 < d.p; f0 += FCH) {
        for (int e = threadIdx.x; e < RT * FCH; e += 256) {
            const int r = e / FCH, f = e % FCH;
            const int64_t i = i0 + r, j = j0 + r;
            ra[r][f] = (i < r1 && f0 + f < d.p) ? pooled_row(d, i)[f0 + f] : 0.f;
            rb[r][f] = (j < d.n && f0 + f < d.p) ? pooled_row(d, j)[f0 + f] : 0.f;
        }
        __syncthreads();
#pragma unroll 2
        for (int f = 0; f < FCH; ++f) {
            float x[4], y[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) x[a] = ra[ty * 4 + a][f];
#pragma unroll
            for (int b = 0; b < 4; ++b) y[b] = rb[tx * 4 + b][f];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    // x - y = s + e exactly
                    const float sd = __fsub_rn(x[a], y[b]);
                    const float bb = __fsub_rn(sd, x[a]);
                    const float e = __fadd_rn(__fsub_rn(x[a], __fsub_rn(sd, bb)), __fsub_rn(-y[b], bb));
                    // (s + e)^2 = p + pe + (2 s e + e^2), p + pe = s^2 exactly
                    const float pq = __fmul_rn(sd, sd);
                    const float pe = __fmaf_rn(sd, sd, -pq);
                    const float tl = __fmaf_rn(2.f * sd, e, __fmul_rn(e, e));
                    // (hi, lo) += p + (pe + tl)
                    const float h2 = __fadd_rn(ahi[a][b], pq);
                    const float hb = __fsub_rn(h2, ahi[a][b]);
                    const float he = __fadd_rn(__fsub_rn(ahi[a][b], __fsub_rn(h2, hb)), __fsub_rn(pq, hb));
                    ahi[a][b] = h2;
                    alo[a][b] = __fadd_rn(alo[a][b], __fadd_rn(he, __fadd_rn(pe, tl)));
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
            if (j < d.n) W64[(i - r0) * d.n + j] = refine_entry((double)ahi[a][b] + (double)alo[a][b], d.stat, sigma);
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
    const int64_t k = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= nflag) return;
    const TestDesc d = bt.desc[t];
    double T = 0.0, L = 0.0, S = 0.0;
    for (int64_t tl = lane; tl < ntiles; tl += 32) {
        T += part[(tl * nflag + k) * 2];
        L += part[(tl * nflag + k) * 2 + 1];
        S += spart[tl];
    }
    for (int off = 16; off; off >>= 1) {
        T += __shfl_xor_sync(0xFFFFFFFFu, T, off);
        L += __shfl_xor_sync(0xFFFFFFFFu, L, off);
        S += __shfl_xor_sync(0xFFFFFFFFu, S, off);
    }
    if (lane != 0) return;
    // sums over the contracted group G (size m) and the other group H (size o)
    const double sGG = T, sGH = L - T, sHH = S - 2.0 * L + T;
    const double sxx = d.comp ? sHH : sGG, syy = d.comp ? sGG : sHH;
    const double fx = (double)d.nx, fy = (double)d.ny;
    const double ed = 2.0 * sGH / (fx * fy) - sxx / (fx * fx) - syy / (fy * fy);
    bt.stats[d.col0 + list[k]] = d.stat == EPT_STAT_ED ? ed : -ed;
}

// ---- exact re-summation of the packed operand (the accumulation part) ----
// For flagged columns whose representation term is small, the statistic is
// recomputed from the packed, centred operand the contraction read, T = s'Cs, with
// no accumulation error: on the tensor-core path every entry is c C_ij = hi + lo, two
// FP16 numbers that are both multiples of 2^-24 with |hi + lo| < 2^15, so 2^24 c C_ij
// is an integer below 2^39 and a row of up to 2^22 entries sums exactly in int64; on
// the plain path the FP32 entries are summed with TwoSum-compensated FP32 pairs.  The
// rows' sums meet in FP64.  One launch serves every flagged test of a run: a job is
// a group of up to 16 flagged columns of one test; CTA = (row panel I, chunk of RK
// K-blocks) x job; thread = (row r of a 64-row quarter, 4 of the 16 columns).
constexpr int PCOLS = REFINE_JOB_COLS;
constexpr int RK = 8;   // K-blocks per CTA

// 2^24 x (an FP16 number), exactly, from its bits with integer operations: a normal
// number (exponent field e >= 1) is (1024 + f) 2^(e - 25), a subnormal one f 2^-24
// (f the 10-bit fraction); infinities and NaNs do not occur in the packed operand
__device__ __forceinline__ long long fp16_fixed24(uint16_t bits) {
    const int e = (bits >> 10) & 31, f = bits & 1023;
    const long long mag = e ? (long long)(1024 + f) << (e - 1) : (long long)f;
    return (bits & 0x8000u) ? -mag : mag;
}

__global__ void __launch_bounds__(256) k_refine_packed(const Batch bt, const RefineJob *__restrict__ jobs,
                                                       const int32_t *__restrict__ list, double *__restrict__ part) {
    // the values of 64 rows x 64 columns (int64 fixed point or FP32), then the sums
    __shared__ __align__(16) uint8_t sm[PANEL * (PCOLS + 1) * 8];
    long long(*vi)[KB + 1] = reinterpret_cast<long long(*)[KB + 1]>(sm);
    float(*vf)[KB + 1] = reinterpret_cast<float(*)[KB + 1]>(sm);
    double(*red)[PCOLS + 1] = reinterpret_cast<double(*)[PCOLS + 1]>(sm);
    static_assert(64 * (KB + 1) * 8 <= PANEL * (PCOLS + 1) * 8, "value buffer");
    const RefineJob J = jobs[blockIdx.y];
    if ((int64_t)blockIdx.x >= (int64_t)J.np * J.nkc) return;
    const int t = J.t;
    const TestDesc d = bt.desc[t];
    const int64_t nkc = J.nkc;
    const int64_t I = blockIdx.x / nkc, kc = blockIdx.x % nkc;
    const int r = threadIdx.x & 63, cg = threadIdx.x >> 6;   // row r of a 64-row quarter, columns 4 cg ..
    const bool split = d.scaled != 0;
    const int64_t nkb = contract_nkb(d);
    const int64_t kb_lo = KB_PER_PANEL * I + kc * RK;
    const int64_t kb_hi = kb_lo + RK < nkb ? kb_lo + RK : nkb;
    int64_t col[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = 4 * cg + q;
        col[q] = k < J.ncol ? (int64_t)list[J.list0 + k] : -1;
    }
    double rowT[4][4];   // [quarter][column]
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) rowT[a][q] = 0.0;
#pragma unroll
    for (int qr = 0; qr < 4; ++qr) {   // the panel's four 64-row quarters
        const int64_t i = I * PANEL + 64 * qr + r;
        long long si[4] = {0, 0, 0, 0};
        float sf[4] = {0.f, 0.f, 0.f, 0.f}, ef[4] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t kb = kb_lo; kb < kb_hi; ++kb) {
            const int64_t blk = d.blk0 + blk_index(I, kb, d.NKB);
            __syncthreads();
            for (int x = threadIdx.x; x < 64 * KB; x += 256) {
                const int rr = x / KB, cc = x % KB;
                const int64_t off = (int64_t)(64 * qr + rr) * KB + cc;
                if (split) {
                    vi[rr][cc] = fp16_fixed24(bt.Chi[blk * bt.c_stride + off]) +
                                 fp16_fixed24(bt.Clo[blk * bt.c_stride + off]);
                } else {
                    vf[rr][cc] = bt.D[blk * (int64_t)(PANEL * KB) + off];
                }
            }
            __syncthreads();
            const int64_t w0 = kb * KB / 32;
            uint32_t mw[4][2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                mw[q][0] = col[q] < 0 ? 0u : bt.maskT[d.mask0 + w0 * d.Bp + col[q]];
                mw[q][1] = col[q] < 0 ? 0u : bt.maskT[d.mask0 + (w0 + 1) * d.Bp + col[q]];
            }
            if (split) {
                // each value read once from shared memory for the four columns
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
#pragma unroll 8
                    for (int sh = 0; sh < 32; ++sh) {
                        const long long x = vi[r][32 * h2 + sh];
#pragma unroll
                        for (int q = 0; q < 4; ++q) si[q] += ((mw[q][h2] >> sh) & 1u) ? x : 0ll;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4 && !split; ++q) {
                if (col[q] < 0) continue;
                const uint32_t m0 = mw[q][0], m1 = mw[q][1];
                {
                    float sq = sf[q], eq = ef[q];
                    for (int cc = 0; cc < KB; ++cc) {
                        const uint32_t bit = cc < 32 ? (m0 >> cc) & 1u : (m1 >> (cc - 32)) & 1u;
                        const float a = bit ? vf[r][cc] : 0.f;
                        const float t2 = sq + a;   // TwoSum
                        const float bb = t2 - sq;
                        eq += (sq - (t2 - bb)) + (a - bb);
                        sq = t2;
                    }
                    sf[q] = sq;
                    ef[q] = eq;
                }
            }
        }
        // this row's masked sum counts when the row is in the column's group
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (col[q] < 0 || i >= d.n) continue;
            const uint32_t bit = (bt.maskT[d.mask0 + (i / 32) * d.Bp + col[q]] >> (i & 31)) & 1u;
            if (bit) rowT[qr][q] = split ? ldexp((double)si[q], -24) : (double)sf[q] + (double)ef[q];
        }
    }
    __syncthreads();
    // rows in order: red[row of the panel][column]
#pragma unroll
    for (int qr = 0; qr < 4; ++qr)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[64 * qr + r][4 * cg + q] = rowT[qr][q];
    __syncthreads();
    if (threadIdx.x < J.ncol) {
        double T = 0.0;
        for (int rr = 0; rr < PANEL; ++rr) T += red[rr][threadIdx.x];
        const double inv_c = split ? 1.0 / (double)packed_scale(bt.ctr[t]) : 1.0;
        part[J.part0 + (I * nkc + kc) * J.ncol + threadIdx.x] = T * inv_c;
    }
}

// the statistics of the listed columns from the exact T: stat = sign (cT T + S~ / o^2)
// (CTA = job, a warp per column of the job: lanes take every 32nd partial, then a
// fixed butterfly -- the same order on every run)
__global__ void __launch_bounds__(32 * REFINE_JOB_COLS) k_refine_packed_finish(const Batch bt,
                                                                             const RefineJob *__restrict__ jobs,
                                                                             const int32_t *__restrict__ list,
                                                                             const double *__restrict__ part) {
    const RefineJob J = jobs[blockIdx.x];
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= J.ncol) return;
    const TestDesc d = bt.desc[J.t];
    double T = 0.0, St = 0.0;
    for (int64_t g = lane; g < (int64_t)J.np * J.nkc; g += 32) T += part[J.part0 + g * J.ncol + k];
    for (int64_t I = lane; I < d.NP; I += 32) St += bt.Stpart[d.pan0 + I];
    for (int off = 16; off; off >>= 1) {
        T += __shfl_xor_sync(0xFFFFFFFFu, T, off);
        St += __shfl_xor_sync(0xFFFFFFFFu, St, off);
    }
    if (lane == 0) bt.stats[d.col0 + list[J.list0 + k]] = d.sign * (d.cT * T + St * d.inv_o2);
}

}  // namespace

int64_t refine_packed_chunks(int64_t NKB) { return (NKB + RK - 1) / RK; }

void launch_refine_packed(const Batch &b, const RefineJob *jobs, int64_t njobs, int64_t max_ctas,
                          const int32_t *list, double *part, cudaStream_t s) {
    for (int64_t j0 = 0; j0 < njobs; j0 += 65535) {   // grid.y holds at most 65535 jobs
        const int64_t nj = njobs - j0 < 65535 ? njobs - j0 : 65535;
        k_refine_packed<<<dim3((unsigned)max_ctas, (unsigned)nj), 256, 0, s>>>(b, jobs + j0, list, part);
        k_refine_packed_finish<<<(unsigned)nj, 32 * REFINE_JOB_COLS, 0, s>>>(b, jobs + j0, list, part);
    }
}

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
    k_refine_finish<<<(unsigned)((nflag + 7) / 8), 256, 0, s>>>(b, t, list, nflag, part, spart, ntiles);
}

}  // namespace ept

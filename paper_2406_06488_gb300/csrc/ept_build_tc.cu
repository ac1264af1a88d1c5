// ept_build_tc.cu -- the block build (phase 1) on tcgen05 tensor cores.
//
// Algorithm 1 builds D_XX, D_YY and D_XY once (Algorithm 3 entries; the Gaussian
// kernel of Appendix A.1 for MMD).  Here the distinct entries of the pooled upper
// storage are built from the norm expansion d^2 = ||z_i||^2 + ||z_j||^2 - 2 z_i.z_j
// with the Gram term on the tensor cores in split FP16: every pooled row i is scaled
// by its own power of two c_i (so that max_k |c_i z_ik| < 2^14, inside FP16's range;
// exact) and split c_i z_i = hi_i + lo_i (hi = fp16(c z), lo = fp16(c z - hi)); then
//     c_i c_j z_i.z_j ~ hi_i.hi_j + hi_i.lo_j + lo_i.hi_j
// (three MMAs per K-step into one FP32 accumulator in tensor memory; the dropped
// lo_i.lo_j term and the residual of the split are below 2^-21 of each product, so
// the entries are about as accurate as an FP32 Gram), and the epilogue multiplies
// by 1/c_i and 1/c_j (exact).
// The epilogue forms d^2, recomputes cancellation-prone near-duplicate pairs
// (d^2 < tau (||z_i||^2 + ||z_j||^2)) directly in FP64, applies sqrt (distances),
// exp(-d^2 / (2 sigma^2)) (Gaussian) or exp(-d / sigma) (Laplacian), forces the
// diagonal to 0 / 1, zeroes padding, and
// writes the FP32 entries into the packed upper blocks.
//
// Tile = 128 rows (half of a 256-row panel I) x 256 columns (panel J >= I, four
// K-blocks); K loop over p in steps of 64 with TMA loads of the four operand tiles
// (A hi/lo 128 x 64, B hi/lo 256 x 64, 128-byte swizzle); two TMEM accumulators so
// the epilogue of one tile overlaps the main loop of the next.  Roles (320
// threads): warp 0 TMA, warp 1 MMA + TMEM owner, warps 2-9 epilogue (two per TMEM
// lane quarter, each taking half of the tile's columns).  All waits are bounded as
// in the contraction kernel.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstdio>
#include <cstring>

#include "ept_internal.cuh"
#include "ept_tc_common.cuh"

namespace ept {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int STAGES = 2;
constexpr int A_BYTES = BM * BK * 2;                  // 16 KB
constexpr int B_BYTES = BN * BK * 2;                  // 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // 96 KB: A hi, A lo, B hi, B lo
constexpr int NUM_THREADS = 320;   // TMA warp, MMA warp, 8 epilogue warps
constexpr int EPI_THREADS = 256;
// stages | barriers (1 KB) | per-epilogue-warp column norms and scales (8 x 1 KB) | alignment slack
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 8 * (PANEL / 2) * 8 + 1024;
// kind::f16 instruction descriptor with A = B = FP16 (format 0), D = FP32, K-major
constexpr uint32_t IDESC = idesc_f16_f32(BM, BN);

constexpr unsigned long long ERR_WAIT_TMA = 0x201, ERR_WAIT_MMA = 0x202, ERR_WAIT_EPI = 0x203, ERR_DRAIN = 0x205;

struct Bars {
    unsigned long long full[STAGES];      // 1 arrival + TMA transaction bytes
    unsigned long long empty[STAGES];     // 1 arrival (tcgen05.commit)
    unsigned long long acc_full[2];       // 1 arrival (tcgen05.commit)
    unsigned long long acc_empty[2];      // 128 epilogue-thread arrivals
    unsigned long long drain;
    uint32_t tmem_base;
    int abort_flag;
};

__device__ __forceinline__ const float *row_ptr(const TestDesc &d, int64_t i) {
    return (i < d.nx) ? d.X + i * d.p : d.Y + (i - d.nx) * d.p;
}

// Pooled row i of a test -> FP16 hi / lo parts of c_i z_i (zero padding up to the
// test's p_pad), the inverse scale 1/c_i, and the squared norm of the unscaled row
// (each product split exactly into p + e by an FMA, the p summed with TwoSum and
// every rounding error carried in a second FP32 sum: about FP64 accuracy without
// FP64 arithmetic per element; the lanes' pairs are added in FP64 and rounded once).
// c_i = 2^k with
// max |c_i z_i| < 2^14, k clamped to [-60, 60] so that 1/c_i 1/c_j stays a normal
// FP32 number (rows above 2^74 would overflow the FP32 norms in any case).
// Non-finite inputs are counted.  One warp per row of the batch.
__global__ void __launch_bounds__(256) k_split_rows(const Batch bt) {
    const int lane = threadIdx.x & 31;
    const int64_t gr = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gr >= bt.nrows_total) return;
    const int t = find_test(bt.pre.rows, bt.n_tests, gr);
    const TestDesc &d = bt.desc[t];
    const int64_t i = gr - d.row0;
    const int64_t p = d.p, p_pad = d.p_pad;
    const float *z = (i < d.n) ? row_ptr(d, i) : nullptr;
    uint32_t mx = 0;
    bool bad = false;
    if (z) {
        for (int64_t k = lane; k < p; k += 32) {
            const float v = z[k];
            if (isfinite(v)) mx = max(mx, __float_as_uint(fabsf(v)));
            else bad = true;
        }
    }
    for (int off = 16; off; off >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    if (__any_sync(0xFFFFFFFFu, bad)) {
        if (lane == 0) atomicAdd(&bt.ctr[t].nonfinite, 1ull);
    }
    int k2 = 0;
    if (mx) {
        int e;
        frexpf(__uint_as_float(mx), &e);   // max = f 2^e, 0.5 <= f < 1
        k2 = 14 - e;
        k2 = k2 < -60 ? -60 : (k2 > 60 ? 60 : k2);
    }
    const float c = ldexpf(1.f, k2);
    __half *zh = (__half *)bt.Zh + gr * bt.p_stride, *zl = (__half *)bt.Zl + gr * bt.p_stride;
    float sh = 0.f, sl = 0.f;
    for (int64_t k = 2 * lane; k < p_pad; k += 64) {
        float v0 = 0.f, v1 = 0.f;
        if (z && k < p) v0 = z[k];
        if (z && k + 1 < p) v1 = z[k + 1];
        if (!isfinite(v0)) v0 = 0.f;
        if (!isfinite(v1)) v1 = 0.f;
        {
            const float p0 = v0 * v0, e0 = fmaf(v0, v0, -p0);
            const float p1 = v1 * v1, e1 = fmaf(v1, v1, -p1);
            float s2, f;
            two_sum(sh, p0, s2, f);
            sh = s2;
            sl += f + e0;
            two_sum(sh, p1, s2, f);
            sh = s2;
            sl += f + e1;
        }
        const float w0 = v0 * c, w1 = v1 * c;
        const __half h0 = __float2half_rn(w0), h1 = __float2half_rn(w1);
        const __half l0 = __float2half_rn(w0 - __half2float(h0));
        const __half l1 = __float2half_rn(w1 - __half2float(h1));
        *reinterpret_cast<__half2 *>(zh + k) = __halves2half2(h0, h1);
        *reinterpret_cast<__half2 *>(zl + k) = __halves2half2(l0, l1);
    }
    double acc = (double)sh + (double)sl;
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if (lane == 0) {
        bt.norms[gr] = (float)acc;
        bt.iscale[gr] = ldexpf(1.f, -k2);
    }
}

// One row's 32 entries of a column group from the Gram accumulator v (scaled by
// c_i c_j): d^2 = n_i + n_j - 2 G_ij, the entry for kernel kind KERN (0 distance,
// 1 Gaussian, 2 Laplacian; the approximate square root is within 2^-22 of the
// exact one, below the split Gram's own error), and the bit mask of the entries
// that need the FP64 recomputation (d^2 < tau (n_i + n_j)).
template <int KERN>
__device__ __forceinline__ uint32_t group_entries(const uint32_t (&v)[32], const float2 *cg, float ni, float si,
                                                  float tau, float neg_inv_2s2, float inv_sigma, float (&out)[32]) {
    uint32_t fix = 0;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        const float2 cj = cg[e];
        const float gij = (__uint_as_float(v[e]) * si) * cj.y;   // exact rescaling
        const float sn = ni + cj.x;
        const float d2 = fmaxf(0.f, sn - 2.f * gij);
        fix |= (d2 < tau * sn) ? (1u << e) : 0u;
        if (KERN == 1) {
            out[e] = exp_cw(d2 * neg_inv_2s2);
        } else {
            float dist;
            asm("sqrt.approx.f32 %0, %1;" : "=f"(dist) : "f"(d2));
            out[e] = (KERN == 0) ? dist : exp_cw(-dist * inv_sigma);
        }
    }
    return fix;
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_build_tc(const __grid_constant__ CUtensorMap tm_ah, const __grid_constant__ CUtensorMap tm_al,
               const __grid_constant__ CUtensorMap tm_bh, const __grid_constant__ CUtensorMap tm_bl, const Batch bt) {
    Counters *ctr = bt.ctr;   // bounded-wait errors are recorded in test 0's counters
    const unsigned long long wait_ns = bt.wait_ns ? bt.wait_ns : WAIT_NS;   // limit of every bounded wait
    const int ntiles = (int)bt.ntiles;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Bars *bars = reinterpret_cast<Bars *>(smem + STAGES * STAGE_BYTES);
    volatile int *abort_flag = &bars->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(su32(&bars->full[s]), 1);
            mbar_init(su32(&bars->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(su32(&bars->acc_full[a]), 1);
            mbar_init(su32(&bars->acc_empty[a]), EPI_THREADS);
        }
        mbar_init(su32(&bars->drain), 1);
        bars->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         su32(&bars->tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = bars->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int armed[STAGES];
            for (int s2 = 0; s2 < STAGES; ++s2) armed[s2] = -1;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const Tile tile = bt.tiles[t];
                const int64_t row0 = bt.desc[tile.t].row0;
                const int rowA = (int)row0 + tile.I * PANEL + tile.h * BM;
                const int rowB = (int)row0 + tile.J * PANEL;
                const int kblocks = bt.desc[tile.t].kblocks;
                for (int kk = 0; kk < kblocks; ++kk) {
                    if (!mbar_wait(su32(&bars->empty[stage]), phase ^ 1u, abort_flag, ctr, ERR_WAIT_TMA, wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t full = su32(&bars->full[stage]);
                    mbar_arrive_tx(full, STAGE_BYTES);
                    uint8_t *st = smem + stage * STAGE_BYTES;
                    tma_load_2d(su32(st), &tm_ah, kk * BK, rowA, full);
                    tma_load_2d(su32(st + A_BYTES), &tm_al, kk * BK, rowA, full);
                    tma_load_2d(su32(st + 2 * A_BYTES), &tm_bh, kk * BK, rowB, full);
                    tma_load_2d(su32(st + 2 * A_BYTES + B_BYTES), &tm_bl, kk * BK, rowB, full);
                    armed[stage] = (int)phase;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                for (int s2 = 0; s2 < STAGES; ++s2) {
                    if (armed[s2] < 0) continue;
                    const unsigned long long t0 = gtimer();
                    while (!mbar_try(su32(&bars->full[s2]), (uint32_t)armed[s2])) {
                        if (gtimer() - t0 > wait_ns) {
                            atomicCAS(&ctr->err_code, 0ull, ERR_DRAIN);
                            break;
                        }
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0, acc = 0;
            uint32_t phase = 0, acc_phase = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int kblocks = bt.desc[bt.tiles[t].t].kblocks;
                if (!mbar_wait(su32(&bars->acc_empty[acc]), acc_phase ^ 1u, abort_flag, ctr, ERR_WAIT_MMA, wait_ns)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
                for (int kk = 0; kk < kblocks; ++kk) {
                    if (!mbar_wait(su32(&bars->full[stage]), phase, abort_flag, ctr, ERR_WAIT_MMA, wait_ns)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t sa = su32(smem + stage * STAGE_BYTES);
                    const uint64_t dah = desc_sw128(sa), dal = desc_sw128(sa + A_BYTES);
                    const uint64_t dbh = desc_sw128(sa + 2 * A_BYTES), dbl = desc_sw128(sa + 2 * A_BYTES + B_BYTES);
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k) {
                        mma_f16(d_tmem, dah + 2 * k, dbh + 2 * k, IDESC, (kk == 0 && k == 0) ? 0u : 1u);
                        mma_f16(d_tmem, dah + 2 * k, dbl + 2 * k, IDESC, 1u);
                        mma_f16(d_tmem, dal + 2 * k, dbh + 2 * k, IDESC, 1u);
                    }
                    mma_commit(su32(&bars->empty[stage]));
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(su32(&bars->acc_full[acc]));
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1u;
                }
            }
            mma_commit(su32(&bars->drain));
            const unsigned long long t0 = gtimer();
            while (!mbar_try(su32(&bars->drain), 0)) {
                if (gtimer() - t0 > wait_ns) {
                    atomicCAS(&ctr->err_code, 0ull, ERR_DRAIN);
                    break;
                }
            }
        }
    } else {
        // ---------------- epilogue: one tile row per thread ----------------
        // Each warp stages the tile's 256 column norms and inverse scales in its own
        // shared-memory slice (read back as broadcasts), computes each group of 32
        // entries without branches, patches padding and the diagonal with selects, and
        // recomputes the rare cancellation-prone entries afterwards (same thread, so
        // its later store wins).
        // two warps per TMEM lane quarter: each takes one half (128 columns) of the tile
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int rt = quarter * 32 + lane;   // row within the 128-row tile
        float2 *colv = reinterpret_cast<float2 *>(smem + STAGES * STAGE_BYTES + 1024) + (warp - 2) * (PANEL / 2);
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const Tile tile = bt.tiles[t];
            const TestDesc &d = bt.desc[tile.t];
            const int64_t n = d.n, p = d.p, NKB = d.NKB, nx = d.nx;
            const float *X = d.X, *Y = d.Y;
            const int kern = d.kern;
            const float neg_inv_2s2 = d.neg_inv_2s2, inv_sigma = d.inv_sigma, tau = d.tau;
            const float diag_val = (kern == 0) ? 0.f : 1.f;
            const float *norms = bt.norms + d.row0, *inv_scale = bt.iscale + d.row0;
            float *Dblk = bt.D + (d.blk0 + blk_index(tile.I, (int64_t)tile.J * KB_PER_PANEL, NKB)) * PANEL * KB;
            unsigned fixups = 0;
            const int rp = tile.h * BM + rt;                 // row within panel I
            const int64_t i = (int64_t)tile.I * PANEL + rp;  // pooled row of the test
            const float ni = (i < n) ? norms[i] : 0.f;
            const float si = (i < n) ? inv_scale[i] : 0.f;
            __syncwarp();
#pragma unroll
            for (int c = lane; c < PANEL / 2; c += 32) {
                const int64_t j = (int64_t)tile.J * PANEL + half * (PANEL / 2) + c;
                colv[c] = (j < n) ? make_float2(norms[j], inv_scale[j]) : make_float2(0.f, 0.f);
            }
            __syncwarp();
            if (!mbar_wait(su32(&bars->acc_full[acc]), acc_phase, abort_flag, ctr, ERR_WAIT_EPI, wait_ns)) break;
            fence_after();
            const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * BN);
#pragma unroll 1
            for (int gl = 0; gl < BN / 64; ++gl) {
                const int g = half * (BN / 64) + gl;   // column group of the tile
                uint32_t v[32];
                tmem_ld32(tbase + (uint32_t)(g * 32), v);
                const int64_t j0 = (int64_t)tile.J * PANEL + g * 32;
                float out[32];
                const float2 *cg = colv + gl * 32;
                uint32_t fix = (kern == 0)   ? group_entries<0>(v, cg, ni, si, tau, neg_inv_2s2, inv_sigma, out)
                               : (kern == 1) ? group_entries<1>(v, cg, ni, si, tau, neg_inv_2s2, inv_sigma, out)
                                             : group_entries<2>(v, cg, ni, si, tau, neg_inv_2s2, inv_sigma, out);
                // padding rows / columns hold 0; the diagonal is exactly 0 (ED) / 1 (MMD)
                const uint32_t jvalid =
                    (j0 >= n) ? 0u : ((j0 + 32 <= n) ? 0xFFFFFFFFu : ((1u << (uint32_t)(n - j0)) - 1u));
                const uint32_t valid = (i < n) ? jvalid : 0u;
                const int64_t dj = i - j0;
                const uint32_t diag = (dj >= 0 && dj < 32 && i < n) ? (1u << (uint32_t)dj) : 0u;
                if (valid != 0xFFFFFFFFu || diag) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        if (!((valid >> e) & 1u)) out[e] = 0.f;
                        if ((diag >> e) & 1u) out[e] = diag_val;
                    }
                }
                fix &= valid & ~diag;
                float *dst = Dblk + ((int64_t)(g >> 1) * PANEL + rp) * KB + (g & 1) * 32;
#pragma unroll
                for (int e = 0; e < 32; e += 4)
                    *reinterpret_cast<float4 *>(dst + e) = make_float4(out[e], out[e + 1], out[e + 2], out[e + 3]);
                // cancellation-prone pairs: d^2 directly in FP64
                while (fix) {
                    const int e = __ffs(fix) - 1;
                    fix &= fix - 1u;
                    const int64_t j = j0 + e;
                    const float *zi = (i < nx) ? X + i * p : Y + (i - nx) * p;
                    const float *zj = (j < nx) ? X + j * p : Y + (j - nx) * p;
                    double sq = 0.0;
                    for (int64_t k = 0; k < p; ++k) {
                        const double df = (double)zi[k] - (double)zj[k];
                        sq = fma(df, df, sq);
                    }
                    ++fixups;
                    dst[e] = (float)entry_from_d2(sq, kern, neg_inv_2s2, inv_sigma);
                }
            }
            fence_before();
            mbar_arrive(su32(&bars->acc_empty[acc]));
            if (fixups) atomicAdd(&bt.ctr[tile.t].n_fixup, (unsigned long long)fixups);
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
            }
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
    }
}

}  // namespace

void launch_split_rows(const Batch &b, cudaStream_t s) {
    if (b.nrows_total <= 0) return;
    k_split_rows<<<(unsigned)((b.nrows_total + 7) / 8), 256, 0, s>>>(b);
}

cudaError_t launch_build_tc(const Batch &b, const void *tmaps, int num_sms, cudaStream_t s) {
    static unsigned long long smem_set = 0;   // one bit per device
    cudaError_t e = smem_limit_once((const void *)k_build_tc, SMEM_BYTES, &smem_set);
    if (e != cudaSuccess) return e;
    if (b.ntiles < 1) return cudaSuccess;
    const CUtensorMap *tm = (const CUtensorMap *)tmaps;
    const int grid = b.ntiles < num_sms ? (int)b.ntiles : num_sms;
    k_build_tc<<<grid, NUM_THREADS, SMEM_BYTES, s>>>(tm[0], tm[1], tm[2], tm[3], b);
    return cudaGetLastError();
}

}  // namespace ept

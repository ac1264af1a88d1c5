// ept_contract_tc.cu -- the permutation contraction on 5th-generation tensor cores.
//
// What it computes (Algorithm 1, permutation loop, rewritten as quadratic forms):
// for relabeling column b with indicator s_b (s_b[t] = 1 iff pooled row t goes to
// x*), the statistic needs Q_b = s_b' C s_b, where C is the packed, centred,
// upper-scaled pooled matrix (see ept_kernels.cu, packing).  Work unit (q, m, h):
// chunk q = (panel I, K-blocks [kb0, kb1)), relabeling tile m (256 columns), half h
// of the panel's rows (128 rows):
//     U[i, b]              = sum_{j in chunk} C[i, j] s_b[j]     (tensor cores)
//     partial[2q + h][b]   = sum_{i in half h} s_b[i] U[i, b]    (epilogue)
// and Q_b = sum over parts (FP64, ept_kernels.cu).
//
// Mapping onto tcgen05 (kind::f16, cta_group::1), M = 128 rows of C, N = 256
// relabelings, K = 64 pooled columns per stage:
//   A (128 x 64): the packed C half-block, the test's C scaled by a power of two and
//     split hi + lo in FP16, loaded by TMA (two 16 KB boxes, 128-byte swizzle);
//   B (256 x 64): 0/1 relabeling values, exact in FP16, expanded from the bit masks
//     by eight producer warps straight into the 128-byte-swizzled K-major layout;
//   D (128 x 256 FP32) in tensor memory: D += A_hi * B, then D += A_lo * B.
//   With the relabelings as N, one stage moves 32 KB through TMA for 2 x 128 x 256 x
//   64 multiply-adds (half of what the relabelings-as-M mapping needs), and three
//   64 KB stages fit in shared memory.  Two accumulators (512 TMEM columns) let the
//   epilogue of one unit overlap the main loop of the next.
//   Epilogue: TMEM lane = row i; a warp reads 32 relabelings at a time, takes the
//   mask bits of its 32 rows for them with a 32 x 32 bit transpose (shuffles), masks
//   its values, and sums over its 32 rows with a butterfly transpose-reduce (lane e
//   ends with relabeling e's sum).  The four warps' sums meet in shared memory and
//   are added in a fixed order.
//
// Roles (576 threads): warp 0 = TMA producer, warp 1 = MMA issuer (and TMEM
// owner), warps 2-9 = epilogue (two warps per TMEM lane quarter, each taking half
// of the relabelings), warps 10-17 = relabeling-tile producers (one B row each).
// Every role takes its units from the precomputed 64-byte records of the schedule
// (UnitRec) and reads the next unit's record while it works on the current one, so
// that no role waits on the schedule, test and chunk tables at a unit boundary.
// Two epilogue and two producer warps per SM sub-partition hide each other's
// shared-memory and L2 latencies.  Every wait on an mbarrier is bounded (2 s unless
// the context sets another limit), and a waiting thread sleeps in the wait until its
// phase completes; on expiry the kernel records an error code, raises a CTA-wide
// abort flag, drains its own copies and MMAs (bounded again), frees its tensor
// memory and returns.
#include <cuda.h>
#include <cstdio>
#include <cstring>

#include "ept_internal.cuh"
#include "ept_tc_common.cuh"

namespace ept {

namespace {

using namespace tc;

constexpr int TC_M = 128;                         // rows of C per unit (half a panel)
constexpr int TC_N = TC_TILE_N;                   // relabelings per unit (256)
constexpr int STAGES = 3;
constexpr int A_BYTES = TC_M * KB * 2;            // 16 KB (hi or lo)
constexpr int B_BYTES = TC_N * KB * 2;            // 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + B_BYTES;   // A hi | A lo | B
constexpr int RED_BYTES = 2 * 4 * TC_N * 4;       // epilogue sums: 2 buffers x 4 warps x 256 floats
constexpr int NUM_THREADS = 576;
constexpr int EPI_THREADS = 256;                  // warps 2-9
constexpr int PROD_THREADS = 256;                 // warps 10-17
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*barriers*/ + RED_BYTES + 1024 /*alignment*/;

// error codes recorded in Counters::err_code
constexpr unsigned long long ERR_WAIT_TMA = 0x101, ERR_WAIT_MMA = 0x102, ERR_WAIT_EPI = 0x103,
                             ERR_WAIT_MASK = 0x104, ERR_DRAIN = 0x105, ERR_INJECTED = 0x1FF;

constexpr uint32_t IDESC = idesc_f16_f32(TC_M, TC_N);

// the barrier region (1 KB): Bars at its start, the 128-byte nibble table at byte 512
struct Bars {
    unsigned long long b_full[STAGES];   // 256 producer-thread arrivals (relabeling tile)
    unsigned long long a_full[STAGES];   // 1 arrival + TMA transaction bytes (C half-block)
    unsigned long long empty[STAGES];    // 1 arrival (tcgen05.commit)
    unsigned long long acc_full[2];      // 1 arrival (tcgen05.commit)
    unsigned long long acc_empty[2];     // 256 epilogue-thread arrivals
    unsigned long long red;              // 256 epilogue-thread arrivals per unit
    unsigned long long drain;            // 1 arrival (final tcgen05.commit)
    uint32_t tmem_base;
    int abort_flag;
};
static_assert(sizeof(Bars) <= 512, "barriers overlap the nibble table");

// MMA N for a unit: the tile's existing relabeling columns, rounded up to 16
__device__ __forceinline__ int mma_n(const UnitRec &x) { return x.left >= TC_N ? TC_N : (x.left + 15) / 16 * 16; }

__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_contract_tc(const __grid_constant__ CUtensorMap tmap_hi, const __grid_constant__ CUtensorMap tmap_lo,
                  const Batch bt) {
    Counters *ctr = bt.ctr;   // bounded-wait errors are recorded in test 0's counters
    const unsigned long long wait_ns = bt.wait_ns ? bt.wait_ns : WAIT_NS;   // limit of every bounded wait
    const int64_t nunits = bt.nunits_total;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Bars *bars = reinterpret_cast<Bars *>(smem + STAGES * STAGE_BYTES);
    float *red = reinterpret_cast<float *>(smem + STAGES * STAGE_BYTES + 1024);
    volatile int *abort_flag = &bars->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's units: its slice of the schedule, or every gridDim.x-th unit; every
    // role reads the record of its next unit while it works on the current one
    const int64_t k_first = bt.sched ? bt.sched_off[blockIdx.x] : (int64_t)blockIdx.x;
    const int64_t k_end = bt.sched ? bt.sched_off[blockIdx.x + 1] : nunits;
    const int64_t k_step = bt.sched ? 1 : (int64_t)gridDim.x;
    auto record = [&bt, k_end](int64_t k) { return k < k_end ? unit_at_position(bt, k) : UnitRec{}; };

    // nibble -> four FP16 values (1.0 where the bit is set), for the relabeling producers
    uint2 *lut = reinterpret_cast<uint2 *>(smem + STAGES * STAGE_BYTES + 512);
    if (threadIdx.x < 16) {
        const uint32_t n = threadIdx.x;
        lut[n] = make_uint2((n & 1u) * 0x3C00u + (n & 2u) * 0x1E000000u,
                            ((n >> 2) & 1u) * 0x3C00u + ((n >> 2) & 2u) * 0x1E000000u);
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(su32(&bars->b_full[s]), PROD_THREADS);
            mbar_init(su32(&bars->a_full[s]), 1);
            mbar_init(su32(&bars->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(su32(&bars->acc_full[a]), 1);
            mbar_init(su32(&bars->acc_empty[a]), EPI_THREADS);
        }
        mbar_init(su32(&bars->red), EPI_THREADS);
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
        // ---------------- TMA producer: packed C hi / lo half-blocks ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int armed[STAGES];   // parity of the last phase armed on each stage, -1 = none
            for (int s2 = 0; s2 < STAGES; ++s2) armed[s2] = -1;
            bool ok = true;
            UnitRec nx = record(k_first);
            for (int64_t k = k_first; k < k_end && ok; k += k_step) {
                const UnitRec x = nx;
                nx = record(k + k_step);
                const int row = x.h * TC_M;
                for (int kb = x.kb0; kb < x.kb1; ++kb) {
                    if (!mbar_wait(su32(&bars->empty[stage]), phase ^ 1u, abort_flag, ctr, ERR_WAIT_TMA, wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t afull = su32(&bars->a_full[stage]);
                    mbar_arrive_tx(afull, 2 * A_BYTES);
                    const int blk = (int)(x.blk0 + blk_index(x.I, kb, x.NKB));
                    uint8_t *st = smem + stage * STAGE_BYTES;
                    tma_load_3d(su32(st), &tmap_hi, 0, row, blk, afull);
                    tma_load_3d(su32(st + A_BYTES), &tmap_lo, 0, row, blk, afull);
                    armed[stage] = (int)phase;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // drain: the copies armed last on each stage complete that phase of
                // a_full; wait for it (bounded) before the CTA may exit
                for (int s2 = 0; s2 < STAGES; ++s2) {
                    if (armed[s2] < 0) continue;
                    const unsigned long long t0 = gtimer();
                    while (!mbar_try(su32(&bars->a_full[s2]), (uint32_t)armed[s2])) {
                        if (gtimer() - t0 > wait_ns) {
                            atomicCAS(&ctr->err_code, 0ull, ERR_DRAIN);
                            break;
                        }
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int stage = 0, acc = 0;
            uint32_t phase = 0, acc_phase = 0;
            bool ok = true;
            // failure-path test hook: wait (bounded) on a flag that nothing sets; the
            // expiry takes the same abort path as any other expired wait
            if (bt.inject_stall && !flag_wait(&ctr->never_set, abort_flag, ctr, ERR_INJECTED, wait_ns)) ok = false;
            UnitRec nx = record(k_first);
            for (int64_t k = k_first; k < k_end && ok; k += k_step) {
                const UnitRec x = nx;
                nx = record(k + k_step);
                const int ncols = mma_n(x);
                const uint32_t idesc = (ncols == TC_N) ? IDESC : idesc_f16_f32(TC_M, ncols);
                if (!mbar_wait(su32(&bars->acc_empty[acc]), acc_phase ^ 1u, abort_flag, ctr, ERR_WAIT_MMA, wait_ns)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * TC_N);
                bool first = true;
                for (int kb = x.kb0; kb < x.kb1; ++kb) {
                    if (!mbar_wait(su32(&bars->a_full[stage]), phase, abort_flag, ctr, ERR_WAIT_MMA, wait_ns) ||
                        !mbar_wait(su32(&bars->b_full[stage]), phase, abort_flag, ctr, ERR_WAIT_MMA, wait_ns)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t sa = su32(smem + stage * STAGE_BYTES);
                    const uint64_t dhi = desc_sw128(sa);
                    const uint64_t dlo = desc_sw128(sa + A_BYTES);
                    const uint64_t db = desc_sw128(sa + 2 * A_BYTES);
#pragma unroll
                    for (int k = 0; k < KB / 16; ++k)
                        mma_f16(d_tmem, dhi + 2 * k, db + 2 * k, idesc, (first && k == 0) ? 0u : 1u);
#pragma unroll
                    for (int k = 0; k < KB / 16; ++k) mma_f16(d_tmem, dlo + 2 * k, db + 2 * k, idesc, 1u);
                    mma_commit(su32(&bars->empty[stage]));
                    first = false;
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
            // drain every MMA this thread issued before the CTA frees its tensor memory
            mma_commit(su32(&bars->drain));
            unsigned long long t0 = gtimer();
            while (!mbar_try(su32(&bars->drain), 0)) {
                if (gtimer() - t0 > wait_ns) {
                    atomicCAS(&ctr->err_code, 0ull, ERR_DRAIN);
                    break;
                }
            }
        }
    } else if (warp < 10) {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3;           // TMEM lanes (rows) this warp may access
        const int g0 = ((warp - 2) >> 2) * 4;   // this warp's four groups of 32 relabelings
        const int et = threadIdx.x - 64;        // 0..255
        int acc = 0;
        uint32_t acc_phase = 0, red_phase = 0;
        int rbuf = 0;
        UnitRec nx = record(k_first);
        for (int64_t k = k_first; k < k_end; k += k_step) {
            const UnitRec x = nx;
            nx = record(k + k_step);
            const int64_t Bp = x.Bp;
            // mask word of this warp's 32 rows, for the warp's 128 relabelings
            const uint32_t *wrow = bt.maskT + x.mask_col + ((int64_t)x.I * 8 + x.h * 4 + quarter) * Bp + g0 * 32;
            uint32_t words[4];
#pragma unroll
            for (int g = 0; g < 4; ++g) words[g] = wrow[g * 32 + lane];
            if (!mbar_wait(su32(&bars->acc_full[acc]), acc_phase, abort_flag, ctr, ERR_WAIT_EPI, wait_ns)) break;
            fence_after();
            const uint32_t tbase =
                tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * TC_N) + (uint32_t)(g0 * 32);
            float *myred = red + (rbuf * 4 + quarter) * TC_N + g0 * 32;
#pragma unroll 1
            for (int g = 0; g < 4; ++g) {
                uint32_t v[32];
                tmem_ld32(tbase + (uint32_t)(g * 32), v);
                // bit e of `mine` = s_{b_e}[row of this lane], b_e = relabeling 32 (g0 + g) + e:
                // the 32 x 32 bit matrix (lane = relabeling, bit = row) transposed in five
                // butterfly stages, each swapping the off-diagonal halves of 2j x 2j blocks
                uint32_t mine = words[g];
#pragma unroll
                for (int j = 16; j >= 1; j >>= 1) {
                    const uint32_t m = j == 16 ? 0x0000FFFFu
                                     : j == 8  ? 0x00FF00FFu
                                     : j == 4  ? 0x0F0F0F0Fu
                                     : j == 2  ? 0x33333333u
                                               : 0x55555555u;
                    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, mine, j);
                    mine = (lane & j) ? ((mine & ~m) | ((y & ~m) >> j)) : ((mine & m) | ((y & m) << j));
                }
                float xv[32];
#pragma unroll
                for (int e = 0; e < 32; ++e) xv[e] = ((mine >> e) & 1u) ? __uint_as_float(v[e]) : 0.f;
                // butterfly transpose-reduce: lane e ends with the sum over the warp's rows of column e
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) {
                    const bool upper = (lane & off) != 0;
#pragma unroll
                    for (int k = 0; k < off; ++k) {
                        const float send = upper ? xv[k] : xv[k + off];
                        const float keep = upper ? xv[k + off] : xv[k];
                        xv[k] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, off);
                    }
                }
                myred[g * 32 + lane] = xv[0];
            }
            fence_before();
            mbar_arrive(su32(&bars->acc_empty[acc]));
            // the four row quarters' sums, added in a fixed order
            mbar_arrive(su32(&bars->red));
            if (!mbar_wait(su32(&bars->red), red_phase, abort_flag, ctr, ERR_WAIT_EPI, wait_ns)) break;
            const float *rb = red + rbuf * 4 * TC_N;
            float *out = bt.partial + x.out_off;
            out[et] = (rb[et] + rb[TC_N + et]) + (rb[2 * TC_N + et] + rb[3 * TC_N + et]);
            red_phase ^= 1u;
            rbuf ^= 1;
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
            }
        }
    } else {
        // ---------------- relabeling-tile producers ----------------
        // The mask words of a stage are loaded two stages ahead, so that their L2
        // latency overlaps the expansion of the stages before.
        const int r = threadIdx.x - 320;   // 0..255: row r of the B tile
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        UnitRec nx = record(k_first);
        for (int64_t k = k_first; k < k_end && ok; k += k_step) {
            const UnitRec x = nx;
            nx = record(k + k_step);
            const int64_t Bp = x.Bp;
            const uint32_t *maskT = bt.maskT + x.mask_col + r;
            // words 2 kb and 2 kb + 1 of relabeling r
            auto load2 = [&](int kb, uint2 &w) {
                const uint32_t *p0 = maskT + (int64_t)(2 * kb) * Bp;
                w.x = p0[0];
                w.y = p0[Bp];
            };
            uint2 cur = make_uint2(0, 0), nxt = make_uint2(0, 0);
            load2(x.kb0, cur);
            if (x.kb0 + 1 < x.kb1) load2(x.kb0 + 1, nxt);
            const int ncols = mma_n(x);
            for (int kb = x.kb0; kb < x.kb1; ++kb) {
                uint2 nn = make_uint2(0, 0);
                if (kb + 2 < x.kb1) load2(kb + 2, nn);
                if (!mbar_wait(su32(&bars->empty[stage]), phase ^ 1u, abort_flag, ctr, ERR_WAIT_MASK, wait_ns)) {
                    ok = false;
                    break;
                }
                uint8_t *brow = smem + stage * STAGE_BYTES + 2 * A_BYTES + r * 128;
                if (r < ncols) {   // rows past the tile's columns are not read by the MMA
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const uint32_t w = c < 4 ? cur.x : cur.y;
                        const uint2 lo = lut[(w >> (8 * (c & 3))) & 15u];
                        const uint2 hi = lut[(w >> (8 * (c & 3) + 4)) & 15u];
                        const uint32_t dst = su32(brow + ((c ^ (r & 7)) << 4));
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(lo.x), "r"(lo.y),
                                     "r"(hi.x), "r"(hi.y)
                                     : "memory");
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(su32(&bars->b_full[stage]));
                cur = nxt;
                nxt = nn;
                if (++stage == STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
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

cudaError_t launch_contract_tc(const Batch &b, const void *tmap_hi, const void *tmap_lo, int num_sms,
                               cudaStream_t s) {
    static unsigned long long smem_set = 0;   // one bit per device
    cudaError_t e = smem_limit_once((const void *)k_contract_tc, SMEM_BYTES, &smem_set);
    if (e != cudaSuccess) return e;
    int64_t grid = b.sched ? (int64_t)b.tc_grid : (int64_t)num_sms;
    if (grid > b.nunits_total) grid = b.nunits_total;
    if (grid < 1) return cudaSuccess;
    CUtensorMap th, tl;
    memcpy(&th, tmap_hi, sizeof(CUtensorMap));
    memcpy(&tl, tmap_lo, sizeof(CUtensorMap));
    k_contract_tc<<<(unsigned)grid, NUM_THREADS, SMEM_BYTES, s>>>(th, tl, b);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled is a driver-API call; it is looked up through the runtime
// so that libept does not link libcuda (and still loads on machines without a GPU).
using EncodeTiledFn = decltype(&cuTensorMapEncodeTiled);

static EncodeTiledFn encode_fn(char *err, size_t errlen) {
    static EncodeTiledFn fn = nullptr;
    if (fn) return fn;
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !ptr) {
        snprintf(err, errlen, "cuTensorMapEncodeTiled unavailable (%s, query %d)", cudaGetErrorString(e), (int)q);
        return nullptr;
    }
    fn = reinterpret_cast<EncodeTiledFn>(ptr);
    return fn;
}

bool encode_rows_tmaps(void *tmaps4, const uint16_t *Zh, const uint16_t *Zl, int64_t nrows, int64_t p_stride,
                       char *err, size_t errlen) {
    EncodeTiledFn enc = encode_fn(err, errlen);
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)p_stride, (cuuint64_t)nrows};
    const cuuint64_t strides[1] = {(cuuint64_t)p_stride * 2};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint32_t box_a[2] = {64, 128}, box_b[2] = {64, 256};
    CUtensorMap *out = (CUtensorMap *)tmaps4;
    const void *srcs[4] = {Zh, Zl, Zh, Zl};
    const cuuint32_t *boxes[4] = {box_a, box_a, box_b, box_b};
    for (int k = 0; k < 4; ++k) {
        CUresult r = enc(&out[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void *)srcs[k], dims, strides, boxes[k], estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            snprintf(err, errlen, "cuTensorMapEncodeTiled (rows) failed (%d)", (int)r);
            return false;
        }
    }
    return true;
}

bool encode_block_tmaps(void *tmap_hi, void *tmap_lo, const uint16_t *Chi, const uint16_t *Clo, int64_t nblk,
                        int64_t c_stride, char *err, size_t errlen) {
    EncodeTiledFn enc = encode_fn(err, errlen);
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)KB, (cuuint64_t)PANEL, (cuuint64_t)nblk};
    const cuuint64_t strides[2] = {(cuuint64_t)KB * 2, (cuuint64_t)c_stride * 2};
    const cuuint32_t box[3] = {(cuuint32_t)KB, (cuuint32_t)TC_M, 1};   // 128 rows of a block per copy
    const cuuint32_t estr[3] = {1, 1, 1};
    void *ptrs[2] = {(void *)Chi, (void *)Clo};
    void *outs[2] = {tmap_hi, tmap_lo};
    for (int k = 0; k < 2; ++k) {
        CUresult r = enc((CUtensorMap *)outs[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, ptrs[k], dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            snprintf(err, errlen, "cuTensorMapEncodeTiled failed (%d)", (int)r);
            return false;
        }
    }
    return true;
}

}  // namespace ept

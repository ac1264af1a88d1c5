// ept_contract_tm.cu -- the permutation contraction with the relabeling tile as the
// tensor-memory operand: Q_b = s_b' C s_b (Algorithm 1's permutation loop written
// as quadratic forms), the same work units, partial sums and summation depth as
// ept_contract_tc.cu, with the roles of the two MMA operands exchanged.
//
// Mapping (tcgen05 kind::f16, cta_group::1), per sub-unit (chunk q of K-blocks, 128
// relabelings of the unit's 256-relabeling tile, row half h of the panel):
//   A (128 x 64, tensor memory): the 0/1 relabeling values in FP16, row = relabeling.
//     Producer threads expand their own relabeling's mask bits in registers and store
//     them with tcgen05.st (TMEM lane = relabeling), so the relabeling tile never
//     passes through shared memory;
//   B (128 x 64, shared memory): the packed C half-block (FP16 hi and lo, TMA,
//     128-byte swizzle, the same copies as ept_contract_tc.cu), read as N = 128 rows;
//   D (128 x 128 FP32, tensor memory): D[b, i] = sum_j s_b[j] C[i, j], hi pass then
//     lo pass, K = 64 pooled columns per stage.
// Epilogue: TMEM lane = relabeling b, column = row i.  Each thread reads its
// relabeling's 128 values, keeps those of the rows in its group (its own mask bits,
// no transposes) and sums them in a fixed pairwise tree (groups of 32 rows, then
// ((g0 + g1) + (g2 + g3)): the depth of ept_contract_tc.cu's butterfly and
// four-quarter sum); no reduction across threads.
//
// Shared-memory traffic per K-block and 2 x 128 x 256 x 64 multiply-adds: the MMAs
// read 64 KB and TMA writes 64 KB, against about 96 KB of MMA reads, 32 KB of TMA
// writes and 32 KB of relabeling-tile stores (plus their table reads) when the
// relabelings are the shared-memory operand.  The price is twice the L2 reads of
// the C blocks: a unit of the schedule (q, 256-relabeling tile m, h) runs as its two
// 128-relabeling sub-units one after the other, each loading its chunk's blocks (two
// accumulators of 128 columns let the epilogue of one sub-unit overlap the main
// loop of the next; the relabeling stages take another 32 columns each).
//
// Measured on a GB300 (n = 5000, B = 10^4): 451 us against 303 us for
// ept_contract_tc.cu.  The MMAs alone (no copies, producers or epilogue) take 366 us
// here against 254 us there for the same multiply-adds: an MMA with N = 128 does
// less work per cycle than one with N = 256 (with the C half-block as the
// shared-memory A operand and N = 128 relabelings, 410 us), and N = 256 rows of C
// would need 2 x 256 accumulator columns beside the relabeling stages, more than the
// 512 columns of tensor memory.  Kept as EPT_OPT_CONTRACTION = 3.
//
// Roles (448 threads): warp 0 TMA, warp 1 MMA issuer and TMEM owner, warps 2-5
// epilogue (one per TMEM lane quarter), warps 6-13 relabeling producers (two per lane
// quarter, taking alternate K-blocks).  Every wait on an mbarrier is bounded (the
// abort protocol of ept_tc_common.cuh).
#include <cuda.h>
#include <cstdio>
#include <cstring>

#include "ept_internal.cuh"
#include "ept_tc_common.cuh"

namespace ept {

namespace {

using namespace tc;

constexpr int TM_M = 128;                         // relabelings per sub-unit (the MMA's M)
constexpr int TM_N = 128;                         // rows of C per sub-unit (the MMA's N)
constexpr int STAGES = 6;
constexpr int C_BYTES = TM_N * KB * 2;            // 16 KB (hi or lo)
constexpr int STAGE_BYTES = 2 * C_BYTES;          // C hi | C lo
constexpr int NUM_THREADS = 448;
constexpr int EPI_THREADS = 128;                  // warps 2-5
constexpr int PROD_THREADS = 128;                 // arrivals per stage: the four producer warps of its parity
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*barriers*/ + 1024 /*alignment*/;
constexpr uint32_t D_COLS = TM_N;                 // TMEM columns of one accumulator
constexpr uint32_t A_COL0 = 2 * D_COLS;           // first TMEM column of the relabeling stages
constexpr uint32_t A_COLS = KB / 2;               // TMEM columns of one relabeling stage (64 FP16 per lane)
static_assert(A_COL0 + STAGES * A_COLS <= 512, "tensor memory");

constexpr unsigned long long ERR_WAIT_TMA = 0x301, ERR_WAIT_MMA = 0x302, ERR_WAIT_EPI = 0x303,
                             ERR_WAIT_MASK = 0x304, ERR_DRAIN = 0x305, ERR_INJECTED = 0x3FF;

constexpr uint32_t IDESC = idesc_f16_f32(TM_M, TM_N);

struct Bars {
    unsigned long long c_full[STAGES];   // 1 arrival + TMA transaction bytes (C half-block)
    unsigned long long a_full[STAGES];   // 128 producer arrivals (relabeling stage in TMEM)
    unsigned long long empty[STAGES];    // 1 arrival (tcgen05.commit): the stage's MMAs are done
    unsigned long long acc_full[2];      // 1 arrival (tcgen05.commit)
    unsigned long long acc_empty[2];     // 128 epilogue arrivals
    unsigned long long drain;            // 1 arrival (final tcgen05.commit)
    uint32_t tmem_base;
    int abort_flag;
};
static_assert(sizeof(Bars) <= 1024, "barrier region");

// D (tensor memory) += A (tensor memory) * B (shared memory)^T, or D = A * B^T when
// accumulate == 0; issued by one thread.
__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
        ::"r"(d_tmem), "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 32 consecutive TMEM columns of this thread's lane from 32 registers; returns when
// the stores are done
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
        ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
        "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
        "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// the test fields, chunk, 256-relabeling tile and row half of global work unit u
// (the numbering of ept_contract_tc.cu), read once into registers
struct Unit {
    Chunk ch;
    int64_t q, m, h, Bp, mask0, part0, blk0, NKB;
    int left;   // relabeling columns of the tile that exist (more than 256: a full tile)
};

__device__ __forceinline__ Unit decode_unit(const Batch &bt, int64_t u) {
    const int t = find_test(bt.pre.units, bt.n_tests, u);
    const TestDesc *d = &bt.desc[t];
    Unit x;
    const int64_t lu = u - bt.pre.units[t];
    const int64_t MT = d->MT;
    x.h = lu & 1;
    x.q = (lu >> 1) / MT;
    x.m = (lu >> 1) % MT;
    x.Bp = d->Bp;
    x.mask0 = d->mask0;
    x.part0 = d->part0;
    x.blk0 = d->blk0;
    x.NKB = d->NKB;
    x.ch = bt.chunks[d->chunk0 + x.q];
    // the first two K-blocks of a panel's diagonal square lie below the diagonal for
    // the second row half: all zero in C, skipped
    if (x.h == 1 && x.ch.kb0 == KB_PER_PANEL * x.ch.I && x.ch.kb1 - x.ch.kb0 > 2) x.ch.kb0 += 2;
    const int64_t left = d->ncols - x.m * TC_TILE_N;
    x.left = left > TC_TILE_N ? TC_TILE_N : (int)left;
    return x;
}

// sub-unit s (relabelings 128 s .. 128 s + 127 of the tile) has columns to compute
__device__ __forceinline__ bool has_sub(const Unit &x, int s) { return x.left > TM_M * s; }

// FP16 pair of 0/1 values (1.0 = 0x3C00) from bits 2c and 2c + 1 of w
__device__ __forceinline__ uint32_t pair_of(uint32_t w, int c) {
    const uint32_t t = (w >> (2 * c)) & 3u;
    return ((t * 0x8001u) & 0x10001u) * 0x3C00u;
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_contract_tm(const __grid_constant__ CUtensorMap tmap_hi, const __grid_constant__ CUtensorMap tmap_lo,
                  const Batch bt) {
    Counters *ctr = bt.ctr;   // bounded-wait errors are recorded in test 0's counters
    const unsigned long long wait_ns = bt.wait_ns ? bt.wait_ns : WAIT_NS;
    const int64_t nunits = bt.nunits_total;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Bars *bars = reinterpret_cast<Bars *>(smem + STAGES * STAGE_BYTES);
    volatile int *abort_flag = &bars->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t k_first = bt.sched ? bt.sched_off[blockIdx.x] : (int64_t)blockIdx.x;
    const int64_t k_end = bt.sched ? bt.sched_off[blockIdx.x + 1] : nunits;
    const int64_t k_step = bt.sched ? 1 : (int64_t)gridDim.x;
    const int64_t *sched = bt.sched;
    auto unit_at = [sched](int64_t k) { return sched ? sched[k] : k; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(su32(&bars->c_full[s]), 1);
            mbar_init(su32(&bars->a_full[s]), PROD_THREADS);
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
        // ---------------- TMA producer: packed C hi / lo half-blocks ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int armed[STAGES];   // parity of the last phase armed on each stage, -1 = none
            for (int s2 = 0; s2 < STAGES; ++s2) armed[s2] = -1;
            bool ok = true;
            for (int64_t k = k_first; k < k_end && ok; k += k_step) {
                const Unit x = decode_unit(bt, unit_at(k));
                const int row = (int)x.h * TM_N;
                for (int s = 0; s < 2 && ok; ++s) {
                    if (!has_sub(x, s)) continue;
                    for (int kb = x.ch.kb0; kb < x.ch.kb1; ++kb) {
                        if (!mbar_wait(su32(&bars->empty[stage]), phase ^ 1u, abort_flag, ctr, ERR_WAIT_TMA,
                                       wait_ns)) {
                            ok = false;
                            break;
                        }
                        const uint32_t cfull = su32(&bars->c_full[stage]);
                        mbar_arrive_tx(cfull, 2 * C_BYTES);
                        const int blk = (int)(x.blk0 + blk_index(x.ch.I, kb, x.NKB));
                        uint8_t *st = smem + stage * STAGE_BYTES;
                        tma_load_3d(su32(st), &tmap_hi, 0, row, blk, cfull);
                        tma_load_3d(su32(st + C_BYTES), &tmap_lo, 0, row, blk, cfull);
                        armed[stage] = (int)phase;
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {
                // drain: the copies armed last on each stage complete that phase of
                // c_full; wait for it (bounded) before the CTA may exit
                for (int s2 = 0; s2 < STAGES; ++s2) {
                    if (armed[s2] < 0) continue;
                    const unsigned long long t0 = gtimer();
                    while (!mbar_try(su32(&bars->c_full[s2]), (uint32_t)armed[s2])) {
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
            for (int64_t k = k_first; k < k_end && ok; k += k_step) {
                const Unit x = decode_unit(bt, unit_at(k));
                for (int s = 0; s < 2 && ok; ++s) {
                    if (!has_sub(x, s)) continue;
                    if (!mbar_wait(su32(&bars->acc_empty[acc]), acc_phase ^ 1u, abort_flag, ctr, ERR_WAIT_MMA,
                                   wait_ns)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)acc * D_COLS;
                    bool first = true;
                    for (int kb = x.ch.kb0; kb < x.ch.kb1; ++kb) {
                        if (!mbar_wait(su32(&bars->c_full[stage]), phase, abort_flag, ctr, ERR_WAIT_MMA, wait_ns) ||
                            !mbar_wait(su32(&bars->a_full[stage]), phase, abort_flag, ctr, ERR_WAIT_MMA, wait_ns)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t sb = su32(smem + stage * STAGE_BYTES);
                        const uint64_t dhi = desc_sw128(sb);
                        const uint64_t dlo = desc_sw128(sb + C_BYTES);
                        const uint32_t a_tmem = tmem_base + A_COL0 + (uint32_t)stage * A_COLS;
#pragma unroll
                        for (int kk = 0; kk < KB / 16; ++kk)
                            mma_f16_ts(d_tmem, a_tmem + 8u * kk, dhi + 2 * kk, IDESC, (first && kk == 0) ? 0u : 1u);
#pragma unroll
                        for (int kk = 0; kk < KB / 16; ++kk) mma_f16_ts(d_tmem, a_tmem + 8u * kk, dlo + 2 * kk, IDESC, 1u);
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
            }
            // drain every MMA this thread issued before the CTA frees its tensor memory
            mma_commit(su32(&bars->drain));
            const unsigned long long t0 = gtimer();
            while (!mbar_try(su32(&bars->drain), 0)) {
                if (gtimer() - t0 > wait_ns) {
                    atomicCAS(&ctr->err_code, 0ull, ERR_DRAIN);
                    break;
                }
            }
        }
    } else if (warp < 6) {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3;   // TMEM lanes (relabelings) this warp may access
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        for (int64_t k = k_first; k < k_end && ok; k += k_step) {
            const Unit x = decode_unit(bt, unit_at(k));
            for (int s = 0; s < 2; ++s) {
                if (!has_sub(x, s)) continue;
                const int64_t col = x.m * TC_TILE_N + TM_M * s + 32 * quarter + lane;   // this thread's relabeling
                // its mask words of the row half's four groups of 32 rows
                const uint32_t *wcol = bt.maskT + x.mask0 + ((int64_t)x.ch.I * 8 + x.h * 4) * x.Bp + col;
                uint32_t words[4];
#pragma unroll
                for (int g = 0; g < 4; ++g) words[g] = wcol[g * x.Bp];
                if (!mbar_wait(su32(&bars->acc_full[acc]), acc_phase, abort_flag, ctr, ERR_WAIT_EPI, wait_ns)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)acc * D_COLS;
                // groups of 32 rows: (g0 + g1) + (g2 + g3), each group a pairwise tree
                float s01 = 0.f, s23 = 0.f;
#pragma unroll 1
                for (int g = 0; g < 4; ++g) {
                    const uint32_t wg = g == 0 ? words[0] : g == 1 ? words[1] : g == 2 ? words[2] : words[3];
                    uint32_t v[32];
                    tmem_ld32(tbase + (uint32_t)(g * 32), v);
                    float xv[32];
#pragma unroll
                    for (int e = 0; e < 32; ++e) xv[e] = ((wg >> e) & 1u) ? __uint_as_float(v[e]) : 0.f;
#pragma unroll
                    for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
                        for (int e = 0; e < w; ++e) xv[e] = xv[e] + xv[e + w];
                    if (g == 0) s01 = xv[0];
                    else if (g == 1) s01 = s01 + xv[0];
                    else if (g == 2) s23 = xv[0];
                    else s23 = s23 + xv[0];
                }
                fence_before();
                mbar_arrive(su32(&bars->acc_empty[acc]));
                float *out = bt.partial + x.part0 + (2 * x.q + x.h) * x.Bp;
                out[col] = s01 + s23;
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1u;
                }
            }
        }
    } else {
        // ---------------- relabeling producers ----------------
        // Warp 6 + 4 par + quarter writes the relabeling stages of the K-blocks at odd
        // (par = 1) or even positions of the CTA's K-block sequence, for the 32
        // relabelings of its TMEM lane quarter.
        const int quarter = warp & 3, par = (warp - 6) >> 2;
        int stage = 0;
        uint32_t phase = 0;
        int64_t pos = 0;
        bool ok = true;
        for (int64_t k = k_first; k < k_end && ok; k += k_step) {
            const Unit x = decode_unit(bt, unit_at(k));
            for (int s = 0; s < 2 && ok; ++s) {
                if (!has_sub(x, s)) continue;
                const int64_t col = x.m * TC_TILE_N + TM_M * s + 32 * quarter + lane;
                const uint32_t *mcol = bt.maskT + x.mask0 + col;
                for (int kb = x.ch.kb0; kb < x.ch.kb1; ++kb, ++pos) {
                    if ((pos & 1) == par) {
                        const uint32_t w0 = mcol[(int64_t)(2 * kb) * x.Bp];
                        const uint32_t w1 = mcol[(int64_t)(2 * kb + 1) * x.Bp];
                        uint32_t v[32];
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            v[c] = pair_of(w0, c);
                            v[16 + c] = pair_of(w1, c);
                        }
                        if (!mbar_wait(su32(&bars->empty[stage]), phase ^ 1u, abort_flag, ctr, ERR_WAIT_MASK,
                                       wait_ns)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        tmem_st32(tmem_base + ((uint32_t)(quarter * 32) << 16) + A_COL0 + (uint32_t)stage * A_COLS, v);
                        fence_before();
                        mbar_arrive(su32(&bars->a_full[stage]));
                    }
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
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

cudaError_t launch_contract_tm(const Batch &b, const void *tmap_hi, const void *tmap_lo, int num_sms,
                               cudaStream_t s) {
    static unsigned long long smem_set = 0;   // one bit per device
    cudaError_t e = smem_limit_once((const void *)k_contract_tm, SMEM_BYTES, &smem_set);
    if (e != cudaSuccess) return e;
    int64_t grid = b.sched ? (int64_t)b.tc_grid : (int64_t)num_sms;
    if (grid > b.nunits_total) grid = b.nunits_total;
    if (grid < 1) return cudaSuccess;
    CUtensorMap th, tl;
    memcpy(&th, tmap_hi, sizeof(CUtensorMap));
    memcpy(&tl, tmap_lo, sizeof(CUtensorMap));
    k_contract_tm<<<(unsigned)grid, NUM_THREADS, SMEM_BYTES, s>>>(th, tl, b);
    return cudaGetLastError();
}

}  // namespace ept

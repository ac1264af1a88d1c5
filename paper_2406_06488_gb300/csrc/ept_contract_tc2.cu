// ept_contract_tc2.cu -- the permutation contraction on pairs of SMs (tcgen05
// cta_group::2): the same quadratic forms as ept_contract_tc.cu, Q_b = s_b' C s_b
// (Algorithm 1's permutation loop), with a work unit of (chunk q of K-blocks,
// relabeling tile m of 256 columns, the whole 256-row panel) shared by a cluster of
// two CTAs.
//
// Mapping (kind::f16, cta_group::2), M = 256 rows of C across the pair, N = 256
// relabelings, K = 64 pooled columns per stage:
//   A: each CTA loads its own 128 rows of the packed C block (FP16 hi and lo, TMA,
//     128-byte swizzle): CTA rank h holds rows 128 h .. 128 h + 127 of the panel;
//   B: each CTA expands its own half of the relabeling tile (rank h: relabelings
//     128 h .. 128 h + 127 of the tile) from the bit masks into its shared memory;
//   D: the leader CTA (rank 0) issues the MMAs for the pair; each CTA's tensor
//     memory receives its 128 rows x 256 relabelings, two accumulators (512 columns)
//     so that the epilogue of one unit overlaps the main loop of the next.
// Per CTA and K-block the MMAs read 64 KB of shared memory instead of 96 KB, and
// each CTA expands 128 instead of 256 relabelings, for the same multiply-adds.
//
// Synchronisation.  Each CTA's TMA copies and relabeling producers complete local
// barriers; in the peer CTA a forwarding thread waits for them and arrives on the
// leader's `peer_ready` barrier (cluster scope), so the leader's MMA issuer starts a
// stage when both halves are in place.  The MMA commits arrive on both CTAs'
// barriers (multicast): stage free, accumulator full.  Both CTAs' epilogues arrive
// on the leader's accumulator-empty barrier.  The epilogue of each CTA is that of
// ept_contract_tc.cu for its row half.  Every mbarrier wait is bounded (the abort
// protocol of ept_tc_common.cuh); the pair meets at cluster barriers after set-up
// and before it frees its tensor memory.
#include <cuda.h>
#include <cstdio>
#include <cstring>

#include "ept_internal.cuh"
#include "ept_tc_common.cuh"

namespace ept {

namespace {

using namespace tc;

constexpr int TC_M = 128;                         // rows of C per CTA
constexpr int TC_N = TC_TILE_N;                   // relabelings per unit (256)
constexpr int BH = TC_N / 2;                      // relabelings per CTA's half of the tile
constexpr int STAGES = 4;
constexpr int A_BYTES = TC_M * KB * 2;            // 16 KB (hi or lo)
constexpr int B_BYTES = BH * KB * 2;              // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + B_BYTES;   // A hi | A lo | B half
constexpr int RED_BYTES = 2 * 4 * TC_N * 4;       // epilogue sums: 2 buffers x 4 warps x 256 floats
constexpr int NUM_THREADS = 448;
constexpr int EPI_THREADS = 256;                  // warps 2-9
constexpr int PROD_THREADS = 128;                 // warps 10-13
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*barriers*/ + RED_BYTES + 1024 /*alignment*/;

constexpr unsigned long long ERR_WAIT_TMA = 0x201, ERR_WAIT_MMA = 0x202, ERR_WAIT_EPI = 0x203,
                             ERR_WAIT_MASK = 0x204, ERR_DRAIN = 0x205, ERR_WAIT_PEER = 0x206, ERR_INJECTED = 0x2FF;

constexpr uint32_t IDESC = idesc_f16_f32(2 * TC_M, TC_N);   // M = 256 across the pair

struct Bars {
    unsigned long long b_full[STAGES];       // local relabeling producers (128 arrivals)
    unsigned long long a_full[STAGES];       // local TMA copies (1 arrival + transaction bytes)
    unsigned long long peer_ready[STAGES];   // leader: the peer's stage is in place (1 remote arrival)
    unsigned long long empty[STAGES];        // both: the pair's MMAs of the stage are done (commit)
    unsigned long long acc_full[2];          // both: the pair's accumulator is complete (commit)
    unsigned long long acc_empty[2];         // leader: both epilogues have read it (2 x 256 arrivals)
    unsigned long long red;                  // local epilogue (256 arrivals per unit)
    unsigned long long drain;                // leader: every MMA issued is done (commit)
    uint32_t tmem_base;
    int abort_flag;
};
static_assert(sizeof(Bars) <= 512, "barriers overlap the nibble table");

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// arrive (release, cluster scope) on the barrier at the same offset in CTA `cta` of the cluster
__device__ __forceinline__ void mbar_arrive_cta(uint32_t bar, uint32_t cta) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(bar), "r"(cta));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(r) : "memory");
}

// one test of a phase with acquire at cluster scope (arrivals that come from the peer)
__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "n"(TRY_WAIT_NS)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                                  Counters *ctr, unsigned long long code, unsigned long long limit) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_cluster(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag) return false;
            const unsigned long long now = gtimer();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > limit) {
                *abort_flag = 1;
                atomicCAS(&ctr->err_code, 0ull, code);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mma2_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the commit arrives on the barrier at this offset in both CTAs of the pair
__device__ __forceinline__ void mma2_commit_both(uint32_t bar) {
    const uint16_t mask = 3;
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"(mask)
        : "memory");
}

// the commit arrives on the barrier at this offset in the leader CTA alone
__device__ __forceinline__ void mma2_commit_leader(uint32_t bar) {
    const uint16_t mask = 1;
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"(mask)
        : "memory");
}

// the test fields, chunk and relabeling tile of a pair unit, in registers: from the
// record of unit 2 pu (row half 0 of the single-CTA numbering), with the mask and
// partial offsets of the tile folded into mask0 and part0 (so q = m = 0)
struct Unit {
    Chunk ch;
    int64_t q, m, Bp, mask0, part0, blk0, NKB;
};

__device__ __forceinline__ UnitRec pair_record(const Batch &bt, int64_t pu, int64_t npu) {
    if (pu >= npu) return UnitRec{};
    if (bt.urec_pair) return bt.urec_pair[pu];
    const int64_t u = 2 * pu;
    const int t = find_test(bt.pre.units, bt.n_tests, u);
    const TestDesc &d = bt.desc[t];
    const int64_t lu = u - bt.pre.units[t];
    return unit_record(d, lu, bt.chunks[d.chunk0 + (lu >> 1) / d.MT]);
}

__device__ __forceinline__ Unit unit_of(const UnitRec &r) {
    Unit x;
    x.ch = Chunk{r.I, r.kb0, r.kb1, 0};
    x.q = 0;
    x.m = 0;
    x.Bp = r.Bp;
    x.mask0 = r.mask_col;
    x.part0 = r.out_off;
    x.blk0 = r.blk0;
    x.NKB = r.NKB;
    return x;
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_contract_tc2(const __grid_constant__ CUtensorMap tmap_hi, const __grid_constant__ CUtensorMap tmap_lo,
                   const Batch bt) {
    Counters *ctr = bt.ctr;
    const unsigned long long wait_ns = bt.wait_ns ? bt.wait_ns : WAIT_NS;
    const int64_t npu = bt.nunits_total / 2;   // pair units
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Bars *bars = reinterpret_cast<Bars *>(smem + STAGES * STAGE_BYTES);
    float *red = reinterpret_cast<float *>(smem + STAGES * STAGE_BYTES + 1024);
    volatile int *abort_flag = &bars->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();   // row half of the panel this CTA holds
    const bool leader = rank == 0;
    const int64_t pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;

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
            mbar_init(su32(&bars->peer_ready[s]), 1);
            mbar_init(su32(&bars->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(su32(&bars->acc_full[a]), 1);
            mbar_init(su32(&bars->acc_empty[a]), 2 * EPI_THREADS);
        }
        mbar_init(su32(&bars->red), EPI_THREADS);
        mbar_init(su32(&bars->drain), 1);
        bars->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         su32(&bars->tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    cluster_sync();   // both CTAs' barriers exist before any arrival from the peer
    fence_after();
    const uint32_t tmem_base = bars->tmem_base;

    if (warp == 0) {
        // ---------------- TMA: this CTA's 128 rows of the packed C block ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int armed[STAGES];
            for (int s2 = 0; s2 < STAGES; ++s2) armed[s2] = -1;
            bool ok = true;
            UnitRec nr = pair_record(bt, pair, npu);
            for (int64_t pu = pair; pu < npu && ok; pu += npairs) {
                const Unit x = unit_of(nr);
                nr = pair_record(bt, pu + npairs, npu);   // the next unit's record, read while this one runs
                const Chunk ch = x.ch;
                const int row = (int)rank * TC_M;
                for (int kb = ch.kb0; kb < ch.kb1; ++kb) {
                    if (!mbar_wait(su32(&bars->empty[stage]), phase ^ 1u, abort_flag, ctr, ERR_WAIT_TMA, wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t afull = su32(&bars->a_full[stage]);
                    mbar_arrive_tx(afull, 2 * A_BYTES);
                    const int blk = (int)(x.blk0 + blk_index(ch.I, kb, x.NKB));
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
        if (lane == 0 && leader) {
            // ---------------- MMA issuer for the pair ----------------
            int stage = 0, acc = 0;
            uint32_t phase = 0, acc_phase = 0;
            bool ok = true;
            if (bt.inject_stall && !flag_wait(&ctr->never_set, abort_flag, ctr, ERR_INJECTED, wait_ns)) ok = false;
            UnitRec nr = pair_record(bt, pair, npu);
            for (int64_t pu = pair; pu < npu && ok; pu += npairs) {
                const Unit x = unit_of(nr);
                nr = pair_record(bt, pu + npairs, npu);   // the next unit's record, read while this one runs
                const Chunk ch = x.ch;
                if (!mbar_wait_cluster(su32(&bars->acc_empty[acc]), acc_phase ^ 1u, abort_flag, ctr, ERR_WAIT_MMA,
                                       wait_ns)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * TC_N);
                bool first = true;
                for (int kb = ch.kb0; kb < ch.kb1; ++kb) {
                    if (!mbar_wait(su32(&bars->a_full[stage]), phase, abort_flag, ctr, ERR_WAIT_MMA, wait_ns) ||
                        !mbar_wait(su32(&bars->b_full[stage]), phase, abort_flag, ctr, ERR_WAIT_MMA, wait_ns) ||
                        !mbar_wait_cluster(su32(&bars->peer_ready[stage]), phase, abort_flag, ctr, ERR_WAIT_PEER,
                                           wait_ns)) {
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
                        mma2_f16(d_tmem, dhi + 2 * k, db + 2 * k, IDESC, (first && k == 0) ? 0u : 1u);
#pragma unroll
                    for (int k = 0; k < KB / 16; ++k) mma2_f16(d_tmem, dlo + 2 * k, db + 2 * k, IDESC, 1u);
                    mma2_commit_both(su32(&bars->empty[stage]));
                    first = false;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma2_commit_both(su32(&bars->acc_full[acc]));
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1u;
                }
            }
            mma2_commit_leader(su32(&bars->drain));
            unsigned long long t0 = gtimer();
            while (!mbar_try(su32(&bars->drain), 0)) {
                if (gtimer() - t0 > wait_ns) {
                    atomicCAS(&ctr->err_code, 0ull, ERR_DRAIN);
                    break;
                }
            }
        } else if (lane == 0) {
            // ---------------- the peer's stage-ready forwarder ----------------
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            UnitRec nr = pair_record(bt, pair, npu);
            for (int64_t pu = pair; pu < npu && ok; pu += npairs) {
                const Unit x = unit_of(nr);
                nr = pair_record(bt, pu + npairs, npu);   // the next unit's record, read while this one runs
                for (int kb = x.ch.kb0; kb < x.ch.kb1; ++kb) {
                    if (!mbar_wait(su32(&bars->a_full[stage]), phase, abort_flag, ctr, ERR_WAIT_PEER, wait_ns) ||
                        !mbar_wait(su32(&bars->b_full[stage]), phase, abort_flag, ctr, ERR_WAIT_PEER, wait_ns)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cta(su32(&bars->peer_ready[stage]), 0);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
    } else if (warp < 10) {
        // ---------------- epilogue: this CTA's row half ----------------
        const int quarter = warp & 3;
        const int g0 = ((warp - 2) >> 2) * 4;
        const int et = threadIdx.x - 64;
        int acc = 0;
        uint32_t acc_phase = 0, red_phase = 0;
        int rbuf = 0;
        UnitRec nr = pair_record(bt, pair, npu);
        for (int64_t pu = pair; pu < npu; pu += npairs) {
            const Unit x = unit_of(nr);
            nr = pair_record(bt, pu + npairs, npu);   // the next unit's record, read while this one runs
            const Chunk ch = x.ch;
            const int64_t Bp = x.Bp;
            const uint32_t *wrow =
                bt.maskT + x.mask0 + ((int64_t)ch.I * 8 + rank * 4 + quarter) * Bp + x.m * TC_N + g0 * 32;
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
            // the leader's accumulator is free once both CTAs' epilogues have read it
            if (leader) mbar_arrive(su32(&bars->acc_empty[acc]));
            else mbar_arrive_cta(su32(&bars->acc_empty[acc]), 0);
            mbar_arrive(su32(&bars->red));
            if (!mbar_wait(su32(&bars->red), red_phase, abort_flag, ctr, ERR_WAIT_EPI, wait_ns)) break;
            const float *rb = red + rbuf * 4 * TC_N;
            float *out = bt.partial + x.part0 + (2 * x.q + rank) * Bp + x.m * TC_N;
            out[et] = (rb[et] + rb[TC_N + et]) + (rb[2 * TC_N + et] + rb[3 * TC_N + et]);
            red_phase ^= 1u;
            rbuf ^= 1;
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
            }
        }
    } else {
        // ---------------- relabeling producers: this CTA's half of the tile ----------------
        const int r = threadIdx.x - 320;   // 0..127: row r of the half = relabeling 128 rank + r of the tile
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        UnitRec nr = pair_record(bt, pair, npu);
        for (int64_t pu = pair; pu < npu && ok; pu += npairs) {
            const Unit x = unit_of(nr);
            nr = pair_record(bt, pu + npairs, npu);   // the next unit's record, read while this one runs
            const Chunk ch = x.ch;
            const int64_t Bp = x.Bp;
            const uint32_t *maskT = bt.maskT + x.mask0 + x.m * TC_N + rank * BH + r;
            auto load2 = [&](int kb, uint2 &w) {
                const uint32_t *p0 = maskT + (int64_t)(2 * kb) * Bp;
                w.x = p0[0];
                w.y = p0[Bp];
            };
            uint2 cur = make_uint2(0, 0), nxt = make_uint2(0, 0);
            load2(ch.kb0, cur);
            if (ch.kb0 + 1 < ch.kb1) load2(ch.kb0 + 1, nxt);
            for (int kb = ch.kb0; kb < ch.kb1; ++kb) {
                uint2 nn = make_uint2(0, 0);
                if (kb + 2 < ch.kb1) load2(kb + 2, nn);
                if (!mbar_wait(su32(&bars->empty[stage]), phase ^ 1u, abort_flag, ctr, ERR_WAIT_MASK, wait_ns)) {
                    ok = false;
                    break;
                }
                uint8_t *brow = smem + stage * STAGE_BYTES + 2 * A_BYTES + r * 128;
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
    cluster_sync();   // no arrival from the peer is still on its way; the pair frees its tensor memory together
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
    }
}

}  // namespace

cudaError_t launch_contract_tc2(const Batch &b, const void *tmap_hi, const void *tmap_lo, int num_sms,
                                cudaStream_t s) {
    static unsigned long long smem_set = 0;   // one bit per device
    cudaError_t e = smem_limit_once((const void *)k_contract_tc2, SMEM_BYTES, &smem_set);
    if (e != cudaSuccess) return e;
    const int64_t npu = b.nunits_total / 2;
    int64_t pairs = num_sms / 2;
    if (pairs > npu) pairs = npu;
    if (pairs < 1) return cudaSuccess;
    CUtensorMap th, tl;
    memcpy(&th, tmap_hi, sizeof(CUtensorMap));
    memcpy(&tl, tmap_lo, sizeof(CUtensorMap));
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(2 * pairs));
    cfg.blockDim = dim3(NUM_THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_contract_tc2, th, tl, b);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace ept

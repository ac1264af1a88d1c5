// ept_contract_tc.cu -- the permutation contraction on 5th-generation tensor cores.
//
// What it computes (Algorithm 1, permutation loop, rewritten as quadratic forms):
// for relabeling column b with indicator s_b (s_b[t] = 1 iff pooled row t goes to
// x*), the statistic needs Q_b = s_b' C s_b, where C is the packed, centred,
// upper-scaled pooled matrix (see ept_kernels.cu, packing).  Work unit (q, m):
// chunk q = (panel I, K-blocks [kb0, kb1)), relabeling tile m (128 columns):
//     U[b, i]        = sum_{j in chunk} s_b[j] * C[i, j]        (tensor cores)
//     partial[q][b]  = sum_{i in panel I} s_b[i] * U[b, i]      (epilogue)
// and Q_b = sum_q partial[q][b] (FP64, ept_kernels.cu).
//
// Mapping onto tcgen05 (kind::f16, cta_group::1):
//   A (M = 128 relabelings x K = 64 pooled columns): 0/1 values, exact in BF16,
//     expanded from the bit masks by four producer warps straight into the
//     128-byte-swizzled K-major shared-memory layout;
//   B (N = 256 panel rows x K = 64): the packed C block, split C = hi + lo in BF16,
//     loaded by TMA (two 32 KB boxes per K-block);
//   D (128 x 256 FP32) in tensor memory: D += A * B_hi, then D += A * B_lo, so the
//     hi and lo products accumulate in one FP32 accumulator.
//   Two accumulators (512 TMEM columns) let the epilogue of one unit overlap the
//   main loop of the next.  The epilogue lane owns one relabeling: it reads its
//   256 columns, keeps those whose panel row is in x* for that relabeling, and sums.
//
// Roles (320 threads): warp 0 = TMA producer, warp 1 = MMA issuer (and TMEM
// owner), warps 2-5 = epilogue, warps 6-9 = relabeling-tile producers.  Every
// wait on an mbarrier is bounded (2 s); on expiry the kernel records an error
// code, raises a CTA-wide abort flag, drains its own copies and MMAs (bounded
// again), frees its tensor memory and returns.
#include <cuda.h>
#include <cstdio>
#include <cstring>

#include "ept_internal.cuh"
#include "ept_tc_common.cuh"

namespace ept {

namespace {

using namespace tc;

constexpr int TC_M = 128;
constexpr int TC_N = PANEL;                       // 256
constexpr int STAGES = 2;
constexpr int A_BYTES = TC_M * KB * 2;            // 16 KB
constexpr int B_BYTES = TC_N * KB * 2;            // 32 KB
constexpr int STAGE_BYTES = A_BYTES + 2 * B_BYTES;
constexpr int NUM_THREADS = 320;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*barriers*/ + 1024 /*alignment*/;

// error codes recorded in Counters::err_code
constexpr unsigned long long ERR_WAIT_TMA = 0x101, ERR_WAIT_MMA = 0x102, ERR_WAIT_EPI = 0x103,
                             ERR_WAIT_MASK = 0x104, ERR_DRAIN = 0x105;

// kind::f16 instruction descriptor with A = B = FP16 (format 0), D = FP32, K-major
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

struct Bars {
    unsigned long long a_full[STAGES];   // 128 producer-thread arrivals
    unsigned long long b_full[STAGES];   // 1 arrival + TMA transaction bytes
    unsigned long long empty[STAGES];    // 1 arrival (tcgen05.commit)
    unsigned long long acc_full[2];      // 1 arrival (tcgen05.commit)
    unsigned long long acc_empty[2];     // 128 epilogue-thread arrivals
    unsigned long long drain;            // 1 arrival (final tcgen05.commit)
    uint32_t tmem_base;
    int abort_flag;
};

// the test fields, chunk and relabeling tile of global work unit u, read once into
// registers (the asm statements' memory clobbers would otherwise force reloads)
struct Unit {
    Chunk ch;
    int64_t q, m, Bp, mask0, part0, blk0, NKB;
};

__device__ __forceinline__ Unit decode_unit(const Batch &bt, int64_t u) {
    const int t = find_test(bt.pre.units, bt.n_tests, u);
    const TestDesc *d = &bt.desc[t];
    Unit x;
    const int64_t lu = u - bt.pre.units[t];
    const int64_t MT = d->MT;
    x.q = lu / MT;
    x.m = lu % MT;
    x.Bp = d->Bp;
    x.mask0 = d->mask0;
    x.part0 = d->part0;
    x.blk0 = d->blk0;
    x.NKB = d->NKB;
    x.ch = bt.chunks[d->chunk0 + x.q];
    return x;
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_contract_tc(const __grid_constant__ CUtensorMap tmap_hi, const __grid_constant__ CUtensorMap tmap_lo,
                  const Batch bt) {
    Counters *ctr = bt.ctr;   // bounded-wait errors are recorded in test 0's counters
    const int64_t nunits = bt.nunits_total;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Bars *bars = reinterpret_cast<Bars *>(smem + STAGES * STAGE_BYTES);
    volatile int *abort_flag = &bars->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(su32(&bars->a_full[s]), 128);
            mbar_init(su32(&bars->b_full[s]), 1);
            mbar_init(su32(&bars->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(su32(&bars->acc_full[a]), 1);
            mbar_init(su32(&bars->acc_empty[a]), 128);
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
        // ---------------- TMA producer: packed C hi / lo blocks ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int armed[STAGES];   // parity of the last phase armed on each stage, -1 = none
            for (int s2 = 0; s2 < STAGES; ++s2) armed[s2] = -1;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                const Unit x = decode_unit(bt, u);
                const Chunk ch = x.ch;
                for (int kb = ch.kb0; kb < ch.kb1; ++kb) {
                    if (!mbar_wait(su32(&bars->empty[stage]), phase ^ 1u, abort_flag, ctr, ERR_WAIT_TMA)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bfull = su32(&bars->b_full[stage]);
                    mbar_arrive_tx(bfull, 2 * B_BYTES);
                    const int blk = (int)(x.blk0 + blk_index(ch.I, kb, x.NKB));
                    uint8_t *st = smem + stage * STAGE_BYTES;
                    tma_load_3d(su32(st + A_BYTES), &tmap_hi, 0, 0, blk, bfull);
                    tma_load_3d(su32(st + A_BYTES + B_BYTES), &tmap_lo, 0, 0, blk, bfull);
                    armed[stage] = (int)phase;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // drain: the copies armed last on each stage complete that phase of
                // b_full; wait for it (bounded) before the CTA may exit
                for (int s2 = 0; s2 < STAGES; ++s2) {
                    if (armed[s2] < 0) continue;
                    const unsigned long long t0 = gtimer();
                    while (!mbar_try(su32(&bars->b_full[s2]), (uint32_t)armed[s2])) {
                        if (gtimer() - t0 > WAIT_NS) {
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
            for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                const Chunk ch = decode_unit(bt, u).ch;
                if (!mbar_wait(su32(&bars->acc_empty[acc]), acc_phase ^ 1u, abort_flag, ctr, ERR_WAIT_MMA)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * TC_N);
                bool first = true;
                for (int kb = ch.kb0; kb < ch.kb1; ++kb) {
                    if (!mbar_wait(su32(&bars->a_full[stage]), phase, abort_flag, ctr, ERR_WAIT_MMA) ||
                        !mbar_wait(su32(&bars->b_full[stage]), phase, abort_flag, ctr, ERR_WAIT_MMA)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t sa = su32(smem + stage * STAGE_BYTES);
                    const uint64_t da = desc_sw128(sa);
                    const uint64_t dhi = desc_sw128(sa + A_BYTES);
                    const uint64_t dlo = desc_sw128(sa + A_BYTES + B_BYTES);
#pragma unroll
                    for (int k = 0; k < KB / 16; ++k)
                        mma_bf16(d_tmem, da + 2 * k, dhi + 2 * k, IDESC, (first && k == 0) ? 0u : 1u);
#pragma unroll
                    for (int k = 0; k < KB / 16; ++k) mma_bf16(d_tmem, da + 2 * k, dlo + 2 * k, IDESC, 1u);
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
                if (gtimer() - t0 > WAIT_NS) {
                    atomicCAS(&ctr->err_code, 0ull, ERR_DRAIN);
                    break;
                }
            }
        }
    } else if (warp < 6) {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3;           // TMEM lanes this warp may access
        const int row = quarter * 32 + lane;    // relabeling within the tile
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
            const Unit x = decode_unit(bt, u);
            const Chunk ch = x.ch;
            const int64_t Bp = x.Bp;
            const uint32_t *maskT = bt.maskT + x.mask0;
            const int64_t b = x.m * TC_M + row;
            uint32_t bits[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) bits[g] = maskT[((int64_t)ch.I * 8 + g) * Bp + b];
            if (!mbar_wait(su32(&bars->acc_full[acc]), acc_phase, abort_flag, ctr, ERR_WAIT_EPI)) break;
            fence_after();
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * TC_N);
#pragma unroll 1
            for (int g = 0; g < 8; ++g) {
                uint32_t v[32];
                tmem_ld32(tbase + (uint32_t)(g * 32), v);
                const uint32_t w = bits[g];
#pragma unroll
                for (int e = 0; e < 32; e += 4) {
                    s0 += ((w >> e) & 1u) ? __uint_as_float(v[e]) : 0.f;
                    s1 += ((w >> (e + 1)) & 1u) ? __uint_as_float(v[e + 1]) : 0.f;
                    s2 += ((w >> (e + 2)) & 1u) ? __uint_as_float(v[e + 2]) : 0.f;
                    s3 += ((w >> (e + 3)) & 1u) ? __uint_as_float(v[e + 3]) : 0.f;
                }
            }
            fence_before();
            mbar_arrive(su32(&bars->acc_empty[acc]));
            bt.partial[x.part0 + x.q * Bp + b] = (s0 + s1) + (s2 + s3);
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
            }
        }
    } else {
        // ---------------- relabeling-tile producers ----------------
        const int r = threadIdx.x - 192;   // 0..127: row of the A tile
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            const Unit x = decode_unit(bt, u);
            const Chunk ch = x.ch;
            const int64_t Bp = x.Bp;
            const uint32_t *maskT = bt.maskT + x.mask0;
            const int64_t b = x.m * TC_M + r;
            for (int kb = ch.kb0; kb < ch.kb1; ++kb) {
                const uint32_t w0 = maskT[(int64_t)(2 * kb) * Bp + b];
                const uint32_t w1 = maskT[(int64_t)(2 * kb + 1) * Bp + b];
                if (!mbar_wait(su32(&bars->empty[stage]), phase ^ 1u, abort_flag, ctr, ERR_WAIT_MASK)) {
                    ok = false;
                    break;
                }
                uint8_t *arow = smem + stage * STAGE_BYTES + r * 128;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint32_t byte = ((c < 4 ? w0 : w1) >> (8 * (c & 3))) & 0xFFu;
                    const uint4 v = expand8(byte);
                    const uint32_t dst = su32(arow + ((c ^ (r & 7)) << 4));
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(v.x), "r"(v.y),
                                 "r"(v.z), "r"(v.w)
                                 : "memory");
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(su32(&bars->a_full[stage]));
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
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int64_t grid = num_sms;
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
                        char *err, size_t errlen) {
    EncodeTiledFn enc = encode_fn(err, errlen);
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)KB, (cuuint64_t)PANEL, (cuuint64_t)nblk};
    const cuuint64_t strides[2] = {(cuuint64_t)KB * 2, (cuuint64_t)KB * 2 * PANEL};
    const cuuint32_t box[3] = {(cuuint32_t)KB, (cuuint32_t)PANEL, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    void *ptrs[2] = {(void *)Chi, (void *)Clo};
    void *outs[2] = {tmap_hi, tmap_lo};
    for (int k = 0; k < 2; ++k) {
        CUresult r = enc((CUtensorMap *)outs[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ptrs[k], dims,
                                            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            snprintf(err, errlen, "cuTensorMapEncodeTiled failed (%d)", (int)r);
            return false;
        }
    }
    return true;
}

}  // namespace ept

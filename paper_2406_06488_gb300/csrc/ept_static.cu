// ept_static.cu -- ept_test_static: the split-BF16 permutation test for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host application whose memory pool already
// owns all of the GPU's memory (a framework that reserves the device up front), or a
// latency-critical loop where an allocation -- which may synchronise the whole
// device and take unbounded time -- is not acceptable.  For them this entry point
// keeps all of its scratch in one file-scope device array of a fixed, modest size
// (EPT_STATIC_SCRATCH_BYTES), which every GPU that loads libept holds until the
// process exits.  The caller still provides the inputs and the output buffer.
//
// Host code cannot use the array's name as a device address (in host code it names
// a host-side stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress while that device is current, checked, cached, and passed
// to the kernels.  The first call on a device performs that set-up.
//
// Every call shares the one array and leaves its contents behind: the counters that
// must start at zero are cleared by each call, everything else is fully rewritten.
// Calls that overlap on the GPU (for instance from several processes, or threads
// driving different streams without ordering) race on the array; calls from this
// process are serialised by a mutex and each returns only after its work finished.
#include <cuda.h>
#include <cuda_runtime.h>

#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/ept.h"
#include "ept_internal.cuh"

namespace ept {

namespace {

__device__ __align__(256) uint8_t g_static_scratch[EPT_STATIC_SCRATCH_BYTES];

struct StaticDevice {
    bool ready = false;
    uint8_t *scratch = nullptr;   // device address of g_static_scratch on this device
    int num_sms = 0;
};

constexpr int MAX_DEVICES = 64;
StaticDevice g_static_dev[MAX_DEVICES];
std::mutex g_static_mu;

inline size_t up(size_t v) { return (v + 255) / 256 * 256; }

// Layout of one test's scratch inside the static array (byte offsets).
struct StaticPlan {
    size_t desc, pre, blk, chunks, norms, iscale, u, D, rowpart, colpart, r, Spart, dcorr, Upart, Stpart,
        maskT, partial, stats, observed, ctr, total;
};

StaticPlan static_plan(const TestDesc &d) {
    StaticPlan P;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = up(o + (bytes ? bytes : 1));
        return at;
    };
    const size_t elems = (size_t)d.nblk * PANEL * KB;
    P.desc = take(sizeof(TestDesc));
    P.pre = take(5 * 2 * sizeof(int64_t));
    P.blk = take((size_t)d.nblk * sizeof(BlkInfo));
    P.chunks = take((size_t)d.nchunks * sizeof(Chunk));
    P.norms = take((size_t)d.n_pad * 4);
    P.iscale = take((size_t)d.n_pad * 4);
    P.u = take((size_t)d.n_pad * 4);
    P.D = take(elems * 4);
    P.rowpart = take((size_t)d.nblk * PANEL * 8);
    P.colpart = take((size_t)d.nblk * KB * 8);
    P.r = take((size_t)d.n_pad * 8);
    P.Spart = take((size_t)(d.n_pad / 32) * 8);
    P.dcorr = take((size_t)d.n_pad * 8);
    P.Upart = take((size_t)d.NP * 8);
    P.Stpart = take((size_t)d.NP * 8);
    P.maskT = take((size_t)d.nw * d.Bp * 4);
    P.partial = take((size_t)d.nparts * d.Bp * 4);
    P.stats = take((size_t)d.ncols * 8);
    P.observed = take(8);
    P.ctr = take(sizeof(Counters));
    P.total = o;
    return P;
}

// Writes the test's descriptor, the prefix sums of a batch of one, the block table
// and the chunk table into the static array, on the device (no host staging).
__global__ void k_static_tables(const TestDesc d, TestDesc *desc, int64_t *pre, BlkInfo *blk, Chunk *chunks) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < d.nblk) {
        int I = 0;
        while (I + 1 < d.NP && blk_off(I + 1, d.NKB) <= b) ++I;
        blk[b] = BlkInfo{0, I, (int)(b - blk_off(I, d.NKB)) + KB_PER_PANEL * I, 0};
    }
    if (b == 0) {
        *desc = d;
        const int64_t tot[5] = {d.n_pad, d.NP, d.Bp, tc_units(d), d.nchunks * 2 * (d.Bp / 64)};
        for (int k = 0; k < 5; ++k) {
            pre[2 * k] = 0;
            pre[2 * k + 1] = tot[k];
        }
        // the chunk table of ept_test's planner (chunks end at the last K-block with real
        // columns), at the default unit length
        int64_t q = 0;
        for (int64_t I = 0; I < d.NP; ++I) {
            const int64_t nq = panel_chunks(d, I, CHUNK_KB_DEFAULT);
            for (int64_t k = 0; k < nq; ++k) chunks[q++] = panel_chunk(d, I, k, CHUNK_KB_DEFAULT);
        }
    }
}

ept_status err(ept_status st, const char *fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

#define SCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return err(EPT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

// Set-up of the calling thread's current device (first call on that device only).
ept_status static_setup(int dev, StaticDevice **out) {
    if (dev < 0 || dev >= MAX_DEVICES) return err(EPT_EUNSUPPORTED, "device %d out of range", dev);
    StaticDevice &d = g_static_dev[dev];
    if (!d.ready) {
        int major = 0, minor = 0, sms = 0;
        SCK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
        SCK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
        SCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (!(major == 10 && minor == 3))
            return err(EPT_EUNSUPPORTED, "device %d is sm_%d%d; libept is built for sm_103a only", dev, major, minor);
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || ptr == nullptr)
            return err(EPT_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        d.scratch = static_cast<uint8_t *>(ptr);
        d.num_sms = sms;
        d.ready = true;
    }
    *out = &d;
    return EPT_OK;
}

}  // namespace
}  // namespace ept

using namespace ept;

extern "C" ept_status ept_test_static(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p, int stat,
                                      double sigma, int64_t B, uint64_t seed, double *perm_stats, ept_result *out,
                                      void *stream) {
    const auto t_start = std::chrono::steady_clock::now();
    if (!X || !Y || !out) return err(EPT_EINVAL, "null X, Y or result pointer");
    if (nx < 1 || ny < 1 || p < 1) return err(EPT_EINVAL, "nx, ny and p must be >= 1");
    if (p > ((int64_t)1 << 30)) return err(EPT_EINVAL, "p exceeds 2^30");
    if (B < 0 || B > ((int64_t)1 << 31)) return err(EPT_EINVAL, "B must be in [0, 2^31]");
    if (nx + ny > ((int64_t)1 << 22)) return err(EPT_EINVAL, "nx + ny exceeds 2^22");
    if (stat != EPT_STAT_ED && stat != EPT_STAT_MMD_GAUSS && stat != EPT_STAT_MMD_LAPLACE)
        return err(EPT_EINVAL, "unknown statistic %d", stat);
    if (stat != EPT_STAT_ED && !(sigma > 0.0 && sigma < 1e300))
        return err(EPT_EINVAL, "MMD needs a finite bandwidth sigma > 0 (ept_test_static has no median heuristic)");
    // the test, described by ept_test's planner as a batch of one
    TestDesc d;
    describe_test(d, nx, ny, p, B, stat, sigma, seed, true);
    d.X = X;
    d.Y = Y;
    d.out_stats = perm_stats;
    for (int64_t I = 0; I < d.NP; ++I) d.nchunks += panel_chunks(d, I, CHUNK_KB_DEFAULT);
    d.nparts = 2 * d.nchunks;
    const StaticPlan P = static_plan(d);
    if (P.total > (size_t)EPT_STATIC_SCRATCH_BYTES)
        return err(EPT_EINVAL,
                   "this test needs %zu bytes of scratch; ept_test_static has %zu (EPT_STATIC_SCRATCH_BYTES): "
                   "use ept_test for larger tests",
                   P.total, (size_t)EPT_STATIC_SCRATCH_BYTES);

    std::lock_guard<std::mutex> lock(g_static_mu);
    int dev = 0;
    SCK(cudaGetDevice(&dev));
    StaticDevice *sd = nullptr;
    ept_status st = static_setup(dev, &sd);
    if (st != EPT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *A = sd->scratch;

    Batch b;
    memset(&b, 0, sizeof(b));
    b.n_tests = 1;
    b.desc = (const TestDesc *)(A + P.desc);
    int64_t *pre = (int64_t *)(A + P.pre);
    b.pre.rows = pre;
    b.pre.panels = pre + 2;
    b.pre.cols = pre + 4;
    b.pre.units = pre + 6;
    b.pre.simt = pre + 8;
    b.blk = (const BlkInfo *)(A + P.blk);
    b.chunks = (const Chunk *)(A + P.chunks);
    b.nblk_total = d.nblk;
    b.nrows_total = d.n_pad;
    b.npan_total = d.NP;
    b.ncols_total = d.Bp;
    b.nunits_total = tc_units(d);
    b.norms = (float *)(A + P.norms);
    b.iscale = (float *)(A + P.iscale);
    b.u = (float *)(A + P.u);
    b.D = (float *)(A + P.D);
    b.Chi = (uint16_t *)(A + P.D);   // the split parts are written over the blocks' FP32 storage
    b.Clo = b.Chi + (size_t)PANEL * KB;
    b.c_stride = 2 * (int64_t)PANEL * KB;
    b.rowpart = (double *)(A + P.rowpart);
    b.colpart = (double *)(A + P.colpart);
    b.r = (double *)(A + P.r);
    b.Spart = (double *)(A + P.Spart);
    b.dcorr = (double *)(A + P.dcorr);
    b.Upart = (double *)(A + P.Upart);
    b.Stpart = (double *)(A + P.Stpart);
    b.maskT = (uint32_t *)(A + P.maskT);
    b.partial = (float *)(A + P.partial);
    b.stats = (double *)(A + P.stats);
    b.observed = (double *)(A + P.observed);
    b.ctr = (Counters *)(A + P.ctr);

    SCK(cudaMemsetAsync(b.ctr, 0, sizeof(Counters), s));
    k_static_tables<<<(unsigned)((d.nblk + 255) / 256), 256, 0, s>>>(d, (TestDesc *)(A + P.desc), pre,
                                                                      (BlkInfo *)(A + P.blk), (Chunk *)(A + P.chunks));
    launch_norms(b, s);
    launch_build_simt(b, s);
    launch_blocksums(b, s);
    launch_rowsum_reduce(b, s);
    launch_center(b, s);
    launch_pack(b, true, s);
    launch_masks(b, sd->num_sms, DRAW_WARPS, s);
    SCK(cudaGetLastError());
    alignas(64) CUtensorMap th, tl;
    char emsg[160];
    if (!encode_block_tmaps(&th, &tl, b.Chi, b.Clo, d.nblk, b.c_stride, emsg, sizeof(emsg)))
        return err(EPT_ECUDA, "%s", emsg);
    SCK(launch_contract_tc(b, &th, &tl, sd->num_sms, s));
    launch_combine(b, s);
    SCK(cudaGetLastError());
    Counters h;
    double observed = 0.0;
    SCK(cudaMemcpyAsync(&h, b.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    SCK(cudaMemcpyAsync(&observed, b.observed, 8, cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    if (h.nonfinite) return err(EPT_EINVAL, "X or Y holds NaN or Inf");
    if (h.err_code)
        return err(EPT_ETIMEOUT, "device-side bounded wait gave up (code 0x%llx)", (unsigned long long)h.err_code);
    out->observed = observed;
    out->n_ge = (int64_t)h.n_ge;
    out->n_near_tie = (int64_t)h.n_near;
    out->n_fixup = (int64_t)h.n_fixup;
    out->p_value = (1.0 + (double)out->n_ge) / (1.0 + (double)B);
    out->ms_build = out->ms_perm = out->ms_masks = out->ms_contract = 0.0;
    out->sigma = (stat == EPT_STAT_ED) ? 0.0 : sigma;
    out->n_windows = 0;
    out->n_refined = 0;   // no FP64 refinement here (it needs scratch beyond the array)
    out->tuning = 0;
    out->tune_candidates = 0;
    out->refine_launches = 0;
    out->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return EPT_OK;
}

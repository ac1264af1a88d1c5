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

void set_last_error(const char *msg);  // ept_api.cu

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

inline size_t up(size_t v) { return (v + 1023) / 1024 * 1024; }

struct StaticPlan {
    size_t norms, blkinfo, chunks, D, rowpart, colpart, r, u, dcorr, sc, hi, lo, maskT, partial, stats, ctr, total;
    size_t Spart, Upart, Stpart;
};

StaticPlan static_plan(const Geom &g) {
    StaticPlan P;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = up(o + (bytes ? bytes : 1));
        return at;
    };
    const size_t elems = (size_t)g.nblk * PANEL * KB;
    P.norms = take((size_t)g.n_pad * 4);
    P.blkinfo = take((size_t)g.nblk * sizeof(int2));
    P.chunks = take((size_t)g.nchunks * sizeof(Chunk));
    P.D = take(elems * 4);
    P.rowpart = take((size_t)g.nblk * PANEL * 8);
    P.colpart = take((size_t)g.nblk * KB * 8);
    P.r = take((size_t)g.n_pad * 8);
    P.u = take((size_t)g.n_pad * 4);
    P.dcorr = take((size_t)g.n_pad * 8);
    P.sc = take(sizeof(StatConst));
    P.Spart = take((size_t)(g.n_pad / 32) * 8);
    P.Upart = take((size_t)g.NP * 8);
    P.Stpart = take((size_t)g.NP * 8);
    P.hi = take(elems * 2);
    P.lo = take(elems * 2);
    P.maskT = take((size_t)g.nw * g.Bp * 4);
    P.partial = take((size_t)g.nchunks * g.Bp * 4);
    P.stats = take((size_t)g.ncols * 8);
    P.ctr = take(sizeof(Counters));
    P.total = o;
    return P;
}

// The block table (stored block -> panel, K-block) and the chunk table, written on
// the device so that no host staging memory is needed.
__global__ void k_static_tables(int NP, int NKB, int64_t nblk, int2 *blk_info, Chunk *chunks) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nblk) {
        int I = 0;
        while (I + 1 < NP && blk_off(I + 1, NKB) <= b) ++I;
        blk_info[b] = make_int2(I, (int)(b - blk_off(I, NKB)) + KB_PER_PANEL * I);
    }
    if (b == 0) {
        int q = 0;
        for (int I = 0; I < NP; ++I)
            for (int kb = KB_PER_PANEL * I; kb < NKB; kb += CHUNK_KB) {
                Chunk ch;
                ch.I = I;
                ch.kb0 = kb;
                ch.kb1 = (kb + CHUNK_KB < NKB) ? kb + CHUNK_KB : NKB;
                ch.pad = 0;
                chunks[q++] = ch;
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
    if (B < 0 || B > ((int64_t)1 << 31)) return err(EPT_EINVAL, "B must be in [0, 2^31]");
    if (nx + ny > ((int64_t)1 << 22)) return err(EPT_EINVAL, "nx + ny exceeds 2^22");
    if (stat != EPT_STAT_ED && stat != EPT_STAT_MMD_GAUSS) return err(EPT_EINVAL, "unknown statistic %d", stat);
    if (stat == EPT_STAT_MMD_GAUSS && !(sigma > 0.0 && sigma < 1e300))
        return err(EPT_EINVAL, "MMD needs a finite bandwidth sigma > 0");
    const Geom g = make_geom(nx, ny, p, B + 1);
    const StaticPlan P = static_plan(g);
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

    Counters *ctr = (Counters *)(A + P.ctr);
    SCK(cudaMemsetAsync(ctr, 0, sizeof(Counters), s));
    int2 *blkinfo = (int2 *)(A + P.blkinfo);
    Chunk *chunks = (Chunk *)(A + P.chunks);
    k_static_tables<<<(unsigned)((g.nblk + 255) / 256), 256, 0, s>>>((int)g.NP, (int)g.NKB, g.nblk, blkinfo, chunks);
    float *norms = (float *)(A + P.norms);
    float *D = (float *)(A + P.D);
    launch_check_finite(X, nx * p, ctr, s);
    launch_check_finite(Y, ny * p, ctr, s);
    launch_norms(X, Y, g, norms, s);
    launch_build_simt(X, Y, norms, g, stat, sigma, 1.0 / 16.0, blkinfo, D, ctr, s);
    double *rowpart = (double *)(A + P.rowpart), *colpart = (double *)(A + P.colpart);
    double *r = (double *)(A + P.r), *dcorr = (double *)(A + P.dcorr);
    float *u = (float *)(A + P.u);
    StatConst *sc = (StatConst *)(A + P.sc);
    uint16_t *hi = (uint16_t *)(A + P.hi), *lo = (uint16_t *)(A + P.lo);
    double *Spart = (double *)(A + P.Spart), *Upart = (double *)(A + P.Upart), *Stpart = (double *)(A + P.Stpart);
    launch_blocksums(D, g, rowpart, colpart, s);
    launch_rowsum_reduce(rowpart, colpart, g, r, Spart, s);
    launch_center(r, Spart, g, u, dcorr, Upart, Stpart, sc, stat, s);
    launch_pack_bf16(D, u, dcorr, g, blkinfo, hi, lo, s);
    uint32_t *maskT = (uint32_t *)(A + P.maskT);
    launch_perm_masks(seed, (int)nx, (int)ny, 0, g.ncols, g.Bp, (int)g.nw, g.comp, maskT, s);
    SCK(cudaGetLastError());
    alignas(64) CUtensorMap th, tl;
    char emsg[160];
    if (!encode_block_tmaps(&th, &tl, hi, lo, g.nblk, emsg, sizeof(emsg))) return err(EPT_ECUDA, "%s", emsg);
    float *partial = (float *)(A + P.partial);
    SCK(launch_contract_tc(&th, &tl, maskT, chunks, g, partial, ctr, sd->num_sms, s));
    double *stats = (double *)(A + P.stats);
    launch_combine(partial, g.nchunks, g, sc, Stpart, stats, ctr, s);
    SCK(cudaGetLastError());
    if (perm_stats && B > 0)
        SCK(cudaMemcpyAsync(perm_stats, stats + 1, (size_t)B * 8, cudaMemcpyDeviceToDevice, s));
    Counters h;
    double observed = 0.0;
    SCK(cudaMemcpyAsync(&h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    SCK(cudaMemcpyAsync(&observed, stats, 8, cudaMemcpyDeviceToHost, s));
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
    out->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return EPT_OK;
}

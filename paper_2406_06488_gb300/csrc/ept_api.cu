// ept_api.cu -- host side of the libept C ABI (include/ept.h): contexts, device
// scratch, validation, and the order of the kernels of one permutation test.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/ept.h"
#include "ept_internal.cuh"

using namespace ept;

namespace {

thread_local std::string g_err = "no error";

ept_status fail(ept_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(EPT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device scratch layout of one test, as byte offsets into the context's arena.
struct Plan {
    Geom g;
    int prec;
    bool host_in;
    int64_t n_user_masks;
    size_t off_X, off_Y, off_norms, off_blkinfo, off_chunks, off_D, off_rowpart, off_colpart, off_r, off_u,
        off_dcorr, off_sc, off_hi, off_lo, off_maskT, off_umask, off_partial, off_stats, off_ctr, total;
    size_t off_zh, off_zl, off_tiles, off_Spart, off_Upart, off_Stpart, off_iscale;
    int64_t nparts, p_pad, ntiles;
};

Plan make_plan(const Geom &g, int prec, bool host_in, int64_t n_user_masks) {
    Plan P;
    P.g = g;
    P.prec = prec;
    P.host_in = host_in;
    P.n_user_masks = n_user_masks;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + std::max<size_t>(bytes, 1), 1024);
        return at;
    };
    const size_t blk_elems = (size_t)g.nblk * PANEL * KB;
    P.off_X = host_in ? take((size_t)g.nx * g.p * 4) : 0;
    P.off_Y = host_in ? take((size_t)g.ny * g.p * 4) : 0;
    P.off_norms = take((size_t)g.n_pad * 4);
    P.off_blkinfo = take((size_t)g.nblk * sizeof(int2));
    P.off_chunks = take((size_t)g.nchunks * sizeof(Chunk));
    P.off_D = take(blk_elems * 4);
    P.off_rowpart = take((size_t)g.nblk * PANEL * 8);
    P.off_colpart = take((size_t)g.nblk * KB * 8);
    P.off_r = take((size_t)g.n_pad * 8);
    P.off_u = take((size_t)g.n_pad * 4);
    P.off_dcorr = take((size_t)g.n_pad * 8);
    P.off_sc = take(sizeof(StatConst));
    P.off_Spart = take((size_t)(g.n_pad / 32) * 8);
    P.off_iscale = take((size_t)g.n_pad * 4);
    P.off_Upart = take((size_t)g.NP * 8);
    P.off_Stpart = take((size_t)g.NP * 8);
    P.p_pad = (g.p + BUILD_KB - 1) / BUILD_KB * BUILD_KB;
    P.ntiles = g.NP * (g.NP + 1);
    if (prec == EPT_PREC_SPLIT_BF16) {
        P.off_hi = take(blk_elems * 2);
        P.off_lo = take(blk_elems * 2);
        P.off_zh = take((size_t)g.n_pad * P.p_pad * 2);
        P.off_zl = take((size_t)g.n_pad * P.p_pad * 2);
        P.off_tiles = take((size_t)P.ntiles * sizeof(int4));
    } else {
        P.off_hi = P.off_lo = 0;
        P.off_zh = P.off_zl = P.off_tiles = 0;
    }
    P.off_maskT = take((size_t)g.nw * g.Bp * 4);
    const int64_t nwu = (g.n + 31) / 32;
    P.off_umask = (host_in && n_user_masks > 0) ? take((size_t)n_user_masks * nwu * 4) : 0;
    P.nparts = (prec == EPT_PREC_SPLIT_BF16) ? g.nchunks : 2 * g.nchunks;
    P.off_partial = take((size_t)P.nparts * g.Bp * 4);
    P.off_stats = take((size_t)g.ncols * 8);
    P.off_ctr = take(sizeof(Counters));
    P.total = o;
    return P;
}

}  // namespace

namespace ept {
// lets other translation units of the library report an error message
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace ept

struct ept_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;        // relabeling draws run here, beside the block build
    cudaEvent_t ev_side[3] = {};        // fork, draws start, draws done
    std::mutex mu;
    uint8_t *arena = nullptr;
    size_t arena_cap = 0;
    uint8_t *pinned = nullptr;
    size_t pinned_cap = 0;
    cudaEvent_t ev[7] = {};
    std::vector<int2> h_blkinfo;
    std::vector<Chunk> h_chunks;
    std::vector<int4> h_tiles;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

ept_status ensure_arena(ept_ctx *c, size_t bytes, cudaStream_t s) {
    if (c->budget && bytes > c->budget)
        return fail(EPT_ENOMEM, "test needs %zu bytes of device scratch, over the context budget of %zu", bytes,
                    c->budget);
    if (bytes <= c->arena_cap) return EPT_OK;
    CK(cudaStreamSynchronize(s));
    if (c->arena) {
        cudaFree(c->arena);
        c->arena = nullptr;
        c->arena_cap = 0;
    }
    const size_t cap = align_up(bytes + bytes / 8, 1 << 20);
    cudaError_t e = cudaMalloc(&c->arena, cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->arena = nullptr;
        return fail(EPT_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", cap, cudaGetErrorString(e));
    }
    c->arena_cap = cap;
    return EPT_OK;
}

ept_status ensure_pinned(ept_ctx *c, size_t bytes) {
    if (bytes <= c->pinned_cap) return EPT_OK;
    if (c->pinned) cudaFreeHost(c->pinned);
    c->pinned = nullptr;
    c->pinned_cap = 0;
    const size_t cap = align_up(bytes + bytes / 8, 1 << 20);
    cudaError_t e = cudaHostAlloc(&c->pinned, cap, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->pinned = nullptr;
        return fail(EPT_ENOMEM, "cudaHostAlloc(%zu bytes) failed: %s", cap, cudaGetErrorString(e));
    }
    c->pinned_cap = cap;
    return EPT_OK;
}

bool is_pinned_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// host -> device copy of `bytes` from `src`, through the pinned staging area at
// `stage` when src is pageable
ept_status h2d(void *dst, const void *src, size_t bytes, uint8_t *stage, cudaStream_t s) {
    if (bytes == 0) return EPT_OK;
    if (is_pinned_host(src)) {
        CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    } else {
        memcpy(stage, src, bytes);
        CK(cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyHostToDevice, s));
    }
    return EPT_OK;
}

ept_status validate(int64_t nx, int64_t ny, int64_t p, int stat, double sigma, int prec) {
    if (nx < 1 || ny < 1) return fail(EPT_EINVAL, "nx and ny must be >= 1 (got %lld, %lld)", (long long)nx, (long long)ny);
    if (p < 1) return fail(EPT_EINVAL, "p must be >= 1 (got %lld)", (long long)p);
    if (nx + ny > (int64_t)1 << 22) return fail(EPT_EINVAL, "nx + ny = %lld exceeds 2^22", (long long)(nx + ny));
    if (stat != EPT_STAT_ED && stat != EPT_STAT_MMD_GAUSS) return fail(EPT_EINVAL, "unknown statistic %d", stat);
    if (stat == EPT_STAT_MMD_GAUSS && !(sigma > 0.0 && std::isfinite(sigma)))
        return fail(EPT_EINVAL, "MMD needs a finite bandwidth sigma > 0");
    if (prec != EPT_PREC_PLAIN_FP32 && prec != EPT_PREC_SPLIT_BF16) return fail(EPT_EINVAL, "unknown precision %d", prec);
    return EPT_OK;
}

void fill_tables(ept_ctx *c, const Geom &g) {
    c->h_blkinfo.resize((size_t)g.nblk);
    c->h_chunks.clear();
    c->h_tiles.clear();
    for (int64_t I = 0; I < g.NP; ++I)
        for (int64_t J = I; J < g.NP; ++J)
            for (int h = 0; h < 2; ++h) c->h_tiles.push_back(make_int4((int)I, h, (int)J, 0));
    for (int64_t I = 0; I < g.NP; ++I) {
        for (int64_t kb = KB_PER_PANEL * I; kb < g.NKB; ++kb)
            c->h_blkinfo[(size_t)blk_index(I, kb, g.NKB)] = make_int2((int)I, (int)kb);
        for (int64_t kb = KB_PER_PANEL * I; kb < g.NKB; kb += CHUNK_KB) {
            Chunk ch;
            ch.I = (int)I;
            ch.kb0 = (int)kb;
            ch.kb1 = (int)std::min<int64_t>(kb + CHUNK_KB, g.NKB);
            ch.pad = 0;
            c->h_chunks.push_back(ch);
        }
    }
}

const double NEAR_DUP_TAU = 1.0 / 16.0;

// Phase 1: blocks, centring constants and the packed contraction operand.
ept_status run_blocks(ept_ctx *c, const Plan &P, const float *X, const float *Y, int stat, double sigma,
                      bool pack, cudaStream_t s) {
    const Geom &g = P.g;
    uint8_t *A = c->arena;
    float *norms = (float *)(A + P.off_norms);
    int2 *blkinfo = (int2 *)(A + P.off_blkinfo);
    float *D = (float *)(A + P.off_D);
    Counters *ctr = (Counters *)(A + P.off_ctr);
    if (P.prec == EPT_PREC_SPLIT_BF16) {
        uint16_t *zh = (uint16_t *)(A + P.off_zh), *zl = (uint16_t *)(A + P.off_zl);
        float *iscale = (float *)(A + P.off_iscale);
        launch_split_rows(X, Y, g, P.p_pad, zh, zl, norms, iscale, ctr, s);   // also counts non-finite inputs
        alignas(64) CUtensorMap tm[4];
        char emsg[160];
        if (!encode_rows_tmaps(tm, zh, zl, g.n_pad, P.p_pad, emsg, sizeof(emsg))) return fail(EPT_ECUDA, "%s", emsg);
        CK(launch_build_tc(tm, (const int4 *)(A + P.off_tiles), (int)P.ntiles, P.p_pad, norms, iscale, X, Y, g, stat,
                           sigma, NEAR_DUP_TAU, D, ctr, c->num_sms, s));
    } else {
        launch_check_finite(X, g.nx * g.p, ctr, s);
        launch_check_finite(Y, g.ny * g.p, ctr, s);
        launch_norms(X, Y, g, norms, s);
        launch_build_simt(X, Y, norms, g, stat, sigma, NEAR_DUP_TAU, blkinfo, D, ctr, s);
    }
    CK(cudaGetLastError());
    if (!pack) return EPT_OK;
    double *rowpart = (double *)(A + P.off_rowpart), *colpart = (double *)(A + P.off_colpart);
    double *r = (double *)(A + P.off_r), *dcorr = (double *)(A + P.off_dcorr);
    float *u = (float *)(A + P.off_u);
    StatConst *sc = (StatConst *)(A + P.off_sc);
    double *Spart = (double *)(A + P.off_Spart), *Upart = (double *)(A + P.off_Upart);
    double *Stpart = (double *)(A + P.off_Stpart);
    launch_blocksums(D, g, rowpart, colpart, s);
    launch_rowsum_reduce(rowpart, colpart, g, r, Spart, s);
    launch_center(r, Spart, g, u, dcorr, Upart, Stpart, sc, stat, s);
    if (P.prec == EPT_PREC_SPLIT_BF16)
        launch_pack_bf16(D, u, dcorr, g, blkinfo, (uint16_t *)(A + P.off_hi), (uint16_t *)(A + P.off_lo), s);
    else
        launch_pack_fp32(D, u, dcorr, g, blkinfo, D, s);
    CK(cudaGetLastError());
    return EPT_OK;
}

// The whole test.  user_masks == nullptr: draws 1..B of the stream of `seed`.
ept_status run_test(ept_ctx *c, const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p, int on_device,
                    int stat, double sigma, int64_t B, uint64_t seed, const uint32_t *user_masks, int prec,
                    double *perm_stats, ept_result *out, void *stream) {
    if (!c) return fail(EPT_EINVAL, "null context");
    if (!X || !Y || !out) return fail(EPT_EINVAL, "null X, Y or result pointer");
    if (B < 0) return fail(EPT_EINVAL, "B must be >= 0");
    if (B > ((int64_t)1 << 31)) return fail(EPT_EINVAL, "B exceeds 2^31");
    ept_status st = validate(nx, ny, p, stat, sigma, prec);
    if (st != EPT_OK) return st;
    std::lock_guard<std::mutex> lock(c->mu);
    DeviceGuard dg(c->device);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const Geom g = make_geom(nx, ny, p, B + 1);
    const bool host_in = !on_device;
    const Plan P = make_plan(g, prec, host_in, user_masks ? B : 0);
    if ((st = ensure_arena(c, P.total, s)) != EPT_OK) return st;
    fill_tables(c, g);
    const int64_t nwu = (g.n + 31) / 32;
    // pinned staging: tables + (host inputs) + results
    const size_t tab_bytes = align_up(c->h_blkinfo.size() * sizeof(int2), 256) +
                             align_up(c->h_chunks.size() * sizeof(Chunk), 256) +
                             align_up(c->h_tiles.size() * sizeof(int4), 256);
    const size_t xin = align_up((size_t)nx * p * 4, 256), yin = align_up((size_t)ny * p * 4, 256);
    const size_t in_bytes = host_in ? xin + yin + (user_masks ? align_up((size_t)B * nwu * 4, 256) : 0) : 0;
    const size_t res_bytes = align_up((size_t)g.ncols * 8, 256) + align_up(sizeof(Counters), 256);
    if ((st = ensure_pinned(c, tab_bytes + in_bytes + res_bytes)) != EPT_OK) return st;
    uint8_t *A = c->arena;
    uint8_t *pin = c->pinned;
    uint8_t *pin_tab = pin, *pin_in = pin + tab_bytes, *pin_res = pin + tab_bytes + in_bytes;

    CK(cudaEventRecord(c->ev[0], s));
    const float *dX = X, *dY = Y;
    const uint32_t *dmasks = user_masks;
    if (host_in) {
        float *xx = (float *)(A + P.off_X), *yy = (float *)(A + P.off_Y);
        if ((st = h2d(xx, X, (size_t)nx * p * 4, pin_in, s)) != EPT_OK) return st;
        if ((st = h2d(yy, Y, (size_t)ny * p * 4, pin_in + xin, s)) != EPT_OK) return st;
        dX = xx;
        dY = yy;
        if (user_masks && B > 0) {
            uint32_t *um = (uint32_t *)(A + P.off_umask);
            if ((st = h2d(um, user_masks, (size_t)B * nwu * 4, pin_in + xin + yin, s)) != EPT_OK) return st;
            dmasks = um;
        }
    }
    // tables
    memcpy(pin_tab, c->h_blkinfo.data(), c->h_blkinfo.size() * sizeof(int2));
    memcpy(pin_tab + align_up(c->h_blkinfo.size() * sizeof(int2), 256), c->h_chunks.data(),
           c->h_chunks.size() * sizeof(Chunk));
    CK(cudaMemcpyAsync(A + P.off_blkinfo, pin_tab, c->h_blkinfo.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(A + P.off_chunks, pin_tab + align_up(c->h_blkinfo.size() * sizeof(int2), 256),
                       c->h_chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice, s));
    if (prec == EPT_PREC_SPLIT_BF16) {
        uint8_t *tsrc = pin_tab + align_up(c->h_blkinfo.size() * sizeof(int2), 256) +
                        align_up(c->h_chunks.size() * sizeof(Chunk), 256);
        memcpy(tsrc, c->h_tiles.data(), c->h_tiles.size() * sizeof(int4));
        CK(cudaMemcpyAsync(A + P.off_tiles, tsrc, c->h_tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    }
    Counters *ctr = (Counters *)(A + P.off_ctr);
    CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), s));
    CK(cudaEventRecord(c->ev[1], s));

    // relabelings on the side stream, beside the block build: column 0 identity, then
    // draws 1..B or the caller's masks (they need only the uploads recorded in ev[1])
    cudaStream_t s2 = c->side;
    CK(cudaStreamWaitEvent(s2, c->ev[1], 0));
    CK(cudaEventRecord(c->ev_side[1], s2));
    uint32_t *maskT = (uint32_t *)(A + P.off_maskT);
    if (user_masks) {
        launch_perm_masks(seed, (int)nx, (int)ny, 0, 1, g.Bp, (int)g.nw, g.comp, maskT, s2);
        launch_user_masks(dmasks, B, (int)nwu, (int)nx, (int)g.n, g.Bp, (int)g.nw, g.comp, maskT, ctr, s2);
    } else {
        launch_perm_masks(seed, (int)nx, (int)ny, 0, g.ncols, g.Bp, (int)g.nw, g.comp, maskT, s2);
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(c->ev_side[2], s2));

    if ((st = run_blocks(c, P, dX, dY, stat, sigma, true, s)) != EPT_OK) return st;
    CK(cudaEventRecord(c->ev[2], s));
    CK(cudaStreamWaitEvent(s, c->ev_side[2], 0));
    CK(cudaEventRecord(c->ev[5], s));
    float *partial = (float *)(A + P.off_partial);
    const Chunk *chunks = (const Chunk *)(A + P.off_chunks);
    if (prec == EPT_PREC_SPLIT_BF16) {
        alignas(64) CUtensorMap th, tl;
        char emsg[160];
        if (!encode_block_tmaps(&th, &tl, (const uint16_t *)(A + P.off_hi), (const uint16_t *)(A + P.off_lo), g.nblk,
                                emsg, sizeof(emsg)))
            return fail(EPT_ECUDA, "%s", emsg);
        CK(launch_contract_tc(&th, &tl, maskT, chunks, g, partial, ctr, c->num_sms, s));
    } else {
        launch_contract_simt((const float *)(A + P.off_D), maskT, chunks, g, partial, s);
        CK(cudaGetLastError());
    }
    CK(cudaEventRecord(c->ev[6], s));
    double *stats = (double *)(A + P.off_stats);
    launch_combine(partial, P.nparts, g, (const StatConst *)(A + P.off_sc), (const double *)(A + P.off_Stpart), stats,
                   ctr, s);
    CK(cudaGetLastError());
    CK(cudaEventRecord(c->ev[3], s));

    double *h_stats = (double *)pin_res;
    Counters *h_ctr = (Counters *)(pin_res + align_up((size_t)g.ncols * 8, 256));
    CK(cudaMemcpyAsync(h_ctr, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    if (on_device) {
        CK(cudaMemcpyAsync(h_stats, stats, 8, cudaMemcpyDeviceToHost, s));
        if (perm_stats && B > 0)
            CK(cudaMemcpyAsync(perm_stats, stats + 1, (size_t)B * 8, cudaMemcpyDeviceToDevice, s));
    } else {
        CK(cudaMemcpyAsync(h_stats, stats, (size_t)g.ncols * 8, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaEventRecord(c->ev[4], s));
    CK(cudaStreamSynchronize(s));

    if (h_ctr->nonfinite) return fail(EPT_EINVAL, "X or Y holds NaN or Inf");
    if (h_ctr->bad_mask)
        return fail(EPT_EINVAL, "%llu relabeling(s) do not have exactly nx = %lld members among the n rows",
                    (unsigned long long)h_ctr->bad_mask, (long long)nx);
    if (h_ctr->err_code)
        return fail(EPT_ETIMEOUT, "device-side bounded wait gave up (code 0x%llx)", (unsigned long long)h_ctr->err_code);
    if (!on_device && perm_stats && B > 0) memcpy(perm_stats, h_stats + 1, (size_t)B * 8);
    out->observed = h_stats[0];
    out->n_ge = (int64_t)h_ctr->n_ge;
    out->n_near_tie = (int64_t)h_ctr->n_near;
    out->n_fixup = (int64_t)h_ctr->n_fixup;
    out->p_value = (1.0 + (double)out->n_ge) / (1.0 + (double)B);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]);
    out->ms_build = ms;
    cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);
    out->ms_perm = ms;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[4]);
    out->ms_total = ms;
    cudaEventElapsedTime(&ms, c->ev_side[1], c->ev_side[2]);
    out->ms_masks = ms;
    cudaEventElapsedTime(&ms, c->ev[5], c->ev[6]);
    out->ms_contract = ms;
    return EPT_OK;
}

}  // namespace

extern "C" {

int ept_abi_version(void) { return EPT_ABI_VERSION; }

const char *ept_last_error(void) { return g_err.c_str(); }

ept_status ept_create(ept_ctx **out, int device, size_t mem_budget_bytes) {
    if (!out) return fail(EPT_EINVAL, "null output pointer");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(EPT_EUNSUPPORTED, "no CUDA device");
    }
    if (device < 0 || device >= ndev) return fail(EPT_EINVAL, "device %d out of range (%d devices)", device, ndev);
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, device));
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(EPT_EUNSUPPORTED, "device %d is sm_%d%d; libept is built for sm_103a only", device, prop.major,
                    prop.minor);
    ept_ctx *c = new (std::nothrow) ept_ctx();
    if (!c) return fail(EPT_ENOMEM, "host allocation failed");
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    c->budget = mem_budget_bytes;
    DeviceGuard dg(device);
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    for (int k = 0; k < 7 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->ev[k]);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->ev_side[k]);
    if (e != cudaSuccess) {
        ept_destroy(c);
        return fail(EPT_ECUDA, "stream/event creation failed: %s", cudaGetErrorString(e));
    }
    *out = c;
    return EPT_OK;
}

ept_status ept_destroy(ept_ctx *c) {
    if (!c) return EPT_OK;
    {
        DeviceGuard dg(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        if (c->arena) cudaFree(c->arena);
        if (c->pinned) cudaFreeHost(c->pinned);
        for (int k = 0; k < 7; ++k)
            if (c->ev[k]) cudaEventDestroy(c->ev[k]);
        if (c->side) cudaStreamSynchronize(c->side);
        for (int k = 0; k < 3; ++k)
            if (c->ev_side[k]) cudaEventDestroy(c->ev_side[k]);
        if (c->side) cudaStreamDestroy(c->side);
        if (c->stream) cudaStreamDestroy(c->stream);
    }
    delete c;
    return EPT_OK;
}

size_t ept_estimate_bytes(int64_t nx, int64_t ny, int64_t p, int64_t B, int prec) {
    if (nx < 1 || ny < 1 || p < 1 || B < 0 || nx + ny > ((int64_t)1 << 22)) return 0;
    if (prec != EPT_PREC_PLAIN_FP32 && prec != EPT_PREC_SPLIT_BF16) return 0;
    const Geom g = make_geom(nx, ny, p, B + 1);
    return make_plan(g, prec, true, 0).total;
}

ept_status ept_test(ept_ctx *ctx, const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p, int on_device,
                    int stat, double sigma, int64_t B, uint64_t seed, int prec, double *perm_stats, ept_result *out,
                    void *stream) {
    return run_test(ctx, X, nx, Y, ny, p, on_device, stat, sigma, B, seed, nullptr, prec, perm_stats, out, stream);
}

ept_status ept_test_masks(ept_ctx *ctx, const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p,
                          int on_device, int stat, double sigma, const uint32_t *masks, int64_t n_masks, int prec,
                          double *perm_stats, ept_result *out, void *stream) {
    if (n_masks > 0 && !masks) return fail(EPT_EINVAL, "null masks");
    static const uint32_t dummy = 0;
    return run_test(ctx, X, nx, Y, ny, p, on_device, stat, sigma, n_masks, 0, masks ? masks : &dummy, prec,
                    perm_stats, out, stream);
}

ept_status ept_perm_masks(ept_ctx *c, uint64_t seed, int64_t nx, int64_t ny, int64_t b0, int64_t count,
                          uint32_t *out, int on_device, void *stream) {
    if (!c) return fail(EPT_EINVAL, "null context");
    if (nx < 1 || ny < 1 || nx + ny > ((int64_t)1 << 22)) return fail(EPT_EINVAL, "bad nx / ny");
    if (b0 < 0 || count < 0) return fail(EPT_EINVAL, "b0 and count must be >= 0");
    if (count == 0) return EPT_OK;
    if (!out) return fail(EPT_EINVAL, "null output");
    std::lock_guard<std::mutex> lock(c->mu);
    DeviceGuard dg(c->device);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const int64_t n = nx + ny;
    const int64_t nwu = (n + 31) / 32;
    const int64_t nw = (n + PANEL - 1) / PANEL * (PANEL / 32);
    const size_t bytesT = align_up((size_t)nw * count * 4, 1024);
    const size_t bytesR = (size_t)count * nwu * 4;
    ept_status st = ensure_arena(c, bytesT + bytesR, s);
    if (st != EPT_OK) return st;
    uint32_t *maskT = (uint32_t *)c->arena;
    uint32_t *rows = on_device ? out : (uint32_t *)(c->arena + bytesT);
    launch_perm_masks(seed, (int)nx, (int)ny, b0, count, count, (int)nw, false, maskT, s);
    launch_masks_to_rows(maskT, count, (int)nw, count, (int)nwu, rows, s);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpyAsync(out, rows, bytesR, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return EPT_OK;
}

ept_status ept_build_blocks(ept_ctx *c, const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p,
                            int on_device, int stat, double sigma, int prec, float *D_out, void *stream) {
    if (!c) return fail(EPT_EINVAL, "null context");
    if (!X || !Y || !D_out) return fail(EPT_EINVAL, "null pointer");
    ept_status st = validate(nx, ny, p, stat, sigma, prec);
    if (st != EPT_OK) return st;
    std::lock_guard<std::mutex> lock(c->mu);
    DeviceGuard dg(c->device);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const Geom g = make_geom(nx, ny, p, 1);
    const bool host_in = !on_device;
    const Plan P = make_plan(g, prec, host_in, 0);
    const size_t out_bytes = (size_t)g.n * g.n * 4;
    const size_t total = P.total + (on_device ? 0 : align_up(out_bytes, 1024));
    if ((st = ensure_arena(c, total, s)) != EPT_OK) return st;
    fill_tables(c, g);
    const size_t tab_bytes = align_up(c->h_blkinfo.size() * sizeof(int2), 256) +
                             align_up(c->h_tiles.size() * sizeof(int4), 256);
    const size_t xin = align_up((size_t)nx * p * 4, 256);
    const size_t in_bytes = host_in ? xin + align_up((size_t)ny * p * 4, 256) : 0;
    if ((st = ensure_pinned(c, tab_bytes + in_bytes + 256)) != EPT_OK) return st;
    uint8_t *A = c->arena;
    const float *dX = X, *dY = Y;
    if (host_in) {
        float *xx = (float *)(A + P.off_X), *yy = (float *)(A + P.off_Y);
        if ((st = h2d(xx, X, (size_t)nx * p * 4, c->pinned + tab_bytes, s)) != EPT_OK) return st;
        if ((st = h2d(yy, Y, (size_t)ny * p * 4, c->pinned + tab_bytes + xin, s)) != EPT_OK) return st;
        dX = xx;
        dY = yy;
    }
    memcpy(c->pinned, c->h_blkinfo.data(), c->h_blkinfo.size() * sizeof(int2));
    CK(cudaMemcpyAsync(A + P.off_blkinfo, c->pinned, c->h_blkinfo.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    if (prec == EPT_PREC_SPLIT_BF16) {
        uint8_t *tsrc = c->pinned + align_up(c->h_blkinfo.size() * sizeof(int2), 256);
        memcpy(tsrc, c->h_tiles.data(), c->h_tiles.size() * sizeof(int4));
        CK(cudaMemcpyAsync(A + P.off_tiles, tsrc, c->h_tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    }
    Counters *ctr = (Counters *)(A + P.off_ctr);
    CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), s));
    if ((st = run_blocks(c, P, dX, dY, stat, sigma, false, s)) != EPT_OK) return st;
    float *dout = on_device ? D_out : (float *)(A + P.total);
    launch_expand_blocks((const float *)(A + P.off_D), g, dout, s);
    CK(cudaGetLastError());
    Counters h;
    CK(cudaMemcpyAsync(&h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    if (!on_device) CK(cudaMemcpyAsync(D_out, dout, out_bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h.nonfinite) return fail(EPT_EINVAL, "X or Y holds NaN or Inf");
    return EPT_OK;
}

}  // extern "C"

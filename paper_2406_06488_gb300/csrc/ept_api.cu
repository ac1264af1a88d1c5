// ept_api.cu -- host side of the libept C ABI (include/ept.h): contexts, device
// scratch, validation, batch planning, the order of the kernels of a batched run,
// CUDA-graph replay of repeated batches, and the contraction-chunk autotuner.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <nvtx3/nvToolsExt.h>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
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

// pairs with d^2 < tau (||x||^2 + ||y||^2) are recomputed directly in FP64: the norm
// expansion amplifies rounding by at most 1/tau on the pairs it keeps
const double NEAR_DUP_TAU = 1.0 / 4.0;
// relabeling masks above this size (a quarter of the L2) change the contraction's unit order
const int64_t MASKS_IN_L2_BYTES = (int64_t)32 << 20;

// Host description of one test of a batch.
struct TestSpec {
    const float *X, *Y;
    int64_t nx, ny, p, B;
    int stat;
    double sigma;
    uint64_t seed;
    int64_t b0 = 1;               // first draw of the stream (column 1)
    const uint32_t *user_masks;   // B relabelings (ept_test_masks), same memory space as X
    double *perm_stats;           // B doubles or null, same memory space as X
};

// The tunable parameters of a run: contraction unit length in K-blocks, the
// relabeling-draw kernel (0 automatic, DRAW_WARPS, DRAW_LANES, DRAW_SCAN) and the order of the
// contraction schedule's units (0 automatic, 1 by length, 2 by first K-block, then
// length).  Every choice computes the same statistics bit for bit except the unit
// length, which changes the FP32 accumulation order (every length offered keeps the
// error criterion's calibration, at most 8 K-blocks unless EPT_OPT_MAX_CHUNK allows more).
struct Tuning {
    int chunk_kb = CHUNK_KB_DEFAULT, draw_mode = 0, order = 0;
    int kernel = 0;   // tensor-core contraction kernel (1..3; 0: the context's choice)
    int64_t code() const { return (int64_t)kernel * 10000 + (int64_t)chunk_kb * 100 + draw_mode * 10 + order; }
};

ept_status validate(int64_t nx, int64_t ny, int64_t p, int stat, double sigma, int prec, bool single = false) {
    if (nx < 1 || ny < 1) return fail(EPT_EINVAL, "nx and ny must be >= 1 (got %lld, %lld)", (long long)nx, (long long)ny);
    if (p < 1 || p > ((int64_t)1 << 30)) return fail(EPT_EINVAL, "p must be in [1, 2^30] (got %lld)", (long long)p);
    if (nx + ny > (int64_t)1 << 22) return fail(EPT_EINVAL, "nx + ny = %lld exceeds 2^22", (long long)(nx + ny));
    if (stat != EPT_STAT_ED && stat != EPT_STAT_MMD_GAUSS && stat != EPT_STAT_MMD_LAPLACE)
        return fail(EPT_EINVAL, "unknown statistic %d", stat);
    if (stat != EPT_STAT_ED && sigma != EPT_SIGMA_MEDIAN && !(sigma > 0.0 && std::isfinite(sigma)))
        return fail(EPT_EINVAL, "MMD needs a finite bandwidth sigma > 0 or EPT_SIGMA_MEDIAN");
    if (prec == EPT_PREC_POOLED_FP32) {
        if (!single) return fail(EPT_EUNSUPPORTED, "the pre-computation baseline runs single tests only");
        if (stat != EPT_STAT_ED && sigma == EPT_SIGMA_MEDIAN)
            return fail(EPT_EUNSUPPORTED, "the pre-computation baseline needs a given sigma");
        return EPT_OK;
    }
    if (prec != EPT_PREC_PLAIN_FP32 && prec != EPT_PREC_SPLIT_BF16) return fail(EPT_EINVAL, "unknown precision %d", prec);
    return EPT_OK;
}

// Geometry, offsets, tables and device-scratch layout of one batched run.
struct Plan {
    int n_tests = 0;
    int prec = 0;
    bool host_in = false;
    std::vector<TestDesc> desc;
    std::vector<int64_t> pre_rows, pre_panels, pre_cols, pre_units, pre_simt;
    std::vector<BlkInfo> blk;
    std::vector<Tile> tiles;
    std::vector<Chunk> chunks;
    std::vector<int64_t> sched, sched_off;   // contraction schedule: units of CTA c = sched[sched_off[c] ..)
    std::vector<UnitRec> urec;               // the scheduled units' records, in schedule order
    std::vector<UnitRec> urec_pair;          // pair contraction (kernel 2): the record of unit 2 pu for pair unit pu
    uint64_t serial = 0;                     // distinct for every plan_batch (the records are uploaded once per plan)
    bool user_masks = false;                 // some test brings its own relabelings
    int draw_mode = 0;                       // relabeling-draw kernel of the run (0: the context's choice)
    int contraction = 0;                     // tensor-core contraction kernel of the run (0: the context's choice)
    bool any_median = false;                 // some test takes its bandwidth from the median heuristic
    bool debug = false;                      // guard bands around the scratch regions
    GuardList guards{};
    size_t off_sel_hist = 0;
    int tc_grid = 0;                         // contraction CTAs
    std::vector<size_t> in_off;       // per test: byte offset of its X (then Y, then masks) in the input region
    int64_t nrows = 0, npan = 0, ncols_pad = 0, nunits = 0, nsimt = 0, nblk = 0, nmask = 0, nchunk = 0, npart = 0,
            nstats = 0, p_stride = 0;
    size_t in_bytes = 0;              // host inputs copied into the arena
    // byte offsets in the arena; the first tab_bytes are the uploaded tables
    size_t off_desc, off_pre_rows, off_pre_panels, off_pre_cols, off_pre_units, off_pre_simt, off_blk, off_tiles,
        off_chunks, off_sched, off_sched_off, off_urec, off_urec_pair, tab_bytes;
    size_t off_in, off_norms, off_iscale, off_u, off_Zh, off_Zl, off_D, off_Chi, off_rowpart, off_colpart,
        off_r, off_Spart, off_dcorr, off_Upart, off_Stpart, off_maskT, off_partial, off_stats, off_observed, off_ctr,
        total;
    size_t off_errest = 0, off_flags = 0;   // error estimates and refinement flags (0: none)
    // streaming mode (one test, windows of row panels): per window its panels
    // [I0, I1), its first stored block and block count, its build tiles, the test's
    // descriptor seen through the window and its contraction units; the window's
    // capacity in blocks and partial floats
    bool stream = false;
    std::vector<TestDesc> gdesc;
    std::vector<int64_t> gI0, gI1, gblk0, gnblk, gtile0, gntile, gpre;
    int64_t win_blk = 0, win_part = 0;
    size_t off_gdesc = 0, off_gpre = 0, off_sacc = 0;
};

// The fields of a test's descriptor that do not depend on its shape (statistic,
// bandwidth, seed); a cached plan is refreshed with them on every run.
void set_params(TestDesc &d, int stat, double sigma, uint64_t seed) {
    d.stat = stat;
    d.seed = seed;
    d.median = (stat != EPT_STAT_ED && sigma == EPT_SIGMA_MEDIAN) ? 1 : 0;
    // the build writes kernel values directly unless the bandwidth is still unknown
    d.kern = (stat == EPT_STAT_ED || d.median) ? 0 : stat;
    d.neg_inv_2s2 = (d.kern == EPT_STAT_MMD_GAUSS) ? (float)(-1.0 / (2.0 * sigma * sigma)) : 0.f;
    d.inv_sigma = (d.kern == EPT_STAT_MMD_LAPLACE) ? (float)(1.0 / sigma) : 0.f;
    d.sign = (stat == EPT_STAT_ED) ? -1.0 : 1.0;
    d.sigma64 = (stat != EPT_STAT_ED && !d.median) ? sigma : 0.0;
}

void set_test_params(TestDesc &d, const TestSpec &s) {
    set_params(d, s.stat, s.sigma, s.seed);
    d.b0 = s.b0;
}

// Static schedule of the tensor-core contraction: units sorted by length (K-blocks,
// longest first; stable, so that the units of one chunk stay together), then dealt
// to the CTAs in snake order, which balances the CTAs' total work far better than a
// plain stride when each CTA gets few units.  The CTAs take their units round by
// round, so the units in flight together are neighbours in this order and share
// their chunk's operand blocks in L2.  When a test's relabeling masks outgrow a
// quarter of L2 (n above about 25,000 at B = 10^4), units of equal length are also
// ordered by the first K-block of their chunk, so that the units in flight share
// the mask words of nearby K-ranges across panels (in panel order every panel
// sweeps all of the masks: measured at n = 60,000, 22.8 GB of DRAM reads for 7.3 GB
// of operand, 18.6 GB in K-block order; the smaller bench shapes are unchanged).
// order: 0 automatic (by first K-block only when the masks outgrow a quarter of L2),
// 1 by length alone, 2 by first K-block, then length.
void plan_schedule(Plan &P, int num_sms, int unit_order = 0) {
    P.sched.clear();
    P.sched_off.clear();
    P.urec.clear();
    P.tc_grid = 0;
    if (P.nunits <= 0) return;
    const int64_t G = std::min<int64_t>(std::max(num_sms, 1), P.nunits);
    P.tc_grid = (int)G;
    // unit lengths and first K-blocks
    std::vector<int> len((size_t)P.nunits), kb((size_t)P.nunits);
    int maxlen = 0, maxkb = 0;
    for (int t = 0; t < P.n_tests; ++t) {
        const TestDesc &d = P.desc[t];
        const int64_t u0 = P.pre_units[t], nu = P.pre_units[t + 1] - u0;
        for (int64_t lu = 0; lu < nu; ++lu) {
            const Chunk &ch = P.chunks[(size_t)(d.chunk0 + (lu >> 1) / d.MT)];
            int l = ch.kb1 - ch.kb0;
            if ((lu & 1) && ch.kb0 == KB_PER_PANEL * ch.I && l > 2) l -= 2;   // zero blocks the kernel skips
            len[(size_t)(u0 + lu)] = l;
            kb[(size_t)(u0 + lu)] = ch.kb0;
            maxlen = std::max(maxlen, l);
            maxkb = std::max(maxkb, ch.kb0);
        }
    }
    // counting sorts (stable): by first K-block when the masks are large, then by
    // length, longest first
    bool big_masks = false;
    for (const TestDesc &d : P.desc) big_masks |= d.nw * d.Bp * 4 > MASKS_IN_L2_BYTES;
    if (unit_order != 0) big_masks = unit_order == 2;
    std::vector<int64_t> by_kb((size_t)P.nunits);
    if (!big_masks) {
        for (int64_t u = 0; u < P.nunits; ++u) by_kb[(size_t)u] = u;
    } else {
        std::vector<int64_t> start((size_t)maxkb + 2, 0);
        for (int64_t u = 0; u < P.nunits; ++u) start[(size_t)kb[(size_t)u] + 1]++;
        for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
        for (int64_t u = 0; u < P.nunits; ++u) by_kb[(size_t)start[(size_t)kb[(size_t)u]]++] = u;
    }
    std::vector<int64_t> start((size_t)maxlen + 2, 0);
    for (int64_t u = 0; u < P.nunits; ++u) start[(size_t)(maxlen - len[(size_t)u]) + 1]++;
    for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
    std::vector<int64_t> order((size_t)P.nunits);
    for (int64_t u : by_kb) order[(size_t)start[(size_t)(maxlen - len[(size_t)u])]++] = u;
    // snake deal: position k goes to CTA (k % G) on even rounds, G - 1 - (k % G) on odd ones
    auto cta_of = [G](int64_t k) {
        const int64_t r = k / G, c = k % G;
        return (r & 1) ? G - 1 - c : c;
    };
    P.sched_off.assign((size_t)G + 1, 0);
    for (int64_t k = 0; k < P.nunits; ++k) P.sched_off[(size_t)cta_of(k) + 1]++;
    for (int64_t c = 0; c < G; ++c) P.sched_off[(size_t)c + 1] += P.sched_off[(size_t)c];
    std::vector<int64_t> fill(P.sched_off.begin(), P.sched_off.end() - 1);
    P.sched.resize((size_t)P.nunits);
    for (int64_t k = 0; k < P.nunits; ++k) P.sched[(size_t)fill[(size_t)cta_of(k)]++] = order[(size_t)k];
    // the records of the scheduled units, in schedule order
    P.urec.resize((size_t)P.nunits);
    for (int64_t k = 0; k < P.nunits; ++k) {
        const int64_t u = P.sched[(size_t)k];
        const int t = (int)(std::upper_bound(P.pre_units.begin(), P.pre_units.end(), u) - P.pre_units.begin()) - 1;
        const TestDesc &d = P.desc[t];
        const int64_t lu = u - P.pre_units[t];
        P.urec[(size_t)k] = unit_record(d, lu, P.chunks[(size_t)(d.chunk0 + (lu >> 1) / d.MT)]);
    }
}

void plan_batch(Plan &P, const std::vector<TestSpec> &specs, int prec, bool host_in, int chunk_kb,
                int num_sms = 160, bool debug = false, bool schedule = true, int order = 0, bool pair_records = false) {
    P = Plan();
    static std::atomic<uint64_t> plans{0};
    P.serial = ++plans;
    P.debug = debug;
    P.n_tests = (int)specs.size();
    P.prec = prec;
    P.host_in = host_in;
    const bool tc = prec == EPT_PREC_SPLIT_BF16;
    auto push_pre = [](std::vector<int64_t> &v, int64_t add) { v.push_back(v.back() + add); };
    P.pre_rows = P.pre_panels = P.pre_cols = P.pre_units = P.pre_simt = std::vector<int64_t>(1, 0);
    size_t in_bytes = 0;
    for (int t = 0; t < P.n_tests; ++t) {
        const TestSpec &s = specs[t];
        TestDesc d;
        describe_test(d, s.nx, s.ny, s.p, s.B, s.stat, s.sigma, s.seed, tc);
        d.b0 = s.b0;
        d.ka = refine_ka(chunk_kb);
        d.row0 = P.nrows;
        d.blk0 = P.nblk;
        d.pan0 = P.npan;
        d.sp0 = P.nrows / 32;
        d.mask0 = P.nmask;
        d.chunk0 = P.nchunk;
        d.col0 = P.nstats;
        for (int64_t I = 0; I < d.NP; ++I) {
            for (int64_t kb = KB_PER_PANEL * I; kb < d.NKB; ++kb) P.blk.push_back(BlkInfo{t, (int)I, (int)kb, 0});
            const int64_t nq = panel_chunks(d, I, chunk_kb);
            for (int64_t q = 0; q < nq; ++q) P.chunks.push_back(panel_chunk(d, I, q, chunk_kb));
            if (tc)
                for (int64_t J = I; J < d.NP; ++J)
                    for (int h = 0; h < 2; ++h) P.tiles.push_back(Tile{t, (int)I, (int)J, h});
        }
        d.nchunks = (int64_t)P.chunks.size() - d.chunk0;
        d.nparts = 2 * d.nchunks;   // (chunk, row half)
        d.part0 = P.npart;
        P.nrows += d.n_pad;
        P.nblk += d.nblk;
        P.npan += d.NP;
        P.nmask += d.nw * d.Bp;
        P.nchunk += d.nchunks;
        P.npart += d.nparts * d.Bp;
        P.nstats += d.ncols;
        P.p_stride = std::max(P.p_stride, d.p_pad);
        push_pre(P.pre_rows, d.n_pad);
        push_pre(P.pre_panels, d.NP);
        push_pre(P.pre_cols, d.Bp);
        push_pre(P.pre_units, tc_units(d));
        push_pre(P.pre_simt, d.nchunks * 2 * (d.Bp / 64));
        P.user_masks |= s.user_masks != nullptr;
        P.any_median |= d.median != 0;
        P.in_off.push_back(in_bytes);
        if (host_in) {
            in_bytes += align_up((size_t)d.nx * d.p * 4, 256) + align_up((size_t)d.ny * d.p * 4, 256);
            if (s.user_masks) in_bytes += align_up((size_t)s.B * d.nwu * 4, 256);
        }
        P.desc.push_back(d);
    }
    P.ncols_pad = P.pre_cols.back();
    P.nunits = P.pre_units.back();
    if (tc && schedule) plan_schedule(P, num_sms, order);
    if (tc && pair_records) {   // the pair kernel takes pair units in order (unit 2 pu: row half 0)
        P.urec_pair.resize((size_t)(P.nunits / 2));
        for (int64_t pu = 0; pu < P.nunits / 2; ++pu) {
            const int64_t u = 2 * pu;
            const int t = (int)(std::upper_bound(P.pre_units.begin(), P.pre_units.end(), u) - P.pre_units.begin()) - 1;
            const TestDesc &d = P.desc[t];
            const int64_t lu = u - P.pre_units[t];
            P.urec_pair[(size_t)pu] = unit_record(d, lu, P.chunks[(size_t)(d.chunk0 + (lu >> 1) / d.MT)]);
        }
    }
    P.nsimt = P.pre_simt.back();
    P.in_bytes = in_bytes;

    size_t o = 0;
    bool in_data = false;   // guard bands follow the data regions (the tables are uploaded whole)
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + std::max<size_t>(bytes, 1), 256);
        if (P.debug && in_data && P.guards.n < MAX_GUARDS) {
            P.guards.off[P.guards.n++] = o;
            o += GUARD_BYTES;
        }
        return at;
    };
    const size_t nt1 = (size_t)P.n_tests + 1;
    P.off_desc = take(sizeof(TestDesc) * P.n_tests);
    P.off_pre_rows = take(8 * nt1);
    P.off_pre_panels = take(8 * nt1);
    P.off_pre_cols = take(8 * nt1);
    P.off_pre_units = take(8 * nt1);
    P.off_pre_simt = take(8 * nt1);
    P.off_blk = take(sizeof(BlkInfo) * P.blk.size());
    P.off_tiles = take(sizeof(Tile) * P.tiles.size());
    P.off_chunks = take(sizeof(Chunk) * P.chunks.size());
    P.off_sched = take(8 * P.sched.size());
    P.off_sched_off = take(8 * P.sched_off.size());
    P.tab_bytes = o;
    o = align_up(o, 1024);
    in_data = true;
    // the unit records: uploaded with the first run of the plan, not with every run
    P.off_urec = take(sizeof(UnitRec) * P.urec.size());
    P.off_urec_pair = take(sizeof(UnitRec) * P.urec_pair.size());
    if (P.debug) {   // a band right after the tables as well
        P.guards.off[P.guards.n++] = o;
        o += GUARD_BYTES;
    }
    const size_t elems = (size_t)P.nblk * PANEL * KB;
    P.off_in = take(P.in_bytes);
    P.off_norms = take((size_t)P.nrows * 4);
    P.off_iscale = take((size_t)P.nrows * 4);
    P.off_u = take((size_t)P.nrows * 4);
    P.off_Zh = tc ? take((size_t)P.nrows * P.p_stride * 2) : 0;
    P.off_Zl = tc ? take((size_t)P.nrows * P.p_stride * 2) : 0;
    P.off_D = take(elems * 4);
    P.off_Chi = P.off_D;   // the split parts are written over the blocks' FP32 storage
    P.off_rowpart = take((size_t)P.nblk * PANEL * 8);
    P.off_colpart = take((size_t)P.nblk * KB * 8);
    P.off_r = take((size_t)P.nrows * 8);
    P.off_Spart = take((size_t)(P.nrows / 32) * 8);
    P.off_dcorr = take((size_t)P.nrows * 8);
    P.off_Upart = take((size_t)P.npan * 8);
    P.off_Stpart = take((size_t)P.npan * 8);
    P.off_maskT = take((size_t)P.nmask * 4);
    P.off_partial = take((size_t)P.npart * 4);
    P.off_stats = take((size_t)P.nstats * 8);
    P.off_errest = take((size_t)P.nstats * 8);
    P.off_flags = take((size_t)P.nstats);
    P.off_observed = take((size_t)P.n_tests * 8);
    P.off_ctr = take(sizeof(Counters) * P.n_tests);
    P.off_sel_hist = P.any_median ? take((size_t)P.n_tests * 2048 * 4) : 0;
    P.total = o;
}

// Debug checks on the host: invariants of a plan that the kernels rely on.
ept_status check_plan(const Plan &P) {
    auto bad = [](const char *what) { return fail(EPT_EINTERNAL, "debug checks: plan invariant broken: %s", what); };
    for (int t = 0; t < P.n_tests; ++t) {
        const TestDesc &d = P.desc[t];
        if (d.n != d.nx + d.ny || d.n_pad < d.n || d.n_pad % PANEL) return bad("row padding");
        if (d.Bp < d.ncols || d.Bp % COL_PAD || d.MT * TC_TILE_N != d.Bp) return bad("column padding");
        if (P.pre_rows[t + 1] - P.pre_rows[t] != d.n_pad || d.row0 != P.pre_rows[t]) return bad("row prefix");
        if (P.pre_cols[t + 1] - P.pre_cols[t] != d.Bp) return bad("column prefix");
        for (int64_t q = 0; q < d.nchunks; ++q) {
            const Chunk &ch = P.chunks[(size_t)(d.chunk0 + q)];
            if (ch.I < 0 || ch.I >= d.NP || ch.kb0 < KB_PER_PANEL * ch.I || ch.kb1 <= ch.kb0 || ch.kb1 > d.NKB)
                return bad("chunk range");
        }
        if (d.nparts != 2 * d.nchunks) return bad("partials");
    }
    if (!P.sched.empty()) {
        std::vector<char> seen((size_t)P.nunits, 0);
        if ((int64_t)P.sched.size() != P.nunits || P.sched_off.back() != P.nunits) return bad("schedule size");
        for (int64_t u : P.sched) {
            if (u < 0 || u >= P.nunits || seen[(size_t)u]) return bad("schedule covers every unit once");
            seen[(size_t)u] = 1;
        }
        // the unit records: each one the unit the schedule names, its offsets inside its test's arrays
        if ((int64_t)P.urec.size() != P.nunits) return bad("one record per scheduled unit");
        for (int64_t k = 0; k < P.nunits; ++k) {
            const int64_t u = P.sched[(size_t)k];
            int t = 0;
            while (t + 1 < P.n_tests && P.pre_units[t + 1] <= u) ++t;
            const TestDesc &d = P.desc[t];
            const int64_t lu = u - P.pre_units[t], h = lu & 1, q = (lu >> 1) / d.MT, m = (lu >> 1) % d.MT;
            const Chunk &ch = P.chunks[(size_t)(d.chunk0 + q)];
            const bool skip = h == 1 && ch.kb0 == KB_PER_PANEL * ch.I && ch.kb1 - ch.kb0 > 2;
            const UnitRec &r = P.urec[(size_t)k];
            if (r.I != ch.I || r.kb0 != ch.kb0 + (skip ? 2 : 0) || r.kb1 != ch.kb1 || r.h != h)
                return bad("unit record chunk");
            if (r.left < 1 || r.left > TC_TILE_N || r.left != std::min<int64_t>(TC_TILE_N, d.ncols - m * TC_TILE_N))
                return bad("unit record columns");
            if (r.NKB != d.NKB || r.Bp != d.Bp || r.blk0 != d.blk0) return bad("unit record test fields");
            if (r.mask_col < d.mask0 || r.mask_col + TC_TILE_N > d.mask0 + d.Bp) return bad("unit record mask offset");
            if (r.out_off < d.part0 || r.out_off + TC_TILE_N > d.part0 + d.nparts * d.Bp ||
                r.out_off != d.part0 + (2 * q + h) * d.Bp + m * TC_TILE_N)
                return bad("unit record partial offset");
        }
    }
    for (int k = 0; k < P.guards.n; ++k)
        if (P.guards.off[k] + GUARD_BYTES > P.total || P.guards.off[k] % 256) return bad("guard band");
    return EPT_OK;
}

std::vector<TestSpec> one_test(const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p, int stat,
                               double sigma, int64_t B, uint64_t seed, const uint32_t *masks, double *perm_stats) {
    TestSpec s;
    s.X = X;
    s.Y = Y;
    s.nx = nx;
    s.ny = ny;
    s.p = p;
    s.B = B;
    s.stat = stat;
    s.sigma = sigma;
    s.seed = seed;
    s.user_masks = masks;
    s.perm_stats = perm_stats;
    return std::vector<TestSpec>(1, s);
}

}  // namespace

namespace ept {
// lets other translation units of the library report an error message
void set_last_error(const char *msg) { g_err = msg; }

void describe_test(TestDesc &d, int64_t nx, int64_t ny, int64_t p, int64_t B, int stat, double sigma,
                   uint64_t seed, bool split) {
    memset(&d, 0, sizeof(d));
    d.nx = nx;
    d.ny = ny;
    d.n = nx + ny;
    d.p = p;
    d.B = B;
    d.n_pad = (d.n + PANEL - 1) / PANEL * PANEL;
    d.NP = d.n_pad / PANEL;
    d.NKB = d.n_pad / KB;
    d.nblk = blk_off(d.NP, d.NKB);
    d.nw = d.n_pad / 32;
    d.nwu = (int)((d.n + 31) / 32);
    d.ncols = B + 1;
    d.Bp = (d.ncols + COL_PAD - 1) / COL_PAD * COL_PAD;
    d.MT = d.Bp / TC_TILE_N;
    d.p_pad = (d.p + BUILD_KB - 1) / BUILD_KB * BUILD_KB;
    d.kblocks = (int)(d.p_pad / BUILD_KB);
    d.comp = d.ny < d.nx;
    d.m = d.comp ? d.ny : d.nx;
    d.other = d.comp ? d.nx : d.ny;
    set_params(d, stat, sigma, seed);
    d.b0 = 1;
    d.tau = (float)NEAR_DUP_TAU;
    const double fn = (double)d.n, q = fn / ((double)d.nx * (double)d.ny);
    d.cT = q * q;
    d.inv_o2 = 1.0 / ((double)d.other * (double)d.other);
    d.kappa = 2.0 * (double)d.m / fn;
    d.inv_n = 1.0 / fn;
    d.inv_2n2 = 1.0 / (2.0 * fn * fn);
    d.scaled = split ? 1 : 0;
    d.ka = refine_ka(CHUNK_KB_DEFAULT);
}

cudaError_t smem_limit_once(const void *func, int bytes, unsigned long long *done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (__atomic_load_n(done, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) __atomic_fetch_or(done, bit, __ATOMIC_RELEASE);
    return e;
}
}  // namespace ept

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> key;    // shapes + precision + memory space + chunk length
    uint8_t *arena = nullptr;
    cudaStream_t stream = nullptr;
};

namespace {
struct Server;

// Host memory copies spread over a small pool of worker threads (the caller works
// too), used to gather pageable inputs into the pinned staging area at several times
// the bandwidth of one core.  run() returns when every byte is copied.
class HostCopier {
public:
    struct Job {
        void *dst;
        const void *src;
        size_t bytes;
    };
    explicit HostCopier(int workers) {
        for (int k = 0; k < workers; ++k) th_.emplace_back([this] { worker(); });
    }
    ~HostCopier() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (std::thread &t : th_) t.join();
    }
    void run(const std::vector<Job> &jobs) {
        constexpr size_t PIECE = 1 << 20;
        {
            std::unique_lock<std::mutex> lk(mu_);
            cv_done_.wait(lk, [this] { return active_ == 0; });   // a late worker of the last run has left
            pieces_.clear();
            for (const Job &j : jobs)
                for (size_t o = 0; o < j.bytes; o += PIECE)
                    pieces_.push_back({(uint8_t *)j.dst + o, (const uint8_t *)j.src + o, std::min(PIECE, j.bytes - o)});
            next_.store(0);
            remaining_.store(pieces_.size());
            ++gen_;
        }
        cv_.notify_all();
        work();
        std::unique_lock<std::mutex> lk(mu_);
        cv_done_.wait(lk, [this] { return remaining_.load() == 0 && active_ == 0; });
    }

private:
    void work() {
        const size_t n = pieces_.size();
        for (;;) {
            const size_t k = next_.fetch_add(1);
            if (k >= n) break;
            memcpy(pieces_[k].dst, pieces_[k].src, pieces_[k].bytes);
            if (remaining_.fetch_sub(1) == 1) {
                std::lock_guard<std::mutex> lk(mu_);
                cv_done_.notify_all();
            }
        }
    }
    void worker() {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = gen_;
                ++active_;
            }
            work();
            {
                std::lock_guard<std::mutex> lk(mu_);
                --active_;
            }
            cv_done_.notify_all();
        }
    }
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_, cv_done_;
    std::vector<Job> pieces_;
    std::atomic<size_t> next_{0}, remaining_{0};
    int active_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};
}  // namespace

struct ept_ctx {
    Server *server = nullptr;           // serving scheduler, started by the first ept_submit
    int device = 0;
    int num_sms = 0;
    size_t total_mem = 0;               // the device's memory (cudaDeviceProp::totalGlobalMem)
    size_t budget = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;        // relabeling draws run here, beside the block build
    cudaEvent_t ev[7] = {};
    cudaEvent_t ev_side[3] = {};
    std::mutex mu;
    uint8_t *arena = nullptr;
    size_t arena_cap = 0;
    uint8_t *pinned = nullptr;
    size_t pinned_cap = 0;
    GraphCache graph;
    std::map<std::vector<int64_t>, Tuning> tuned;   // autotuner cache: batch shape -> parameters
    bool autotune = true;
    bool graphs = true;                 // replay captured graphs of repeated batches
    bool debug = false;                 // guard bands around scratch regions, plan invariants checked
    int draw_mode = 0;                  // relabeling draws: 0 automatic, DRAW_WARPS, DRAW_LANES, DRAW_SCAN
    int64_t stream_blocks = 0;          // streaming mode: 0 automatic, k > 0 windows of <= k blocks, -1 never
    unsigned long long wait_ns = 0;     // limit of the kernels' bounded waits (0: their default, 2 s)
    int max_chunk = 32;                 // longest contraction unit the autotuner may pick
    int unit_kb = 0;                    // unit length of every run (EPT_OPT_UNIT_KB; 0: the default / autotuner)
    bool refine = true;                 // recompute flagged statistics (EPT_OPT_REFINE)
    int contraction = 0;                // tensor-core contraction kernel (EPT_OPT_CONTRACTION; 0: default)
    uint8_t *refine_buf = nullptr;      // scratch of the recomputation (grows, kept until ept_destroy)
    size_t refine_cap = 0;
    ept_allocator alloc{};              // caller-supplied device memory (alloc.alloc == nullptr: cudaMalloc)
    std::atomic<int> inject_alloc{0};   // test hook: the next N scratch acquisitions fail (host side)
    bool inject_stall = false;          // test hook: the next run's contraction waits out its limit
    int serve_lanes = 3;                // serving: batches in flight at once
    int serve_slots = 256;              // serving: requests in flight at once
    cudaEvent_t ev_user = nullptr;      // orders the context's stream after a caller's stream
    cudaStream_t copy = nullptr;        // host-to-device input copies, beside the relabeling draws
    cudaEvent_t ev_in = nullptr;        // the run's inputs are on the device
    std::vector<cudaEvent_t> ev_win;    // streaming mode: around each window's contraction (first 64 windows)
    // plan of the last run, reused while the batch shape repeats; tables_staged: the
    // pinned staging area still holds its constant tables
    Plan *plan = nullptr;
    std::vector<int64_t> plan_key;
    bool tables_staged = false;
    uint64_t urec_serial = 0;           // plan whose unit records the arena holds (0: none)
    uint8_t *urec_arena = nullptr;      // the arena they were uploaded to
    // host-to-device copies of this run's inputs: from the caller's buffers when they
    // are page-locked, else from the pinned staging area
    struct InputCopy {
        size_t dst;          // byte offset in the arena
        const void *src;
        size_t bytes;
    };
    std::vector<InputCopy> in_copies;
    std::unique_ptr<HostCopier> copier;   // started by the first large pageable input
    std::string tune_file;
};

// the tensor-core contraction kernel of a run: 1 relabelings in shared memory (the
// default: measured fastest), 2 the same on pairs of SMs, 3 relabelings in tensor memory
static int contraction_kernel(const ept_ctx *c) { return c->contraction ? c->contraction : 1; }

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

// NVTX range on the host timeline (shown by Nsight tools; no cost without them)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// fault-injection hook (EPT_OPT_FAULT_INJECT_ALLOC): consume one injected failure
bool injected_failure(ept_ctx *c) {
    int v = c->inject_alloc.load();
    while (v > 0)
        if (c->inject_alloc.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

void drop_graph(ept_ctx *c) {
    if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
    c->graph = GraphCache();
}

// device memory through the context's allocator (or cudaMalloc / cudaFree); memory
// from a caller's allocator must be 256-byte aligned (the tensor maps and the
// arena's own alignment rely on it)
ept_status device_alloc(ept_ctx *c, size_t bytes, cudaStream_t s, void **out) {
    *out = nullptr;
    if (c->alloc.alloc) {
        void *p = c->alloc.alloc(bytes, (void *)s, c->alloc.user);
        if (!p) return fail(EPT_ENOMEM, "the caller's allocator returned no memory for %zu bytes", bytes);
        if ((uintptr_t)p % 256) {
            c->alloc.free(p, (void *)s, c->alloc.user);
            return fail(EPT_EINVAL, "the caller's allocator returned an address not aligned to 256 bytes");
        }
        *out = p;
        return EPT_OK;
    }
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return fail(EPT_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    return EPT_OK;
}

void device_free(ept_ctx *c, void *p, cudaStream_t s) {
    if (!p) return;
    if (c->alloc.alloc) c->alloc.free(p, (void *)s, c->alloc.user);
    else cudaFree(p);
}

// exact: allocate just `bytes` (the streaming mode sizes its window to the memory
// there is), else 1/8 more, so that slightly larger runs reuse the arena
ept_status ensure_arena(ept_ctx *c, size_t bytes, cudaStream_t s, bool exact = false) {
    if (c->budget && bytes > c->budget)
        return fail(EPT_ENOMEM, "this run needs %zu bytes of device scratch, over the context budget of %zu", bytes,
                    c->budget);
    if (bytes <= c->arena_cap) return EPT_OK;
    CK(cudaStreamSynchronize(s));
    CK(cudaStreamSynchronize(c->stream));
    drop_graph(c);
    if (c->arena) {
        device_free(c, c->arena, c->stream);
        c->arena = nullptr;
        c->arena_cap = 0;
    }
    const size_t cap = align_up(exact ? bytes : bytes + bytes / 8, 1 << 20);
    void *p = nullptr;
    ept_status st = device_alloc(c, cap, c->stream, &p);
    if (st != EPT_OK) return st;
    c->arena = (uint8_t *)p;
    c->arena_cap = cap;
    c->urec_serial = 0;   // a new arena holds no unit records
    return EPT_OK;
}

ept_status ensure_pinned(ept_ctx *c, size_t bytes) {
    if (bytes <= c->pinned_cap) return EPT_OK;
    drop_graph(c);   // a captured graph reads the old staging area
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
    c->tables_staged = false;
    return EPT_OK;
}

// Pinned staging layout: [tables (tab_bytes)] [inputs (in_bytes)] [results].
struct Staging {
    size_t tables, inputs, res_ctr, res_obs, res_stats, total;
};

Staging staging_layout(const Plan &P) {
    Staging S;
    size_t o = 0;
    S.tables = o;
    o = align_up(o + P.tab_bytes, 256);
    S.inputs = o;
    o = align_up(o + P.in_bytes, 256);
    S.res_ctr = o;
    o = align_up(o + sizeof(Counters) * P.n_tests, 256);
    S.res_obs = o;
    o = align_up(o + 8 * (size_t)P.n_tests, 256);
    S.res_stats = o;
    o = align_up(o + (P.host_in ? 8 * (size_t)P.nstats : 0), 256);
    S.total = o;
    return S;
}

bool page_locked(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Host-side staging of one run: device pointers into the descriptors and the tables
// into the pinned area (everything a captured graph reads from the host goes through
// it, so the graph can be replayed after re-staging), and the list of input copies:
// host inputs in page-locked memory are copied to the device directly, others are
// first gathered into the pinned area.
void stage_host(ept_ctx *c, Plan &P, const std::vector<TestSpec> &specs, bool on_device, bool tables = true) {
    const Staging S = staging_layout(P);
    uint8_t *A = c->arena, *pin = c->pinned;
    c->in_copies.clear();
    bool all_staged = true;
    std::vector<HostCopier::Job> gather;
    size_t gather_bytes = 0;
    auto input = [&](size_t off, const void *src, size_t bytes) {
        if (bytes == 0) return;
        if (page_locked(src)) {
            c->in_copies.push_back({P.off_in + off, src, bytes});
            all_staged = false;
        } else {
            gather.push_back({pin + S.inputs + off, src, bytes});
            gather_bytes += bytes;
            c->in_copies.push_back({P.off_in + off, pin + S.inputs + off, bytes});
        }
    };
    for (int t = 0; t < P.n_tests; ++t) {
        TestDesc &d = P.desc[t];
        const TestSpec &s = specs[t];
        if (on_device) {
            d.X = s.X;
            d.Y = s.Y;
            d.user_masks = s.user_masks;
            d.out_stats = s.perm_stats;
        } else {
            const size_t xo = P.in_off[t], yo = xo + align_up((size_t)d.nx * d.p * 4, 256);
            const size_t mo = yo + align_up((size_t)d.ny * d.p * 4, 256);
            input(xo, s.X, (size_t)d.nx * d.p * 4);
            input(yo, s.Y, (size_t)d.ny * d.p * 4);
            d.X = (const float *)(A + P.off_in + xo);
            d.Y = (const float *)(A + P.off_in + yo);
            if (s.user_masks) {
                input(mo, s.user_masks, (size_t)s.B * d.nwu * 4);
                d.user_masks = (const uint32_t *)(A + P.off_in + mo);
            } else {
                d.user_masks = nullptr;
            }
            d.out_stats = nullptr;   // copied back to the host and scattered there
        }
    }
    if (gather_bytes >= ((size_t)4 << 20)) {
        if (!c->copier) {
            const unsigned hw = std::thread::hardware_concurrency();
            c->copier.reset(new HostCopier((int)std::max(1u, std::min(8u, hw / 2))));
        }
        c->copier->run(gather);
    } else {
        for (const HostCopier::Job &j : gather) memcpy(j.dst, j.src, j.bytes);
    }
    if (!on_device && all_staged && P.in_bytes) {
        // everything went through the staging area: one copy of the whole input region
        c->in_copies.clear();
        c->in_copies.push_back({P.off_in, pin + S.inputs, P.in_bytes});
    }
    uint8_t *tab = pin + S.tables;
    memcpy(tab + P.off_desc, P.desc.data(), sizeof(TestDesc) * P.n_tests);
    if (!tables) return;   // the shape-dependent tables are already in place
    memcpy(tab + P.off_pre_rows, P.pre_rows.data(), 8 * P.pre_rows.size());
    memcpy(tab + P.off_pre_panels, P.pre_panels.data(), 8 * P.pre_panels.size());
    memcpy(tab + P.off_pre_cols, P.pre_cols.data(), 8 * P.pre_cols.size());
    memcpy(tab + P.off_pre_units, P.pre_units.data(), 8 * P.pre_units.size());
    memcpy(tab + P.off_pre_simt, P.pre_simt.data(), 8 * P.pre_simt.size());
    if (!P.blk.empty()) memcpy(tab + P.off_blk, P.blk.data(), sizeof(BlkInfo) * P.blk.size());
    if (!P.tiles.empty()) memcpy(tab + P.off_tiles, P.tiles.data(), sizeof(Tile) * P.tiles.size());
    if (!P.chunks.empty()) memcpy(tab + P.off_chunks, P.chunks.data(), sizeof(Chunk) * P.chunks.size());
    if (!P.sched.empty()) {
        memcpy(tab + P.off_sched, P.sched.data(), 8 * P.sched.size());
        memcpy(tab + P.off_sched_off, P.sched_off.data(), 8 * P.sched_off.size());
    }
}

Batch device_view(ept_ctx *c, const Plan &P) {
    uint8_t *A = c->arena;
    Batch b;
    memset(&b, 0, sizeof(b));
    b.n_tests = P.n_tests;
    b.desc = (const TestDesc *)(A + P.off_desc);
    b.pre.rows = (const int64_t *)(A + P.off_pre_rows);
    b.pre.panels = (const int64_t *)(A + P.off_pre_panels);
    b.pre.cols = (const int64_t *)(A + P.off_pre_cols);
    b.pre.units = (const int64_t *)(A + P.off_pre_units);
    b.pre.simt = (const int64_t *)(A + P.off_pre_simt);
    b.blk = (const BlkInfo *)(A + P.off_blk);
    b.tiles = (const Tile *)(A + P.off_tiles);
    b.chunks = (const Chunk *)(A + P.off_chunks);
    b.sched = P.sched.empty() ? nullptr : (const int64_t *)(A + P.off_sched);
    b.sched_off = P.sched.empty() ? nullptr : (const int64_t *)(A + P.off_sched_off);
    b.urec = P.urec.empty() ? nullptr : (const UnitRec *)(A + P.off_urec);
    b.urec_pair = P.urec_pair.empty() ? nullptr : (const UnitRec *)(A + P.off_urec_pair);
    b.tc_grid = P.tc_grid;
    b.nblk_total = P.nblk;
    b.ntiles = (int64_t)P.tiles.size();
    b.nrows_total = P.nrows;
    b.npan_total = P.npan;
    b.ncols_total = P.ncols_pad;
    b.nunits_total = P.nunits;
    b.nsimt_total = P.nsimt;
    b.p_stride = P.p_stride;
    b.norms = (float *)(A + P.off_norms);
    b.iscale = (float *)(A + P.off_iscale);
    b.u = (float *)(A + P.off_u);
    b.Zh = (uint16_t *)(A + P.off_Zh);
    b.Zl = (uint16_t *)(A + P.off_Zl);
    b.Chi = (uint16_t *)(A + P.off_D);            // block b: hi at its first 32 KB,
    b.Clo = b.Chi + (size_t)PANEL * KB;           //          lo at its second 32 KB
    b.c_stride = 2 * (int64_t)PANEL * KB;
    b.D = (float *)(A + P.off_D);
    b.partial = (float *)(A + P.off_partial);
    b.rowpart = (double *)(A + P.off_rowpart);
    b.colpart = (double *)(A + P.off_colpart);
    b.r = (double *)(A + P.off_r);
    b.Spart = (double *)(A + P.off_Spart);
    b.dcorr = (double *)(A + P.off_dcorr);
    b.Upart = (double *)(A + P.off_Upart);
    b.Stpart = (double *)(A + P.off_Stpart);
    b.stats = (double *)(A + P.off_stats);
    b.errest = P.off_errest ? (double *)(A + P.off_errest) : nullptr;
    b.flags = P.off_flags ? (uint8_t *)(A + P.off_flags) : nullptr;
    b.observed = (double *)(A + P.off_observed);
    b.maskT = (uint32_t *)(A + P.off_maskT);
    b.ctr = (Counters *)(A + P.off_ctr);
    b.sel_hist = P.any_median ? (uint32_t *)(A + P.off_sel_hist) : nullptr;
    b.sacc = nullptr;
    b.inject_stall = c->inject_stall ? 1 : 0;
    b.wait_ns = c->wait_ns;
    return b;
}

// relabeling-draw kernel of a run: the context's choice, else a thread per column
// when there are at least 1024 columns per SM and a warp per column otherwise (the
// producer / scanner kernel is an option: slower beside the block build, whose SMs
// have no room left for its 32 KB of shared memory); caller relabelings always take
// the warp kernel (it validates them)
int draw_mode_for(const ept_ctx *c, const Plan &P) {
    int mode = P.draw_mode ? P.draw_mode : c->draw_mode;
    if (mode == 0)
        mode = P.ncols_pad >= DRAW_LANES_MIN_COLS_PER_SM * (int64_t)c->num_sms ? DRAW_LANES : DRAW_WARPS;
    return P.user_masks ? DRAW_WARPS : mode;
}

// The device work of one run, enqueued on s (and the side stream).  With `timed`,
// events mark the phases (not used while capturing a graph).
// The run's input copies on the copy stream (after `after`'s prior work), then ev_in:
// the relabeling draws, which do not read the inputs, start while the copies run.
ept_status enqueue_inputs(ept_ctx *c, cudaStream_t after) {
    CK(cudaEventRecord(c->ev_user, after));
    CK(cudaStreamWaitEvent(c->copy, c->ev_user, 0));
    for (const ept_ctx::InputCopy &k : c->in_copies)
        CK(cudaMemcpyAsync(c->arena + k.dst, k.src, k.bytes, cudaMemcpyHostToDevice, c->copy));
    CK(cudaEventRecord(c->ev_in, c->copy));
    return EPT_OK;
}

// The run's host-to-device traffic: the tables on s first (the copy engine takes
// copies in order, so the small upload that the draws wait for goes ahead), then the
// inputs on the copy stream.
ept_status enqueue_uploads(ept_ctx *c, const Plan &P, cudaStream_t s) {
    const Staging S = staging_layout(P);
    CK(cudaMemcpyAsync(c->arena, c->pinned + S.tables, P.tab_bytes, cudaMemcpyHostToDevice, s));
    // the unit records stay in the arena while the same plan runs on it; a run of any
    // other plan may overwrite them
    if (P.urec.empty() && P.urec_pair.empty()) {
        c->urec_serial = 0;
    } else if (c->urec_serial != P.serial || c->urec_arena != c->arena) {
        if (!P.urec.empty())
            CK(cudaMemcpyAsync(c->arena + P.off_urec, P.urec.data(), sizeof(UnitRec) * P.urec.size(),
                               cudaMemcpyHostToDevice, s));
        if (!P.urec_pair.empty())
            CK(cudaMemcpyAsync(c->arena + P.off_urec_pair, P.urec_pair.data(), sizeof(UnitRec) * P.urec_pair.size(),
                               cudaMemcpyHostToDevice, s));
        c->urec_serial = P.serial;
        c->urec_arena = c->arena;
    }
    return enqueue_inputs(c, s);
}

// with_inputs: also issue the uploads; a captured graph leaves them out (they are
// issued before each replay, the inputs from wherever the caller's buffers are) and
// waits for the inputs through ev_in as an external event.
ept_status enqueue_device(ept_ctx *c, const Plan &P, cudaStream_t s, bool timed, bool with_inputs = true) {
    ept_status st = EPT_OK;
    const Staging S = staging_layout(P);
    uint8_t *pin = c->pinned;
    const Batch b = device_view(c, P);
    const bool tc = P.prec == EPT_PREC_SPLIT_BF16;
    if (timed) CK(cudaEventRecord(c->ev[0], s));
    if (with_inputs && (st = enqueue_uploads(c, P, s)) != EPT_OK) return st;
    CK(cudaMemsetAsync(b.ctr, 0, sizeof(Counters) * P.n_tests, s));
    if (P.any_median) CK(cudaMemsetAsync(b.sel_hist, 0, (size_t)P.n_tests * 2048 * 4, s));
    if (P.debug) launch_guards(c->arena, P.guards, false, b.ctr, s);
    CK(cudaEventRecord(c->ev[1], s));

    // relabelings on the side stream, beside the block build
    cudaStream_t s2 = c->side;
    CK(cudaStreamWaitEvent(s2, c->ev[1], 0));
    if (timed) CK(cudaEventRecord(c->ev_side[1], s2));
    launch_masks(b, c->num_sms, draw_mode_for(c, P), s2);
    CK(cudaGetLastError());
    CK(cudaEventRecord(c->ev_side[2], s2));

    // phase 1: blocks, centring, packing (after the inputs have arrived)
    CK(cudaStreamWaitEvent(s, c->ev_in, with_inputs ? cudaEventWaitDefault : cudaEventWaitExternal));
    if (tc) {
        launch_split_rows(b, s);
        alignas(64) CUtensorMap tm[4];
        char emsg[160];
        if (!encode_rows_tmaps(tm, b.Zh, b.Zl, P.nrows, P.p_stride, emsg, sizeof(emsg)))
            return fail(EPT_ECUDA, "%s", emsg);
        CK(launch_build_tc(b, tm, c->num_sms, s));
    } else {
        launch_norms(b, s);
        launch_build_simt(b, s);
    }
    launch_median_select(b, s);
    launch_blocksums(b, s);
    launch_rowsum_reduce(b, s);
    launch_center(b, s);
    launch_pack(b, tc, s);
    CK(cudaGetLastError());
    if (timed) CK(cudaEventRecord(c->ev[2], s));

    // phase 2: contraction, combination
    CK(cudaStreamWaitEvent(s, c->ev_side[2], 0));
    if (timed) CK(cudaEventRecord(c->ev[5], s));
    if (tc) {
        alignas(64) CUtensorMap th, tl;
        char emsg[160];
        if (!encode_block_tmaps(&th, &tl, b.Chi, b.Clo, P.nblk, b.c_stride, emsg, sizeof(emsg)))
            return fail(EPT_ECUDA, "%s", emsg);
        switch (P.contraction ? P.contraction : contraction_kernel(c)) {
        case 2: CK(launch_contract_tc2(b, &th, &tl, c->num_sms, s)); break;
        case 3: CK(launch_contract_tm(b, &th, &tl, c->num_sms, s)); break;
        default: CK(launch_contract_tc(b, &th, &tl, c->num_sms, s)); break;
        }
    } else {
        launch_contract_simt(b, s);
        CK(cudaGetLastError());
    }
    if (timed) CK(cudaEventRecord(c->ev[6], s));
    launch_combine(b, s);
    CK(cudaGetLastError());
    if (P.debug) launch_guards(c->arena, P.guards, true, b.ctr, s);   // after every write of the run
    if (timed) CK(cudaEventRecord(c->ev[3], s));

    CK(cudaMemcpyAsync(pin + S.res_ctr, b.ctr, sizeof(Counters) * P.n_tests, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pin + S.res_obs, b.observed, 8 * (size_t)P.n_tests, cudaMemcpyDeviceToHost, s));
    if (P.host_in) CK(cudaMemcpyAsync(pin + S.res_stats, b.stats, 8 * (size_t)P.nstats, cudaMemcpyDeviceToHost, s));
    if (timed) CK(cudaEventRecord(c->ev[4], s));
    return EPT_OK;
}

// Results of a finished run (host side).
// With `per_test`, a test whose input was rejected on the device gets its own
// status and message there and the others are still returned (serving); without
// it, the first such test fails the whole call.
struct TestError {
    ept_status st;
    std::string msg;
};

float median_sigma(const Counters &k) {
    float v;
    memcpy(&v, &k.sel_prefix, 4);
    return v;
}

ept_status test_error(const Plan &P, const Counters *ctr, int t) {
    if (ctr[t].nonfinite) return fail(EPT_EINVAL, "test %d: X or Y holds NaN or Inf", t);
    if (P.desc[t].median) {
        const float sg = median_sigma(ctr[t]);
        if (!(sg > 0.f) || !std::isfinite(sg))
            return fail(EPT_EINVAL, "test %d: the median-heuristic bandwidth is %g (more than half of the pooled "
                                    "pairs coincide)", t, (double)sg);
    }
    if (ctr[t].bad_mask)
        return fail(EPT_EINVAL, "test %d: %llu relabeling(s) do not have exactly nx = %lld members among the n rows", t,
                    (unsigned long long)ctr[t].bad_mask, (long long)P.desc[t].nx);
    return EPT_OK;
}

ept_status collect(ept_ctx *c, const Plan &P, const std::vector<TestSpec> &specs, ept_result *out, bool timed,
                   std::vector<TestError> *per_test = nullptr) {
    const Staging S = staging_layout(P);
    const Counters *ctr = (const Counters *)(c->pinned + S.res_ctr);
    const double *obs = (const double *)(c->pinned + S.res_obs);
    const double *stats = (const double *)(c->pinned + S.res_stats);
    if (P.n_tests > 0 && ctr[0].err_code)
        return fail(EPT_ETIMEOUT, "device-side bounded wait gave up (code 0x%llx)", (unsigned long long)ctr[0].err_code);
    if (P.debug && P.n_tests > 0 && ctr[0].guard_bad)
        return fail(EPT_EINTERNAL, "debug checks: %llu words of the scratch guard bands were overwritten",
                    (unsigned long long)ctr[0].guard_bad);
    if (per_test) per_test->assign(P.n_tests, TestError{EPT_OK, std::string()});
    for (int t = 0; t < P.n_tests; ++t) {
        const ept_status st = test_error(P, ctr, t);
        if (st == EPT_OK) continue;
        if (!per_test) return st;
        (*per_test)[t] = TestError{st, g_err};
    }
    float ms_build = 0.f, ms_perm = 0.f, ms_total = 0.f, ms_masks = 0.f, ms_contract = 0.f;
    if (timed) {
        cudaEventElapsedTime(&ms_build, c->ev[1], c->ev[2]);
        cudaEventElapsedTime(&ms_perm, c->ev[2], c->ev[3]);
        cudaEventElapsedTime(&ms_total, c->ev[0], c->ev[4]);
        cudaEventElapsedTime(&ms_masks, c->ev_side[1], c->ev_side[2]);
        cudaEventElapsedTime(&ms_contract, c->ev[5], c->ev[6]);
    }
    for (int t = 0; t < P.n_tests; ++t) {
        const TestDesc &d = P.desc[t];
        ept_result &r = out[t];
        r.observed = obs[t];
        r.n_ge = (int64_t)ctr[t].n_ge;
        r.n_near_tie = (int64_t)ctr[t].n_near;
        r.n_fixup = (int64_t)ctr[t].n_fixup;
        r.p_value = (1.0 + (double)r.n_ge) / (1.0 + (double)d.B);
        r.sigma = d.median ? (double)median_sigma(ctr[t]) : (d.stat == EPT_STAT_ED ? 0.0 : specs[t].sigma);
        r.ms_build = ms_build;
        r.ms_perm = ms_perm;
        r.ms_total = ms_total;
        r.ms_masks = ms_masks;
        r.ms_contract = ms_contract;
        r.n_windows = P.stream ? (int64_t)P.gI0.size() : 0;
        r.n_refined = (int64_t)ctr[t].n_flag;
        r.tuning = 0;
        r.tune_candidates = 0;
        r.refine_launches = 0;
        if (P.host_in && specs[t].perm_stats && d.B > 0)
            memcpy(specs[t].perm_stats, stats + d.col0 + 1, (size_t)d.B * 8);
    }
    return EPT_OK;
}

std::vector<int64_t> shape_key(const std::vector<TestSpec> &specs, int prec, bool on_device) {
    std::vector<int64_t> k;
    k.push_back(prec);
    k.push_back(on_device ? 1 : 0);
    for (const TestSpec &s : specs) {
        k.push_back(s.nx);
        k.push_back(s.ny);
        k.push_back(s.p);
        k.push_back(s.B);
        k.push_back(s.user_masks ? 1 : 0);
        k.push_back(s.perm_stats ? 1 : 0);
        k.push_back(s.stat != EPT_STAT_ED && s.sigma == EPT_SIGMA_MEDIAN ? 1 : 0);   // selection buffers
    }
    return k;
}

// key of the autotuner: the batch's padded shapes (what the unit decomposition sees)
// and the longest unit allowed
std::vector<int64_t> tune_key(const std::vector<TestSpec> &specs, int prec, int max_chunk) {
    std::vector<int64_t> k;
    k.push_back(prec);
    k.push_back(max_chunk);
    for (const TestSpec &s : specs) {
        k.push_back((s.nx + s.ny + PANEL - 1) / PANEL);
        k.push_back((s.B + 1 + COL_PAD - 1) / COL_PAD);
    }
    return k;
}

void save_tune_file(ept_ctx *c) {
    if (c->tune_file.empty()) return;
    FILE *f = fopen(c->tune_file.c_str(), "w");
    if (!f) return;
    for (auto &kv : c->tuned) {
        fprintf(f, "%d %d %d %d", kv.second.chunk_kb, kv.second.draw_mode, kv.second.order, kv.second.kernel);
        for (int64_t v : kv.first) fprintf(f, " %lld", (long long)v);
        fprintf(f, "\n");
    }
    fclose(f);
}

void load_tune_file(ept_ctx *c) {
    if (c->tune_file.empty()) return;
    FILE *f = fopen(c->tune_file.c_str(), "r");
    if (!f) return;
    char line[1 << 16];
    while (fgets(line, sizeof(line), f)) {
        char *p = line, *end = nullptr;
        long head[4];
        int k = 0;
        for (; k < 4; ++k) {
            head[k] = strtol(p, &end, 10);
            if (end == p) break;
            p = end;
        }
        if (k < 4) continue;
        std::vector<int64_t> key;
        for (;;) {
            const long long v = strtoll(p, &end, 10);
            if (end == p) break;
            key.push_back(v);
            p = end;
        }
        Tuning tn;
        tn.chunk_kb = (int)head[0];
        tn.draw_mode = (int)head[1];
        tn.order = (int)head[2];
        tn.kernel = (int)head[3];
        const bool ok = (tn.chunk_kb == 4 || tn.chunk_kb == 8 || tn.chunk_kb == 16 || tn.chunk_kb == 32) &&
                        tn.draw_mode >= 0 && tn.draw_mode <= 3 && tn.order >= 0 && tn.order <= 2 &&
                        tn.kernel >= 0 && tn.kernel <= 3;
        if (ok) c->tuned[key] = tn;
    }
    fclose(f);
}

// Recomputation of the statistics the error criterion flagged (ept_refine.cu), after
// a finished run whose scratch is still in place: the flags of every flagged test are
// read back together; the columns flagged for an exact re-summation of the packed
// operand, of all tests, in one launch (a job per group of up to 16 columns of a
// test); then, test by test, those flagged for entries rebuilt in FP64 (W64 in row
// windows of at most REFINE_W64_BYTES); then the counts again and the results read
// back as the run itself does, with one synchronisation for all of it.  Statistics
// that were not flagged keep their values.
const size_t REFINE_W64_BYTES = (size_t)2 << 30;

// the recomputation's scratch: the context's buffer, grown when needed (the previous
// recomputation has finished with it: it waits for its work before returning); kept
// between calls up to 256 MiB
ept_status refine_scratch(ept_ctx *c, size_t bytes, cudaStream_t s, uint8_t **out) {
    if (bytes > c->refine_cap) {
        if (c->refine_buf) device_free(c, c->refine_buf, s);
        c->refine_buf = nullptr;
        c->refine_cap = 0;
        void *p = nullptr;
        const size_t cap = align_up(bytes + bytes / 4, 1 << 20);
        ept_status st = device_alloc(c, cap, s, &p);
        if (st != EPT_OK) return st;
        c->refine_buf = (uint8_t *)p;
        c->refine_cap = cap;
    }
    *out = c->refine_buf;
    return EPT_OK;
}

ept_status refine_after(ept_ctx *c, const Plan &P, const std::vector<TestSpec> &specs, ept_result *out, bool timed,
                        cudaStream_t s, std::vector<TestError> *per_test = nullptr) {
    if (!c->refine || P.off_flags == 0) return EPT_OK;
    const Staging S = staging_layout(P);
    const Counters *ctr = (const Counters *)(c->pinned + S.res_ctr);
    std::vector<int> tl;   // tests with flagged statistics
    size_t nfl = 0;
    for (int t = 0; t < P.n_tests; ++t) {
        if (ctr[t].n_flag == 0 || test_error(P, ctr, t) != EPT_OK) continue;
        if (per_test && (*per_test)[t].st != EPT_OK) continue;
        tl.push_back(t);
        nfl += (size_t)P.desc[t].ncols;
    }
    if (tl.empty()) return EPT_OK;
    NvtxRange range("ept.refine");
    const Batch b = device_view(c, P);
    // the flags of those tests, read back together
    std::vector<uint8_t> fl(nfl);
    std::vector<size_t> fl_off;
    for (size_t k = 0, o = 0; k < tl.size(); ++k) {
        const TestDesc &d = P.desc[tl[k]];
        fl_off.push_back(o);
        CK(cudaMemcpyAsync(fl.data() + o, b.flags + d.col0, (size_t)d.ncols, cudaMemcpyDeviceToHost, s));
        o += (size_t)d.ncols;
    }
    CK(cudaStreamSynchronize(s));
    // level 1: exact re-summation of the packed operand (the accumulation part), every
    // test's groups of flagged columns in one launch; level 2: the entries rebuilt in
    // FP64 from the raw rows (the representation part), test by test.  The host lists
    // live until the final synchronisation.
    std::vector<int32_t> list1, list2;
    std::vector<RefineJob> jobs;
    std::vector<int64_t> l2_first(tl.size() + 1, 0);
    int64_t part1 = 0, max_ctas = 0;
    size_t l2_bytes = 0;
    for (size_t k = 0; k < tl.size(); ++k) {
        const int t = tl[k];
        const TestDesc &d = P.desc[t];
        const uint8_t *f = fl.data() + fl_off[k];
        const int64_t first1 = (int64_t)list1.size();
        for (int64_t j = 0; j < d.ncols; ++j) {
            if (f[j] == 1) list1.push_back((int32_t)j);
            if (f[j] == 2) list2.push_back((int32_t)j);
        }
        const int32_t nkc = (int32_t)refine_packed_chunks(d.NKB);
        for (int64_t j = first1; j < (int64_t)list1.size(); j += REFINE_JOB_COLS) {
            RefineJob J;
            J.t = t;
            J.ncol = (int32_t)std::min<int64_t>(REFINE_JOB_COLS, (int64_t)list1.size() - j);
            J.np = (int32_t)d.NP;
            J.nkc = nkc;
            J.list0 = j;
            J.part0 = part1;
            part1 += (int64_t)J.np * J.nkc * J.ncol;
            max_ctas = std::max<int64_t>(max_ctas, (int64_t)J.np * J.nkc);
            jobs.push_back(J);
        }
        l2_first[k + 1] = (int64_t)list2.size();
        const int64_t n2 = l2_first[k + 1] - l2_first[k];
        if (n2 > 0) {
            const int64_t ntiles = (d.n + 63) / 64;
            int64_t rows_w = (int64_t)(REFINE_W64_BYTES / (8 * (size_t)d.n)) / 64 * 64;
            rows_w = std::max<int64_t>(64, std::min<int64_t>(rows_w, ntiles * 64));
            l2_bytes = std::max(l2_bytes, align_up(16 * (size_t)ntiles * n2, 256) + align_up(8 * (size_t)ntiles, 256) +
                                              8 * (size_t)rows_w * (size_t)d.n);
        }
    }
    const size_t b_list1 = align_up(4 * list1.size() + 4, 256), b_list2 = align_up(4 * list2.size() + 4, 256),
                 b_jobs = align_up(sizeof(RefineJob) * jobs.size() + 16, 256), b_part1 = align_up(8 * (size_t)part1 + 8, 256);
    uint8_t *mem = nullptr;
    ept_status st = refine_scratch(c, b_list1 + b_list2 + b_jobs + b_part1 + l2_bytes, s, &mem);
    if (st != EPT_OK) return st;
    int32_t *dlist1 = (int32_t *)mem, *dlist2 = (int32_t *)(mem + b_list1);
    RefineJob *djobs = (RefineJob *)(mem + b_list1 + b_list2);
    double *dpart1 = (double *)(mem + b_list1 + b_list2 + b_jobs);
    uint8_t *l2mem = mem + b_list1 + b_list2 + b_jobs + b_part1;
    cudaError_t e = cudaSuccess;
    int64_t launches = 2;   // the counts reset and taken again
    if (!jobs.empty()) {
        launches += 2 * (((int64_t)jobs.size() + 65534) / 65535);
        e = cudaMemcpyAsync(dlist1, list1.data(), 4 * list1.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(djobs, jobs.data(), sizeof(RefineJob) * jobs.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            launch_refine_packed(b, djobs, (int64_t)jobs.size(), max_ctas, dlist1, dpart1, s);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && !list2.empty())
        e = cudaMemcpyAsync(dlist2, list2.data(), 4 * list2.size(), cudaMemcpyHostToDevice, s);
    for (size_t k = 0; k < tl.size() && e == cudaSuccess; ++k) {
        const int64_t nflag = l2_first[k + 1] - l2_first[k];
        if (nflag == 0) continue;
        const int t = tl[k];
        const TestDesc &d = P.desc[t];
        const double sigma = d.stat == EPT_STAT_ED ? 0.0 : (d.median ? (double)median_sigma(ctr[t]) : d.sigma64);
        const int64_t ntiles = (d.n + 63) / 64;
        int64_t rows_w = (int64_t)(REFINE_W64_BYTES / (8 * (size_t)d.n)) / 64 * 64;
        rows_w = std::max<int64_t>(64, std::min<int64_t>(rows_w, ntiles * 64));
        const size_t b_part = align_up(16 * (size_t)ntiles * nflag, 256), b_spart = align_up(8 * (size_t)ntiles, 256);
        // the tests' rebuilds reuse one region in stream order
        const int32_t *dlist = dlist2 + l2_first[k];
        double *part = (double *)l2mem, *spart = (double *)(l2mem + b_part);
        double *W64 = (double *)(l2mem + b_part + b_spart);
        for (int64_t r0 = 0; r0 < d.n && e == cudaSuccess; r0 += rows_w) {
            const int64_t r1 = std::min<int64_t>(d.n, r0 + rows_w);
            launch_refine_w(b, t, d.n, sigma, r0, r1, W64, s);
            launch_refine_rows(b, t, r0, r1, W64, dlist, nflag, part, spart, s);
            launches += 2;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            launch_refine_finish(b, t, dlist, nflag, part, spart, ntiles, s);
            launches += 1;
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host lists stay valid until here
    if (e != cudaSuccess) return fail(EPT_ECUDA, "recomputation of flagged statistics failed: %s", cudaGetErrorString(e));
    // large scratch (an FP64 rebuild's window) is not kept between calls
    if (c->refine_cap > ((size_t)256 << 20)) {
        device_free(c, c->refine_buf, s);
        c->refine_buf = nullptr;
        c->refine_cap = 0;
    }
    // counts and outputs again, read back as in the run
    launch_reset_counts(b, s);
    launch_combine_count(b, s);
    CK(cudaGetLastError());
    uint8_t *pin = c->pinned;
    CK(cudaMemcpyAsync(pin + S.res_ctr, b.ctr, sizeof(Counters) * P.n_tests, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pin + S.res_obs, b.observed, 8 * (size_t)P.n_tests, cudaMemcpyDeviceToHost, s));
    if (P.host_in) CK(cudaMemcpyAsync(pin + S.res_stats, b.stats, 8 * (size_t)P.nstats, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const ept_status st2 = collect(c, P, specs, out, timed, per_test);
    for (int t = 0; st2 == EPT_OK && t < P.n_tests; ++t) out[t].refine_launches = launches;
    return st2;
}

// One run of a batch: plan, stage, enqueue (or replay a captured graph), wait, collect.
ept_status run_once(ept_ctx *c, const std::vector<TestSpec> &specs, int prec, bool on_device, const Tuning &tn,
                    bool use_graph, ept_result *out, void *stream, float *device_ms) {
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    ept_status st0 = EPT_OK;
    const int chunk_kb = tn.chunk_kb;
    std::vector<int64_t> pkey = shape_key(specs, prec, on_device);
    pkey.push_back(tn.code());
    pkey.push_back(c->debug ? 1 : 0);
    if (!c->plan) {
        c->plan = new (std::nothrow) Plan();
        if (!c->plan) return fail(EPT_ENOMEM, "host allocation failed");
    }
    if (c->plan_key != pkey) {
        plan_batch(*c->plan, specs, prec, !on_device, chunk_kb, c->num_sms, c->debug, true, tn.order,
                   (tn.kernel ? tn.kernel : contraction_kernel(c)) == 2);
        c->plan->draw_mode = tn.draw_mode;
        c->plan->contraction = tn.kernel;
        c->plan_key = pkey;
        c->tables_staged = false;
        if (c->debug && (st0 = check_plan(*c->plan)) != EPT_OK) {
            c->plan_key.clear();
            return st0;
        }
    }
    Plan &P = *c->plan;
    for (int t = 0; t < P.n_tests; ++t) set_test_params(P.desc[t], specs[t]);
    NvtxRange range(use_graph && c->graphs ? "ept.run (graph)" : "ept.run");
    if (injected_failure(c)) return fail(EPT_ENOMEM, "device scratch not available (injected failure)");
    ept_status st = ensure_arena(c, P.total, s);
    if (st != EPT_OK) return st;
    const Staging S = staging_layout(P);
    if ((st = ensure_pinned(c, S.total)) != EPT_OK) return st;
    if (s != c->stream) CK(cudaStreamSynchronize(c->stream));
    stage_host(c, P, specs, on_device, !c->tables_staged);
    c->tables_staged = true;
    if (c->inject_stall) use_graph = false;   // one direct run with the hook, never captured
    if (use_graph && c->graphs) {
        // the graph runs on the context's stream, after the caller's stream's prior work
        if (s != c->stream) {
            CK(cudaEventRecord(c->ev_user, s));
            CK(cudaStreamWaitEvent(c->stream, c->ev_user, 0));
            s = c->stream;
        }
        std::vector<int64_t> key = shape_key(specs, prec, on_device);
        key.push_back(tn.code());
        key.push_back(c->debug ? 1 : 0);
        if (!(c->graph.exec && c->graph.key == key && c->graph.arena == c->arena)) {
            drop_graph(c);
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            st = enqueue_device(c, P, s, false, false);
            const cudaError_t e_end = cudaStreamEndCapture(s, &g);
            if (st != EPT_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e_end != cudaSuccess) return fail(EPT_ECUDA, "graph capture failed: %s", cudaGetErrorString(e_end));
            cudaGraphExec_t ex = nullptr;
            const cudaError_t e_in = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e_in != cudaSuccess) return fail(EPT_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e_in));
            c->graph.exec = ex;
            c->graph.key = key;
            c->graph.arena = c->arena;
        }
        CK(cudaEventRecord(c->ev[0], s));
        if ((st = enqueue_uploads(c, P, s)) != EPT_OK) return st;   // the graph waits for ev_in
        CK(cudaGraphLaunch(c->graph.exec, s));
        CK(cudaEventRecord(c->ev[4], s));
        CK(cudaStreamSynchronize(s));
        if ((st = collect(c, P, specs, out, false)) != EPT_OK) return st;
        if ((st = refine_after(c, P, specs, out, false, s)) != EPT_OK) return st;
        for (int t = 0; t < P.n_tests; ++t) out[t].tuning = tn.code();
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[4]);
        for (int t = 0; t < P.n_tests; ++t) out[t].ms_total = ms;
        if (device_ms) *device_ms = ms;
        return EPT_OK;
    }
    st = enqueue_device(c, P, s, true);
    c->inject_stall = false;   // the hook is one-shot
    if (st != EPT_OK) return st;
    CK(cudaStreamSynchronize(s));
    if ((st = collect(c, P, specs, out, true)) != EPT_OK) return st;
    const auto r0 = std::chrono::steady_clock::now();
    if ((st = refine_after(c, P, specs, out, true, s)) != EPT_OK) return st;
    if (device_ms) {
        // the whole run on the device, and the recomputation of flagged statistics (its
        // wall time: it waits for its own work)
        cudaEventElapsedTime(device_ms, c->ev[0], c->ev[4]);
        *device_ms += std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - r0).count();
    }
    for (int t = 0; t < P.n_tests; ++t) out[t].tuning = tn.code();
    return EPT_OK;
}

// Contraction chunk length for this batch shape: from the cache, or (first time)
// by timing the contraction with each candidate on this very batch.  Each tuning
// run is a complete, correct test, so the last one's results are returned when it
// is the one chosen.
// Contraction unit length (K-blocks) of a context's untuned runs: the default, or the
// context's precision limit when that is shorter.
int unit_kb(const ept_ctx *c) { return c->unit_kb ? c->unit_kb : std::min(CHUNK_KB_DEFAULT, c->max_chunk); }

Tuning default_tuning(const ept_ctx *c) {
    Tuning tn;
    tn.chunk_kb = unit_kb(c);
    return tn;
}

// batches worth timing several parameter sets on their first call: several tests,
// or a test whose contraction is long enough for the choice to show
// (n^2 B >= 2.5e10: the high-dimensional ED workload has 2.5e11)
bool worth_tuning(const std::vector<TestSpec> &specs) {
    if (specs.size() >= 2) return true;
    const double n = (double)(specs[0].nx + specs[0].ny);
    return n * n * (double)specs[0].B >= 2.5e10;
}

// Parameters for this batch shape (tensor-core path): from the cache, or (first call
// of the shape) by timing whole device runs with each candidate on this very batch:
// the defaults; the other relabeling-draw kernel; the other unit order; units of 4
// K-blocks; and longer units where EPT_OPT_MAX_CHUNK allows them.  Every candidate
// run is a complete, correct test; the chosen one is run once more for the results
// (a captured graph when graphs are on).
ept_status run_tuned(ept_ctx *c, const std::vector<TestSpec> &specs, int prec, bool on_device, bool use_graph,
                     ept_result *out, void *stream) {
    const Tuning def = default_tuning(c);
    if (!c->autotune || prec != EPT_PREC_SPLIT_BF16 || !worth_tuning(specs)) {
        ept_status st = run_once(c, specs, prec, on_device, def, use_graph, out, stream, nullptr);
        for (size_t t = 0; st == EPT_OK && t < specs.size(); ++t) out[t].tune_candidates = 0;
        return st;
    }
    const std::vector<int64_t> key = tune_key(specs, prec, 64 * c->max_chunk + c->unit_kb);
    auto it = c->tuned.find(key);
    if (it != c->tuned.end()) {
        ept_status st = run_once(c, specs, prec, on_device, it->second, use_graph, out, stream, nullptr);
        for (size_t t = 0; st == EPT_OK && t < specs.size(); ++t) out[t].tune_candidates = 0;
        return st;
    }
    // the automatic choices of this batch, and their alternatives
    int64_t cols = 0;
    bool big_masks = false, user_masks = false;
    for (const TestSpec &sp : specs) {
        const int64_t Bp = (sp.B + 1 + COL_PAD - 1) / COL_PAD * COL_PAD;
        const int64_t nw = (sp.nx + sp.ny + PANEL - 1) / PANEL * (PANEL / 32);
        cols += Bp;
        big_masks |= nw * Bp * 4 > MASKS_IN_L2_BYTES;
        user_masks |= sp.user_masks != nullptr;
    }
    const int auto_draw = cols >= DRAW_LANES_MIN_COLS_PER_SM * (int64_t)c->num_sms ? DRAW_LANES : DRAW_WARPS;
    std::vector<Tuning> cand(1, def);
    if (!user_masks && c->draw_mode == 0) {
        Tuning t = def;
        t.draw_mode = auto_draw == DRAW_LANES ? DRAW_WARPS : DRAW_LANES;
        cand.push_back(t);
    }
    {
        Tuning t = def;
        t.order = big_masks ? 1 : 2;
        cand.push_back(t);
    }
    for (int kb : {4, 16, 32})
        if (kb != def.chunk_kb && kb <= c->max_chunk && c->unit_kb == 0) {
            Tuning t = def;
            t.chunk_kb = kb;
            cand.push_back(t);
        }
    // the MMA shape: pairs of SMs (M = 256 across a cluster) and relabelings as the
    // tensor-memory operand (N = 128), unless the context fixes the kernel
    if (c->contraction == 0)
        for (int k : {2, 3}) {
            Tuning t = def;
            t.kernel = k;
            cand.push_back(t);
        }
    Tuning best = def;
    float best_ms = 1e30f;
    for (const Tuning &tn : cand) {
        float ms = 0.f;
        ept_status st = run_once(c, specs, prec, on_device, tn, false, out, stream, &ms);
        if (st != EPT_OK) return st;
        if (ms < best_ms) {
            best_ms = ms;
            best = tn;
        }
    }
    c->tuned[key] = best;
    save_tune_file(c);
    ept_status st = run_once(c, specs, prec, on_device, best, use_graph, out, stream, nullptr);
    for (size_t t = 0; st == EPT_OK && t < specs.size(); ++t) out[t].tune_candidates = (int64_t)cand.size();
    return st;
}

// ---------------------------------------------------------------------------
// Streaming mode (EPT_OPT_STREAM_BLOCKS): one test whose packed blocks do not fit
// in device memory runs one window of row panels at a time, in two passes (the
// first for the exact row sums; ept_stream.cu).  The test's tables are those of a
// resident run (plan_batch, without the contraction schedule: a window's units are
// strided over the grid); each window sees the test through its own descriptor,
// whose block offset maps the window's blocks to the start of the window's memory.

// device bytes of one stored block in a window: its FP32 entries (the FP16 parts
// are written over them) and its row and column sums
constexpr size_t STREAM_BLK_BYTES = (size_t)PANEL * KB * 4 + (size_t)PANEL * 8 + (size_t)KB * 8;

// device bytes of a resident run of one test, without building its tables (the
// dominant terms of plan_batch's layout, rounded up)
size_t resident_bytes(const TestSpec &s, int prec) {
    const int64_t n = s.nx + s.ny, n_pad = (n + PANEL - 1) / PANEL * PANEL, NP = n_pad / PANEL, NKB = n_pad / KB;
    const int64_t nblk = blk_off(NP, NKB), Bp = (s.B + 1 + COL_PAD - 1) / COL_PAD * COL_PAD;
    const int64_t p_pad = (s.p + BUILD_KB - 1) / BUILD_KB * BUILD_KB;
    const int64_t nchunks = nblk / 8 + NP;   // chunks of 8 K-blocks or more, one partial one per panel
    const bool tc = prec == EPT_PREC_SPLIT_BF16;
    size_t b = (size_t)nblk * (STREAM_BLK_BYTES + sizeof(BlkInfo) + sizeof(Tile));
    b += (size_t)nchunks * (sizeof(Chunk) + 2 * (size_t)Bp * 4 + 2 * (size_t)(Bp / TC_TILE_N) * 8);
    b += (size_t)n_pad * (4 * 3 + 8 * 4 + (tc ? 4 * (size_t)p_pad : 0));
    b += (size_t)(n_pad / 32) * Bp * 4 + (size_t)Bp * 8;
    b += (size_t)n * s.p * 4 + (s.user_masks ? (size_t)s.B * ((n + 31) / 32) * 4 : 0);
    return b + ((size_t)1 << 20);
}

// device memory a run may take: the context budget, else what is free plus the
// context's own arena, less a margin (3 %, at least 2 GiB) for everything else
size_t available_bytes(ept_ctx *c) {
    if (c->budget) return c->budget;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const size_t have = fr + c->arena_cap;
    const size_t margin = std::max<size_t>((size_t)2 << 30, have / 33);
    return have > margin ? have - margin : 0;
}

// whether a single test runs in the streaming mode.  The free memory is asked of
// the CUDA driver only for tests near the device's size: the query costs tens of
// microseconds, and most tests need a small fraction of the memory.
bool use_stream(ept_ctx *c, const TestSpec &s, int prec) {
    if (c->stream_blocks < 0) return false;
    if (c->stream_blocks > 0) return true;
    if (prec != EPT_PREC_SPLIT_BF16 || (s.stat != EPT_STAT_ED && s.sigma == EPT_SIGMA_MEDIAN)) return false;
    const size_t need = resident_bytes(s, prec);
    if (c->budget) return need > c->budget;
    if (need <= c->arena_cap || need <= c->total_mem / 4) return false;
    return need > available_bytes(c);
}

// Windows of consecutive row panels: a panel joins the current window while the
// window stays within limit_blk stored blocks and limit_bytes of device memory (a
// window holds at least one panel).  Fills the per-window fields of P.
void stream_partition(Plan &P, int64_t limit_blk, size_t limit_bytes) {
    const TestDesc &d = P.desc[0];
    const int64_t NP = d.NP;
    std::vector<int64_t> cfirst((size_t)NP + 1, 0), tfirst((size_t)NP + 1, 0);
    int64_t q = 0;
    for (int64_t I = 0; I < NP; ++I) {
        cfirst[(size_t)I] = q;
        while (q < (int64_t)P.chunks.size() && P.chunks[(size_t)q].I == I) ++q;
        tfirst[(size_t)I + 1] = tfirst[(size_t)I] + 2 * (NP - I);
    }
    cfirst[(size_t)NP] = q;
    P.gdesc.clear();
    P.gI0.clear();
    P.gI1.clear();
    P.gblk0.clear();
    P.gnblk.clear();
    P.gtile0.clear();
    P.gntile.clear();
    P.gpre.clear();
    P.win_blk = P.win_part = 0;
    int64_t I = 0;
    while (I < NP) {
        const int64_t I0 = I;
        int64_t blocks = 0;
        size_t bytes = 0;
        while (I < NP) {
            const int64_t nb = d.NKB - KB_PER_PANEL * I, nc = cfirst[(size_t)I + 1] - cfirst[(size_t)I];
            const size_t add = (size_t)nb * STREAM_BLK_BYTES + (size_t)(2 * nc * d.Bp) * 4;
            if (I > I0 && (blocks + nb > limit_blk || bytes + add > limit_bytes)) break;
            blocks += nb;
            bytes += add;
            ++I;
        }
        TestDesc g = d;
        g.blk0 = -blk_off(I0, d.NKB);
        g.chunk0 = cfirst[(size_t)I0];
        g.nchunks = cfirst[(size_t)I] - cfirst[(size_t)I0];
        g.nparts = 2 * g.nchunks;
        g.part0 = 0;
        P.gdesc.push_back(g);
        P.gI0.push_back(I0);
        P.gI1.push_back(I);
        P.gblk0.push_back(blk_off(I0, d.NKB));
        P.gnblk.push_back(blocks);
        P.gtile0.push_back(tfirst[(size_t)I0]);
        P.gntile.push_back(tfirst[(size_t)I] - tfirst[(size_t)I0]);
        P.gpre.push_back(0);
        P.gpre.push_back(tc_units(g));
        P.win_blk = std::max(P.win_blk, blocks);
        P.win_part = std::max(P.win_part, g.nparts * d.Bp);
    }
}

// Arena layout of a streaming run: the test's tables as plan_batch laid them out,
// the windows' descriptors and unit prefixes, the per-row and per-relabeling arrays
// of the whole test, then the window (blocks, their sums, the partials).
// Debug checks: a guard band after every data region (the tables are uploaded whole).
struct LayoutCursor {
    Plan &P;
    size_t o;
    bool in_data = false;
    size_t take(size_t bytes) {
        const size_t at = o;
        o = align_up(o + std::max<size_t>(bytes, 1), 256);
        if (P.debug && in_data && P.guards.n < MAX_GUARDS) {
            P.guards.off[P.guards.n++] = o;
            o += GUARD_BYTES;
        }
        return at;
    }
    void start_data() {   // after the tables: a band right away, then one after each region
        o = align_up(o, 1024);
        in_data = true;
        if (P.debug && P.guards.n < MAX_GUARDS) {
            P.guards.off[P.guards.n++] = o;
            o += GUARD_BYTES;
        }
    }
};

void stream_layout(Plan &P, size_t tab_bytes_resident) {
    const TestDesc &d = P.desc[0];
    P.guards.n = 0;
    P.off_errest = P.off_flags = 0;   // no FP64 refinement in the streaming mode
    LayoutCursor L{P, tab_bytes_resident};
    auto take = [&](size_t bytes) { return L.take(bytes); };
    P.off_gdesc = take(sizeof(TestDesc) * P.gdesc.size());
    P.off_gpre = take(8 * P.gpre.size());
    P.tab_bytes = L.o;
    L.start_data();
    P.off_in = take(P.in_bytes);
    P.off_norms = take((size_t)P.nrows * 4);
    P.off_iscale = take((size_t)P.nrows * 4);
    P.off_u = take((size_t)P.nrows * 4);
    P.off_Zh = take((size_t)P.nrows * P.p_stride * 2);
    P.off_Zl = take((size_t)P.nrows * P.p_stride * 2);
    P.off_r = take((size_t)P.nrows * 8);
    P.off_Spart = take((size_t)(P.nrows / 32) * 8);
    P.off_dcorr = take((size_t)P.nrows * 8);
    P.off_Upart = take((size_t)P.npan * 8);
    P.off_Stpart = take((size_t)P.npan * 8);
    P.off_maskT = take((size_t)P.nmask * 4);
    P.off_sacc = take((size_t)d.Bp * 8);
    P.off_stats = take((size_t)P.nstats * 8);
    P.off_observed = take(8);
    P.off_ctr = take(sizeof(Counters));
    P.off_D = take((size_t)P.win_blk * PANEL * KB * 4);
    P.off_Chi = P.off_D;
    P.off_rowpart = take((size_t)P.win_blk * PANEL * 8);
    P.off_colpart = take((size_t)P.win_blk * KB * 8);
    P.off_partial = take((size_t)P.win_part * 4);
    P.total = L.o;
}

// Debug checks on the host: the windows of a streaming plan cover the panels in
// order, once, within the window's capacity.
ept_status check_stream_plan(const Plan &P) {
    auto bad = [](const char *what) { return fail(EPT_EINTERNAL, "debug checks: streaming plan broken: %s", what); };
    const TestDesc &d = P.desc[0];
    int64_t next = 0, tiles = 0;
    for (size_t g = 0; g < P.gI0.size(); ++g) {
        if (P.gI0[g] != next || P.gI1[g] <= P.gI0[g] || P.gI1[g] > d.NP) return bad("panel ranges");
        next = P.gI1[g];
        if (P.gblk0[g] != blk_off(P.gI0[g], d.NKB) || P.gnblk[g] != blk_off(P.gI1[g], d.NKB) - P.gblk0[g])
            return bad("block ranges");
        if (P.gnblk[g] > P.win_blk || P.gdesc[g].nparts * d.Bp > P.win_part) return bad("window capacity");
        if (P.gdesc[g].blk0 != -P.gblk0[g] || P.gdesc[g].part0 != 0) return bad("window offsets");
        if (P.gtile0[g] != tiles) return bad("tile ranges");
        tiles += P.gntile[g];
        for (int64_t q = 0; q < P.gdesc[g].nchunks; ++q) {
            const Chunk &ch = P.chunks[(size_t)(P.gdesc[g].chunk0 + q)];
            if (ch.I < P.gI0[g] || ch.I >= P.gI1[g]) return bad("chunks outside their window");
        }
    }
    if (next != d.NP || tiles != (int64_t)P.tiles.size()) return bad("coverage");
    for (int k = 0; k < P.guards.n; ++k)
        if (P.guards.off[k] + GUARD_BYTES > P.total || P.guards.off[k] % 256) return bad("guard band");
    return EPT_OK;
}

// device view of a streaming run: the whole test (g < 0) or window g
Batch stream_view(ept_ctx *c, const Plan &P, int g) {
    uint8_t *A = c->arena;
    Batch b;
    memset(&b, 0, sizeof(b));
    b.n_tests = 1;
    b.desc = g < 0 ? (const TestDesc *)(A + P.off_desc) : (const TestDesc *)(A + P.off_gdesc) + g;
    b.pre.rows = (const int64_t *)(A + P.off_pre_rows);
    b.pre.panels = (const int64_t *)(A + P.off_pre_panels);
    b.pre.cols = (const int64_t *)(A + P.off_pre_cols);
    b.pre.units = g < 0 ? (const int64_t *)(A + P.off_pre_units) : (const int64_t *)(A + P.off_gpre) + 2 * g;
    b.pre.simt = (const int64_t *)(A + P.off_pre_simt);
    b.blk = (const BlkInfo *)(A + P.off_blk) + (g < 0 ? 0 : P.gblk0[(size_t)g]);
    b.tiles = (const Tile *)(A + P.off_tiles) + (g < 0 ? 0 : P.gtile0[(size_t)g]);
    b.chunks = (const Chunk *)(A + P.off_chunks);
    b.nblk_total = g < 0 ? 0 : P.gnblk[(size_t)g];
    b.ntiles = g < 0 ? 0 : P.gntile[(size_t)g];
    b.nrows_total = P.nrows;
    b.npan_total = P.npan;
    b.ncols_total = P.ncols_pad;
    b.nunits_total = g < 0 ? 0 : P.gpre[2 * (size_t)g + 1];
    b.p_stride = P.p_stride;
    b.norms = (float *)(A + P.off_norms);
    b.iscale = (float *)(A + P.off_iscale);
    b.u = (float *)(A + P.off_u);
    b.Zh = (uint16_t *)(A + P.off_Zh);
    b.Zl = (uint16_t *)(A + P.off_Zl);
    b.Chi = (uint16_t *)(A + P.off_D);
    b.Clo = b.Chi + (size_t)PANEL * KB;
    b.c_stride = 2 * (int64_t)PANEL * KB;
    b.D = (float *)(A + P.off_D);
    b.partial = (float *)(A + P.off_partial);
    b.rowpart = (double *)(A + P.off_rowpart);
    b.colpart = (double *)(A + P.off_colpart);
    b.r = (double *)(A + P.off_r);
    b.Spart = (double *)(A + P.off_Spart);
    b.dcorr = (double *)(A + P.off_dcorr);
    b.Upart = (double *)(A + P.off_Upart);
    b.Stpart = (double *)(A + P.off_Stpart);
    b.stats = (double *)(A + P.off_stats);
    b.observed = (double *)(A + P.off_observed);
    b.maskT = (uint32_t *)(A + P.off_maskT);
    b.ctr = (Counters *)(A + P.off_ctr);
    b.sacc = (double *)(A + P.off_sacc);
    b.inject_stall = (g == 0 && c->inject_stall) ? 1 : 0;
    b.wait_ns = c->wait_ns;
    return b;
}

ept_status run_stream(ept_ctx *c, const std::vector<TestSpec> &specs, int prec, bool on_device, ept_result *out,
                      void *stream) {
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const TestSpec &sp = specs[0];
    if (prec != EPT_PREC_SPLIT_BF16) return fail(EPT_EUNSUPPORTED, "the streaming mode runs the split precision only");
    if (sp.stat != EPT_STAT_ED && sp.sigma == EPT_SIGMA_MEDIAN)
        return fail(EPT_EUNSUPPORTED, "the streaming mode needs a given sigma (the median heuristic selects over "
                                      "every pooled distance before the first window)");
    NvtxRange range("ept.run (streaming)");
    std::unique_ptr<Plan> hold(new (std::nothrow) Plan());
    if (!hold) return fail(EPT_ENOMEM, "host allocation failed");
    Plan &P = *hold;
    plan_batch(P, specs, prec, !on_device, unit_kb(c), c->num_sms, c->debug, false);
    P.stream = true;
    const size_t tab0 = P.tab_bytes;
    const TestDesc &d = P.desc[0];
    const size_t panel0 = (size_t)d.NKB * STREAM_BLK_BYTES;
    if (c->stream_blocks > 0) {
        stream_partition(P, c->stream_blocks, SIZE_MAX);
        stream_layout(P, tab0);
    } else {
        const size_t avail = available_bytes(c);
        stream_partition(P, INT64_MAX, panel0);   // the smallest windows: the fixed part of the layout
        stream_layout(P, tab0);
        const size_t win0 = (size_t)P.win_blk * STREAM_BLK_BYTES + (size_t)P.win_part * 4;
        const size_t fixed = P.total - std::min(P.total, win0);
        if (fixed + win0 > avail)
            return fail(EPT_ENOMEM, "the streaming mode needs %zu bytes of device memory for one panel, %zu are "
                                    "available", fixed + win0, avail);
        size_t wb = avail - fixed;
        for (;;) {
            stream_partition(P, INT64_MAX, wb);
            stream_layout(P, tab0);
            if (P.total <= avail || wb <= win0) break;
            wb = std::max(win0, wb / 10 * 9);
        }
        if (P.total > avail)
            return fail(EPT_ENOMEM, "the streaming mode needs %zu bytes of device memory, %zu are available", P.total,
                        avail);
    }
    // Within each window, chunks in order of their first K-block (then panel): a
    // window's units are strided over the grid, so the units in flight together then
    // cover nearby K-ranges of all the window's panels and share the relabeling-mask
    // words of those columns in L2.  In panel order they span many K-ranges, and once
    // the masks outgrow L2 (n of about 50,000 at B = 10^4) every unit read its mask
    // words from DRAM (measured: 1.9 times the algorithmic bytes at n = 60,000).
    for (size_t g = 0; g < P.gdesc.size(); ++g) {
        auto first = P.chunks.begin() + P.gdesc[g].chunk0;
        std::stable_sort(first, first + P.gdesc[g].nchunks,
                         [](const Chunk &a, const Chunk &b) { return a.kb0 < b.kb0; });
    }
    if (c->debug) {
        ept_status st0 = check_plan(P);
        if (st0 == EPT_OK) st0 = check_stream_plan(P);
        if (st0 != EPT_OK) return st0;
    }
    if (injected_failure(c)) return fail(EPT_ENOMEM, "device scratch not available (injected failure)");
    ept_status st = ensure_arena(c, P.total, s, true);
    if (st != EPT_OK) return st;
    const Staging S = staging_layout(P);
    if ((st = ensure_pinned(c, S.total)) != EPT_OK) return st;
    if (s != c->stream) CK(cudaStreamSynchronize(c->stream));
    stage_host(c, P, specs, on_device, true);
    c->tables_staged = false;   // the pinned tables now hold this run's; the cached plan's are staged again
    for (TestDesc &g : P.gdesc) {   // the device addresses of the inputs, as staged
        g.X = P.desc[0].X;
        g.Y = P.desc[0].Y;
        g.user_masks = P.desc[0].user_masks;
        g.out_stats = P.desc[0].out_stats;
    }
    uint8_t *tab = c->pinned + S.tables;
    memcpy(tab + P.off_gdesc, P.gdesc.data(), sizeof(TestDesc) * P.gdesc.size());
    memcpy(tab + P.off_gpre, P.gpre.data(), 8 * P.gpre.size());

    const Batch bf = stream_view(c, P, -1);
    CK(cudaEventRecord(c->ev[0], s));
    if ((st = enqueue_uploads(c, P, s)) != EPT_OK) return st;
    CK(cudaMemsetAsync(bf.ctr, 0, sizeof(Counters), s));
    if (P.debug) launch_guards(c->arena, P.guards, false, bf.ctr, s);
    CK(cudaMemsetAsync(bf.r, 0, (size_t)P.nrows * 8, s));
    CK(cudaMemsetAsync(bf.sacc, 0, (size_t)d.Bp * 8, s));
    CK(cudaEventRecord(c->ev[1], s));
    // relabeling draws on the side stream, beside the first pass
    CK(cudaStreamWaitEvent(c->side, c->ev[1], 0));
    CK(cudaEventRecord(c->ev_side[1], c->side));
    launch_masks(bf, c->num_sms, draw_mode_for(c, P), c->side);
    CK(cudaGetLastError());
    CK(cudaEventRecord(c->ev_side[2], c->side));
    CK(cudaStreamWaitEvent(s, c->ev_in, 0));
    launch_split_rows(bf, s);
    CK(cudaGetLastError());
    alignas(64) CUtensorMap tm[4];
    alignas(64) CUtensorMap th, tl;
    char emsg[160];
    if (!encode_rows_tmaps(tm, bf.Zh, bf.Zl, P.nrows, P.p_stride, emsg, sizeof(emsg)))
        return fail(EPT_ECUDA, "%s", emsg);
    if (!encode_block_tmaps(&th, &tl, bf.Chi, bf.Clo, P.win_blk, bf.c_stride, emsg, sizeof(emsg)))
        return fail(EPT_ECUDA, "%s", emsg);
    const int nwin = (int)P.gI0.size();
    const int ntimed = std::min(nwin, 64);
    while ((int)c->ev_win.size() < 2 * ntimed) {
        cudaEvent_t e = nullptr;
        CK(cudaEventCreate(&e));
        c->ev_win.push_back(e);
    }
    // pass 1: the row sums r (and max |D| for the FP16 scale)
    for (int g = 0; g < nwin; ++g) {
        const Batch gv = stream_view(c, P, g);
        CK(launch_build_tc(gv, tm, c->num_sms, s));
        launch_blocksums(gv, s);
        launch_stream_rowsums(gv, P.gI0[(size_t)g], P.gI1[(size_t)g], d.n_pad, s);
        CK(cudaGetLastError());
    }
    // the resident path's centring: u, r~, the diagonal fold, S~
    launch_stream_spart(bf, s);
    launch_center(bf, s);
    CK(cudaGetLastError());
    CK(cudaStreamWaitEvent(s, c->ev_side[2], 0));
    CK(cudaEventRecord(c->ev[2], s));
    // pass 2: build again, pack, contract, fold the partials
    for (int g = 0; g < nwin; ++g) {
        const Batch gv = stream_view(c, P, g);
        CK(launch_build_tc(gv, tm, c->num_sms, s));
        launch_pack(gv, true, s);
        CK(cudaGetLastError());
        if (g < ntimed) CK(cudaEventRecord(c->ev_win[2 * (size_t)g], s));
        CK(launch_contract_tc(gv, &th, &tl, c->num_sms, s));
        if (g < ntimed) CK(cudaEventRecord(c->ev_win[2 * (size_t)g + 1], s));
        launch_stream_accum(gv, s);
        CK(cudaGetLastError());
    }
    launch_stream_stats(bf, s);
    launch_combine_count(bf, s);
    CK(cudaGetLastError());
    if (P.debug) launch_guards(c->arena, P.guards, true, bf.ctr, s);
    CK(cudaEventRecord(c->ev[3], s));
    CK(cudaMemcpyAsync(c->pinned + S.res_ctr, bf.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->pinned + S.res_obs, bf.observed, 8, cudaMemcpyDeviceToHost, s));
    if (P.host_in) CK(cudaMemcpyAsync(c->pinned + S.res_stats, bf.stats, 8 * (size_t)P.nstats, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(c->ev[4], s));
    c->inject_stall = false;   // the hook is one-shot
    CK(cudaStreamSynchronize(s));
    if ((st = collect(c, P, specs, out, false)) != EPT_OK) return st;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[4]);
    out[0].ms_total = ms;
    // phases: row split + pass 1 + centring (build), pass 2 + combination (perm), the
    // draws, and the contraction launches (summed; 0 beyond 64 windows)
    cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]);
    out[0].ms_build = ms;
    cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);
    out[0].ms_perm = ms;
    cudaEventElapsedTime(&ms, c->ev_side[1], c->ev_side[2]);
    out[0].ms_masks = ms;
    double con = 0.0;
    for (int g = 0; g < ntimed; ++g) {
        cudaEventElapsedTime(&ms, c->ev_win[2 * (size_t)g], c->ev_win[2 * (size_t)g + 1]);
        con += ms;
    }
    out[0].ms_contract = nwin <= 64 ? con : 0.0;
    return EPT_OK;
}

// ---------------------------------------------------------------------------
// Pre-computation baseline (EPT_PREC_POOLED_FP32, Algorithm 5; kernels in
// ept_pooled.cu).  The test's descriptor comes from plan_batch (its tables are not
// used); the relabelings mark x* (no complement).  Arena: the tables, the inputs,
// W (n_pad x n_pad FP32), the masks, the per-chunk sums, the statistics.
void pooled_layout(Plan &P, int num_sms) {
    const TestDesc &d = P.desc[0];
    P.guards.n = 0;
    P.off_errest = P.off_flags = 0;   // the baseline has no error estimate
    LayoutCursor L{P, P.tab_bytes};
    auto take = [&](size_t bytes) { return L.take(bytes); };
    L.start_data();
    P.off_in = take(P.in_bytes);
    P.off_D = take((size_t)d.n_pad * d.n_pad * 4);
    P.off_maskT = take((size_t)P.nmask * 4);
    P.win_part = pooled_row_chunks(d.n, d.ncols, num_sms);   // row chunks of the sums
    P.off_partial = take((size_t)P.win_part * 3 * d.ncols * 8);
    P.off_stats = take((size_t)P.nstats * 8);
    P.off_observed = take(8);
    P.off_ctr = take(sizeof(Counters));
    P.total = L.o;
}

void plan_pooled(Plan &P, const std::vector<TestSpec> &specs, bool host_in, int num_sms, bool debug = false) {
    plan_batch(P, specs, EPT_PREC_PLAIN_FP32, host_in, CHUNK_KB_DEFAULT, num_sms, debug, false);
    TestDesc &d = P.desc[0];
    d.comp = 0;   // the relabelings mark x*
    d.m = d.nx;
    d.other = d.ny;
    pooled_layout(P, num_sms);
}

ept_status run_pooled(ept_ctx *c, const std::vector<TestSpec> &specs, bool on_device, ept_result *out, void *stream) {
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    NvtxRange range("ept.run (pooled baseline)");
    std::unique_ptr<Plan> hold(new (std::nothrow) Plan());
    if (!hold) return fail(EPT_ENOMEM, "host allocation failed");
    Plan &P = *hold;
    plan_pooled(P, specs, !on_device, c->num_sms, c->debug);
    if (injected_failure(c)) return fail(EPT_ENOMEM, "device scratch not available (injected failure)");
    ept_status st = ensure_arena(c, P.total, s);
    if (st != EPT_OK) return st;
    const Staging S = staging_layout(P);
    if ((st = ensure_pinned(c, S.total)) != EPT_OK) return st;
    if (s != c->stream) CK(cudaStreamSynchronize(c->stream));
    stage_host(c, P, specs, on_device, true);
    c->tables_staged = false;   // the pinned tables now hold this run's
    const TestDesc &d = P.desc[0];
    uint8_t *A = c->arena;
    Batch b;
    memset(&b, 0, sizeof(b));
    b.n_tests = 1;
    b.desc = (const TestDesc *)(A + P.off_desc);
    b.pre.rows = (const int64_t *)(A + P.off_pre_rows);
    b.pre.panels = (const int64_t *)(A + P.off_pre_panels);
    b.pre.cols = (const int64_t *)(A + P.off_pre_cols);
    b.ncols_total = P.ncols_pad;
    b.nrows_total = P.nrows;
    b.D = (float *)(A + P.off_D);
    b.maskT = (uint32_t *)(A + P.off_maskT);
    b.stats = (double *)(A + P.off_stats);
    b.observed = (double *)(A + P.off_observed);
    b.ctr = (Counters *)(A + P.off_ctr);
    double *part = (double *)(A + P.off_partial);

    CK(cudaEventRecord(c->ev[0], s));
    if ((st = enqueue_uploads(c, P, s)) != EPT_OK) return st;
    CK(cudaMemsetAsync(b.ctr, 0, sizeof(Counters), s));
    if (P.debug) launch_guards(c->arena, P.guards, false, b.ctr, s);
    CK(cudaEventRecord(c->ev[1], s));
    // the relabelings (Algorithm 5's SampleWithoutReplacement, the library's stream)
    // on the side stream, beside the matrix
    CK(cudaStreamWaitEvent(c->side, c->ev[1], 0));
    CK(cudaEventRecord(c->ev_side[1], c->side));
    launch_masks(b, c->num_sms, draw_mode_for(c, P), c->side);
    CK(cudaGetLastError());
    CK(cudaEventRecord(c->ev_side[2], c->side));
    CK(cudaStreamWaitEvent(s, c->ev_in, 0));
    CK(cudaStreamWaitEvent(s, c->ev_side[2], 0));
    CK(cudaEventRecord(c->ev[2], s));
    CK(launch_pooled(b, d.n, d.n_pad, d.ncols, part, P.win_part, d.nw, s));
    CK(cudaEventRecord(c->ev[3], s));
    launch_combine_count(b, s);
    CK(cudaGetLastError());
    if (P.debug) launch_guards(c->arena, P.guards, true, b.ctr, s);
    CK(cudaMemcpyAsync(c->pinned + S.res_ctr, b.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->pinned + S.res_obs, b.observed, 8, cudaMemcpyDeviceToHost, s));
    if (P.host_in) CK(cudaMemcpyAsync(c->pinned + S.res_stats, b.stats, 8 * (size_t)P.nstats, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(c->ev[4], s));
    CK(cudaStreamSynchronize(s));
    if ((st = collect(c, P, specs, out, false)) != EPT_OK) return st;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[4]);
    out[0].ms_total = ms;
    cudaEventElapsedTime(&ms, c->ev_side[1], c->ev_side[2]);
    out[0].ms_masks = ms;
    cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);
    out[0].ms_perm = ms;   // matrix and sums (the matrix and the extraction are one launch sequence)
    return EPT_OK;
}

// a single test: the pre-computation baseline when asked for; streamed when its
// blocks do not fit (or the option asks for it); else the resident path
ept_status run_single(ept_ctx *c, const std::vector<TestSpec> &specs, int prec, bool on_device, bool tuned,
                      ept_result *out, void *stream) {
    if (prec == EPT_PREC_POOLED_FP32) return run_pooled(c, specs, on_device, out, stream);
    if (use_stream(c, specs[0], prec)) return run_stream(c, specs, prec, on_device, out, stream);
    if (tuned) return run_tuned(c, specs, prec, on_device, true, out, stream);
    return run_once(c, specs, prec, on_device, default_tuning(c), false, out, stream, nullptr);
}

// ---------------------------------------------------------------------------
// Serving (continuous batching).  ept_submit copies a request and queues it.  A
// scheduler thread admits queued requests in arrival order while request slots
// and the device-memory budget allow, packs everything admitted into one batched
// run (all phases as grouped launches over the batch) and starts it on a free
// lane: an internal sub-context with its own streams and pinned staging, whose
// device scratch comes from the server's stream-ordered memory pool and goes back
// to it when the lane's work is done.  Several lanes run at once, so requests that
// arrive while others are on the GPU start in the next batch and overlap with
// them on the device.  A host callback at the end of each lane's work wakes the
// scheduler.
enum ReqState { REQ_PENDING = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_CANCELLED = 3 };

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    TestSpec spec;
    std::vector<float> X, Y;
    std::vector<double> stats;
    ept_result res;
    int prec = 0;
    int state = REQ_PENDING;
    bool cancel_req = false;
    ept_status status = EPT_OK;
    std::string err;
    size_t bytes = 0;   // device scratch of this request alone (admission estimate)
    Clock::time_point t_submit;
};

struct Lane {
    ept_ctx *ctx = nullptr;
    bool busy = false;
    std::vector<Request *> reqs;
    std::vector<TestSpec> specs;
    Plan plan;
    size_t bytes = 0;   // device scratch held by the lane's run
    uint8_t *arena = nullptr;
    cudaEvent_t done = nullptr;
};

struct Server {
    ept_ctx *owner = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::atomic<uint64_t> wakeups{0};
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> reqs;
    std::vector<Lane> lanes;
    cudaMemPool_t pool = nullptr;
    size_t budget = 0, in_use = 0;
    int max_slots = 256, slots = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    size_t max_pending = 1 << 16;
    int64_t peak_busy = 0;         // the most lanes that held a running batch at the same time
    int64_t submits_busy = 0;      // requests submitted while some lane held a running batch
};

void CUDART_CB lane_finished(void *arg) {
    Server *S = (Server *)arg;
    S->wakeups.fetch_add(1);
    S->cv_work.notify_all();   // no lock: the scheduler also wakes on a short timeout
}

// the lane's scratch back to the pool (or the caller's allocator), stream-ordered
// after the lane's work
ept_status lane_release(Server *S, Lane &L) {
    if (!L.arena) return EPT_OK;
    cudaStream_t s = L.ctx->stream;
    const ept_allocator &ua = S->owner->alloc;
    cudaError_t e = cudaSuccess;
    if (ua.alloc) ua.free(L.arena, (void *)s, ua.user);
    else e = cudaFreeAsync(L.arena, s);
    L.arena = nullptr;
    if (e != cudaSuccess) return fail(EPT_ECUDA, "cudaFreeAsync: %s", cudaGetErrorString(e));
    return EPT_OK;
}

ept_status lane_enqueue(Server *S, Lane &L) {
    ept_ctx *c = L.ctx;
    cudaStream_t s = c->stream;
    const Staging SL = staging_layout(L.plan);
    ept_status st = ensure_pinned(c, SL.total);
    if (st != EPT_OK) return st;
    NvtxRange range("ept.serve.batch");
    if (injected_failure(S->owner)) return fail(EPT_ENOMEM, "device scratch not available (injected failure)");
    void *mem = nullptr;
    ept_allocator &ua = S->owner->alloc;
    if (ua.alloc) {
        if ((st = device_alloc(S->owner, L.plan.total, s, &mem)) != EPT_OK) return st;
    } else {
        cudaError_t e = cudaMallocFromPoolAsync(&mem, L.plan.total, S->pool, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(EPT_ENOMEM, "device scratch of %zu bytes not available: %s", (size_t)L.plan.total,
                        cudaGetErrorString(e));
        }
    }
    L.arena = (uint8_t *)mem;
    c->arena = L.arena;   // the kernels and staging address the lane's scratch through the context
    c->arena_cap = L.plan.total;
    c->refine = S->owner->refine;
    c->contraction = S->owner->contraction;
    stage_host(c, L.plan, L.specs, false);
    st = enqueue_device(c, L.plan, s, false);
    c->arena = nullptr;
    c->arena_cap = 0;
    if (st != EPT_OK) {
        lane_release(S, L);
        return st;
    }
    // the scratch stays with the lane until its results (and any FP64 refinement)
    // have been collected
    CK(cudaEventRecord(L.done, s));
    CK(cudaLaunchHostFunc(s, lane_finished, S));
    return EPT_OK;
}

void finish_requests(Server *S, Lane &L, ept_status st, const std::string &msg, const ept_result *out,
                     const std::vector<TestError> *per_test) {
    const Clock::time_point now = Clock::now();
    for (size_t k = 0; k < L.reqs.size(); ++k) {
        Request *r = L.reqs[k];
        r->status = st;
        r->err = msg;
        if (st == EPT_OK && per_test && (*per_test)[k].st != EPT_OK) {
            r->status = (*per_test)[k].st;
            r->err = (*per_test)[k].msg;
        }
        if (r->status == EPT_OK) {
            r->res = out[k];
            r->res.ms_build = r->res.ms_perm = r->res.ms_masks = r->res.ms_contract = 0.f;
            r->res.ms_total = (float)std::chrono::duration<double, std::milli>(now - r->t_submit).count();
        }
        r->state = r->cancel_req ? REQ_CANCELLED : REQ_DONE;
        S->slots -= 1;
    }
    S->in_use -= L.bytes;
    L.bytes = 0;
    L.busy = false;
    L.reqs.clear();
    L.specs.clear();
    S->cv_done.notify_all();
}

// Takes the next batch from the queue for a free lane (lock held): requests of the
// first request's precision in arrival order, while slots and memory allow.  The
// batch's exact scratch size is planned; requests are handed back from the end
// until it fits.
bool form_batch(Server *S, Lane &L) {
    if (S->pending.empty()) return false;
    const int prec = S->pending.front()->prec;
    std::vector<Request *> batch;
    size_t est = 0;
    for (auto it = S->pending.begin(); it != S->pending.end();) {
        Request *r = *it;
        if (r->prec != prec) {
            ++it;
            continue;
        }
        if (S->slots + (int)batch.size() >= S->max_slots) break;
        if (S->in_use + est + r->bytes > S->budget) break;   // arrival order: no overtaking
        batch.push_back(r);
        est += r->bytes;
        it = S->pending.erase(it);
    }
    std::vector<TestSpec> specs;
    for (Request *r : batch) specs.push_back(r->spec);
    while (!batch.empty()) {
        plan_batch(L.plan, specs, prec, true, unit_kb(L.ctx), L.ctx->num_sms, false, true, 0,
                   contraction_kernel(S->owner) == 2);
        if (S->in_use + L.plan.total <= S->budget) break;
        // hand the last one back, at its place in arrival order
        Request *r = batch.back();
        batch.pop_back();
        specs.pop_back();
        auto pos = S->pending.begin();
        while (pos != S->pending.end() && (*pos)->ticket < r->ticket) ++pos;
        S->pending.insert(pos, r);
    }
    if (batch.empty()) return false;
    L.busy = true;
    int64_t busy = 0;
    for (const Lane &o : S->lanes) busy += o.busy ? 1 : 0;
    S->peak_busy = std::max(S->peak_busy, busy);
    L.reqs = batch;
    L.specs = specs;
    L.bytes = L.plan.total;
    S->in_use += L.bytes;
    S->slots += (int)batch.size();
    for (Request *r : batch) r->state = REQ_RUNNING;
    return true;
}

void serve_loop(Server *S, int device) {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        const uint64_t seen = S->wakeups.load();
        bool progressed = false;
        for (Lane &L : S->lanes) {
            if (!L.busy) continue;
            const cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaErrorNotReady) continue;
            std::vector<ept_result> out(L.reqs.size());
            std::vector<TestError> per_test;
            ept_status st = EPT_OK;
            // the lane stays busy (no other thread uses its state) while its results are
            // collected and its flagged statistics recomputed, without the server lock,
            // so that submissions and waits go on meanwhile
            lk.unlock();
            if (q != cudaSuccess) st = fail(EPT_ECUDA, "serving run failed: %s", cudaGetErrorString(q));
            else st = collect(L.ctx, L.plan, L.specs, out.data(), false, &per_test);
            if (st == EPT_OK) {
                L.ctx->arena = L.arena;
                L.ctx->arena_cap = L.plan.total;
                st = refine_after(L.ctx, L.plan, L.specs, out.data(), false, L.ctx->stream, &per_test);
                L.ctx->arena = nullptr;
                L.ctx->arena_cap = 0;
            }
            const std::string msg = st == EPT_OK ? std::string() : g_err;
            const ept_status rst = lane_release(S, L);
            if (st == EPT_OK && rst != EPT_OK) st = rst;
            lk.lock();
            finish_requests(S, L, st, st == EPT_OK ? msg : (msg.empty() ? g_err : msg), out.data(), &per_test);
            progressed = true;
        }
        bool any_busy = false;
        for (Lane &L : S->lanes) any_busy |= L.busy;
        if (S->stop && !any_busy) break;
        if (!S->stop) {
            for (Lane &L : S->lanes) {
                if (L.busy || !form_batch(S, L)) continue;
                lk.unlock();
                const ept_status st = lane_enqueue(S, L);
                const std::string msg = g_err;
                if (st != EPT_OK) cudaStreamSynchronize(L.ctx->stream);   // nothing of it stays in flight
                lk.lock();
                if (st != EPT_OK) finish_requests(S, L, st, msg, nullptr, nullptr);
                progressed = true;
            }
        }
        if (!progressed)
            S->cv_work.wait_for(lk, std::chrono::milliseconds(any_busy ? 1 : 50),
                                [S, seen] { return S->wakeups.load() != seen || S->stop; });
    }
}

ept_status serve_start(ept_ctx *c) {
    if (c->server) return EPT_OK;
    DeviceGuard dg(c->device);
    std::unique_ptr<Server> S(new (std::nothrow) Server());
    if (!S) return fail(EPT_ENOMEM, "host allocation failed");
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
    }
    S->owner = c;
    S->budget = c->budget ? c->budget : (size_t)(0.8 * (double)free_b);
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c->device;
    CK(cudaMemPoolCreate(&S->pool, &props));
    uint64_t keep = S->budget;   // freed scratch stays in the pool for the next batch
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    ept_status st = EPT_OK;
    S->max_slots = c->serve_slots;
    for (int k = 0; k < c->serve_lanes && st == EPT_OK; ++k) {
        Lane L;
        if ((st = ept_create(&L.ctx, c->device, 0)) != EPT_OK) break;
        L.ctx->autotune = false;
        L.ctx->alloc = c->alloc;   // the FP64 refinement's scratch comes from the caller's allocator too
        if (cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            ept_destroy(L.ctx);
            st = fail(EPT_ECUDA, "event creation failed");
            break;
        }
        S->lanes.push_back(L);
    }
    if (st != EPT_OK) {
        for (Lane &M : S->lanes) {
            cudaEventDestroy(M.done);
            ept_destroy(M.ctx);
        }
        cudaMemPoolDestroy(S->pool);
        return st;
    }
    S->th = std::thread(serve_loop, S.get(), c->device);
    c->server = S.release();
    return EPT_OK;
}

void serve_stop(ept_ctx *c) {
    Server *S = c->server;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (Request *r : S->pending) r->state = REQ_CANCELLED;
        S->pending.clear();
        S->cv_done.notify_all();
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    DeviceGuard dg(c->device);
    for (Lane &L : S->lanes) {
        cudaEventDestroy(L.done);
        ept_destroy(L.ctx);
    }
    cudaMemPoolDestroy(S->pool);
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
    c->server = nullptr;
}

}  // namespace

#define EPT_STR2(x) #x
#define EPT_STR(x) EPT_STR2(x)
#if defined(__aarch64__)
#define EPT_HOST_ARCH "aarch64"
#elif defined(__x86_64__)
#define EPT_HOST_ARCH "x86_64"
#else
#define EPT_HOST_ARCH "other"
#endif
#ifndef EPT_DEVICE_ARCH
#define EPT_DEVICE_ARCH unspecified
#endif

extern "C" {

int ept_abi_version(void) { return EPT_ABI_VERSION; }

const char *ept_build_info(void) {
    return "libept abi " EPT_STR(EPT_ABI_VERSION) "; host " EPT_HOST_ARCH "; device " EPT_STR(EPT_DEVICE_ARCH)
           "; nvcc " EPT_STR(__CUDACC_VER_MAJOR__) "." EPT_STR(__CUDACC_VER_MINOR__) "." EPT_STR(
               __CUDACC_VER_BUILD__) "; built " __DATE__ " " __TIME__;
}

const char *ept_last_error(void) { return g_err.c_str(); }

ept_status ept_create(ept_ctx **out, int device, size_t mem_budget_bytes) {
    return ept_create_ex(out, device, mem_budget_bytes, nullptr);
}

ept_status ept_create_ex(ept_ctx **out, int device, size_t mem_budget_bytes, const ept_allocator *alloc) {
    if (!out) return fail(EPT_EINVAL, "null output pointer");
    if (alloc && (!alloc->alloc != !alloc->free))
        return fail(EPT_EINVAL, "an allocator needs both alloc and free (or neither)");
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
    c->total_mem = prop.totalGlobalMem;
    c->budget = mem_budget_bytes;
    if (alloc) c->alloc = *alloc;
    c->autotune = true;
    const char *tf = getenv("EPT_AUTOTUNE_CACHE");
    if (tf) c->tune_file = tf;
    load_tune_file(c);
    DeviceGuard dg(device);
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    for (int k = 0; k < 7 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->ev[k]);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->ev_side[k]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_user, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        ept_destroy(c);
        return fail(EPT_ECUDA, "stream/event creation failed: %s", cudaGetErrorString(e));
    }
    // EPT_<OPTION> environment variables give the options' starting values
    static const struct {
        const char *env;
        int option;
    } env_opts[] = {{"EPT_GRAPHS", EPT_OPT_GRAPHS},           {"EPT_AUTOTUNE", EPT_OPT_AUTOTUNE},
                    {"EPT_DRAW_MODE", EPT_OPT_DRAW_MODE},     {"EPT_DEBUG_CHECKS", EPT_OPT_DEBUG_CHECKS},
                    {"EPT_STREAM_BLOCKS", EPT_OPT_STREAM_BLOCKS}, {"EPT_WAIT_LIMIT_MS", EPT_OPT_WAIT_LIMIT_MS},
                    {"EPT_MAX_CHUNK", EPT_OPT_MAX_CHUNK},     {"EPT_REFINE", EPT_OPT_REFINE},
                    {"EPT_CONTRACTION", EPT_OPT_CONTRACTION}, {"EPT_UNIT_KB", EPT_OPT_UNIT_KB},
                    {"EPT_SERVE_LANES", EPT_OPT_SERVE_LANES}, {"EPT_SERVE_SLOTS", EPT_OPT_SERVE_SLOTS}};
    for (const auto &eo : env_opts) {
        const char *v = getenv(eo.env);
        if (!v || !*v) continue;
        char *end = nullptr;
        const long long x = strtoll(v, &end, 10);
        if (end == v || *end || ept_set_option(c, eo.option, (int64_t)x) != EPT_OK) {
            const std::string msg = g_err;
            ept_destroy(c);
            return fail(EPT_EINVAL, "environment %s=%s: %s", eo.env, v,
                        end == v || *end ? "not an integer" : msg.c_str());
        }
    }
    *out = c;
    return EPT_OK;
}

ept_status ept_destroy(ept_ctx *c) {
    if (!c) return EPT_OK;
    serve_stop(c);
    {
        DeviceGuard dg(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        if (c->side) cudaStreamSynchronize(c->side);
        drop_graph(c);
        if (c->arena) device_free(c, c->arena, c->stream);
        if (c->refine_buf) device_free(c, c->refine_buf, c->stream);
        if (c->pinned) cudaFreeHost(c->pinned);
        delete c->plan;
        for (int k = 0; k < 7; ++k)
            if (c->ev[k]) cudaEventDestroy(c->ev[k]);
        for (int k = 0; k < 3; ++k)
            if (c->ev_side[k]) cudaEventDestroy(c->ev_side[k]);
        if (c->ev_user) cudaEventDestroy(c->ev_user);
        if (c->ev_in) cudaEventDestroy(c->ev_in);
        for (cudaEvent_t e : c->ev_win) cudaEventDestroy(e);
        if (c->copy) {
            cudaStreamSynchronize(c->copy);
            cudaStreamDestroy(c->copy);
        }
        if (c->side) cudaStreamDestroy(c->side);
        if (c->stream) cudaStreamDestroy(c->stream);
    }
    delete c;
    return EPT_OK;
}

size_t ept_estimate_bytes(int64_t nx, int64_t ny, int64_t p, int64_t B, int prec) {
    if (nx < 1 || ny < 1 || p < 1 || p > ((int64_t)1 << 30) || B < 0 || nx + ny > ((int64_t)1 << 22)) return 0;
    if (prec == EPT_PREC_POOLED_FP32) {
        Plan P;
        plan_pooled(P, one_test(nullptr, nx, nullptr, ny, p, 0, 1.0, B, 0, nullptr, nullptr), true, 148);
        return P.total;
    }
    if (prec != EPT_PREC_PLAIN_FP32 && prec != EPT_PREC_SPLIT_BF16) return 0;
    Plan P;
    plan_batch(P, one_test(nullptr, nx, nullptr, ny, p, 0, 1.0, B, 0, nullptr, nullptr), prec, true, 8);
    return P.total;
}

ept_status ept_plan_check(const int64_t *nx, const int64_t *ny, const int64_t *p, const int64_t *B, int n_tests,
                          int unit_kb, int num_sms, int64_t stream_blocks, ept_plan_info *out) {
    if (!nx || !ny || !p || !B || n_tests < 1) return fail(EPT_EINVAL, "null size arrays or n_tests < 1");
    if (unit_kb < 1 || unit_kb > 1024) return fail(EPT_EINVAL, "unit_kb must be in [1, 1024]");
    if (num_sms < 1 || num_sms > 4096) return fail(EPT_EINVAL, "num_sms must be in [1, 4096]");
    if (stream_blocks > 0 && n_tests != 1) return fail(EPT_EINVAL, "streaming windows are planned for one test");
    std::vector<TestSpec> specs;
    for (int t = 0; t < n_tests; ++t) {
        ept_status st = validate(nx[t], ny[t], p[t], EPT_STAT_ED, 1.0, EPT_PREC_SPLIT_BF16);
        if (st != EPT_OK) return st;
        if (B[t] < 0 || B[t] > ((int64_t)1 << 31)) return fail(EPT_EINVAL, "test %d: B must be in [0, 2^31]", t);
        specs.push_back(one_test(nullptr, nx[t], nullptr, ny[t], p[t], EPT_STAT_ED, 1.0, B[t], 0, nullptr, nullptr)[0]);
    }
    std::unique_ptr<Plan> hold(new (std::nothrow) Plan());
    if (!hold) return fail(EPT_ENOMEM, "host allocation failed");
    Plan &P = *hold;
    const bool streaming = stream_blocks > 0;
    plan_batch(P, specs, EPT_PREC_SPLIT_BF16, true, unit_kb, num_sms, true, !streaming);
    if (streaming) {
        // as the streaming run plans it: windows of panels, chunks of each window by first K-block
        P.stream = true;
        const size_t tab0 = P.tab_bytes;
        stream_partition(P, stream_blocks, SIZE_MAX);
        stream_layout(P, tab0);
        for (size_t g = 0; g < P.gdesc.size(); ++g) {
            auto first = P.chunks.begin() + P.gdesc[g].chunk0;
            std::stable_sort(first, first + P.gdesc[g].nchunks,
                             [](const Chunk &a, const Chunk &b) { return a.kb0 < b.kb0; });
        }
    }
    ept_status st = check_plan(P);
    if (st == EPT_OK && streaming) st = check_stream_plan(P);
    if (st != EPT_OK) return st;
    if (out) {
        memset(out, 0, sizeof(*out));
        out->units = P.nunits;
        out->chunks = (int64_t)P.chunks.size();
        out->stored_blocks = P.nblk;
        for (const TestDesc &d : P.desc) out->partials += d.nparts;
        out->windows = streaming ? (int64_t)P.gI0.size() : 0;
        out->scratch_bytes = P.total;
        if (!P.sched.empty()) {
            // MMA work per CTA, with the unit lengths the kernel sees (the all-zero
            // K-blocks of a diagonal square's second row half skipped)
            int64_t mx = 0, mn = INT64_MAX;
            for (size_t c = 0; c + 1 < P.sched_off.size(); ++c) {
                int64_t w = 0;
                for (int64_t k = P.sched_off[c]; k < P.sched_off[c + 1]; ++k) {
                    const int64_t u = P.sched[(size_t)k];
                    int t = 0;
                    while (t + 1 < P.n_tests && P.pre_units[t + 1] <= u) ++t;
                    const TestDesc &d = P.desc[t];
                    const int64_t lu = u - P.pre_units[t];
                    const Chunk &ch = P.chunks[(size_t)(d.chunk0 + (lu >> 1) / d.MT)];
                    int64_t l = ch.kb1 - ch.kb0;
                    if ((lu & 1) && ch.kb0 == KB_PER_PANEL * ch.I && l > 2) l -= 2;
                    w += l;
                }
                mx = std::max(mx, w);
                mn = std::min(mn, w);
            }
            out->cta_kblocks_max = mx;
            out->cta_kblocks_min = mn;
        }
    }
    return EPT_OK;
}

ept_status ept_test(ept_ctx *ctx, const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p, int on_device,
                    int stat, double sigma, int64_t B, uint64_t seed, int prec, double *perm_stats, ept_result *out,
                    void *stream) {
    if (!ctx) return fail(EPT_EINVAL, "null context");
    if (!X || !Y || !out) return fail(EPT_EINVAL, "null X, Y or result pointer");
    if (B < 0 || B > ((int64_t)1 << 31)) return fail(EPT_EINVAL, "B must be in [0, 2^31]");
    ept_status st = validate(nx, ny, p, stat, sigma, prec, true);
    if (st != EPT_OK) return st;
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    return run_single(ctx, one_test(X, nx, Y, ny, p, stat, sigma, B, seed, nullptr, perm_stats), prec, on_device != 0,
                      true, out, stream);
}

ept_status ept_test_range(ept_ctx *ctx, const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p,
                          int on_device, int stat, double sigma, int64_t b_first, int64_t count, uint64_t seed,
                          int prec, double *perm_stats, ept_result *out, void *stream) {
    if (!ctx || !out) return fail(EPT_EINVAL, "null context or result");
    if (!X || !Y) return fail(EPT_EINVAL, "null X or Y");
    if (count < 0 || count > ((int64_t)1 << 31)) return fail(EPT_EINVAL, "count must be in [0, 2^31]");
    if (b_first < 1 || b_first > ((int64_t)1 << 62)) return fail(EPT_EINVAL, "b_first must be >= 1");
    ept_status st = validate(nx, ny, p, stat, sigma, prec, true);
    if (st != EPT_OK) return st;
    std::vector<TestSpec> specs = one_test(X, nx, Y, ny, p, stat, sigma, count, seed, nullptr, perm_stats);
    specs[0].b0 = b_first;
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    return run_single(ctx, specs, prec, on_device != 0, true, out, stream);
}

ept_status ept_test_masks(ept_ctx *ctx, const float *X, int64_t nx, const float *Y, int64_t ny, int64_t p,
                          int on_device, int stat, double sigma, const uint32_t *masks, int64_t n_masks, int prec,
                          double *perm_stats, ept_result *out, void *stream) {
    if (!ctx) return fail(EPT_EINVAL, "null context");
    if (!X || !Y || !out) return fail(EPT_EINVAL, "null X, Y or result pointer");
    if (n_masks < 0 || n_masks > ((int64_t)1 << 31)) return fail(EPT_EINVAL, "n_masks must be in [0, 2^31]");
    if (n_masks > 0 && !masks) return fail(EPT_EINVAL, "null masks");
    ept_status st = validate(nx, ny, p, stat, sigma, prec, true);
    if (st != EPT_OK) return st;
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    return run_single(ctx,
                      one_test(X, nx, Y, ny, p, stat, sigma, n_masks, 0, n_masks > 0 ? masks : nullptr, perm_stats),
                      prec, on_device != 0, false, out, stream);
}

ept_status ept_test_batch(ept_ctx *ctx, const ept_test_desc *tests, int64_t n_tests, int on_device, int prec,
                          ept_result *results, void *stream) {
    if (!ctx) return fail(EPT_EINVAL, "null context");
    if (n_tests < 0 || n_tests > (1 << 20)) return fail(EPT_EINVAL, "n_tests must be in [0, 2^20]");
    if (n_tests == 0) return EPT_OK;
    if (!tests || !results) return fail(EPT_EINVAL, "null tests or results");
    std::vector<TestSpec> specs;
    specs.reserve((size_t)n_tests);
    for (int64_t t = 0; t < n_tests; ++t) {
        const ept_test_desc &q = tests[t];
        if (!q.X || !q.Y) return fail(EPT_EINVAL, "test %lld: null X or Y", (long long)t);
        if (q.B < 0 || q.B > ((int64_t)1 << 31)) return fail(EPT_EINVAL, "test %lld: B must be in [0, 2^31]", (long long)t);
        ept_status st = validate(q.nx, q.ny, q.p, q.stat, q.sigma, prec);
        if (st != EPT_OK) return fail(st, "test %lld: %s", (long long)t, g_err.c_str());
        specs.push_back(one_test(q.X, q.nx, q.Y, q.ny, q.p, q.stat, q.sigma, q.B, q.seed, nullptr, q.perm_stats)[0]);
    }
    std::lock_guard<std::mutex> lock(ctx->mu);
    DeviceGuard dg(ctx->device);
    return run_tuned(ctx, specs, prec, on_device != 0, true, results, stream);
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
    launch_perm_masks_plain(seed, (int)nx, (int)ny, b0, count, (int)nw, maskT, s);
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
    const std::vector<TestSpec> specs = one_test(X, nx, Y, ny, p, stat, sigma, 0, 0, nullptr, nullptr);
    Plan P;
    plan_batch(P, specs, prec, !on_device, CHUNK_KB_DEFAULT);
    const size_t out_bytes = (size_t)(nx + ny) * (nx + ny) * 4;
    if ((st = ensure_arena(c, P.total + (on_device ? 0 : align_up(out_bytes, 1024)), s)) != EPT_OK) return st;
    const Staging S = staging_layout(P);
    if ((st = ensure_pinned(c, S.total)) != EPT_OK) return st;
    if (s != c->stream) CK(cudaStreamSynchronize(c->stream));
    c->tables_staged = false;   // the staging area now holds this call's tables
    stage_host(c, P, specs, on_device != 0);
    uint8_t *A = c->arena;
    const Batch b = device_view(c, P);
    CK(cudaMemcpyAsync(A, c->pinned + S.tables, P.tab_bytes, cudaMemcpyHostToDevice, s));
    if ((st = enqueue_inputs(c, s)) != EPT_OK) return st;
    CK(cudaStreamWaitEvent(s, c->ev_in, 0));
    CK(cudaMemsetAsync(b.ctr, 0, sizeof(Counters), s));
    if (prec == EPT_PREC_SPLIT_BF16) {
        launch_split_rows(b, s);
        alignas(64) CUtensorMap tm[4];
        char emsg[160];
        if (!encode_rows_tmaps(tm, b.Zh, b.Zl, P.nrows, P.p_stride, emsg, sizeof(emsg))) return fail(EPT_ECUDA, "%s", emsg);
        CK(launch_build_tc(b, tm, c->num_sms, s));
    } else {
        launch_norms(b, s);
        launch_build_simt(b, s);
    }
    if (P.any_median) {
        // median bandwidth: select it, then the block-sum pass turns distances into kernel values
        CK(cudaMemsetAsync(b.sel_hist, 0, (size_t)2048 * 4, s));
        launch_median_select(b, s);
        launch_blocksums(b, s);
    }
    float *dout = on_device ? D_out : (float *)(A + P.total);
    launch_expand_blocks(b.D, nx + ny, P.desc[0].NKB, dout, s);
    CK(cudaGetLastError());
    Counters *h = (Counters *)(c->pinned + S.res_ctr);
    CK(cudaMemcpyAsync(h, b.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    if (!on_device) CK(cudaMemcpyAsync(D_out, dout, out_bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->nonfinite) return fail(EPT_EINVAL, "X or Y holds NaN or Inf");
    return EPT_OK;
}

ept_status ept_set_option(ept_ctx *c, int option, int64_t value) {
    if (!c) return fail(EPT_EINVAL, "null context");
    std::lock_guard<std::mutex> lock(c->mu);
    switch (option) {
    case EPT_OPT_GRAPHS:
        c->graphs = value != 0;
        if (!c->graphs) {
            DeviceGuard dg(c->device);
            drop_graph(c);
        }
        return EPT_OK;
    case EPT_OPT_AUTOTUNE:
        c->autotune = value != 0;
        return EPT_OK;
    case EPT_OPT_FAULT_INJECT_ALLOC:
        if (value < 0 || value > (1 << 20)) return fail(EPT_EINVAL, "injected failure count must be in [0, 2^20]");
        c->inject_alloc.store((int)value);
        return EPT_OK;
    case EPT_OPT_FAULT_INJECT_STALL:
        c->inject_stall = value != 0;
        return EPT_OK;
    case EPT_OPT_DEBUG_CHECKS:
        c->debug = value != 0;
        c->plan_key.clear();
        drop_graph(c);
        return EPT_OK;
    case EPT_OPT_DRAW_MODE:
        if (value < 0 || value > 3) return fail(EPT_EINVAL, "draw mode must be 0, 1, 2 or 3");
        c->draw_mode = (int)value;
        c->plan_key.clear();   // a captured graph holds the previous draw kernel
        drop_graph(c);
        return EPT_OK;
    case EPT_OPT_STREAM_BLOCKS:
        if (value < -1) return fail(EPT_EINVAL, "stream blocks must be -1, 0 or a block count");
        c->stream_blocks = value;
        return EPT_OK;
    case EPT_OPT_REFINE:
        if (value != 0 && value != 1) return fail(EPT_EINVAL, "refine must be 0 or 1");
        c->refine = value != 0;
        return EPT_OK;
    case EPT_OPT_CONTRACTION:
        if (value < 0 || value > 3) return fail(EPT_EINVAL, "contraction must be 0, 1, 2 or 3");
        c->contraction = (int)value;
        c->plan_key.clear();   // a captured graph holds the previous contraction kernel
        drop_graph(c);
        return EPT_OK;
    case EPT_OPT_UNIT_KB:
        if (value != 0 && value != 4 && value != 8 && value != 16 && value != 32)
            return fail(EPT_EINVAL, "the unit length must be 0, 4, 8, 16 or 32");
        c->unit_kb = (int)value;
        return EPT_OK;
    case EPT_OPT_MAX_CHUNK:
        if (value != 4 && value != 8 && value != 16 && value != 32)
            return fail(EPT_EINVAL, "the longest unit must be 4, 8, 16 or 32");
        c->max_chunk = (int)value;
        return EPT_OK;
    case EPT_OPT_WAIT_LIMIT_MS:
        if (value < 10 || value > 600000) return fail(EPT_EINVAL, "the wait limit must be in [10, 600000] ms");
        c->wait_ns = (unsigned long long)value * 1000000ull;
        c->plan_key.clear();   // a captured graph holds the previous limit
        drop_graph(c);
        return EPT_OK;
    case EPT_OPT_SERVE_LANES:
    case EPT_OPT_SERVE_SLOTS:
        if (c->server) return fail(EPT_EINVAL, "serving options must be set before the first ept_submit");
        if (option == EPT_OPT_SERVE_LANES) {
            if (value < 1 || value > 16) return fail(EPT_EINVAL, "serving lanes must be in [1, 16]");
            c->serve_lanes = (int)value;
        } else {
            if (value < 1 || value > (1 << 16)) return fail(EPT_EINVAL, "serving slots must be in [1, 65536]");
            c->serve_slots = (int)value;
        }
        return EPT_OK;
    default:
        return fail(EPT_EINVAL, "unknown option %d", option);
    }
}

ept_status ept_submit(ept_ctx *c, const ept_test_desc *q, int prec, uint64_t *ticket) {
    if (!c || !q || !ticket) return fail(EPT_EINVAL, "null context, request or ticket");
    if (!q->X || !q->Y) return fail(EPT_EINVAL, "null X or Y");
    if (q->B < 0 || q->B > ((int64_t)1 << 31)) return fail(EPT_EINVAL, "B must be in [0, 2^31]");
    ept_status st = validate(q->nx, q->ny, q->p, q->stat, q->sigma, prec);
    if (st != EPT_OK) return st;
    {
        std::lock_guard<std::mutex> lock(c->mu);
        if ((st = serve_start(c)) != EPT_OK) return st;
    }
    Server *S = c->server;
    Request *r = new (std::nothrow) Request();
    if (!r) return fail(EPT_ENOMEM, "host allocation failed");
    r->X.assign(q->X, q->X + q->nx * q->p);
    r->Y.assign(q->Y, q->Y + q->ny * q->p);
    r->stats.assign((size_t)q->B, 0.0);
    r->spec = one_test(r->X.data(), q->nx, r->Y.data(), q->ny, q->p, q->stat, q->sigma, q->B, q->seed, nullptr,
                       q->B > 0 ? r->stats.data() : nullptr)[0];
    r->prec = prec;
    Plan P;
    plan_batch(P, std::vector<TestSpec>(1, r->spec), prec, true, unit_kb(c));
    r->bytes = P.total;
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->bytes > S->budget) {
        delete r;
        return fail(EPT_ENOMEM, "request needs %zu bytes of device scratch, over the serving budget of %zu",
                    (size_t)P.total, S->budget);
    }
    if (S->pending.size() >= S->max_pending) {
        delete r;
        return fail(EPT_EBUSY, "serving queue is full (%zu pending requests)", S->pending.size());
    }
    r->ticket = S->next_ticket++;
    r->t_submit = Clock::now();
    for (const Lane &L : S->lanes)
        if (L.busy) {
            ++S->submits_busy;
            break;
        }
    S->reqs[r->ticket] = r;
    S->pending.push_back(r);
    *ticket = r->ticket;
    S->wakeups.fetch_add(1);
    S->cv_work.notify_all();
    return EPT_OK;
}

ept_status ept_poll(ept_ctx *c, uint64_t ticket, int *done) {
    if (!c || !done) return fail(EPT_EINVAL, "null context or output");
    Server *S = c->server;
    if (!S) return fail(EPT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(EPT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    *done = it->second->state >= REQ_DONE;
    return EPT_OK;
}

ept_status ept_wait(ept_ctx *c, uint64_t ticket, double *perm_stats, ept_result *out, int64_t timeout_ms) {
    if (!c) return fail(EPT_EINVAL, "null context");
    Server *S = c->server;
    if (!S) return fail(EPT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(EPT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    const auto pred = [r] { return r->state >= REQ_DONE; };
    if (timeout_ms < 0) S->cv_done.wait(lk, pred);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return fail(EPT_ETIMEOUT, "request %llu not finished after %lld ms", (unsigned long long)ticket,
                    (long long)timeout_ms);
    S->reqs.erase(it);
    const int state = r->state;
    const ept_status st = r->status;
    const std::string msg = r->err;
    if (state == REQ_DONE && st == EPT_OK) {
        if (out) *out = r->res;
        if (perm_stats && !r->stats.empty()) memcpy(perm_stats, r->stats.data(), r->stats.size() * 8);
    }
    delete r;
    if (state == REQ_CANCELLED) return fail(EPT_ECANCELLED, "request %llu was cancelled", (unsigned long long)ticket);
    if (st != EPT_OK) return fail(st, "%s", msg.c_str());
    return EPT_OK;
}

ept_status ept_serving_stats(ept_ctx *c, size_t *bytes_in_use, int64_t *running, int64_t *queued,
                             int64_t *finished) {
    if (!c) return fail(EPT_EINVAL, "null context");
    size_t b = 0;
    int64_t run = 0, q = 0, fin = 0;
    if (Server *S = c->server) {
        std::lock_guard<std::mutex> lk(S->mu);
        b = S->in_use;
        run = S->slots;
        q = (int64_t)S->pending.size();
        for (auto &kv : S->reqs) fin += kv.second->state >= REQ_DONE;
    }
    if (bytes_in_use) *bytes_in_use = b;
    if (running) *running = run;
    if (queued) *queued = q;
    if (finished) *finished = fin;
    return EPT_OK;
}

ept_status ept_serving_lanes(ept_ctx *c, int64_t *busy, int64_t *peak_busy, int64_t *submits_while_busy) {
    if (!c) return fail(EPT_EINVAL, "null context");
    int64_t b = 0, pk = 0, sb = 0;
    if (Server *S = c->server) {
        std::lock_guard<std::mutex> lk(S->mu);
        for (const Lane &L : S->lanes) b += L.busy ? 1 : 0;
        pk = S->peak_busy;
        sb = S->submits_busy;
    }
    if (busy) *busy = b;
    if (peak_busy) *peak_busy = pk;
    if (submits_while_busy) *submits_while_busy = sb;
    return EPT_OK;
}

ept_status ept_cancel(ept_ctx *c, uint64_t ticket) {
    if (!c) return fail(EPT_EINVAL, "null context");
    Server *S = c->server;
    if (!S) return fail(EPT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(EPT_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    if (r->state == REQ_PENDING) {
        for (auto p = S->pending.begin(); p != S->pending.end(); ++p)
            if (*p == r) {
                S->pending.erase(p);
                break;
            }
        r->state = REQ_CANCELLED;
        S->cv_done.notify_all();
    } else if (r->state == REQ_RUNNING) {
        r->cancel_req = true;   // its batch finishes; the result is discarded
    }
    return EPT_OK;
}

}  // extern "C"

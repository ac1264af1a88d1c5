// ept_kernels.cu -- SIMT kernels of libept: relabeling draws, the plain FP32 block
// build, centring and packing, the plain FP32 contraction and the final
// combination.  Every kernel processes a batch of tests (ept_internal.cuh).
#include "ept_internal.cuh"

#include <cuda_fp16.h>
#include <cstdint>
#include <cstdlib>

namespace ept {

// ---------------------------------------------------------------------------
// Permutation stream: Philox4x32-10 (Salmon et al., SC'11) drives Knuth's selection
// sampling; see draw_column.

// floor(u * m / 2^64) for a 64-bit u and a 32-bit m, from two 32x32->64 products:
// with u = uh 2^32 + ul, the value is floor((uh m + floor(ul m / 2^32)) / 2^32)
// (the dropped low word of ul m cannot carry across a multiple of 2^32), and
// uh m + floor(ul m / 2^32) < 2^64.  Equal to the high word of the 128-bit product.
__device__ __forceinline__ uint64_t mulhi_64x32(uint64_t u, uint32_t m) {
    const uint64_t a = (uint64_t)(uint32_t)(u >> 32) * m;
    const uint64_t b = (uint64_t)(uint32_t)u * m;
    return (a + (b >> 32)) >> 32;
}

// bits of word w that belong to real pooled rows t < n
__device__ __forceinline__ uint32_t valid_bits(int w, int n) {
    const int lo = w * 32;
    if (lo + 32 <= n) return 0xFFFFFFFFu;
    if (lo >= n) return 0u;
    return (1u << (n - lo)) - 1u;
}

// Philox4x32-10 of counter (c0, 0, blo, bhi) under the precomputed round keys: each
// round multiplies counter words 0 and 2 by the two Philox multipliers (one wide
// multiply gives both halves) and mixes the high halves with words 1 and 3 and the
// round key.  Returns the two 64-bit output words (word 0 = (x1:x0), word 1 = (x3:x2)).
__device__ __forceinline__ void philox_words(uint32_t c0, uint32_t blo, uint32_t bhi, const uint32_t *kx,
                                             const uint32_t *ky, uint64_t &w0, uint64_t &w1) {
    uint32_t x0 = c0, x1 = 0u, x2 = blo, x3 = bhi;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ kx[r];
        const uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ ky[r];
        x1 = (uint32_t)p1;
        x3 = (uint32_t)p0;
        x0 = y0;
        x2 = y2;
    }
    w0 = ((uint64_t)x1 << 32) | x0;
    w1 = ((uint64_t)x3 << 32) | x2;
}

// Decisions of one 64-slot window: lane l holds the ranks r0 (slot base+l) and r1
// (slot base+32+l); returns the two ballots (kept slots) and lowers `need`.  The
// sequential dependence through `need` is resolved by a fixed-point iteration over
// ballots: with every earlier decision known a slot's decision is determined, so
// iterating "decide from the previous guesses" reaches the unique sequential
// solution in at most 65 rounds (almost always 1 or 2).
__device__ __forceinline__ void decide_window(int r0, int r1, unsigned lt, int &need, unsigned &m0, unsigned &m1) {
    m0 = __ballot_sync(0xFFFFFFFFu, r0 < need);
    m1 = __ballot_sync(0xFFFFFFFFu, r1 < need);
    for (int it = 0; it < 70; ++it) {
        const int before0 = __popc(m0 & lt);
        const int before1 = __popc(m0) + __popc(m1 & lt);
        const unsigned nm0 = __ballot_sync(0xFFFFFFFFu, r0 < need - before0);
        const unsigned nm1 = __ballot_sync(0xFFFFFFFFu, r1 < need - before1);
        const bool same = (nm0 == m0) && (nm1 == m1);
        m0 = nm0;
        m1 = nm1;
        if (same) break;
    }
    need -= __popc(m0) + __popc(m1);
}

// One warp writes one relabeling column (words w = 0..nw-1 at col[w * stride]; nw is
// a multiple of 8).  Draw b of the stream: b = 0 is the identity; b >= 1 is Knuth's
// selection sampling (Algorithm S) over the n pooled slots, slot t kept iff
// floor(u_t (n - t) / 2^64) < need, with u_t the 64-bit word (t mod 2) of
// Philox4x32-10(counter = (t/2, 0, b lo, b hi), key = (seed lo, seed hi)).  The warp
// takes 128 consecutive slots per step: lane l runs the Philox calls of slots
// base+2l, base+2l+1 and base+64+2l, base+64+2l+1 (two independent chains, so that
// few warps per SM keep the integer pipes busy) and forms their floor(u (n - t) /
// 2^64) values; shuffles then place slot base+l on lane l (first word) and slot
// base+32+l on lane l (second word) of each 64-slot window, so one ballot is one
// output word.  comp: store the complement (the y* members).
__device__ void draw_column(uint64_t seed, int nx, int n, int64_t b, int nw, bool comp, uint32_t *col,
                            int64_t stride) {
    const int lane = threadIdx.x & 31;
    if (b == 0) {
        for (int w = lane; w < nw; w += 32) {
            const uint32_t v = valid_bits(w, nx);
            col[(int64_t)w * stride] = comp ? (~v & valid_bits(w, n)) : v;
        }
        return;
    }
    uint32_t kx[10], ky[10];
    kx[0] = (uint32_t)seed;
    ky[0] = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        kx[r] = kx[r - 1] + 0x9E3779B9u;
        ky[r] = ky[r - 1] + 0xBB67AE85u;
    }
    const uint32_t blo = (uint32_t)(uint64_t)b, bhi = (uint32_t)((uint64_t)b >> 32);
    const unsigned lt = (1u << lane) - 1u;
    const int src = lane >> 1;
    const bool odd = lane & 1;
    int need = nx;
    for (int base = 0; base < nw * 32; base += 128) {
        // ranks of this lane's four slots ("never kept" past the end or once need is 0)
        uint32_t ra = 0xFFFFFFFFu, rb = 0xFFFFFFFFu, rc = 0xFFFFFFFFu, rd = 0xFFFFFFFFu;
        if (need > 0) {
            const int tp = base + 2 * lane, tq = tp + 64;
            uint64_t u0, u1, u2, u3;
            philox_words((uint32_t)(tp >> 1), blo, bhi, kx, ky, u0, u1);
            philox_words((uint32_t)(tq >> 1), blo, bhi, kx, ky, u2, u3);
            if (tp < n) ra = (uint32_t)mulhi_64x32(u0, (uint32_t)(n - tp));
            if (tp + 1 < n) rb = (uint32_t)mulhi_64x32(u1, (uint32_t)(n - tp - 1));
            if (tq < n) rc = (uint32_t)mulhi_64x32(u2, (uint32_t)(n - tq));
            if (tq + 1 < n) rd = (uint32_t)mulhi_64x32(u3, (uint32_t)(n - tq - 1));
        }
        unsigned m[4];
        {
            const uint32_t a0 = __shfl_sync(0xFFFFFFFFu, ra, src), b0 = __shfl_sync(0xFFFFFFFFu, rb, src);
            const uint32_t a1 = __shfl_sync(0xFFFFFFFFu, ra, src + 16), b1 = __shfl_sync(0xFFFFFFFFu, rb, src + 16);
            const int r0 = (int)min(odd ? b0 : a0, 0x7FFFFFFFu);
            const int r1 = (int)min(odd ? b1 : a1, 0x7FFFFFFFu);
            decide_window(r0, r1, lt, need, m[0], m[1]);
        }
        {
            const uint32_t a0 = __shfl_sync(0xFFFFFFFFu, rc, src), b0 = __shfl_sync(0xFFFFFFFFu, rd, src);
            const uint32_t a1 = __shfl_sync(0xFFFFFFFFu, rc, src + 16), b1 = __shfl_sync(0xFFFFFFFFu, rd, src + 16);
            const int r0 = (int)min(odd ? b0 : a0, 0x7FFFFFFFu);
            const int r1 = (int)min(odd ? b1 : a1, 0x7FFFFFFFu);
            decide_window(r0, r1, lt, need, m[2], m[3]);
        }
        if (lane < 4) {
            const int w = (base >> 5) + lane;
            uint32_t v = lane == 0 ? m[0] : lane == 1 ? m[1] : lane == 2 ? m[2] : m[3];
            if (comp) v = ~v & valid_bits(w, n);
            col[(int64_t)w * stride] = v;
        }
    }
}

// Relabeling columns of the batch, one warp per column: column 0 of a test is the
// identity, columns 1..B its draws 1..B (or the caller's relabelings, validated:
// exactly nx members among the n rows), padding columns are zero.  Warps stride over
// the columns, so the grid may be capped (MASK_CTAS_PER_SM).
__global__ void __launch_bounds__(128) k_masks(const Batch bt) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t gc = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gc < bt.ncols_total;
         gc += nwarps) {
        const int t = find_test(bt.pre.cols, bt.n_tests, gc);
        const TestDesc &d = bt.desc[t];
        const int64_t c = gc - bt.pre.cols[t];
        const int n = (int)d.n, nw = (int)d.nw;
        const int64_t Bp = d.Bp;
        uint32_t *col = bt.maskT + d.mask0 + c;
        if (c >= d.ncols) {
            for (int w = lane; w < nw; w += 32) col[(int64_t)w * Bp] = 0u;
            continue;
        }
        if (c >= 1 && d.user_masks) {
            const int nwu = d.nwu, nx = (int)d.nx;
            const bool comp = d.comp != 0;
            const uint32_t *row = d.user_masks + (c - 1) * nwu;
            int cnt = 0;
            bool bad = false;
            for (int w = lane; w < nw; w += 32) {
                uint32_t v = (w < nwu) ? row[w] : 0u;
                const uint32_t valid = valid_bits(w, n);
                if (v & ~valid) bad = true;
                v &= valid;
                cnt += __popc(v);
                col[(int64_t)w * Bp] = comp ? (~v & valid) : v;
            }
            for (int off = 16; off; off >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, off);
            bad = __any_sync(0xFFFFFFFFu, bad);
            if (lane == 0 && (bad || cnt != nx)) atomicAdd(&bt.ctr[t].bad_mask, 1ull);
            continue;
        }
        // column 0: the identity (draw 0); column c >= 1: draw b0 + c - 1
        draw_column(d.seed, (int)d.nx, n, c == 0 ? 0 : d.b0 + c - 1, nw, d.comp != 0, col, Bp);
    }
}

// One thread per relabeling column (used when the batch has enough columns to fill
// the GPU this way, and no caller relabelings): the thread runs Algorithm S over
// its column's slots one at a time, from the same Philox words as draw_column, so
// the two kernels write identical bits.  Without the warp's ballots, shuffles and
// fixed-point rounds a slot costs about half the instructions, and the 32 lanes of
// a warp write 32 neighbouring columns of a word with one coalesced store.
__global__ void __launch_bounds__(256) k_masks_lanes(const Batch bt) {
    const int64_t gc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gc >= bt.ncols_total) return;
    const int t = find_test(bt.pre.cols, bt.n_tests, gc);
    const TestDesc &d = bt.desc[t];
    const int64_t c = gc - bt.pre.cols[t];
    const int n = (int)d.n, nw = (int)d.nw, nx = (int)d.nx;
    const int64_t Bp = d.Bp;
    const bool comp = d.comp != 0;
    uint32_t *col = bt.maskT + d.mask0 + c;
    if (c >= d.ncols) {
        for (int w = 0; w < nw; ++w) col[(int64_t)w * Bp] = 0u;
        return;
    }
    if (c == 0) {
        for (int w = 0; w < nw; ++w) {
            const uint32_t v = valid_bits(w, nx);
            col[(int64_t)w * Bp] = comp ? (~v & valid_bits(w, n)) : v;
        }
        return;
    }
    const uint64_t seed = d.seed;
    uint32_t kx[10], ky[10];
    kx[0] = (uint32_t)seed;
    ky[0] = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        kx[r] = kx[r - 1] + 0x9E3779B9u;
        ky[r] = ky[r - 1] + 0xBB67AE85u;
    }
    const uint64_t bdraw = (uint64_t)(d.b0 + c - 1);   // column c >= 1 holds draw b0 + c - 1
    const uint32_t blo = (uint32_t)bdraw, bhi = (uint32_t)(bdraw >> 32);
    int need = nx;
    for (int w = 0; w < nw; ++w) {
        uint32_t bits = 0;
        const int t0 = w * 32;
        if (need > 0 && t0 < n) {
            // two Philox calls per step (slots tp .. tp + 3): independent chains for the
            // scheduler to interleave
#pragma unroll 2
            for (int j = 0; j < 16; j += 2) {
                const int tp = t0 + 2 * j;
                uint64_t u0, u1, u2, u3;
                philox_words((uint32_t)(tp >> 1), blo, bhi, kx, ky, u0, u1);
                philox_words((uint32_t)(tp >> 1) + 1u, blo, bhi, kx, ky, u2, u3);
                const uint64_t uu[4] = {u0, u1, u2, u3};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int ts = tp + q;
                    if (ts < n && (int)mulhi_64x32(uu[q], (uint32_t)(n - ts)) < need) {
                        bits |= 1u << (2 * j + q);
                        --need;
                    }
                }
            }
        }
        col[(int64_t)w * Bp] = comp ? (~bits & valid_bits(w, n)) : bits;
    }
}

// Relabeling columns in groups of 32 per CTA, with Algorithm S split into its two
// parts: a slot's rank r_t = floor(u_t (n - t) / 2^64) depends only on the stream
// (the same Philox words as draw_column), and only the decisions "keep slot t iff
// r_t < need" depend on each other.  Eight producer warps compute the ranks of the
// next 128 slots of all 32 columns into shared memory (two buffers) while one
// scanner warp, a lane per column, runs the sequential decisions over the previous
// 128 (a compare and a subtraction per slot) and writes each 32-slot word, the 32
// lanes storing neighbouring columns of a word together.  No ballots, shuffles or
// fixed-point rounds: about half the instructions per slot of the warp kernel, with
// the columns' Philox work spread over eight times as many threads as the thread
// kernel.  The identity (column 0) and padding columns are written by the scanner
// lane; caller relabelings take the warp kernel.  A group never straddles two tests
// (every test's column count Bp is a multiple of 32).
constexpr int SCAN_SLOTS = 128;                    // slots per chunk
constexpr int SCAN_PRODUCERS = 256;                // eight producer warps
constexpr int SCAN_THREADS = SCAN_PRODUCERS + 32;  // and the scanner warp
static_assert(COL_PAD % 32 == 0, "column groups of 32 stay inside one test");

__global__ void __launch_bounds__(SCAN_THREADS) k_masks_scan(const Batch bt) {
    __shared__ uint32_t rank[2][SCAN_SLOTS][32];   // [buffer][slot in chunk][column in group]
    const int64_t gc0 = (int64_t)blockIdx.x * 32;  // first batch column of the group
    if (gc0 >= bt.ncols_total) return;             // uniform over the CTA, before any barrier
    const int t = find_test(bt.pre.cols, bt.n_tests, gc0);
    const TestDesc &d = bt.desc[t];
    const int64_t c0 = gc0 - bt.pre.cols[t];       // first column of the group within the test
    const int n = (int)d.n, nw = (int)d.nw;
    const int nchunks = nw * 32 / SCAN_SLOTS;      // nw is a multiple of 8
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = c0 + lane;                   // this lane's column (producers and scanner)

    // producer state: round keys and the draw of this thread's column
    uint32_t kx[10], ky[10];
    kx[0] = (uint32_t)d.seed;
    ky[0] = (uint32_t)(d.seed >> 32);
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        kx[r] = kx[r - 1] + 0x9E3779B9u;
        ky[r] = ky[r - 1] + 0xBB67AE85u;
    }
    const uint64_t bdraw = (uint64_t)(d.b0 + c - 1);   // column c >= 1 holds draw b0 + c - 1
    const uint32_t blo = (uint32_t)bdraw, bhi = (uint32_t)(bdraw >> 32);
    const bool drawn = c >= 1 && c < d.ncols;
    // ranks of chunk k into buffer buf: this thread's column, slot pairs warp + 8 i
    auto produce = [&](int k, int buf) {
        if (!drawn) return;
#pragma unroll 2
        for (int i = 0; i < SCAN_SLOTS / 2 / 8; ++i) {
            const int jp = warp + 8 * i;                 // slot pair within the chunk
            const int ts = k * SCAN_SLOTS + 2 * jp;      // its first slot
            uint64_t u0, u1;
            philox_words((uint32_t)(ts >> 1), blo, bhi, kx, ky, u0, u1);
            rank[buf][2 * jp][lane] = ts < n ? (uint32_t)mulhi_64x32(u0, (uint32_t)(n - ts)) : 0xFFFFFFFFu;
            rank[buf][2 * jp + 1][lane] =
                ts + 1 < n ? (uint32_t)mulhi_64x32(u1, (uint32_t)(n - ts - 1)) : 0xFFFFFFFFu;
        }
    };

    // scanner state
    uint32_t *col = bt.maskT + d.mask0 + c;
    const int64_t Bp = d.Bp;
    const bool comp = d.comp != 0;
    uint32_t need = (uint32_t)d.nx;

    if (warp < 8) produce(0, 0);
    __syncthreads();
    for (int k = 0; k < nchunks; ++k) {
        if (warp == 8) {
            const int buf = k & 1;
#pragma unroll 1
            for (int q = 0; q < SCAN_SLOTS / 32; ++q) {
                const int w = k * (SCAN_SLOTS / 32) + q;   // output word
                uint32_t bits;
                if (drawn) {
                    uint32_t r[32];
#pragma unroll
                    for (int e = 0; e < 32; ++e) r[e] = rank[buf][q * 32 + e][lane];
                    bits = 0;
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const uint32_t keep = r[e] < need ? 1u : 0u;
                        bits |= keep << e;
                        need -= keep;
                    }
                } else {
                    bits = (c == 0) ? valid_bits(w, (int)d.nx) : 0u;   // identity, or padding
                }
                if (c < d.ncols) bits = comp ? (~bits & valid_bits(w, n)) : bits;
                col[(int64_t)w * Bp] = bits;
            }
        } else if (k + 1 < nchunks) {
            produce(k + 1, (k + 1) & 1);
        }
        __syncthreads();
    }
}

// Blocks per SM of the draw kernel: MASK_CTAS_PER_SM, or the environment's
// EPT_MASK_BLOCKS_PER_SM (0: one warp per column, no cap).
static int mask_blocks_per_sm() {
    static const int v = [] {
        const char *e = getenv("EPT_MASK_BLOCKS_PER_SM");
        if (!e || !*e) return MASK_CTAS_PER_SM;
        const int k = atoi(e);
        return k < 0 ? MASK_CTAS_PER_SM : (k > 64 ? 64 : k);
    }();
    return v;
}

void launch_masks(const Batch &b, int num_sms, int mode, cudaStream_t s) {
    if (b.ncols_total <= 0) return;
    if (mode == DRAW_SCAN) {
        k_masks_scan<<<(unsigned)((b.ncols_total + 31) / 32), SCAN_THREADS, 0, s>>>(b);
        return;
    }
    if (mode == DRAW_LANES) {
        // few columns: small blocks, so that they spread over the SMs beside the build
        const int threads = (b.ncols_total >= 1024 * (int64_t)(num_sms > 0 ? num_sms : 1)) ? 256 : 64;
        k_masks_lanes<<<(unsigned)((b.ncols_total + threads - 1) / threads), threads, 0, s>>>(b);
        return;
    }
    int64_t blocks = (b.ncols_total + 3) / 4;
    const int per_sm = mask_blocks_per_sm();
    if (per_sm > 0) {
        const int64_t cap = (int64_t)(num_sms > 0 ? num_sms : 1) * per_sm;
        if (blocks > cap) blocks = cap;
    }
    k_masks<<<(unsigned)blocks, 128, 0, s>>>(b);
}

// the stream itself, for export: column c = draw b0 + c
__global__ void __launch_bounds__(256) k_perm_masks_plain(uint64_t seed, int nx, int ny, int64_t b0, int64_t count,
                                                          int nw, uint32_t *__restrict__ maskT) {
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= count) return;
    draw_column(seed, nx, nx + ny, b0 + c, nw, false, maskT + c, count);
}

void launch_perm_masks_plain(uint64_t seed, int nx, int ny, int64_t b0, int64_t count, int nw, uint32_t *maskT,
                             cudaStream_t s) {
    if (count <= 0) return;
    k_perm_masks_plain<<<(unsigned)((count + 7) / 8), 256, 0, s>>>(seed, nx, ny, b0, count, nw, maskT);
}

// maskT columns 0..count-1 -> row-major [count][nwu]
__global__ void k_masks_to_rows(const uint32_t *__restrict__ maskT, int64_t ncols, int nw, int64_t count, int nwu,
                                uint32_t *__restrict__ rows) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count * nwu) return;
    const int64_t c = idx / nwu;
    const int w = (int)(idx % nwu);
    rows[idx] = maskT[(int64_t)w * ncols + c];
}

void launch_masks_to_rows(const uint32_t *maskT, int64_t ncols, int nw, int64_t count, int nwu, uint32_t *rows,
                          cudaStream_t s) {
    const int64_t tot = count * nwu;
    if (tot <= 0) return;
    k_masks_to_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(maskT, ncols, nw, count, nwu, rows);
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ const float *pooled_row(const TestDesc &d, int64_t i) {
    return (i < d.nx) ? d.X + i * d.p : d.Y + (i - d.nx) * d.p;
}

// Plain path: squared row norms ||z_i||^2 of the pooled rows, exact products summed
// in FP64 and rounded once to FP32 (padded rows: 0), and the count of non-finite
// inputs.  One warp per row of the batch.
__global__ void __launch_bounds__(256) k_norms(const Batch bt) {
    const int lane = threadIdx.x & 31;
    const int64_t gr = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gr >= bt.nrows_total) return;
    const int t = find_test(bt.pre.rows, bt.n_tests, gr);
    const TestDesc d = bt.desc[t];
    const int64_t i = gr - d.row0;
    double acc = 0.0;
    bool bad = false;
    if (i < d.n) {
        const float *z = pooled_row(d, i);
        for (int64_t k = lane; k < d.p; k += 32) {
            const float v = z[k];
            bad |= !isfinite(v);
            acc = fma((double)v, (double)v, acc);
        }
    }
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicAdd(&bt.ctr[t].nonfinite, 1ull);
    if (lane == 0) bt.norms[gr] = (float)acc;
}

void launch_norms(const Batch &b, cudaStream_t s) {
    if (b.nrows_total <= 0) return;
    k_norms<<<(unsigned)((b.nrows_total + 7) / 8), 256, 0, s>>>(b);
}

// ---------------------------------------------------------------------------
// Plain block build, SIMT FP32 (Algorithm 1 block construction; Algorithm 3 entries
// through the expansion ||x||^2 + ||y||^2 - 2 x.y).  One CTA computes half of a
// stored 256x64 block (128 rows x 64 columns): 256 threads, 8x4 outputs each,
// K-loop over p in steps of 16 staged through shared memory.
// Epilogue: d2 = max(0, n_i + n_j - 2 g_ij); a pair with d2 < tau (n_i + n_j)
// (cancellation-prone near-duplicate) is recomputed directly as sum (x - y)^2 in
// FP64; then the distance, exp(-d2 / (2 sigma^2)) (Gaussian) or exp(-d / sigma)
// (Laplacian); the diagonal is exactly 0 (distances) or 1 (kernels); padded rows and
// columns are 0.
__global__ void __launch_bounds__(256) k_build_simt(const Batch bt) {
    __shared__ float As[16][128 + 4];
    __shared__ float Bs[16][64 + 4];
    const int64_t gb = blockIdx.x;
    const int h = blockIdx.y;
    const BlkInfo bi = bt.blk[gb];
    const TestDesc d = bt.desc[bi.t];
    const int64_t n = d.n, p = d.p;
    const int64_t row0 = (int64_t)bi.I * PANEL + h * 128;
    const int64_t col0 = (int64_t)bi.kb * KB;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;

    for (int64_t k0 = 0; k0 < p; k0 += 16) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int idx = e * 256 + t, r = idx >> 4, k = idx & 15;
            const int64_t i = row0 + r;
            float v = 0.f;
            if (i < n && k0 + k < p) v = __ldg(pooled_row(d, i) + k0 + k);
            As[k][r] = v;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = e * 256 + t, cc = idx >> 4, k = idx & 15;
            const int64_t j = col0 + cc;
            float v = 0.f;
            if (j < n && k0 + k < p) v = __ldg(pooled_row(d, j) + k0 + k);
            Bs[k][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[k][ty * 8 + 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(av[a], bv[c], acc[a][c]);
        }
        __syncthreads();
    }
    const float neg = d.neg_inv_2s2, inv_sigma = d.inv_sigma, tau = d.tau;
    const int kern = d.kern;
    unsigned fixups = 0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int64_t i = row0 + ty * 8 + a;
        float out[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t j = col0 + tx * 4 + c;
            float v = 0.f;
            if (i < n && j < n) {
                if (i == j) {
                    v = (kern == 0) ? 0.f : 1.f;
                } else {
                    const float ni = __ldg(bt.norms + d.row0 + i), nj = __ldg(bt.norms + d.row0 + j);
                    const float d2 = fmaxf(0.f, ni + nj - 2.f * acc[a][c]);
                    if (d2 < tau * (ni + nj)) {
                        const float *zi = pooled_row(d, i), *zj = pooled_row(d, j);
                        double s = 0.0;
                        for (int64_t k = 0; k < p; ++k) {
                            const double df = (double)zi[k] - (double)zj[k];
                            s = fma(df, df, s);
                        }
                        ++fixups;
                        v = (float)entry_from_d2(s, kern, neg, inv_sigma);
                    } else {
                        v = (kern == 0) ? sqrtf(d2) : (kern == 1) ? exp_cw(d2 * neg) : exp_cw(-sqrtf(d2) * inv_sigma);
                    }
                }
            }
            out[c] = v;
        }
        const int64_t off = (gb * PANEL + h * 128 + ty * 8 + a) * KB + tx * 4;
        *reinterpret_cast<float4 *>(bt.D + off) = make_float4(out[0], out[1], out[2], out[3]);
    }
    if (fixups) atomicAdd(&bt.ctr[bi.t].n_fixup, (unsigned long long)fixups);
}

void launch_build_simt(const Batch &b, cudaStream_t s) {
    if (b.nblk_total <= 0) return;
    k_build_simt<<<dim3((unsigned)b.nblk_total, 2), 256, 0, s>>>(b);
}

// ---------------------------------------------------------------------------
// Row and column partial sums of each stored block, for the row sums r = W 1
// (the lower part of W is the transpose of the stored strictly-upper blocks, so
// their column sums supply it).  Sums are accumulated as unevaluated FP32 pairs
// (hi, lo) with Knuth's TwoSum, an error-free transformation (the rounding error of
// every addition is carried in lo), then widened to FP64: about twice the FP32
// precision at FP32 cost.  One CTA per stored block of the batch, taking the block
// in four quarters of 64 rows: each quarter is read once with coalesced 16-byte loads
// into shared memory (rows padded to 65 words, so that threads walking rows or
// columns hit distinct banks), then four threads per row and four per column each
// sum 16 values, and the four pairs meet in a fixed order.

// (h, l) += (h2, l2), the rounding error of the hi addition kept in l
__device__ __forceinline__ void pair_add(float &h, float &l, float h2, float l2) {
    float s2, e;
    two_sum(h, h2, s2, e);
    h = s2;
    l += l2 + e;
}

__global__ void __launch_bounds__(256) k_blocksums(const Batch bt) {
    constexpr int QR = 64, LD = KB + 1;   // rows per quarter, padded row length
    __shared__ float tile[QR * LD];
    __shared__ float wmax[8];
    const int64_t gb = blockIdx.x;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    float *base = bt.D + gb * (int64_t)(PANEL * KB);
    const BlkInfo bi = bt.blk[gb];
    const TestDesc &d = bt.desc[bi.t];
    // median-heuristic tests: the build wrote distances; now that the bandwidth is
    // known, they become kernel values in place as they are read (padding stays 0)
    const bool median = d.median != 0;
    float neg = 0.f, inv = 0.f;
    if (median) {
        const float sigma = __uint_as_float(bt.ctr[bi.t].sel_prefix);
        neg = -1.f / (2.f * sigma * sigma);
        inv = 1.f / sigma;
    }
    const bool gauss = d.stat == 1;
    const int64_t n = d.n;
    float mx = 0.f;
    const int rr = t >> 2, part = t & 3;   // row rr (or column rr) of the quarter, its quarter `part`
    float ch = 0.f, cl = 0.f;               // this thread's column partial over the block's quarters
    for (int qtr = 0; qtr < PANEL / QR; ++qtr) {
        float *qbase = base + (int64_t)qtr * QR * KB;
        // coalesced load: float4 k = t + 256 i covers row k / 16, columns 4 (k % 16) ..
#pragma unroll
        for (int i = 0; i < QR * KB / 4 / 256; ++i) {
            const int k = t + 256 * i, row = k >> 4, c4 = (k & 15) * 4;
            float4 v = reinterpret_cast<const float4 *>(qbase)[k];
            if (median) {
                const int64_t gi = (int64_t)bi.I * PANEL + qtr * QR + row, gj = (int64_t)bi.kb * KB + c4;
                float e4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (gi < n && gj + e < n) e4[e] = gauss ? exp_cw(e4[e] * e4[e] * neg) : exp_cw(-e4[e] * inv);
                v = make_float4(e4[0], e4[1], e4[2], e4[3]);
                reinterpret_cast<float4 *>(qbase)[k] = v;
            }
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            float *dst = tile + row * LD + c4;
            dst[0] = v.x;
            dst[1] = v.y;
            dst[2] = v.z;
            dst[3] = v.w;
        }
        __syncthreads();
        // row rr of the quarter: columns 16 part .. 16 part + 15, then the four parts in order
        {
            float h = 0.f, l = 0.f;
            const float *src = tile + rr * LD + 16 * part;
#pragma unroll
            for (int j = 0; j < 16; ++j) pair_add(h, l, src[j], 0.f);
            float h1 = __shfl_xor_sync(0xFFFFFFFFu, h, 1), l1 = __shfl_xor_sync(0xFFFFFFFFu, l, 1);
            if (part & 1) { const float th = h, tl = l; h = h1; l = l1; h1 = th; l1 = tl; }
            pair_add(h, l, h1, l1);   // (part 0 + part 1), (part 2 + part 3)
            float h2 = __shfl_xor_sync(0xFFFFFFFFu, h, 2), l2 = __shfl_xor_sync(0xFFFFFFFFu, l, 2);
            if (part & 2) { const float th = h, tl = l; h = h2; l = l2; h2 = th; l2 = tl; }
            pair_add(h, l, h2, l2);   // (0 + 1) + (2 + 3)
            if (part == 0) bt.rowpart[gb * PANEL + qtr * QR + rr] = (double)h + (double)l;
        }
        // column rr: rows 16 part .. 16 part + 15 of the quarter, into this thread's pair
        {
            const float *src = tile + (16 * part) * LD + rr;
#pragma unroll
            for (int i = 0; i < 16; ++i) pair_add(ch, cl, src[i * LD], 0.f);
        }
        __syncthreads();
    }
    // the column's four parts in order: (0 + 1) + (2 + 3)
    {
        float h = ch, l = cl;
        float h1 = __shfl_xor_sync(0xFFFFFFFFu, h, 1), l1 = __shfl_xor_sync(0xFFFFFFFFu, l, 1);
        if (part & 1) { const float th = h, tl = l; h = h1; l = l1; h1 = th; l1 = tl; }
        pair_add(h, l, h1, l1);
        float h2 = __shfl_xor_sync(0xFFFFFFFFu, h, 2), l2 = __shfl_xor_sync(0xFFFFFFFFu, l, 2);
        if (part & 2) { const float th = h, tl = l; h = h2; l = l2; h2 = th; l2 = tl; }
        pair_add(h, l, h2, l2);
        if (part == 0) bt.colpart[gb * KB + rr] = (double)h + (double)l;
    }
    for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    if (lane == 0) wmax[warp] = mx;
    __syncthreads();
    if (t == 0) {
        float m = wmax[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) m = fmaxf(m, wmax[w]);
        atomicMax(&bt.ctr[bi.t].max_d_bits, __float_as_uint(m));
    }
}

void launch_blocksums(const Batch &b, cudaStream_t s) {
    if (b.nblk_total <= 0) return;
    k_blocksums<<<(unsigned)b.nblk_total, 256, 0, s>>>(b);
}

// ---------------------------------------------------------------------------
// Median heuristic (bandwidth of the MMD kernels): the lower median, rank
// k = floor((N - 1) / 2) in ascending order, of the N = n (n - 1) / 2 distances
// between distinct pooled rows (the strictly upper entries of the stored blocks).
// Exact radix selection on the FP32 bit patterns (non-negative floats order like
// their bits): three passes over digits of 11, 11 and 10 bits, most significant
// first; each pass histograms the digit of the entries whose higher bits match the
// prefix found so far (k_median_hist, one CTA per stored block, lanes with equal
// digits aggregated before the shared-memory atomics) and then finds the bin that
// holds rank k (k_median_pick, one CTA per test), which extends the prefix.  After
// the last pass the prefix is the median's bit pattern (Counters::sel_prefix).
__device__ __forceinline__ void sel_digit(int pass, uint32_t &mask, int &shift, uint32_t &dmask) {
    mask = pass == 0 ? 0u : (pass == 1 ? 0xFFE00000u : 0xFFFFFC00u);
    shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
    dmask = pass == 2 ? 0x3FFu : 0x7FFu;
}

__global__ void __launch_bounds__(256) k_median_hist(const Batch bt, int pass) {
    __shared__ uint32_t hist[2048];
    const int64_t gb = blockIdx.x;
    const BlkInfo bi = bt.blk[gb];
    const TestDesc &d = bt.desc[bi.t];
    if (!d.median) return;
    for (int k = threadIdx.x; k < 2048; k += 256) hist[k] = 0u;
    __syncthreads();
    uint32_t mask, dmask;
    int shift;
    sel_digit(pass, mask, shift, dmask);
    const uint32_t prefix = bt.ctr[bi.t].sel_prefix;
    const int64_t n = d.n;
    const float *base = bt.D + gb * (int64_t)(PANEL * KB);
    for (int e = threadIdx.x; e < PANEL * KB; e += 256) {
        const int64_t i = (int64_t)bi.I * PANEL + (e >> 6), j = (int64_t)bi.kb * KB + (e & 63);
        const uint32_t v = __float_as_uint(base[e]);
        const bool take = i < n && j < n && j > i && (v & mask) == prefix;
        const uint32_t bin = take ? ((v >> shift) & dmask) : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, bin);
        if (take && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
    }
    __syncthreads();
    uint32_t *gh = bt.sel_hist + (int64_t)bi.t * 2048;
    for (int k = threadIdx.x; k < 2048; k += 256)
        if (hist[k]) atomicAdd(&gh[k], hist[k]);
}

__global__ void __launch_bounds__(256) k_median_pick(const Batch bt, int pass) {
    __shared__ unsigned long long part[256];
    __shared__ int owner;
    __shared__ unsigned long long before;
    const int t = blockIdx.x;
    const TestDesc &d = bt.desc[t];
    if (!d.median) return;
    uint32_t mask, dmask;
    int shift;
    sel_digit(pass, mask, shift, dmask);
    const int nbins = (int)dmask + 1, per = nbins / 256;
    uint32_t *gh = bt.sel_hist + (int64_t)t * 2048;
    Counters *c = bt.ctr + t;
    const unsigned long long npairs = (unsigned long long)d.n * (unsigned long long)(d.n - 1) / 2ull;
    const unsigned long long k = pass == 0 ? (npairs - 1ull) / 2ull : c->sel_k;
    unsigned long long mine = 0;
    for (int q = 0; q < per; ++q) mine += gh[threadIdx.x * per + q];
    part[threadIdx.x] = mine;
    if (threadIdx.x == 0) owner = -1;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long cum = 0;
        for (int q = 0; q < 256; ++q) {
            if (k < cum + part[q]) {
                owner = q;
                before = cum;
                break;
            }
            cum += part[q];
        }
    }
    __syncthreads();
    if ((int)threadIdx.x == owner) {
        unsigned long long cum = before;
        for (int q = 0; q < per; ++q) {
            const unsigned long long h = gh[threadIdx.x * per + q];
            if (k < cum + h) {
                c->sel_prefix |= (uint32_t)(threadIdx.x * per + q) << shift;
                c->sel_k = k - cum;
                break;
            }
            cum += h;
        }
    }
    if (owner < 0 && threadIdx.x == 0) c->sel_prefix = 0u;   // counts do not add up: reported as a zero bandwidth
    __syncthreads();
    for (int q = 0; q < per; ++q) gh[threadIdx.x * per + q] = 0u;   // ready for the next pass
}

void launch_median_select(const Batch &b, cudaStream_t s) {
    if (!b.sel_hist || b.nblk_total <= 0) return;
    for (int pass = 0; pass < 3; ++pass) {
        k_median_hist<<<(unsigned)b.nblk_total, 256, 0, s>>>(b, pass);
        k_median_pick<<<(unsigned)b.n_tests, 256, 0, s>>>(b, pass);
    }
}

// r_i = sum over the stored blocks of row i's panel (its own row segments) + sum
// over the earlier panels J < panel(i) of column i's segments.  Eight threads per
// row take every eighth term and combine by a fixed shuffle tree (deterministic).
// CTA = 32 rows of one test (256 threads); Spart[CTA] = sum of its rows' r_i.
__global__ void __launch_bounds__(256) k_rowsum_reduce(const Batch bt) {
    __shared__ double sh[32];
    const int sub = threadIdx.x & 7, rl = threadIdx.x >> 3;
    const int64_t gr = (int64_t)blockIdx.x * 32 + rl;
    const int t = find_test(bt.pre.rows, bt.n_tests, (int64_t)blockIdx.x * 32);
    const TestDesc d = bt.desc[t];
    const int64_t i = gr - d.row0;
    const int64_t I = i / PANEL, rr = i % PANEL, NKB = d.NKB;
    double acc = 0.0;
    if (i < d.n) {
        const int64_t nkb = NKB - KB_PER_PANEL * I;
        const int64_t base = d.blk0 + blk_off(I, NKB);
        for (int64_t k = sub; k < nkb; k += 8) acc += bt.rowpart[(base + k) * PANEL + rr];
        const int64_t kbi = i / KB, ci = i % KB;
        for (int64_t J = sub; J < I; J += 8) acc += bt.colpart[(d.blk0 + blk_index(J, kbi, NKB)) * KB + ci];
    }
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
    if (sub == 0) {
        bt.r[gr] = acc;
        sh[rl] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 32; ++k) s += sh[k];
        bt.Spart[blockIdx.x] = s;
    }
}

void launch_rowsum_reduce(const Batch &b, cudaStream_t s) {
    if (b.nrows_total <= 0) return;
    k_rowsum_reduce<<<(unsigned)(b.nrows_total / 32), 256, 0, s>>>(b);
}

// Deterministic sum of a short array in fixed order (one warp: strided lane sums,
// then a fixed shuffle tree).
__device__ __forceinline__ double warp_ordered_sum(const double *a, int64_t m) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int64_t k = lane; k < m; k += 32) s += a[k];
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
    return s;
}

__device__ __forceinline__ double block_sum_256(double v, double *sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 128; off; off >>= 1) {
        if (t < off) sh[t] += sh[t + off];
        __syncthreads();
    }
    return sh[0];
}

// Centring.  u_i = r_i / n - S / (2 n^2) (double centring, S = 1'W1), rounded to FP32;
// the centred matrix is W~ = W - u 1' - 1 u'.  Let s mark the contracted group (size
// m, the other group has size o; see ept_internal.cuh).  Writing Eq. 1 with
// T = s'W~s, L = s'W~1 and S~ = 1'W~1 (the sums over the other group are
// S~ - 2L + T, the cross sums L - T) gives, whatever u is,
//     ED = -cT T + cL L - S~/o^2,  cT = (n/(nx ny))^2,  cL = 2n/(m o^2),
// and MMD^2 (Eq. 2) is the same expression with the opposite sign.  Because
// s_i^2 = s_i, L = s' diag(r~) s with r~ = W~ 1 = r - n u - (1'u) 1, so
//     stat = sign * (cT s'Cs + S~/o^2),  C = W~ - kappa diag(r~),  kappa = cL/cT = 2m/n,
// sign = -1 (ED) or +1 (MMD).  dcorr_i = kappa r~_i.
// Only r~ must be exact (it is, in FP64, for the FP32 u actually stored); u itself
// may be any value, so it is formed with multiplications by precomputed reciprocals.
// Step 1 (one CTA per panel of the batch): u_i, Upart[panel] = sum of the u_i.
__global__ void __launch_bounds__(256) k_center_u(const Batch bt) {
    __shared__ double sh[256];
    __shared__ double bS;
    const int64_t gp = blockIdx.x;
    const int t = find_test(bt.pre.panels, bt.n_tests, gp);
    const TestDesc d = bt.desc[t];
    if (threadIdx.x < 32) {
        const double S = warp_ordered_sum(bt.Spart + d.sp0, d.n_pad / 32);
        if (threadIdx.x == 0) bS = S;
    }
    __syncthreads();
    const int64_t i = (gp - d.pan0) * PANEL + threadIdx.x;
    float ui = 0.f;
    if (i < d.n) ui = (float)(bt.r[d.row0 + i] * d.inv_n - bS * d.inv_2n2);
    bt.u[d.row0 + i] = ui;
    float mx = fabsf(ui);
    for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&bt.ctr[t].max_u_bits, __float_as_uint(mx));
    const double tot = block_sum_256((double)ui, sh);
    if (threadIdx.x == 0) bt.Upart[gp] = tot;
}

// Step 2 (one CTA per panel): r~_i, dcorr_i = kappa r~_i, Stpart[panel] = sum of r~_i.
__global__ void __launch_bounds__(256) k_center_r(const Batch bt) {
    __shared__ double sh[256];
    __shared__ double bU;
    const int64_t gp = blockIdx.x;
    const int t = find_test(bt.pre.panels, bt.n_tests, gp);
    const TestDesc d = bt.desc[t];
    if (threadIdx.x < 32) {
        const double U = warp_ordered_sum(bt.Upart + d.pan0, d.NP);
        if (threadIdx.x == 0) bU = U;
    }
    __syncthreads();
    const int64_t i = (gp - d.pan0) * PANEL + threadIdx.x;
    double rt = 0.0;
    if (i < d.n) rt = bt.r[d.row0 + i] - (double)d.n * (double)bt.u[d.row0 + i] - bU;
    bt.dcorr[d.row0 + i] = d.kappa * rt;
    float mx = (float)fabs(d.kappa * rt);
    for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&bt.ctr[t].max_dc_bits, __float_as_uint(mx));
    const double tot = block_sum_256(rt, sh);
    if (threadIdx.x == 0) bt.Stpart[gp] = tot;
}

void launch_center(const Batch &b, cudaStream_t s) {
    if (b.npan_total <= 0) return;
    k_center_u<<<(unsigned)b.npan_total, 256, 0, s>>>(b);
    k_center_r<<<(unsigned)b.npan_total, 256, 0, s>>>(b);
}

// Packing.  Stored entry (i, j), j >= 256*panel(i):
//   j > i:  2 * ((D_ij - u_i) - u_j)      (upper triangle counted twice: s'Cs over
//                                           the upper triangle = the full form)
//   j = i:  D_ii - 2 u_i - dcorr_i
//   j < i or padding: 0
// FP32 in place (plain path), or (tuned path) c C split into FP16 hi + lo parts,
// hi = fp16(c C), lo = fp16(c C - hi), with the test's power-of-two scale c
// (packed_scale): |c C - hi - lo| <= 2^-22 |c C|, written over the block's own FP32
// storage (Batch::Chi / Clo with block stride c_stride), so the packed operand needs
// no memory of its own.  One CTA per block.
template <bool SPLIT>
__global__ void __launch_bounds__(512) k_pack(const Batch bt) {
    const int64_t gb = blockIdx.x;
    const BlkInfo bi = bt.blk[gb];
    const TestDesc d = bt.desc[bi.t];
    const int64_t n = d.n;
    const float *u = bt.u + d.row0;
    const double *dcorr = bt.dcorr + d.row0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j0 = (int64_t)bi.kb * KB + 2 * lane;
    const float uj[2] = {(j0 < n) ? u[j0] : 0.f, (j0 + 1 < n) ? u[j0 + 1] : 0.f};
    const int64_t row0 = (int64_t)bi.I * PANEL + warp * 16;   // 16 warps x 16 rows
    const float cs = SPLIT ? packed_scale(bt.ctr[bi.t]) : 1.f;
    // the whole block is read before any of it is rewritten: the split parts are
    // written over the block's own FP32 storage (hi in its first half, lo in its second)
    float2 dv[16];
#pragma unroll
    for (int q = 0; q < 16; ++q)
        dv[q] = *reinterpret_cast<const float2 *>(bt.D + (gb * PANEL + warp * 16 + q) * KB + 2 * lane);
    if (SPLIT) __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int64_t i = row0 + q;
        const float ui = (i < n) ? u[i] : 0.f;
        const float dq[2] = {dv[q].x, dv[q].y};
        float w[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t j = j0 + e;
            float v = 0.f;
            if (i < n && j < n && j >= i) {
                if (j == i) v = (float)((double)dq[e] - 2.0 * (double)ui - dcorr[i]);
                else v = 2.f * ((dq[e] - ui) - uj[e]);
            }
            w[e] = v;
        }
        const int64_t r = warp * 16 + q;
        if (SPLIT) {
            const float a0 = w[0] * cs, a1 = w[1] * cs;   // exact: cs is a power of two
            const __half h0 = __float2half_rn(a0), h1 = __float2half_rn(a1);
            const __half l0 = __float2half_rn(a0 - __half2float(h0));
            const __half l1 = __float2half_rn(a1 - __half2float(h1));
            const uint32_t hv = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
            const uint32_t lv = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
            const int64_t off = gb * bt.c_stride + r * KB + 2 * lane;
            *reinterpret_cast<uint32_t *>(bt.Chi + off) = hv;
            *reinterpret_cast<uint32_t *>(bt.Clo + off) = lv;
        } else {
            *reinterpret_cast<float2 *>(bt.D + (gb * PANEL + r) * KB + 2 * lane) = make_float2(w[0], w[1]);
        }
    }
}

void launch_pack(const Batch &b, bool split, cudaStream_t s) {
    if (b.nblk_total <= 0) return;
    if (split) k_pack<true><<<(unsigned)b.nblk_total, 512, 0, s>>>(b);
    else k_pack<false><<<(unsigned)b.nblk_total, 512, 0, s>>>(b);
}

// ---------------------------------------------------------------------------
// Plain FP32 contraction (the comparison path).  Work item = (test, chunk q =
// (panel I, K-blocks [kb0, kb1)), half h of the panel's rows, 64 relabeling columns):
//   U[b, i] = sum_{j in chunk} s_b[j] C[i, j]     (FP32 FMA, masks as 0/1 floats)
//   partial[(2q + h)][b] = sum_{i in half} s_b[i] U[b, i]
// 256 threads, each 4 relabelings x 8 rows; columns staged 32 at a time.
__global__ void __launch_bounds__(256) k_contract_simt(const Batch bt) {
    __shared__ float Cs[32][128 + 4];
    __shared__ uint32_t Ms[64];
    const int64_t w = blockIdx.x;
    const int tt = find_test(bt.pre.simt, bt.n_tests, w);
    const TestDesc d = bt.desc[tt];
    const int64_t lw = w - bt.pre.simt[tt];
    const int64_t tiles = d.Bp / 64;
    const int64_t q = lw / (2 * tiles), rem = lw % (2 * tiles);
    const int h = (int)(rem / tiles);
    const int64_t b0 = (rem % tiles) * 64;
    const Chunk ch = bt.chunks[d.chunk0 + q];
    const uint32_t *maskT = bt.maskT + d.mask0;
    const int64_t Bp = d.Bp;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[a][r] = 0.f;

    for (int kb = ch.kb0; kb < ch.kb1; ++kb) {
        const float *blkp = bt.D + (d.blk0 + blk_index(ch.I, kb, d.NKB)) * (int64_t)(PANEL * KB) + (int64_t)h * 128 * KB;
        for (int sub = 0; sub < 2; ++sub) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int idx = e * 256 + t, r = idx >> 5, j = idx & 31;
                Cs[j][r] = blkp[(int64_t)r * KB + sub * 32 + j];
            }
            if (t < 64) Ms[t] = maskT[(int64_t)(2 * kb + sub) * Bp + b0 + t];
            __syncthreads();
            uint32_t mw[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) mw[a] = Ms[ty * 4 + a];
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const float4 c0 = *reinterpret_cast<const float4 *>(&Cs[j][tx * 8]);
                const float4 c1 = *reinterpret_cast<const float4 *>(&Cs[j][tx * 8 + 4]);
                const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float f = ((mw[a] >> j) & 1u) ? 1.f : 0.f;
#pragma unroll
                    for (int r = 0; r < 8; ++r) acc[a][r] = fmaf(f, cv[r], acc[a][r]);
                }
            }
            __syncthreads();
        }
    }
    // rows tx*8 .. tx*8+7 of this half lie in one mask word
    const int64_t word = (int64_t)ch.I * (PANEL / 32) + h * 4 + (tx >> 2);
    const int shift = (tx & 3) * 8;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t b = b0 + ty * 4 + a;
        const uint32_t bits = (maskT[word * Bp + b] >> shift) & 0xFFu;
        float v = 0.f;
#pragma unroll
        for (int r = 0; r < 8; ++r) v += ((bits >> r) & 1u) ? acc[a][r] : 0.f;
        for (int off = 8; off; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
        if (tx == 0) bt.partial[d.part0 + (2 * q + h) * Bp + b] = v;
    }
}

void launch_contract_simt(const Batch &b, cudaStream_t s) {
    if (b.nsimt_total <= 0) return;
    k_contract_simt<<<(unsigned)b.nsimt_total, 256, 0, s>>>(b);
}

// ---------------------------------------------------------------------------
// Final combination (Algorithm 1, statistic and p-value lines): per relabeling
// column b, Q_b = sum of its partials, stat_b = sign * (cT Q_b + S~/o^2).  A CTA
// covers 32 columns of one test (the column padding is a multiple of 256): lane l of
// each of its 16 warps reads column l of every 16th partial (one coalesced 128-byte
// row per load, eight loads in flight), and the 16 warp sums are added in a fixed
// order (deterministic).
// Then k_combine_count compares against stat_0 (the identity, evaluated by the same
// kernels): stat_b >= stat_0 and near-ties |stat_b - stat_0| <= 1e-5 |stat_0|.
__global__ void __launch_bounds__(512) k_combine_stats(const Batch bt) {
    constexpr int NW = 16;   // warps: parts k = warp, warp + NW, ...
    __shared__ double bSt;
    __shared__ double ws[NW][32], wa[NW][32];
    const int64_t gc0 = (int64_t)blockIdx.x * 32;
    const int t = find_test(bt.pre.cols, bt.n_tests, gc0);
    const TestDesc &d = bt.desc[t];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        const double St = warp_ordered_sum(bt.Stpart + d.pan0, d.NP);
        if (lane == 0) bSt = St;
    }
    const int64_t c = gc0 + lane - bt.pre.cols[t];
    const int64_t Bp = d.Bp, nparts = d.nparts;
    const float *part = bt.partial + d.part0 + c;
    // a warp's parts summed as an unevaluated FP32 pair (TwoSum: each addition's
    // rounding error is kept exactly), so that no FP64 operation runs per partial;
    // the pairs of the warps then meet in FP64 in a fixed order
    float h = 0.f, l = 0.f, aabs = 0.f;
#pragma unroll 8
    for (int64_t k = warp; k < nparts; k += NW) {
        const float v = part[k * Bp];
        float s2, e;
        two_sum(h, v, s2, e);
        h = s2;
        l += e;
        aabs += fabsf(v);
    }
    ws[warp][lane] = (double)h + (double)l;
    wa[warp][lane] = (double)aabs;
    __syncthreads();
    if (warp == 0) {
        double q = 0.0, a = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            q += ws[w][lane];
            a += wa[w][lane];
        }
        // the tensor-core path accumulates c Q (packed operand scaled by c); 1/c is exact
        const double inv_c = d.scaled ? 1.0 / (double)packed_scale(bt.ctr[t]) : 1.0;
        if (c < d.ncols) {
            bt.stats[d.col0 + c] = d.sign * (d.cT * (q * inv_c) + bSt * d.inv_o2);
            // accumulation part of the error estimate (ept_internal.cuh, refine_ka)
            if (bt.errest) bt.errest[d.col0 + c] = d.ka * REFINE_U * d.cT * (a * inv_c);
        }
    }
}

// Errors of test t that the host will report: non-finite data, malformed
// relabelings, a median bandwidth that is not positive and finite.
__device__ __forceinline__ bool test_failed(const Batch &bt, int t) {
    const Counters &k = bt.ctr[t];
    bool f = k.nonfinite || k.bad_mask;
    if (bt.desc[t].median) {
        const float sg = __uint_as_float(k.sel_prefix);
        f = f || !(sg > 0.f) || !isfinite(sg);
    }
    return f;
}

// Whether any test of a batch failed (one CTA): a batched call that returns an
// error writes none of its device outputs.
__global__ void __launch_bounds__(256) k_batch_status(const Batch bt) {
    int bad = 0;
    for (int t = threadIdx.x; t < bt.n_tests; t += blockDim.x) bad |= test_failed(bt, t) ? 1 : 0;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0 && bad) bt.ctr[0].batch_failed = 1ull;
}

// Counting and outputs: a CTA covers 256 columns of one test.  A caller's device
// buffer of permuted statistics is written only when the call will succeed (no
// error in any test of the call, no expired wait), so that output buffers are
// written only on success.
// With `flag` (the first count of a run), also the error criterion: statistic c is
// flagged for FP64 recomputation when E_c > REFINE_TOL |stat_c| (ept_internal.cuh).
__global__ void __launch_bounds__(256) k_combine_count(const Batch bt, int flag) {
    __shared__ double bW;
    const int64_t gc = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int t = find_test(bt.pre.cols, bt.n_tests, (int64_t)blockIdx.x * 256);
    const TestDesc d = bt.desc[t];
    const int64_t c = gc - bt.pre.cols[t];
    const double obs = bt.stats[d.col0];
    if (flag && bt.flags) {
        if (threadIdx.x < 32) {
            const double S = warp_ordered_sum(bt.Spart + d.sp0, d.n_pad / 32);
            if (threadIdx.x == 0) bW = S * d.inv_n * d.inv_n;
        }
        __syncthreads();
        int fl = 0;
        if (c < d.ncols) {
            const double v = bt.stats[d.col0 + c];
            const double rep = REFINE_KR * REFINE_U * fabs(bW) / (double)d.m;
            // errest holds refine_ka u cT A; the observed and aligned statistics take REFINE_KC_RATIO times it
            const double e0 = REFINE_KC_RATIO * bt.errest[d.col0] + rep;
            const bool aligned = c == 0 || fabs(v - obs) <= REFINE_TOL * fabs(obs) + 2.0 * e0;
            const double acc = aligned ? REFINE_KC_RATIO * bt.errest[d.col0 + c] : bt.errest[d.col0 + c];
            const double tol = REFINE_TOL * fabs(v);
            // flagged when the estimate exceeds the tolerance; 2 (rebuild the entries in FP64)
            // when the representation term exceeds REFINE_L2 of it, else 1 (re-sum the
            // packed operand exactly).  NaN-safe: a non-finite estimate takes the rebuild
            const int lvl = !(acc + rep <= tol) ? (!(rep <= REFINE_L2 * tol) ? 2 : 1) : 0;
            fl = lvl != 0;
            bt.flags[d.col0 + c] = (uint8_t)lvl;
        }
        fl = __syncthreads_count(fl);
        if (threadIdx.x == 0 && fl) atomicAdd(&bt.ctr[t].n_flag, (unsigned long long)fl);
    }
    int ge = 0, near = 0;
    if (c >= 1 && c < d.ncols) {
        const double v = bt.stats[d.col0 + c];
        ge = v >= obs;
        near = fabs(v - obs) <= 1e-5 * fabs(obs);
        if (d.out_stats) {
            if (!test_failed(bt, t) && !bt.ctr[0].err_code && !bt.ctr[0].batch_failed) d.out_stats[c - 1] = v;
        }
    }
    if (c == 0) bt.observed[t] = obs;
    ge = __syncthreads_count(ge);
    near = __syncthreads_count(near);
    if (threadIdx.x == 0) {
        if (ge) atomicAdd(&bt.ctr[t].n_ge, (unsigned long long)ge);
        if (near) atomicAdd(&bt.ctr[t].n_near, (unsigned long long)near);
    }
}

void launch_combine(const Batch &b, cudaStream_t s) {
    if (b.ncols_total <= 0) return;
    if (b.n_tests > 1) k_batch_status<<<1, 256, 0, s>>>(b);
    k_combine_stats<<<(unsigned)(b.ncols_total / 32), 512, 0, s>>>(b);
    k_combine_count<<<(unsigned)(b.ncols_total / 256), 256, 0, s>>>(b, 1);
}

void launch_combine_count(const Batch &b, cudaStream_t s) {
    if (b.ncols_total <= 0) return;
    k_combine_count<<<(unsigned)(b.ncols_total / 256), 256, 0, s>>>(b, 0);
}

__global__ void k_reset_counts(Counters *ctr, int n_tests) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tests) {
        ctr[t].n_ge = 0;
        ctr[t].n_near = 0;
    }
}

void launch_reset_counts(const Batch &b, cudaStream_t s) {
    if (b.n_tests <= 0) return;
    k_reset_counts<<<(unsigned)((b.n_tests + 255) / 256), 256, 0, s>>>(b.ctr, b.n_tests);
}

// ---------------------------------------------------------------------------
// Expand one test's packed upper storage into a full row-major n x n matrix
// (checking aid).
__global__ void k_expand(const float *__restrict__ D, int64_t n, int64_t NKB, float *__restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int64_t i = idx / n, j = idx % n;
    if (j / PANEL < i / PANEL) {
        const int64_t tmp = i;
        i = j;
        j = tmp;
    }
    const int64_t I = i / PANEL, kb = j / KB;
    out[idx] = D[(blk_index(I, kb, NKB) * PANEL + (i - I * PANEL)) * KB + (j - kb * KB)];
}

void launch_expand_blocks(const float *D, int64_t n, int64_t NKB, float *out, cudaStream_t s) {
    const int64_t tot = n * n;
    if (tot <= 0) return;
    k_expand<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(D, n, NKB, out);
}

// ---------------------------------------------------------------------------
// Debug checks: one CTA per guard band fills it with a pattern that depends on the
// band's index, or counts the words that no longer hold it.
__global__ void k_guards(uint8_t *arena, GuardList g, int check, Counters *ctr) {
    const int k = blockIdx.x;
    if (k >= g.n) return;
    uint32_t *w = reinterpret_cast<uint32_t *>(arena + g.off[k]);
    const uint32_t pat = 0xA5C3E1F0u ^ (uint32_t)(k * 0x9E3779B9u);
    unsigned bad = 0;
    for (int i = threadIdx.x; i < GUARD_BYTES / 4; i += blockDim.x) {
        if (check) bad += (w[i] != (pat ^ (uint32_t)i));
        else w[i] = pat ^ (uint32_t)i;
    }
    if (check) {
        for (int off = 16; off; off >>= 1) bad += __shfl_xor_sync(0xFFFFFFFFu, bad, off);
        if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&ctr->guard_bad, (unsigned long long)bad);
    }
}

void launch_guards(uint8_t *arena, const GuardList &g, bool check, Counters *ctr, cudaStream_t s) {
    if (g.n <= 0) return;
    k_guards<<<(unsigned)g.n, 32, 0, s>>>(arena, g, check ? 1 : 0, ctr);
}

}  // namespace ept

// ept_kernels.cu -- SIMT kernels of libept: permutation stream, block build,
// centring and packing, the plain FP32 contraction and the final combination.
#include "ept_internal.cuh"

#include <cuda_bf16.h>
#include <cstdint>

namespace ept {

Geom make_geom(int64_t nx, int64_t ny, int64_t p, int64_t ncols) {
    Geom g;
    g.nx = nx; g.ny = ny; g.n = nx + ny; g.p = p;
    g.n_pad = (g.n + PANEL - 1) / PANEL * PANEL;
    g.NP = g.n_pad / PANEL;
    g.NKB = g.n_pad / KB;
    g.nblk = blk_off(g.NP, g.NKB);
    g.nw = g.n_pad / 32;
    g.ncols = ncols;
    g.Bp = (ncols + COL_PAD - 1) / COL_PAD * COL_PAD;
    int64_t q = 0;
    for (int64_t I = 0; I < g.NP; ++I) {
        const int64_t len = g.NKB - KB_PER_PANEL * I;
        q += (len + CHUNK_KB - 1) / CHUNK_KB;
    }
    g.nchunks = q;
    g.comp = ny < nx;
    g.m = g.comp ? ny : nx;
    g.other = g.comp ? nx : ny;
    return g;
}

// ---------------------------------------------------------------------------
// Permutation stream: Philox4x32-10 (Salmon et al., SC'11) drives Knuth's selection
// sampling; see k_perm_masks.
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

// One warp per relabeling column c.  Philox4x32-10: each round multiplies counter
// words 0 and 2 by the two Philox multipliers (one wide multiply gives both
// halves), mixes the high halves with words 1 and 3 and the round key, and the key
// advances by the two Weyl constants between rounds.
// Draw b = b_first + c of the stream:
// b = 0 is the identity; b >= 1 is Knuth's selection sampling (Algorithm S) over
// the n pooled slots, slot t kept iff floor(u_t * (n - t) / 2^64) < need, with
// u_t the 64-bit word (t mod 2) of Philox4x32-10(counter = (t/2, 0, b lo, b hi),
// key = (seed lo, seed hi)).  The warp draws 64 consecutive slots at once: lane l
// runs the Philox call of slots base+2l and base+2l+1 and forms their two
// floor(u (n - t) / 2^64) values; shuffles then place slot base+l on lane l (first
// word) and slot base+32+l on lane l (second word), so one ballot is one output
// word.  The sequential dependence through `need` is resolved by a fixed-point
// iteration over ballots: with every earlier decision known a slot's decision is
// determined, so iterating "decide from the previous guesses" reaches the unique
// sequential solution in at most 65 rounds (almost always 1 or 2).
// comp: store the complement (the y* members) of every real draw.
__global__ void __launch_bounds__(256) k_perm_masks(uint64_t seed, int nx, int ny, int64_t b_first,
                                                    int64_t count, int64_t ncols, int nw, int comp,
                                                    uint32_t *__restrict__ maskT) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= ncols) return;
    const int n = nx + ny;
    uint32_t *col = maskT + c;
    if (c >= count) {
        for (int w = lane; w < nw; w += 32) col[(int64_t)w * ncols] = 0u;
        return;
    }
    const int64_t b = b_first + c;
    if (b == 0) {
        for (int w = lane; w < nw; w += 32) {
            const uint32_t v = valid_bits(w, nx);
            col[(int64_t)w * ncols] = comp ? (~v & valid_bits(w, n)) : v;
        }
        return;
    }
    // Philox round keys of this seed (the key schedule adds the two Weyl constants)
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
    for (int base = 0; base < nw * 32; base += 64) {
        const int tp = base + 2 * lane;   // this lane's Philox slots tp, tp + 1
        uint32_t ra = 0xFFFFFFFFu, rb = 0xFFFFFFFFu;   // "never kept"
        if (tp < n && need > 0) {
            uint32_t x0 = (uint32_t)(tp >> 1), x1 = 0u, x2 = blo, x3 = bhi;
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
            ra = (uint32_t)mulhi_64x32(((uint64_t)x1 << 32) | x0, (uint32_t)(n - tp));
            if (tp + 1 < n) rb = (uint32_t)mulhi_64x32(((uint64_t)x3 << 32) | x2, (uint32_t)(n - tp - 1));
        }
        // slot base + lane  <- (ra or rb) of lane lane/2;  slot base + 32 + lane <- of lane 16 + lane/2
        const uint32_t a0 = __shfl_sync(0xFFFFFFFFu, ra, src), b0 = __shfl_sync(0xFFFFFFFFu, rb, src);
        const uint32_t a1 = __shfl_sync(0xFFFFFFFFu, ra, src + 16), b1 = __shfl_sync(0xFFFFFFFFu, rb, src + 16);
        const int r0 = (int)min(odd ? b0 : a0, 0x7FFFFFFFu);
        const int r1 = (int)min(odd ? b1 : a1, 0x7FFFFFFFu);
        bool s0 = r0 < need, s1 = r1 < need;
        unsigned m0 = __ballot_sync(0xFFFFFFFFu, s0), m1 = __ballot_sync(0xFFFFFFFFu, s1);
        for (int it = 0; it < 70; ++it) {
            const int before0 = __popc(m0 & lt);
            const int before1 = __popc(m0) + __popc(m1 & lt);
            const bool n0 = r0 < need - before0;
            const bool n1 = r1 < need - before1;
            const unsigned nm0 = __ballot_sync(0xFFFFFFFFu, n0), nm1 = __ballot_sync(0xFFFFFFFFu, n1);
            const bool same = (nm0 == m0) && (nm1 == m1);
            m0 = nm0;
            m1 = nm1;
            if (same) break;
        }
        need -= __popc(m0) + __popc(m1);
        if (lane == 0) {
            const int w = base >> 5;
            uint32_t v0 = m0, v1 = m1;
            if (comp) {
                v0 = ~v0 & valid_bits(w, n);
                v1 = ~v1 & valid_bits(w + 1, n);
            }
            col[(int64_t)w * ncols] = v0;
            col[(int64_t)(w + 1) * ncols] = v1;
        }
    }
}

void launch_perm_masks(uint64_t seed, int nx, int ny, int64_t b_first, int64_t count, int64_t ncols,
                       int nw, bool comp, uint32_t *maskT, cudaStream_t s) {
    const int warps = 8;
    const int64_t grid = (ncols + warps - 1) / warps;
    k_perm_masks<<<(unsigned)grid, warps * 32, 0, s>>>(seed, nx, ny, b_first, count, ncols, nw, comp ? 1 : 0,
                                                       maskT);
}

// Caller-given relabelings, row-major [m][nwu], become columns 1..n_masks of maskT;
// column 0 is written as the identity by the caller.  A relabeling with a popcount
// other than nx, or with bits at t >= n, is counted in ctr->bad_mask.
__global__ void k_user_masks(const uint32_t *__restrict__ user, int64_t n_masks, int nwu, int nx, int n,
                             int64_t ncols, int nw, int comp, uint32_t *__restrict__ maskT, Counters *ctr) {
    const int lane = threadIdx.x & 31;
    const int64_t m = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (m >= n_masks) return;
    const uint32_t *row = user + m * nwu;
    uint32_t *col = maskT + (m + 1);
    int cnt = 0;
    bool bad = false;
    for (int w = lane; w < nw; w += 32) {
        uint32_t v = (w < nwu) ? row[w] : 0u;
        const uint32_t valid = valid_bits(w, n);
        if (v & ~valid) bad = true;
        v &= valid;
        cnt += __popc(v);
        col[(int64_t)w * ncols] = comp ? (~v & valid_bits(w, n)) : v;
    }
    for (int off = 16; off; off >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, off);
    bad = __any_sync(0xFFFFFFFFu, bad);
    if (lane == 0 && (bad || cnt != nx)) atomicAdd(&ctr->bad_mask, 1ull);
}

void launch_user_masks(const uint32_t *user, int64_t n_masks, int nwu, int nx, int n, int64_t ncols,
                       int nw, bool comp, uint32_t *maskT, Counters *ctr, cudaStream_t s) {
    if (n_masks <= 0) return;
    const int warps = 8;
    k_user_masks<<<(unsigned)((n_masks + warps - 1) / warps), warps * 32, 0, s>>>(user, n_masks, nwu, nx, n,
                                                                                 ncols, nw, comp ? 1 : 0, maskT, ctr);
}

// maskT columns 0..count-1 -> row-major [count][nwu]
__global__ void k_masks_to_rows(const uint32_t *__restrict__ maskT, int64_t ncols, int nw, int64_t count,
                                int nwu, uint32_t *__restrict__ rows) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count * nwu) return;
    const int64_t c = idx / nwu;
    const int w = (int)(idx % nwu);
    rows[idx] = maskT[(int64_t)w * ncols + c];
}

void launch_masks_to_rows(const uint32_t *maskT, int64_t ncols, int nw, int64_t count, int nwu,
                          uint32_t *rows, cudaStream_t s) {
    const int64_t tot = count * nwu;
    if (tot <= 0) return;
    k_masks_to_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(maskT, ncols, nw, count, nwu, rows);
}

// ---------------------------------------------------------------------------
// Counts non-finite inputs and records max |x| (non-negative FP32 values order like
// their bit patterns, so an integer atomicMax on the bits gives the maximum).
__global__ void k_check_finite(const float *__restrict__ a, int64_t count, Counters *ctr) {
    bool bad = false;
    uint32_t mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = a[i];
        if (isfinite(v)) mx = max(mx, __float_as_uint(fabsf(v)));
        else bad = true;
    }
    for (int off = 16; off; off >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicAdd(&ctr->nonfinite, 1ull);
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&ctr->maxabs_bits, (unsigned long long)mx);
}

void launch_check_finite(const float *a, int64_t count, Counters *ctr, cudaStream_t s) {
    if (count <= 0) return;
    int64_t grid = (count + 255) / 256;
    if (grid > 4096) grid = 4096;
    k_check_finite<<<(unsigned)grid, 256, 0, s>>>(a, count, ctr);
}

__device__ __forceinline__ const float *pooled_row(const float *X, const float *Y, int64_t nx, int64_t i,
                                                   int64_t p) {
    return (i < nx) ? X + i * p : Y + (i - nx) * p;
}

// Squared row norms ||z_i||^2 of the pooled rows, exact products summed in FP64 and
// rounded once to FP32 (padded rows: 0).  One warp per row.
__global__ void k_norms(const float *__restrict__ X, const float *__restrict__ Y, int64_t nx, int64_t n,
                        int64_t n_pad, int64_t p, float *__restrict__ norms) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n_pad) return;
    double acc = 0.0;
    if (i < n) {
        const float *z = pooled_row(X, Y, nx, i, p);
        for (int64_t k = lane; k < p; k += 32) {
            const double v = (double)z[k];
            acc = fma(v, v, acc);
        }
    }
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if (lane == 0) norms[i] = (float)acc;
}

void launch_norms(const float *X, const float *Y, const Geom &g, float *norms, cudaStream_t s) {
    const int warps = 8;
    k_norms<<<(unsigned)((g.n_pad + warps - 1) / warps), warps * 32, 0, s>>>(X, Y, g.nx, g.n, g.n_pad, g.p,
                                                                              norms);
}

// ---------------------------------------------------------------------------
// Block build, SIMT FP32 (Algorithm 1 block construction; Algorithm 3 entries
// through the expansion ||x||^2 + ||y||^2 - 2 x.y).  One CTA computes half of a
// stored 256x64 block (128 rows x 64 columns): 256 threads, 8x4 outputs each,
// K-loop over p in steps of 16 staged through shared memory.
// Epilogue: d2 = max(0, n_i + n_j - 2 g_ij); a pair with d2 < tau (n_i + n_j)
// (cancellation-prone near-duplicate) is recomputed directly as sum (x - y)^2 in
// FP64; then sqrt (ED) or exp(-d2 / (2 sigma^2)) (MMD); the diagonal is exactly 0
// (ED) or 1 (MMD); padded rows and columns are 0.
__device__ __forceinline__ float finish_entry(float d2, int stat, float neg_inv_2s2) {
    return stat == 0 ? sqrtf(d2) : expf(d2 * neg_inv_2s2);
}

__global__ void __launch_bounds__(256) k_build_simt(const float *__restrict__ X, const float *__restrict__ Y,
                                                    const float *__restrict__ norms, int64_t nx, int64_t n,
                                                    int64_t p, int64_t NKB, int stat, float neg_inv_2s2,
                                                    float tau, const int2 *__restrict__ blk_info,
                                                    float *__restrict__ D, Counters *ctr) {
    __shared__ float As[16][128 + 4];
    __shared__ float Bs[16][64 + 4];
    const int64_t blk = blockIdx.x;
    const int h = blockIdx.y;
    const int2 bi = blk_info[blk];
    const int64_t row0 = (int64_t)bi.x * PANEL + h * 128;
    const int64_t col0 = (int64_t)bi.y * KB;
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
            if (i < n && k0 + k < p) v = pooled_row(X, Y, nx, i, p)[k0 + k];
            As[k][r] = v;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = e * 256 + t, cc = idx >> 4, k = idx & 15;
            const int64_t j = col0 + cc;
            float v = 0.f;
            if (j < n && k0 + k < p) v = pooled_row(X, Y, nx, j, p)[k0 + k];
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
                    v = (stat == 0) ? 0.f : 1.f;
                } else {
                    const float ni = norms[i], nj = norms[j];
                    float d2 = fmaxf(0.f, ni + nj - 2.f * acc[a][c]);
                    if (d2 < tau * (ni + nj)) {
                        const float *zi = pooled_row(X, Y, nx, i, p), *zj = pooled_row(X, Y, nx, j, p);
                        double s = 0.0;
                        for (int64_t k = 0; k < p; ++k) {
                            const double d = (double)zi[k] - (double)zj[k];
                            s = fma(d, d, s);
                        }
                        ++fixups;
                        v = (stat == 0) ? (float)sqrt(s) : (float)exp(s * (double)neg_inv_2s2);
                    } else {
                        v = finish_entry(d2, stat, neg_inv_2s2);
                    }
                }
            }
            out[c] = v;
        }
        const int64_t off = (blk * PANEL + h * 128 + ty * 8 + a) * KB + tx * 4;
        *reinterpret_cast<float4 *>(D + off) = make_float4(out[0], out[1], out[2], out[3]);
    }
    if (fixups) atomicAdd(&ctr->n_fixup, (unsigned long long)fixups);
}

void launch_build_simt(const float *X, const float *Y, const float *norms, const Geom &g, int stat,
                       double sigma, double tau, const int2 *blk_info, float *D, Counters *ctr,
                       cudaStream_t s) {
    const float neg = (stat == 0) ? 0.f : (float)(-1.0 / (2.0 * sigma * sigma));
    dim3 grid((unsigned)g.nblk, 2);
    k_build_simt<<<grid, 256, 0, s>>>(X, Y, norms, g.nx, g.n, g.p, g.NKB, stat, neg, (float)tau, blk_info, D,
                                     ctr);
}

// ---------------------------------------------------------------------------
// Row and column partial sums of each stored block, for the row sums r = W 1
// (the lower part of W is the transpose of the stored strictly-upper blocks, so
// their column sums supply it).  Sums are accumulated as unevaluated FP32 pairs
// (hi, lo) with Knuth's TwoSum, an error-free transformation (the rounding error of
// every addition is carried in lo), then widened to FP64: about twice the FP32
// precision at FP32 cost.  One CTA (8 warps) per block, one row per warp step,
// lane l owns columns 2l and 2l+1.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__global__ void __launch_bounds__(256) k_blocksums(const float *__restrict__ D, double *__restrict__ rowpart,
                                                   double *__restrict__ colpart) {
    __shared__ double cs[8][64];
    const int64_t blk = blockIdx.x;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const float *base = D + blk * (int64_t)(PANEL * KB);
    // row sums: thread t owns row t (64 contiguous values, no cross-thread traffic)
    {
        const float4 *row = reinterpret_cast<const float4 *>(base + (int64_t)t * KB);
        float4 v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = row[q];
        float h = 0.f, l = 0.f;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float e4[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float s2, f;
                two_sum(h, e4[k], s2, f);
                h = s2;
                l += f;
            }
        }
        rowpart[blk * PANEL + t] = (double)h + (double)l;
    }
    // column sums: warp w covers rows 32w..32w+31, lane l columns 2l and 2l+1
    {
        const float *cbase = base + (int64_t)(warp * 32) * KB + 2 * lane;
        float ch0 = 0.f, cl0 = 0.f, ch1 = 0.f, cl1 = 0.f;
#pragma unroll 1
        for (int r0 = 0; r0 < 32; r0 += 8) {
            float2 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = *reinterpret_cast<const float2 *>(cbase + (int64_t)(r0 + q) * KB);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float s2, f;
                two_sum(ch0, v[q].x, s2, f);
                ch0 = s2;
                cl0 += f;
                two_sum(ch1, v[q].y, s2, f);
                ch1 = s2;
                cl1 += f;
            }
        }
        cs[warp][2 * lane] = (double)ch0 + (double)cl0;
        cs[warp][2 * lane + 1] = (double)ch1 + (double)cl1;
    }
    __syncthreads();
    if (t < 64) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) acc += cs[w][t];
        colpart[blk * KB + t] = acc;
    }
}

void launch_blocksums(const float *D, const Geom &g, double *rowpart, double *colpart, cudaStream_t s) {
    k_blocksums<<<(unsigned)g.nblk, 256, 0, s>>>(D, rowpart, colpart);
}

// r_i = sum over the stored blocks of row i's panel (its own row segments) + sum
// over the earlier panels J < panel(i) of column i's segments.  Eight threads per
// row take every eighth term and combine by a fixed shuffle tree (deterministic).
// CTA = 32 rows (256 threads); Spart[CTA] = sum of its rows' r_i.
__global__ void __launch_bounds__(256) k_rowsum_reduce(const double *__restrict__ rowpart,
                                                       const double *__restrict__ colpart, int64_t n, int64_t NKB,
                                                       double *__restrict__ r, double *__restrict__ Spart) {
    __shared__ double sh[32];
    const int sub = threadIdx.x & 7, rl = threadIdx.x >> 3;
    const int64_t i = (int64_t)blockIdx.x * 32 + rl;
    const int64_t I = i / PANEL, rr = i % PANEL;
    double acc = 0.0;
    if (i < n) {
        const int64_t nkb = NKB - KB_PER_PANEL * I;          // stored K-blocks of panel I
        const int64_t base = blk_off(I, NKB);
        for (int64_t k = sub; k < nkb; k += 8) acc += rowpart[(base + k) * PANEL + rr];
        const int64_t kbi = i / KB, ci = i % KB;
        for (int64_t J = sub; J < I; J += 8) acc += colpart[blk_index(J, kbi, NKB) * KB + ci];
    }
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
    if (sub == 0) {
        r[i] = acc;
        sh[rl] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 32; ++k) s += sh[k];
        Spart[blockIdx.x] = s;
    }
}

void launch_rowsum_reduce(const double *rowpart, const double *colpart, const Geom &g, double *r, double *Spart,
                          cudaStream_t s) {
    k_rowsum_reduce<<<(unsigned)(g.n_pad / 32), 256, 0, s>>>(rowpart, colpart, g.n, g.NKB, r, Spart);
}

// Deterministic sum of a short array in fixed order.
__device__ __forceinline__ double ordered_sum(const double *a, int64_t m) {
    double s = 0.0;
    for (int64_t k = 0; k < m; ++k) s += a[k];
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
// Step 1 (one CTA per panel): u_i, Upart[panel] = sum of the u_i as doubles.
__global__ void __launch_bounds__(256) k_center_u(const double *__restrict__ r, const double *__restrict__ Spart,
                                                  int64_t nS, int64_t n, double inv_n, double inv_2n2,
                                                  float *__restrict__ u, double *__restrict__ Upart) {
    __shared__ double sh[256];
    __shared__ double bS;
    if (threadIdx.x == 0) bS = ordered_sum(Spart, nS);
    __syncthreads();
    const double S = bS;
    const int64_t i = (int64_t)blockIdx.x * PANEL + threadIdx.x;
    float ui = 0.f;
    if (i < n) ui = (float)(r[i] * inv_n - S * inv_2n2);
    u[i] = ui;
    const double tot = block_sum_256((double)ui, sh);
    if (threadIdx.x == 0) Upart[blockIdx.x] = tot;
}

// Step 2 (one CTA per panel): r~_i, dcorr_i = kappa r~_i, Stpart[panel] = sum of r~_i;
// block 0 also writes the constants of the final combination.
__global__ void __launch_bounds__(256) k_center_r(const double *__restrict__ r, const float *__restrict__ u,
                                                  const double *__restrict__ Upart, int64_t NP, int64_t n,
                                                  double kappa, double cT, double inv_o2, double sign,
                                                  double *__restrict__ dcorr, double *__restrict__ Stpart,
                                                  StatConst *sc) {
    __shared__ double sh[256];
    __shared__ double bU;
    if (threadIdx.x == 0) bU = ordered_sum(Upart, NP);
    __syncthreads();
    const double U = bU;
    const int64_t i = (int64_t)blockIdx.x * PANEL + threadIdx.x;
    double rt = 0.0;
    if (i < n) rt = r[i] - (double)n * (double)u[i] - U;
    dcorr[i] = kappa * rt;
    const double tot = block_sum_256(rt, sh);
    if (threadIdx.x == 0) {
        Stpart[blockIdx.x] = tot;
        if (blockIdx.x == 0) {
            sc->cT = cT;
            sc->inv_o2 = inv_o2;
            sc->sign = sign;
            sc->S_tilde = 0.0;
        }
    }
}

void launch_center(const double *r, const double *Spart, const Geom &g, float *u, double *dcorr, double *Upart,
                   double *Stpart, StatConst *sc, int stat, cudaStream_t s) {
    const double fn = (double)g.n;
    const double q = fn / ((double)g.nx * (double)g.ny);
    k_center_u<<<(unsigned)g.NP, 256, 0, s>>>(r, Spart, g.n_pad / 32, g.n, 1.0 / fn, 1.0 / (2.0 * fn * fn), u,
                                             Upart);
    k_center_r<<<(unsigned)g.NP, 256, 0, s>>>(r, u, Upart, g.NP, g.n, 2.0 * (double)g.m / fn, q * q,
                                             1.0 / ((double)g.other * (double)g.other), stat == 0 ? -1.0 : 1.0, dcorr,
                                             Stpart, sc);
}

// Packing.  Stored entry (i, j), j >= 256*panel(i):
//   j > i:  2 * ((D_ij - u_i) - u_j)      (upper triangle counted twice: s'Cs over
//                                           the upper triangle = the full form)
//   j = i:  D_ii - 2 u_i - dcorr_i
//   j < i or padding: 0
template <bool BF16>
__global__ void __launch_bounds__(256) k_pack(const float *__restrict__ D, const float *__restrict__ u,
                                              const double *__restrict__ dcorr, int64_t n,
                                              const int2 *__restrict__ blk_info, float *__restrict__ C32,
                                              uint16_t *__restrict__ Chi, uint16_t *__restrict__ Clo) {
    const int64_t blk = blockIdx.x;
    const int2 bi = blk_info[blk];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j0 = (int64_t)bi.y * KB + 2 * lane;
    const float uj[2] = {(j0 < n) ? u[j0] : 0.f, (j0 + 1 < n) ? u[j0 + 1] : 0.f};
    const int64_t row0 = (int64_t)bi.x * PANEL + warp * 32;
#pragma unroll 1
    for (int r0 = 0; r0 < 32; r0 += 8) {
        float2 d[8];
        float ui[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            d[q] = *reinterpret_cast<const float2 *>(D + (blk * PANEL + warp * 32 + r0 + q) * KB + 2 * lane);
            const int64_t i = row0 + r0 + q;
            ui[q] = (i < n) ? u[i] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t i = row0 + r0 + q;
            const int64_t off = (blk * PANEL + warp * 32 + r0 + q) * KB + 2 * lane;
            const float dv[2] = {d[q].x, d[q].y};
            float w[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int64_t j = j0 + e;
                float v = 0.f;
                if (i < n && j < n && j >= i) {
                    if (j == i) v = (float)((double)dv[e] - 2.0 * (double)ui[q] - dcorr[i]);
                    else v = 2.f * ((dv[e] - ui[q]) - uj[e]);
                }
                w[e] = v;
            }
            if (BF16) {
                const __nv_bfloat16 h0 = __float2bfloat16_rn(w[0]), h1 = __float2bfloat16_rn(w[1]);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(w[0] - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(w[1] - __bfloat162float(h1));
                const uint32_t hv = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                const uint32_t lv = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                *reinterpret_cast<uint32_t *>(Chi + off) = hv;
                *reinterpret_cast<uint32_t *>(Clo + off) = lv;
            } else {
                *reinterpret_cast<float2 *>(C32 + off) = make_float2(w[0], w[1]);
            }
        }
    }
}

void launch_pack_fp32(const float *D, const float *u, const double *dcorr, const Geom &g,
                      const int2 *blk_info, float *C, cudaStream_t s) {
    k_pack<false><<<(unsigned)g.nblk, 256, 0, s>>>(D, u, dcorr, g.n, blk_info, C, nullptr, nullptr);
}

void launch_pack_bf16(const float *D, const float *u, const double *dcorr, const Geom &g,
                      const int2 *blk_info, uint16_t *Chi, uint16_t *Clo, cudaStream_t s) {
    k_pack<true><<<(unsigned)g.nblk, 256, 0, s>>>(D, u, dcorr, g.n, blk_info, nullptr, Chi, Clo);
}

// ---------------------------------------------------------------------------
// Plain FP32 contraction (the comparison path).  For work chunk q (panel I,
// K-blocks [kb0, kb1)), half h of the panel's rows and 64 relabeling columns:
//   U[b, i] = sum_{j in chunk} s_b[j] C[i, j]     (FP32 FMA, masks as 0/1 floats)
//   partial[(2q + h)][b] = sum_{i in half} s_b[i] U[b, i]
// 256 threads, each 4 relabelings x 8 rows; columns staged 32 at a time.
__global__ void __launch_bounds__(256) k_contract_simt(const float *__restrict__ C, const uint32_t *__restrict__ maskT,
                                                       const Chunk *__restrict__ chunks, int64_t NKB, int64_t Bp,
                                                       float *__restrict__ partial) {
    __shared__ float Cs[32][128 + 4];
    __shared__ uint32_t Ms[64];
    const int q = blockIdx.x >> 1, h = blockIdx.x & 1;
    const Chunk ch = chunks[q];
    const int64_t b0 = (int64_t)blockIdx.y * 64;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[a][r] = 0.f;

    for (int kb = ch.kb0; kb < ch.kb1; ++kb) {
        const float *blkp = C + blk_index(ch.I, kb, NKB) * (int64_t)(PANEL * KB) + (int64_t)h * 128 * KB;
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
        if (tx == 0) partial[(int64_t)(2 * q + h) * Bp + b] = v;
    }
}

void launch_contract_simt(const float *C, const uint32_t *maskT, const Chunk *chunks, const Geom &g,
                          float *partial, cudaStream_t s) {
    dim3 grid((unsigned)(g.nchunks * 2), (unsigned)(g.Bp / 64));
    k_contract_simt<<<grid, 256, 0, s>>>(C, maskT, chunks, g.NKB, g.Bp, partial);
}

// ---------------------------------------------------------------------------
// Final combination (Algorithm 1, statistic and p-value lines): per relabeling
// column b, Q_b = sum of its partials in fixed order (FP64), stat_b =
// sign * (cT Q_b + S~/o^2).  Then, against stat_0 (the identity, evaluated by the
// same kernels), count stat_b >= stat_0 and near-ties |stat_b - stat_0| <= 1e-5 |stat_0|.
__global__ void __launch_bounds__(256) k_combine_stats(const float *__restrict__ partial, int64_t nparts, int64_t Bp,
                                                       int64_t ncols, const StatConst *__restrict__ sc,
                                                       const double *__restrict__ Stpart, int64_t NP,
                                                       double *__restrict__ stats) {
    // four threads per column: thread q of a column sums partials q, q+4, ...; the
    // four sums are combined by a fixed shuffle tree (deterministic)
    __shared__ double bSt;
    if (threadIdx.x == 0) bSt = ordered_sum(Stpart, NP);
    __syncthreads();
    const int q = threadIdx.x & 3;
    const int64_t b = (int64_t)blockIdx.x * 64 + (threadIdx.x >> 2);
    double acc = 0.0;
    if (b < ncols)
        for (int64_t k = q; k < nparts; k += 4) acc += (double)partial[k * Bp + b];
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
    if (b < ncols && q == 0) stats[b] = sc->sign * (sc->cT * acc + bSt * sc->inv_o2);
}

__global__ void k_combine_count(const double *__restrict__ stats, int64_t ncols, Counters *ctr) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double obs = stats[0];
    int ge = 0, near = 0;
    if (b >= 1 && b < ncols) {
        const double v = stats[b];
        ge = v >= obs;
        near = fabs(v - obs) <= 1e-5 * fabs(obs);
    }
    ge = __syncthreads_count(ge);
    near = __syncthreads_count(near);
    if (threadIdx.x == 0) {
        if (ge) atomicAdd(&ctr->n_ge, (unsigned long long)ge);
        if (near) atomicAdd(&ctr->n_near, (unsigned long long)near);
    }
}

void launch_combine(const float *partial, int64_t nparts, const Geom &g, const StatConst *sc,
                    const double *Stpart, double *stats, Counters *ctr, cudaStream_t s) {
    k_combine_stats<<<(unsigned)((g.ncols + 63) / 64), 256, 0, s>>>(partial, nparts, g.Bp, g.ncols, sc, Stpart, g.NP,
                                                                   stats);
    k_combine_count<<<(unsigned)((g.ncols + 255) / 256), 256, 0, s>>>(stats, g.ncols, ctr);
}

// ---------------------------------------------------------------------------
// Expand the packed upper storage into a full row-major n x n matrix (checking aid).
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

void launch_expand_blocks(const float *D, const Geom &g, float *out, cudaStream_t s) {
    const int64_t tot = g.n * g.n;
    k_expand<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(D, g.n, g.NKB, out);
}

}  // namespace ept

// a1: rasterisation of Manhattan clips and the per-clip signatures read by the
// lossless gates (Sec. 2.2.1 step 1; signatures for the pre-screening of
// Sec. 3.1 stage 1).
//
// One CTA per clip, one thread per raster row (blockDim = N <= 512).  The
// clip's rectangles are staged in shared memory in chunks; each thread ORs
// the pixel-centre runs of the rectangles that cover its row centre into its
// row words (registers), then the CTA derives the popcount, row/column
// profiles and the 16x16 block counts from the row words in shared memory.
#include "common.cuh"

namespace pcl {

namespace {

constexpr int kRectChunk = 256;

// Storage position of 16x16 block (by, bx) among the nb x nb blocks (nb a
// multiple of 4): blocks are grouped by (by mod 4, bx mod 4), groups in
// row-major order of that pair, blocks within a group row-major; at nb = 16
// the first 64 positions are the block rows 0, 4, 8 and 12.
__device__ __forceinline__ int blk_pos(int by, int bx, int nb) {
    const int q = nb >> 2;
    return (((by & 3) << 2) | (bx & 3)) * q * q + (by >> 2) * q + (bx >> 2);
}

// grid cell of coordinate v (floor division, clamped to the 64 cells)
__device__ __forceinline__ int cell_of(int v, int csz) {
    const int q = v >= 0 ? v / csz : -((-v + csz - 1) / csz);
    return q < 0 ? 0 : (q > 63 ? 63 : q);
}

// first pixel index i (clamped to [0, N]) whose centre p i + p/2 is >= v:
// ceil((2 v - p) / (2 p)), the pixel-centre rule of a rectangle edge at v
__device__ __forceinline__ int pix_from(int v, long long p, int N) {
    const long long a = 2LL * v - p, b = 2 * p;
    long long q = a / b;
    if (a % b != 0 && a > 0) ++q;
    return (int)(q < 0 ? 0 : (q > N ? N : q));
}

// 32 x 32 bit transpose across a warp: on entry lane l holds row l (bit b =
// column b), on return lane l holds column l (bit b = row b).  Five rounds of
// exchanging the off-diagonal halves of 2s x 2s blocks with lane l ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu
                         : s == 2 ? 0x33333333u : 0x55555555u;  // bit positions b with (b & s) == 0
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
        x = (lane & s) ? ((x & ~m) | ((y & ~m) >> s)) : ((x & m) | ((y & m) << s));
    }
    return x;
}

template <int NW>
__global__ void __launch_bounds__(512) raster_kernel(pcl_params prm, pcl_clipset cs) {
    constexpr int NR = 64 * NW;  // rows (N = 64 NW: 64^2 .. 512^2)
    const Geo g = make_geo(prm);
    const int c = blockIdx.x;
    const int j = threadIdx.x;  // row (y index)
    const int N = g.N;
    __shared__ int4 rs[kRectChunk];          // pixel ranges {i0, i1, j0, j1} of staged rectangles
    __shared__ uint64_t rows[NR * NW];
    __shared__ uint8_t colpart[NR / 32][NR];  // column counts over each warp's 32 rows
    __shared__ uint32_t red[32];

    const uint32_t r0 = cs.rect_off[c], r1 = cs.rect_off[c + 1];
    const long long p = g.p;
    uint64_t w[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) w[k] = 0ull;

    for (uint32_t base = r0; base < r1; base += kRectChunk) {
        const uint32_t cnt = min((uint32_t)kRectChunk, r1 - base);
        __syncthreads();
        // pixel (i, j) is set when x0 <= p i + p/2 < x1 and y0 <= p j + p/2 < y1
        // (doubled: 2 x0 <= 2 p i + p < 2 x1): columns [i0, i1), rows [j0, j1)
        for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int4 q = reinterpret_cast<const int4 *>(cs.rects)[base + t];
            rs[t] = make_int4(pix_from(q.x, p, N), pix_from(q.z, p, N), pix_from(q.y, p, N), pix_from(q.w, p, N));
        }
        __syncthreads();
        if (j < N) {
            for (uint32_t t = 0; t < cnt; ++t) {
                const int4 q = rs[t];
                if (!(q.z <= j && j < q.w)) continue;
                const int i0 = q.x, i1 = q.y;
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    const int lo = max(i0, 64 * k), hi = min(i1, 64 * k + 64);
                    if (lo < hi) {
                        const int len = hi - lo;
                        const uint64_t m = (len == 64) ? ~0ull : (((1ull << len) - 1ull) << (lo - 64 * k));
                        w[k] |= m;
                    }
                }
            }
        }
    }
    uint32_t rowpop = 0;
    if (j < N) {
        uint64_t *dst = cs.bits + ((size_t)c * N + j) * NW;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            dst[k] = w[k];
            rows[j * NW + k] = w[k];
            rowpop += (uint32_t)__popcll(w[k]);
        }
        cs.prof[(size_t)c * 2 * N + j] = (uint16_t)rowpop;
    }
    // total popcount
    uint32_t tot = __reduce_add_sync(0xffffffffu, rowpop);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) s += red[k];
        cs.pop[c] = s;
    }
    // column counts: each warp transposes its 32 rows in 32-column chunks
    // (lane l then holds column l of the chunk) and counts them; the warps'
    // partial counts are summed per column (blockDim = N, a multiple of 32)
    {
        const int lane = threadIdx.x & 31, wr = threadIdx.x >> 5;
#pragma unroll
        for (int h = 0; h < 2 * NW; ++h) {
            const uint32_t x = (h & 1) ? (uint32_t)(w[h >> 1] >> 32) : (uint32_t)w[h >> 1];
            colpart[wr][32 * h + lane] = (uint8_t)__popc(warp_transpose32(x, lane));
        }
    }
    __syncthreads();
    if (j < N) {
        uint32_t q = 0;
        for (int wr = 0; wr < N / 32; ++wr) q += colpart[wr][j];
        cs.prof[(size_t)c * 2 * N + N + j] = (uint16_t)q;
    }
    // 16x16 block counts, then neighbourhood sums, each stored in the order of
    // blk_pos: blocks spread over the whole clip come first, so the gates'
    // chunked density bound sees every part of the clip in its first chunk
    const int nb = g.nb, nb2 = nb * nb;
    uint16_t *blk = cs.blk + (size_t)c * 2 * nb2;
    __shared__ uint16_t cnt_s[32 * 32];
    for (int t = threadIdx.x; t < nb2; t += blockDim.x) {
        const int by = t / nb, bx = t % nb;
        const int k = bx >> 2, sh = (bx & 3) * 16;
        uint32_t s = 0;
        for (int jj = 0; jj < 16; ++jj) s += (uint32_t)__popcll((rows[(by * 16 + jj) * NW + k] >> sh) & 0xffffull);
        cnt_s[t] = (uint16_t)s;
        blk[blk_pos(by, bx, nb)] = (uint16_t)s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb2; t += blockDim.x) {
        const int by = t / nb, bx = t % nb;
        uint32_t s = 0;
        for (int oy = -g.rb; oy <= g.rb; ++oy)
            for (int ox = -g.rb; ox <= g.rb; ++ox) {
                const int yy = by + oy, xx = bx + ox;
                if (yy >= 0 && yy < nb && xx >= 0 && xx < nb) s += cnt_s[yy * nb + xx];
            }
        blk[nb2 + blk_pos(by, bx, nb)] = (uint16_t)min(s, 65535u);
    }
    // edge signature (warp 0): bbox over edges that are not on the window border
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int W = g.W;
        int hasx = 0, hasy = 0, border = 0;
        int lox = INT_MAX, hix = INT_MIN, loy = INT_MAX, hiy = INT_MIN;
        for (uint32_t t = r0 + lane; t < r1; t += 32) {
            const int4 q = reinterpret_cast<const int4 *>(cs.rects)[t];
            if (q.x != 0) { hasx = 1; lox = min(lox, q.x); hix = max(hix, q.x); } else border = 1;
            if (q.z != W) { hasx = 1; lox = min(lox, q.z); hix = max(hix, q.z); } else border = 1;
            if (q.y != 0) { hasy = 1; loy = min(loy, q.y); hiy = max(hiy, q.y); } else border = 1;
            if (q.w != W) { hasy = 1; loy = min(loy, q.w); hiy = max(hiy, q.w); } else border = 1;
        }
        hasx = __reduce_or_sync(0xffffffffu, hasx);
        hasy = __reduce_or_sync(0xffffffffu, hasy);
        border = __reduce_or_sync(0xffffffffu, border);
        lox = __reduce_min_sync(0xffffffffu, lox);
        hix = __reduce_max_sync(0xffffffffu, hix);
        loy = __reduce_min_sync(0xffffffffu, loy);
        hiy = __reduce_max_sync(0xffffffffu, hiy);
        if (lane == 0) {
            int32_t *e = cs.esig + (size_t)c * 8;
            e[ES_N] = (int32_t)(r1 - r0);
            e[ES_HASX] = hasx;
            e[ES_LOX] = hasx ? lox : 0;
            e[ES_HIX] = hasx ? hix : 0;
            e[ES_HASY] = hasy;
            e[ES_LOY] = hasy ? loy : 0;
            e[ES_HIY] = hasy ? hiy : 0;
            e[ES_BORDER] = border;
        }
    }
    // 64 x 64 occupancy grid (cell side W/64): a cell is marked when it holds an
    // integer point of some rectangle's interior, so two rectangles that
    // overlap with positive area always share a marked cell
    // (one thread per rectangle ORs its cells into the grid rows it spans)
    const int csz = g.W / 64;
    const int4 *r4 = reinterpret_cast<const int4 *>(cs.rects);
    __shared__ unsigned long long occ_s[64];
    for (int cy = threadIdx.x; cy < 64; cy += blockDim.x) occ_s[cy] = 0ull;
    __syncthreads();
    for (uint32_t t = r0 + threadIdx.x; t < r1; t += blockDim.x) {
        const int4 q = r4[t];
        if (q.z <= q.x || q.w <= q.y) continue;
        const int y0 = cell_of(q.y, csz), y1 = cell_of(q.w - 1, csz);
        const int x0 = cell_of(q.x, csz), x1 = cell_of(q.z - 1, csz);
        const unsigned long long m = (~0ull >> (63 - (x1 - x0))) << x0;
        for (int cy = y0; cy <= y1; ++cy) atomicOr(&occ_s[cy], m);
    }
    __syncthreads();
    for (int cy = threadIdx.x; cy < 64; cy += blockDim.x) cs.occ[(size_t)c * 64 + cy] = occ_s[cy];
    // rectangles by ascending area (ties by index): rank by counting
    const uint32_t nr = r1 - r0;
    for (uint32_t t = threadIdx.x; t < nr; t += blockDim.x) {
        const int4 q = r4[r0 + t];
        const long long at = (long long)(q.z - q.x) * (long long)(q.w - q.y);
        uint32_t rank = 0;
        for (uint32_t m = 0; m < nr; ++m) {
            const int4 u = r4[r0 + m];
            const long long am = (long long)(u.z - u.x) * (long long)(u.w - u.y);
            rank += (am < at || (am == at && m < t)) ? 1u : 0u;
        }
        cs.rorder[r0 + rank] = (uint16_t)t;
    }
    if (threadIdx.x == 0 && cs.spec_state) cs.spec_state[c] = 0;
}

}  // namespace

cudaError_t launch_raster(const pcl_params &prm, const pcl_clipset &cs, cudaStream_t st) {
    const Geo g = make_geo(prm);
    if (cs.n_clips == 0) return cudaSuccess;
    dim3 grid(cs.n_clips), block(g.N);
    switch (g.nw) {
        case 1: raster_kernel<1><<<grid, block, 0, st>>>(prm, cs); break;
        case 2: raster_kernel<2><<<grid, block, 0, st>>>(prm, cs); break;
        case 4: raster_kernel<4><<<grid, block, 0, st>>>(prm, cs); break;
        case 8: raster_kernel<8><<<grid, block, 0, st>>>(prm, cs); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pcl

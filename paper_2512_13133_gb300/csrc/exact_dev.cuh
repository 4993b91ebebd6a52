// Device code of the exact window scan (Sec. 2.2.1, Eq. 2: c(s) for the
// shifts of the marker window by popcount, the best shift by the exact argmax
// with the tie order), shared by the exact pair kernel (fft.cu) and the
// mixed-batch kernel: the path of 512^2 rasters and the exact-scan engine.
#pragma once

#include "gates.cuh"

namespace pcl {
namespace exact_dev {

// Exact window scan (N = 64 NW: 512^2, where the FFT body's buffers exceed
// shared memory, and 128^2 / 256^2 as the exact-scan engine): c(s) = sum_x
// A(x) B(x - s) counted with AND + popcount for the shifts |dx|, |dy| <= S
// (S <= SMAX <= 32) that the profile bounds do not exclude -- the definition
// itself, so the record is the oracle's.  Both rasters are staged in shared memory (2 N²/8 bytes).  Warps
// take (dy, 8 consecutive dx starting at a multiple of 8); lanes take row pairs
// (A row y, B row y - dy) as 32-bit words and count the 8 shifts of a row pair
// from registers, one funnel shift per word and shift: B's row moved by
// dx = 32 q + r is word w - q funnel-shifted by r with word w - q - 1, and q is
// the same for the 8 shifts of a task because the chunk starts at a multiple
// of 8.  No phase-correlation surface is formed (pcm fields 0).  The caller has
// checked the indices, emptiness and gates.
template <int NW32, int Q>
__device__ __forceinline__ void exact_row_counts(const uint32_t (&a)[NW32], const uint32_t (&bp)[NW32 + 3], int rb,
                                                 uint32_t (&cnt)[8]) {
    // bp[i] = B's word i - 2 (zero outside the row); B moved by 32 Q + r has
    // word w = funnel(b[w - Q - 1], b[w - Q], r) = funnel(bp[w + 1 - Q], bp[w + 2 - Q], r)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int r = rb + u;  // 0..31
        uint32_t x[NW32];
#pragma unroll
        for (int w = 0; w < NW32; ++w) x[w] = a[w] & __funnelshift_l(bp[w + 1 - Q], bp[w + 2 - Q], r);
        cnt[u] += popc_sum<NW32>(x);
    }
}

template <int NW, int SMAX>
__device__ __forceinline__ void exact_body(const pcl_params &prm, const pcl_clipset &A, const pcl_clipset &B,
                                           const pcl_pair pr, pcl_record *dst,
                                           unsigned long long *stats = nullptr) {
    static_assert(SMAX <= 32 && NW >= 2, "shift words: q in {-1, 0, 1}; rows of whole 16-byte vectors");
    constexpr int N = 64 * NW, NW32 = 2 * NW, NV = NW32 / 4;  // 32-bit words and 16-byte vectors per row
    // row stride in shared memory: an odd number of vectors, so that the 8
    // lanes of a quarter-warp reading 8 consecutive rows hit 8 bank groups
    constexpr int SV = NV | 1;
    const Geo g = make_geo(prm);
    const int S = g.S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    extern __shared__ __align__(16) unsigned char smem[];
    uint4 *sa = reinterpret_cast<uint4 *>(smem);
    uint4 *sb = sa + N * SV;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(sb + N * SV);  // [32]
    uint32_t *rbound = reinterpret_cast<uint32_t *>(keys + 32);                      // [2 SMAX + 1]: R(dy)
    uint32_t *cbound = rbound + 2 * SMAX + 1;                                         // [2 SMAX + 1]: C(dx)
    uint32_t *lbest = cbound + 2 * SMAX + 1;  // [0]: L, [1]: tasks evaluated
    uint32_t *order = lbest + 4;                                                      // [1024] sort keys
    uint16_t *prof = reinterpret_cast<uint16_t *>(order + 1024);                      // [2][2N]: A's, B's
    const uint4 *ga = reinterpret_cast<const uint4 *>(A.bits + (size_t)pr.a * N * NW);
    const uint4 *gb = reinterpret_cast<const uint4 *>(B.bits + (size_t)pr.b * N * NW);
    __syncthreads();  // the shared memory may still be read by the previous item
    for (int t = threadIdx.x; t < N * NV; t += blockDim.x) {
        const int st = (t / NV) * SV + t % NV;
        sa[st] = __ldg(ga + t);
        sb[st] = __ldg(gb + t);
    }
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
        prof[t] = __ldg(A.prof + (size_t)pr.a * 2 * N + t);
        prof[2 * N + t] = __ldg(B.prof + (size_t)pr.b * 2 * N + t);
    }
    if (threadIdx.x == 0) lbest[0] = lbest[1] = 0u;
    __syncthreads();
    const int K = 2 * S + 1;
    // Upper bounds from the projection profiles (the bound of gate G2): rows y
    // of A and y - dy of B overlap in at most min(r_A(y), r_B(y - dy)) pixels,
    // so c(dx, dy) <= R(dy) = sum_y min(r_A(y), r_B(y - dy)), and likewise
    // c(dx, dy) <= C(dx) over the columns.
    for (int v = warp; v < 2 * K; v += nwarps) {
        const bool col = v >= K;
        const int d = (col ? v - K : v) - S;
        const uint16_t *pa_ = prof + (col ? N : 0), *pb_ = prof + 2 * N + (col ? N : 0);
        uint32_t sum = 0;
        for (int y = lane; y < N; y += 32) {
            const int yb = y - d;
            if (yb >= 0 && yb < N) sum += min((uint32_t)pa_[y], (uint32_t)pb_[yb]);
        }
        sum = __reduce_add_sync(0xffffffffu, sum);
        if (lane == 0) (col ? cbound : rbound)[d + S] = sum;
    }
    __syncthreads();
    // dx chunks [8 c, 8 c + 7] for c = floor(-S / 8) .. floor(S / 8); a task
    // (dy, chunk) is bounded by min(R(dy), max of C over its shifts)
    const int c0 = -((S + 7) / 8), nch = S / 8 - c0 + 1;
    auto task_bound = [&](int task) -> uint32_t {
        const int dy = task / nch - S, dx0 = (c0 + task % nch) * 8;
        uint32_t cm = 0;
        for (int u = 0; u < 8; ++u) {
            const int dx = dx0 + u;
            if (dx >= -S && dx <= S) cm = max(cm, cbound[dx + S]);
        }
        return min(rbound[dy + S], cm);
    };
    unsigned long long best = 0ull;
    // c(s) for the 8 shifts of one task; returns their largest overlap
    auto eval_task = [&](int task) -> uint32_t {
        const int dy = task / nch - S, dx0 = (c0 + task % nch) * 8;  // -32 <= dx0 <= 32
        const int q = (dx0 + 32) / 32 - 1, rb = dx0 - 32 * q;        // dx0 = 32 q + rb, rb in {0, 8, 16, 24}
        uint32_t cnt[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) cnt[u] = 0;
        const int j0 = dy > 0 ? dy : 0, j1 = dy < 0 ? N + dy : N;
        for (int j = j0 + lane; j < j1; j += 32) {
            uint32_t a[NW32], bp[NW32 + 3];
            bp[0] = bp[1] = bp[NW32 + 2] = 0u;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const uint4 x = sa[j * SV + v], y = sb[(j - dy) * SV + v];
                a[4 * v] = x.x, a[4 * v + 1] = x.y, a[4 * v + 2] = x.z, a[4 * v + 3] = x.w;
                bp[4 * v + 2] = y.x, bp[4 * v + 3] = y.y, bp[4 * v + 4] = y.z, bp[4 * v + 5] = y.w;
            }
            if (q < 0) exact_row_counts<NW32, -1>(a, bp, rb, cnt);
            else if (q == 0) exact_row_counts<NW32, 0>(a, bp, rb, cnt);
            else exact_row_counts<NW32, 1>(a, bp, rb, cnt);
        }
        uint32_t cmax = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int dx = dx0 + u;
            const uint32_t c = __reduce_add_sync(0xffffffffu, cnt[u]);
            if (dx >= -S && dx <= S) {
                const unsigned long long k = shift_key(c, dx, dy, S);
                best = k > best ? k : best;
                cmax = max(cmax, c);
            }
        }
        return cmax;
    };
    // Best first: the tasks sorted by bound, descending (bitonic sort of
    // keys bound << 12 | 4095 - task in shared memory; ties by task index);
    // warp w takes sorted positions w, w + nwarps, ...  The first round (the
    // nwarps largest bounds) sets L, the largest overlap counted so far, and
    // every counted task raises it (shared atomic max).  A warp stops at its
    // first position whose bound is below L: the positions after it have
    // bounds no larger, and a task below L holds no shift whose overlap
    // reaches the best, so the argmax and its ties are the full scan's.
    const int ntask = K * nch;  // <= 65 x 9 = 585
    int nsort = 32;
    while (nsort < ntask) nsort <<= 1;
    for (int t = threadIdx.x; t < nsort; t += blockDim.x)
        order[t] = t < ntask ? (task_bound(t) << 12) | (uint32_t)(4095 - t) : 0u;
    __syncthreads();
    for (int k = 2; k <= nsort; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < nsort; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const uint32_t x = order[i], y = order[l];
                    if (((i & k) == 0) ? (x < y) : (x > y)) {  // descending runs first
                        order[i] = y;
                        order[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (int p = warp; p < ntask; p += nwarps) {
        const uint32_t key = order[p];
        const uint32_t lnow = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile uint32_t *>(lbest), 0);
        if ((key >> 12) < lnow) break;  // warp-uniform
        const uint32_t cm = eval_task(4095 - (int)(key & 4095u));
        if (lane == 0) {
            atomicMax(lbest, cm);
            atomicAdd(lbest + 1, 1u);
        }
    }
    if (lane == 0) keys[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (stats) {
            atomicAdd(stats, (unsigned long long)lbest[1]);
            atomicAdd(stats + 1, (unsigned long long)(K * nch));
        }
        unsigned long long bk = 0ull;
        for (int w = 0; w < nwarps; ++w) bk = keys[w] > bk ? keys[w] : bk;
        const int dx = S - (int)(bk & 0xffu), dy = S - (int)((bk >> 8) & 0xffu);
        const uint32_t cb = (uint32_t)(bk >> 32);
        const uint64_t pa = A.pop[pr.a], pb = B.pop[pr.b];
        pcl_record rec{};
        rec.a = pr.a;
        rec.b = pr.b;
        rec.mode = PCL_MODE_COSINE;
        rec.dx_dbu = dx * g.p;
        rec.dy_dbu = dy * g.p;
        rec.score = cb;
        float sim = (pa && pb) ? (float)cb / sqrtf((float)pa * (float)pb) : 0.0f;
        uint16_t fl = PCL_F_ALIGNED;
        const float T = (float)prm.cos_num / (float)prm.cos_den;
        if (pa && pb && fabsf(sim - T) < prm.near_band) {
            fl |= PCL_F_NEAR_BAND;
            sim = (float)((double)cb / sqrt((double)pa * (double)pb));
        }
        rec.sim = sim;
        rec.flags = fl;
        rec.pass = cos_exceeds(cb, pa, pb, prm.cos_num, prm.cos_den) ? 1 : 0;
        *dst = rec;
    }
    __syncthreads();
}

// shared memory of exact_body
template <int NW>
constexpr size_t exact_smem() {
    // rasters (odd row stride), keys[32], R and C bounds (2 x 65), L and the task count (+ 2 pad),
    // 1024 sort keys, profiles [2][2N] u16
    return 2 * 16 * 64 * NW * ((NW / 2) | 1) + 32 * 8 + 4 * (2 * 65 + 4) + 4 * 1024 + 2 * 2 * 2 * 64 * NW;
}

}  // namespace exact_dev
}  // namespace pcl

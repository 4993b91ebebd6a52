// Cosine mode with the shift of the XY-separation interval competition
// (Sec. 3.2.1 (2)): the geometric alternative to phase correlation.  Instead
// of evaluating every shift of the marker window, the shift is synthesised from
// the tightest per-axis constraint of corresponding polygons, and the overlap
// is counted at that one shift.
//
//  1. pre-alignment s0 from the non-border-edge bboxes (as in edge mode); each
//     polygon k of the clip with fewer polygons (A on a tie) pairs with the one
//     polygon of the other clip that overlaps it at s0 (no pair when none or
//     several do).  A pair's allowable interval on an axis is [d_min, d_max]
//     over the displacements d = e_A - e_B of its edges on that axis, edges on
//     the window border in either clip excluded;
//  2. interval quality Q = d_max - d_min;
//  3. per axis, the pair with the smallest Q wins (ties: the smaller k);
//  4. T = trunc((d_min + d_max) / 2) of the winner, clamped to +/-M (s0 on an
//     axis without intervals); the raster shift is T / p rounded half away
//     from zero, clamped to +/-S.
// The record holds the exact overlap c at that shift, sim and the integer
// decision of Eq. 2, so it can only lose passes of the exact argmax.
//
// One warp per pair.  Lanes take the small clip's polygons (k = lane, lane +
// 32, ...) and scan the large clip's polygons for their partners (every lane
// reads the same large polygon at a time); a 64-bit warp minimum of (Q, k)
// picks each axis' winner; one warp popcount pass gives c.
#include <climits>

#include "gates.cuh"

namespace pcl {

namespace {

__device__ __forceinline__ int clamp_i(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
__device__ __forceinline__ int round_div_away(int v, int p) { return v >= 0 ? (v + p / 2) / p : -((-v + p / 2) / p); }

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

// one record (every lane gets it)
__device__ pcl_record xysep_record(const pcl_params &prm, const pcl_clipset &A, const pcl_clipset &B, pcl_pair pr,
                                   int lane) {
    pcl_record r{};
    r.a = pr.a;
    r.b = pr.b;
    r.mode = PCL_MODE_COSINE;
    if (pr.a >= A.n_clips || pr.b >= B.n_clips) {
        r.flags = PCL_GATE_BAD_INDEX;
        return r;
    }
    const Geo g = make_geo(prm);
    const uint64_t pa = A.pop[pr.a], pb = B.pop[pr.b];
    if (pa == 0 && pb == 0) {
        r.flags = PCL_F_EMPTY;
        r.sim = 1.0f;
        r.pass = 1;
        return r;
    }
    if (!(prm.flags & PCL_P_NO_GATES)) {
        const int gate = warp_cosine_gate(A, pr.a, B, pr.b, g, prm.cos_num, prm.cos_den, lane);
        if (gate) {
            r.flags = (uint16_t)gate;
            return r;
        }
    }
    const int W = prm.window_dbu, M = prm.marker_dbu;
    // edge signatures: {n, hasx, lox, hix}, {hasy, loy, hiy, border}
    const int4 *e4a = reinterpret_cast<const int4 *>(A.esig + (size_t)pr.a * 8);
    const int4 *e4b = reinterpret_cast<const int4 *>(B.esig + (size_t)pr.b * 8);
    const int4 alo = __ldg(e4a), ahi = __ldg(e4a + 1), blo = __ldg(e4b), bhi = __ldg(e4b + 1);
    const int na = alo.x, nb = blo.x;
    const int s0x = (alo.y && blo.y) ? clamp_i(((alo.z + alo.w) - (blo.z + blo.w)) / 2, -M, M) : 0;
    const int s0y = (ahi.x && bhi.x) ? clamp_i(((ahi.y + ahi.z) - (bhi.y + bhi.z)) / 2, -M, M) : 0;
    const bool small_is_a = na <= nb;
    const int4 *ra = reinterpret_cast<const int4 *>(A.rects) + __ldg(A.rect_off + pr.a);
    const int4 *rb = reinterpret_cast<const int4 *>(B.rects) + __ldg(B.rect_off + pr.b);
    const int4 *rs = small_is_a ? ra : rb, *rl = small_is_a ? rb : ra;
    const int ns = small_is_a ? na : nb, nl = small_is_a ? nb : na;
    // A's polygon first and B's moved by s0: with the small clip on side A
    // that is (s, l + s0), otherwise (l, s + s0) -- both the plain overlap of
    // s with l moved by u = +s0 or -s0
    const int ux = small_is_a ? s0x : -s0x, uy = small_is_a ? s0y : -s0y;
    // per lane: best (Q, k) and d_min + d_max of each axis over its polygons
    unsigned long long bx = ~0ull, by = ~0ull;
    int sx = 0, sy = 0;
    const int iters = (ns + 31) / 32;  // warp-uniform
    for (int it = 0; it < iters; ++it) {
        const int k = it * 32 + lane;
        const bool kv = k < ns;
        const int4 s = kv ? __ldg(rs + k) : make_int4(0, 0, 0, 0);
        int cnt = 0, m = -1;
        for (int j = 0; j < nl; ++j) {
            const int4 l = __ldg(rl + j);
            const bool hit = s.x < l.z + ux && l.x + ux < s.z && s.y < l.w + uy && l.y + uy < s.w;
            if (hit) {
                ++cnt;
                m = j;
            }
        }
        if (!kv || cnt != 1) continue;
        const int4 l = __ldg(rl + m);
        const int4 p_a = small_is_a ? s : l, p_b = small_is_a ? l : s;
        // x interval
        {
            const bool o0 = p_a.x != 0 && p_b.x != 0, o1 = p_a.z != W && p_b.z != W;
            const int d0 = p_a.x - p_b.x, d1 = p_a.z - p_b.z;
            if (o0 || o1) {
                const int lo = o0 && o1 ? min(d0, d1) : (o0 ? d0 : d1);
                const int hi = o0 && o1 ? max(d0, d1) : (o0 ? d0 : d1);
                const unsigned long long key = ((unsigned long long)(uint32_t)(hi - lo) << 32) | (uint32_t)k;
                if (key < bx) {
                    bx = key;
                    sx = lo + hi;
                }
            }
        }
        // y interval
        {
            const bool o0 = p_a.y != 0 && p_b.y != 0, o1 = p_a.w != W && p_b.w != W;
            const int d0 = p_a.y - p_b.y, d1 = p_a.w - p_b.w;
            if (o0 || o1) {
                const int lo = o0 && o1 ? min(d0, d1) : (o0 ? d0 : d1);
                const int hi = o0 && o1 ? max(d0, d1) : (o0 ? d0 : d1);
                const unsigned long long key = ((unsigned long long)(uint32_t)(hi - lo) << 32) | (uint32_t)k;
                if (key < by) {
                    by = key;
                    sy = lo + hi;
                }
            }
        }
    }
    const unsigned long long wx = warp_min_u64(bx), wy = warp_min_u64(by);
    // the winner's d_min + d_max sits in lane k mod 32, as that lane's own best
    const int sumx = __shfl_sync(0xffffffffu, sx, (int)(wx & 31u));
    const int sumy = __shfl_sync(0xffffffffu, sy, (int)(wy & 31u));
    const int Tx = wx != ~0ull ? clamp_i(sumx / 2, -M, M) : s0x;
    const int Ty = wy != ~0ull ? clamp_i(sumy / 2, -M, M) : s0y;
    const int dx = clamp_i(round_div_away(Tx, g.p), -g.S, g.S), dy = clamp_i(round_div_away(Ty, g.p), -g.S, g.S);
    const uint32_t c = warp_corr_exact(A.bits + (size_t)pr.a * g.N * g.nw, B.bits + (size_t)pr.b * g.N * g.nw, g.N,
                                       g.nw, dx, dy, lane);
    r.dx_dbu = dx * g.p;
    r.dy_dbu = dy * g.p;
    r.score = c;
    float sim = (pa && pb) ? (float)c / sqrtf((float)pa * (float)pb) : 0.0f;
    uint16_t fl = PCL_F_ALIGNED;
    const float T = (float)prm.cos_num / (float)prm.cos_den;
    if (pa && pb && fabsf(sim - T) < prm.near_band) {
        fl |= PCL_F_NEAR_BAND;
        sim = (float)((double)c / sqrt((double)pa * (double)pb));
    }
    r.sim = sim;
    r.flags = fl;
    r.pass = cos_exceeds(c, pa, pb, prm.cos_num, prm.cos_den) ? 1 : 0;
    return r;
}

// one pair per warp, warps striding the list
__global__ void __launch_bounds__(256) xysep_kernel(pcl_params prm, pcl_clipset A, pcl_clipset B,
                                                    const pcl_pair *pairs, uint64_t n,
                                                    const unsigned long long *d_n, pcl_record *out) {
    if (d_n && *d_n < n) n = *d_n;
    const int lane = threadIdx.x & 31;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t t = w0; t < n; t += nw) {
        const pcl_record r = xysep_record(prm, A, B, pairs[t], lane);
        if (lane == 0) out[t] = r;
    }
}

}  // namespace

cudaError_t launch_xysep(const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b, const pcl_pair *pairs,
                         uint64_t n, const unsigned long long *d_n, pcl_record *out, int num_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint64_t warps = (uint64_t)num_sms * 8 * 8;  // 8 blocks of 8 warps per SM, striding
    const uint64_t need = (n + 7) / 8;
    const uint64_t blocks = need < warps / 8 ? need : warps / 8;
    xysep_kernel<<<(unsigned)blocks, 256, 0, st>>>(prm, a, b, pairs, n, d_n, out);
    return cudaGetLastError();
}

}  // namespace pcl

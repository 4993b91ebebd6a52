// Warp-cooperative evaluation of the lossless cosine gates of one pair
// (Sec. 3.1 stage 1): G1 area, G3 block density, G2 projection profiles.
#pragma once

#include "common.cuh"

namespace pcl {

// warp-cooperative G3 test: true if the density bound (both directions,
// minimum kept) cannot reach the threshold.  Blocks are visited 64 at a time;
// after each chunk the deficits seen so far, sum_k (cnt_A(k) - min(cnt_A(k),
// nbr_B(k))) and the same the other way, already bound c from above by
// min(|A| - def_A, |B| - def_B), so most pairs are rejected before all blocks
// are read.  The last chunk gives exactly the full bound, so the decision is
// the same as evaluating the bound at once.
__device__ __forceinline__ bool warp_g3_rejects(const uint16_t *__restrict__ ba, const uint16_t *__restrict__ bb,
                                                int nb2, uint64_t pa, uint64_t pb, uint32_t num, uint32_t den,
                                                int lane) {
    const uint32_t *ca = reinterpret_cast<const uint32_t *>(ba);
    const uint32_t *da = reinterpret_cast<const uint32_t *>(ba + nb2);
    const uint32_t *cb = reinterpret_cast<const uint32_t *>(bb);
    const uint32_t *db = reinterpret_cast<const uint32_t *>(bb + nb2);
    const int words = nb2 / 2;
    uint32_t defa = 0, defb = 0;
    for (int t0 = 0; t0 < words; t0 += 32) {
        const int t = t0 + lane;
        if (t < words) {
            const uint32_t a = __ldg(ca + t), b = __ldg(cb + t);
            const uint32_t m1 = __vminu2(a, __ldg(db + t));
            const uint32_t m2 = __vminu2(b, __ldg(da + t));
            defa += ((a & 0xffffu) + (a >> 16)) - ((m1 & 0xffffu) + (m1 >> 16));
            defb += ((b & 0xffffu) + (b >> 16)) - ((m2 & 0xffffu) + (m2 >> 16));
        }
        const uint64_t DA = __reduce_add_sync(0xffffffffu, defa);
        const uint64_t DB = __reduce_add_sync(0xffffffffu, defb);
        const uint64_t ua = pa - DA, ub = pb - DB;
        if (!cos_exceeds(ua < ub ? ua : ub, pa, pb, num, den)) return true;
    }
    return false;
}

// warp-cooperative G2 bound: min over (rows, columns) of the max over
// |d| <= S of sum_j min(prof_A(j), prof_B(j - d))
__device__ __forceinline__ uint32_t warp_g2(const uint16_t *__restrict__ pa, const uint16_t *__restrict__ pb,
                                            int N, int S, int lane) {
    uint32_t ur = 0, uc = 0;
    for (int d = -S; d <= S; ++d) {
        uint32_t tr = 0, tc = 0;
        for (int j = lane; j < N; j += 32) {
            const int k = j - d;
            if (k >= 0 && k < N) {
                tr += min((uint32_t)__ldg(pa + j), (uint32_t)__ldg(pb + k));
                tc += min((uint32_t)__ldg(pa + N + j), (uint32_t)__ldg(pb + N + k));
            }
        }
        tr = __reduce_add_sync(0xffffffffu, tr);
        tc = __reduce_add_sync(0xffffffffu, tc);
        ur = max(ur, tr);
        uc = max(uc, tc);
    }
    return ur < uc ? ur : uc;
}

// cosine gates of one pair (warp-uniform result): PCL_GATE_* or 0
__device__ __forceinline__ int warp_cosine_gate(const pcl_clipset &A, uint32_t a, const pcl_clipset &B, uint32_t b,
                                const Geo &g, uint32_t num, uint32_t den, int lane) {
    const uint64_t pa = A.pop[a], pb = B.pop[b];
    const uint64_t mn = pa < pb ? pa : pb, mx = pa < pb ? pb : pa;
    if (!((uint64_t)den * den * mn > (uint64_t)num * num * mx)) return PCL_GATE_G1_AREA;
    const int nb2 = g.nb * g.nb;
    if (warp_g3_rejects(A.blk + (size_t)a * 2 * nb2, B.blk + (size_t)b * 2 * nb2, nb2, pa, pb, num, den, lane))
        return PCL_GATE_G3_DENSITY;
    const uint32_t u2 = warp_g2(A.prof + (size_t)a * 2 * g.N, B.prof + (size_t)b * 2 * g.N, g.N, g.S, lane);
    if (!cos_exceeds(u2, pa, pb, num, den)) return PCL_GATE_G2_PROFILE;
    return PCL_GATE_NONE;
}

}  // namespace pcl

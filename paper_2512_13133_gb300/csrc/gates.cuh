// Warp-cooperative evaluation of the lossless cosine gates of one pair
// (Sec. 3.1 stage 1): G1 area, G3 block density, G2 projection profiles.
#pragma once

#include "common.cuh"

namespace pcl {

// Largest overlap u that does NOT pass the integer rule of Eq. 2 for areas
// pa, pb (cos_exceeds(u) is false exactly for u <= result): a float estimate
// of num sqrt(pa pb) / den corrected by the exact rule (the estimate is off by
// at most one or two).  A gate bound u rejects a pair exactly when u <= this.
__device__ __forceinline__ int64_t cos_umax(uint64_t pa, uint64_t pb, uint32_t num, uint32_t den) {
    uint64_t u = (uint64_t)(sqrtf((float)pa * (float)pb) * ((float)num / (float)den));
    while (u > 0 && cos_exceeds(u, pa, pb, num, den)) --u;
    while (!cos_exceeds(u + 1, pa, pb, num, den)) ++u;
    return (int64_t)u;
}

// warp-cooperative G3 test: true if the density bound (both directions,
// minimum kept) cannot pass Eq. 2, i.e. min(|A| - def_A, |B| - def_B) <= um.
// Blocks are visited 64 at a time; after each chunk the deficits seen so far,
// sum_k (cnt_A(k) - min(cnt_A(k), nbr_B(k))) and the same the other way,
// already bound c from above, so most pairs are rejected before all blocks
// are read.  The last chunk gives exactly the full bound, so the decision is
// the same as evaluating the bound at once.  Deficits accumulate as packed
// 16-bit halves (a chunk's 32-lane sum of one half is at most 32 * 256).
__device__ __forceinline__ bool warp_g3_rejects(const uint16_t *__restrict__ ba, const uint16_t *__restrict__ bb,
                                                int nb2, uint64_t pa, uint64_t pb, int64_t um, int lane) {
    const uint32_t *ca = reinterpret_cast<const uint32_t *>(ba);
    const uint32_t *da = reinterpret_cast<const uint32_t *>(ba + nb2);
    const uint32_t *cb = reinterpret_cast<const uint32_t *>(bb);
    const uint32_t *db = reinterpret_cast<const uint32_t *>(bb + nb2);
    const int words = nb2 / 2;
    const int64_t tA = (int64_t)pa - um, tB = (int64_t)pb - um;  // reject once DA >= tA or DB >= tB
    int64_t DA = 0, DB = 0;
    // the next chunk's words are loaded while the current one is reduced
    uint32_t a = 0u, b = 0u, na = 0u, nb = 0u;
    if (lane < words) {
        a = __ldg(ca + lane);
        b = __ldg(cb + lane);
        na = __ldg(db + lane);
        nb = __ldg(da + lane);
    }
    for (int t0 = 0; t0 < words; t0 += 32) {
        const uint32_t pda = a - __vminu2(a, na), pdb = b - __vminu2(b, nb);
        const int t = t0 + 32 + lane;
        a = b = na = nb = 0u;
        if (t < words) {
            a = __ldg(ca + t);
            b = __ldg(cb + t);
            na = __ldg(db + t);
            nb = __ldg(da + t);
        }
        const uint32_t sa = __reduce_add_sync(0xffffffffu, pda), sb = __reduce_add_sync(0xffffffffu, pdb);
        DA += (sa & 0xffffu) + (sa >> 16);
        DB += (sb & 0xffffu) + (sb >> 16);
        if (DA >= tA || DB >= tB) return true;
    }
    return false;
}

// G2 as a decision (kept out of line: it is rare in the hot loops that call it,
// and inlining it would cost them registers): true if the bound min(max_d R(d), max_d Q(d)) <= um,
// i.e. one axis keeps every shift's profile sum at or below um.  The rows are
// tried first (the columns are skipped when the rows already reject); an axis
// stops at its first shift above um, visiting d = 0, 1, -1, 2, -2, ...  A's
// profile is held in registers (NPL = N / 32 values per lane).
template <int NPL>
__device__ __forceinline__ bool warp_g2_rejects(const uint16_t *__restrict__ pa, const uint16_t *__restrict__ pb,
                                                int S, int64_t um, int lane) {
    constexpr int N = 32 * NPL;
#pragma unroll 1
    for (int ax = 0; ax < 2; ++ax) {
        const uint16_t *A = pa + ax * N, *B = pb + ax * N;
        uint32_t av[NPL];
#pragma unroll
        for (int u = 0; u < NPL; ++u) av[u] = __ldg(A + lane + 32 * u);
        bool above = false;
        for (int i = 0; i <= 2 * S && !above; ++i) {
            const int d = (i & 1) ? (i + 1) >> 1 : -(i >> 1);
            uint32_t t = 0;
#pragma unroll
            for (int u = 0; u < NPL; ++u) {
                const int k = lane + 32 * u - d;
                if (k >= 0 && k < N) t += min(av[u], (uint32_t)__ldg(B + k));
            }
            above = (int64_t)__reduce_add_sync(0xffffffffu, t) > um;
        }
        if (!above) return true;
    }
    return false;
}

static __device__ __noinline__ bool warp_g2_rejects_n(const uint16_t *pa, const uint16_t *pb, int N, int S, int64_t um,
                                                  int lane) {
    switch (N) {
        case 64: return warp_g2_rejects<2>(pa, pb, S, um, lane);
        case 128: return warp_g2_rejects<4>(pa, pb, S, um, lane);
        case 256: return warp_g2_rejects<8>(pa, pb, S, um, lane);
        default: return warp_g2_rejects<16>(pa, pb, S, um, lane);
    }
}

// G2 as a decision with B's two profiles staged by the warp in shared memory
// (scratch: 2 (N + 2S) u16, zero padded by S on both sides, so no bounds
// checks), A's profile in registers; otherwise as warp_g2_rejects.
template <int NPL>
__device__ __forceinline__ bool warp_g2_rejects_smem(const uint16_t *__restrict__ pa,
                                                     const uint16_t *__restrict__ pb, int S, int64_t um, int lane,
                                                     uint16_t *scratch) {
    constexpr int N = 32 * NPL;
    const int L = N + 2 * S;
    __syncwarp();  // the previous pair's reads of scratch are done
    for (int k = lane; k < 2 * L; k += 32) {
        const int ax = k >= L, i = k - ax * L - S;
        scratch[k] = (i >= 0 && i < N) ? __ldg(pb + ax * N + i) : (uint16_t)0;
    }
    __syncwarp();
#pragma unroll 1
    for (int ax = 0; ax < 2; ++ax) {
        const uint16_t *A = pa + ax * N;
        const uint16_t *Bs = scratch + ax * L + S;  // Bs[k] = prof_B(k) for -S <= k < N + S
        uint32_t av[NPL];
#pragma unroll
        for (int u = 0; u < NPL; ++u) av[u] = __ldg(A + lane + 32 * u);
        bool above = false;
        for (int i = 0; i <= 2 * S && !above; ++i) {
            const int d = (i & 1) ? (i + 1) >> 1 : -(i >> 1);
            uint32_t t = 0;
#pragma unroll
            for (int u = 0; u < NPL; ++u) t += min(av[u], (uint32_t)Bs[lane + 32 * u - d]);
            above = (int64_t)__reduce_add_sync(0xffffffffu, t) > um;
        }
        if (!above) return true;
    }
    return false;
}

// shared-memory G2 scratch per warp (u16 elements) for rasters up to N = 512
constexpr int kG2Scratch = 2 * (512 + 2 * 64);

// G2 for a band walk over small rasters (N <= 128, where the density bound of
// 16-px blocks dilated by a block is loose and G2 decides most band pairs).
// Per representative, in the warp's scratch: its row and column counts (As,
// 2N u16) and their maxima over |d| <= S, the dilated profiles rmax(z) = max
// r_A(z + d) (Am, 2N u16).  Since each row sum sum_y min(r_A(y), r_B(y - d))
// is at most sum_z min(rmax(z), r_B(z)), one pass over the member's profiles
// without shifts decides G2 whenever that bound (or the columns') is <= um;
// otherwise the member's profiles are staged (Bs, 2 (N + 2S) u16, zero padded
// by S) and every shift is summed.  The decision is warp_g2_rejects_lite's.
__device__ __forceinline__ void g2_rep_setup(const uint16_t *__restrict__ pr, int N, int S, int lane, uint16_t *As) {
    uint16_t *Am = As + 2 * N;
    __syncwarp();  // the previous representative's reads are done
    for (int k = lane; k < 2 * N; k += 32) As[k] = __ldg(pr + k);
    __syncwarp();
    for (int k = lane; k < 2 * N; k += 32) {
        const int ax = k >= N, j = k - ax * N, lo = j - S < 0 ? 0 : j - S, hi = j + S >= N ? N - 1 : j + S;
        uint32_t m = 0;
        for (int t = lo; t <= hi; ++t) m = max(m, (uint32_t)As[ax * N + t]);
        Am[k] = (uint16_t)m;
    }
    __syncwarp();
}

__device__ __forceinline__ bool g2_rejects_small(uint16_t *As, const uint16_t *__restrict__ pb, int N, int S,
                                                 int64_t um, int lane) {
    const uint16_t *Am = As + 2 * N;
    uint16_t *Bs = As + 4 * N;
    // both dilated bounds in one reduction (each at most N^2 <= 16384)
    uint32_t tr = 0, tc = 0;
    for (int j = lane; j < N; j += 32) {
        tr += min((uint32_t)Am[j], (uint32_t)__ldg(pb + j));
        tc += min((uint32_t)Am[N + j], (uint32_t)__ldg(pb + N + j));
    }
    const uint32_t sr = __reduce_add_sync(0xffffffffu, tr | (tc << 16));
    if ((int64_t)(sr & 0xffffu) <= um || (int64_t)(sr >> 16) <= um) return true;
    const int L = N + 2 * S;
    __syncwarp();  // the previous pair's reads of Bs are done
    for (int k = lane; k < 2 * L; k += 32) {
        const int ax = k >= L, i = k - ax * L - S;
        Bs[k] = (i >= 0 && i < N) ? __ldg(pb + ax * N + i) : (uint16_t)0;
    }
    __syncwarp();
    for (int ax = 0; ax < 2; ++ax) {
        const uint16_t *B = Bs + ax * L + S;  // B[k] = prof_B(k) for -S <= k < N + S
        const uint16_t *A = As + ax * N;
        bool above = false;
        for (int i = 0; i <= 2 * S && !above; ++i) {
            const int d = (i & 1) ? (i + 1) >> 1 : -(i >> 1);
            uint32_t t = 0;
            for (int j = lane; j < N; j += 32) t += min((uint32_t)A[j], (uint32_t)B[j - d]);
            above = (int64_t)__reduce_add_sync(0xffffffffu, t) > um;
        }
        if (!above) return true;
    }
    return false;
}

// per-warp G2 scratch (u16) of a band walk over N <= 128: As, Am, then Bs
__host__ __device__ inline int band_g2_warp(int N, int S) { return 4 * N + 2 * (N + 2 * S); }
// bytes of that scratch for a 256-thread block
__host__ __device__ inline int band_g2_smem(int N, int S) { return N <= 128 ? 8 * band_g2_warp(N, S) * 2 : 0; }

// The same decision with every profile value loaded where it is used and no
// early exit: fewer registers, for callers where G2 is rare and register
// pressure matters more than its speed.
__device__ __forceinline__ bool warp_g2_rejects_lite(const uint16_t *__restrict__ pa,
                                                     const uint16_t *__restrict__ pb, int N, int S, int64_t um,
                                                     int lane) {
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
        ur = max(ur, __reduce_add_sync(0xffffffffu, tr));
        uc = max(uc, __reduce_add_sync(0xffffffffu, tc));
    }
    return (int64_t)(ur < uc ? ur : uc) <= um;
}

// G3 for one band member with the representative's block words in registers
// (WPL u32 words per lane = two 16-bit blocks each).  Deficits accumulate as
// packed 16-bit halves (min <= value, so no borrow crosses halves; a chunk's
// 32-lane sum of one half is at most 32 * 256); after every 32-lane chunk the
// bound min(pa - DA, pb - DB) is compared with the pair's thresholds: it
// fails Eq. 2 exactly when DA >= tA or DB >= tB (tX = pX - cos_umax).  In the
// first chunk A's deficit is summed and tested before B's: on its own it
// rejects most pairs of a band.
template <int WPL>
__device__ __forceinline__ bool g3_rest_rejects(const uint32_t (&ca)[WPL], const uint32_t (&da)[WPL],
                                                const uint32_t *__restrict__ cb, const uint32_t *__restrict__ db,
                                                int words, int tA, int tB, int DA, int DB, int lane);

template <int WPL>
__device__ __forceinline__ bool g3_rejects_thr(const uint32_t (&ca)[WPL], const uint32_t (&da)[WPL],
                                               const uint32_t *__restrict__ cb, const uint32_t *__restrict__ db,
                                               int words, int tA, int tB, int lane) {
    const bool v = lane < words;  // lanes past the words hold zero block counts
    const uint32_t d0 = v ? __ldg(db + lane) : 0u, b0 = v ? __ldg(cb + lane) : 0u;
    uint32_t sr = __reduce_add_sync(0xffffffffu, ca[0] - __vminu2(ca[0], d0));
    int DA = (int)((sr & 0xffffu) + (sr >> 16));
    if (DA >= tA) return true;
    sr = __reduce_add_sync(0xffffffffu, b0 - __vminu2(b0, da[0]));
    const int DB = (int)((sr & 0xffffu) + (sr >> 16));
    if (DB >= tB) return true;
    return g3_rest_rejects<WPL>(ca, da, cb, db, words, tA, tB, DA, DB, lane);
}

// g3_rest_rejects with the second chunk's words of the member (cb, db at
// 32 + lane) already loaded into b1 and d1 (WPL > 1)
template <int WPL>
__device__ __forceinline__ bool g3_rest_pre(const uint32_t (&ca)[WPL], const uint32_t (&da)[WPL],
                                            const uint32_t *__restrict__ cb, const uint32_t *__restrict__ db,
                                            int words, int tA, int tB, int DA, int DB, uint32_t b1, uint32_t d1,
                                            int lane) {
    const uint32_t sa = __reduce_add_sync(0xffffffffu, ca[1] - __vminu2(ca[1], d1));
    const uint32_t sb = __reduce_add_sync(0xffffffffu, b1 - __vminu2(b1, da[1]));
    DA += (int)((sa & 0xffffu) + (sa >> 16));
    DB += (int)((sb & 0xffffu) + (sb >> 16));
    if (DA >= tA || DB >= tB) return true;
#pragma unroll
    for (int c = 2; c < WPL; ++c) {
        const int t = c * 32 + lane;
        uint32_t pda = 0u, pdb = 0u;
        if (t < words) {
            const uint32_t b = __ldg(cb + t);
            pda = ca[c] - __vminu2(ca[c], __ldg(db + t));
            pdb = b - __vminu2(b, da[c]);
        }
        const uint32_t ra = __reduce_add_sync(0xffffffffu, pda), rb = __reduce_add_sync(0xffffffffu, pdb);
        DA += (int)((ra & 0xffffu) + (ra >> 16));
        DB += (int)((rb & 0xffffu) + (rb >> 16));
        if (DA >= tA || DB >= tB) return true;
    }
    return false;
}

// G3 from the second 32-lane chunk on, the first chunk's deficits DA and DB
// (neither at its threshold) already summed: the rest of g3_rejects_thr.
template <int WPL>
__device__ __forceinline__ bool g3_rest_rejects(const uint32_t (&ca)[WPL], const uint32_t (&da)[WPL],
                                                const uint32_t *__restrict__ cb, const uint32_t *__restrict__ db,
                                                int words, int tA, int tB, int DA, int DB, int lane) {
#pragma unroll
    for (int c = 1; c < WPL; ++c) {
        const int t = c * 32 + lane;
        uint32_t pda = 0u, pdb = 0u;
        if (t < words) {
            const uint32_t b = __ldg(cb + t);
            pda = ca[c] - __vminu2(ca[c], __ldg(db + t));
            pdb = b - __vminu2(b, da[c]);
        }
        const uint32_t sa = __reduce_add_sync(0xffffffffu, pda), sb = __reduce_add_sync(0xffffffffu, pdb);
        DA += (int)((sa & 0xffffu) + (sa >> 16));
        DB += (int)((sb & 0xffffu) + (sb >> 16));
        if (DA >= tA || DB >= tB) return true;
    }
    return false;
}

// ---- lane-per-member first chunk (N >= 256: 32 or more u32 words of block
// counts per clip).  In the band join each lane takes one of up to 32 band
// members and sums the member's first-chunk deficits (the first 64 blocks,
// spread over the raster) itself, from member words staged in the warp's
// shared memory by 16-byte asynchronous copies: the test that decides about
// four fifths of band pairs costs a few instructions per pair instead of a
// warp reduction per member.  Per warp: the representative's first 32 words
// of block counts and of neighbourhood sums, then one 32-word row per member.
constexpr int kBjWarpWords = 64 + 32 * 32;
__host__ __device__ inline int band_lp_smem() { return 8 * kBjWarpWords * 4; }  // 8 warps per CTA

__device__ __forceinline__ void cp_async16(uint32_t *dst, const uint32_t *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Stage words [off, off + 32) of the block row of each member m in mask
// (lane m holds its clip index bm) into row m of rows.  16-byte chunk j of
// row m sits at chunk position j ^ (m & 7), so that 8 lanes reading 16-byte
// vectors of their own rows meet 8 different bank groups.  blk must be
// 16-byte aligned (the caller checks).
__device__ __forceinline__ void bj_stage(uint32_t *rows, const uint16_t *blk, int nb2, uint32_t bm, unsigned mask,
                                         int off, int lane) {
    __syncwarp();  // the rows' previous contents are no longer read
    const int g = lane >> 3, j = lane & 7;
    for (int m0 = 0; m0 < 32; m0 += 4) {
        if (((mask >> m0) & 0xfu) == 0u) continue;  // warp-uniform
        const int m = m0 + g;
        const uint32_t b = __shfl_sync(0xffffffffu, bm, m);
        if ((mask >> m) & 1u)
            cp_async16(rows + 32 * m + 4 * (j ^ (m & 7)),
                       reinterpret_cast<const uint32_t *>(blk + (size_t)b * 2 * nb2) + off + 4 * j);
    }
    cp_async_wait_all();
    __syncwarp();
}

// Sum over the 32 words of x - min(x, y), both 16-bit halves added: x from the
// lane's member row m and y from the representative's words (MEMBER_FIRST),
// or the other way round.  Each half of a term is at most 256 (a block
// count), so each half of the running sum stays below 32 * 256.
template <bool MEMBER_FIRST>
__device__ __forceinline__ int bj_deficit(const uint32_t *row, int m, const uint32_t *rep) {
    uint32_t acc = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint4 u = *reinterpret_cast<const uint4 *>(row + 4 * (j ^ (m & 7)));
        const uint4 r = *reinterpret_cast<const uint4 *>(rep + 4 * j);
        if constexpr (MEMBER_FIRST) {
            acc += (u.x - __vminu2(u.x, r.x)) + (u.y - __vminu2(u.y, r.y));
            acc += (u.z - __vminu2(u.z, r.z)) + (u.w - __vminu2(u.w, r.w));
        } else {
            acc += (r.x - __vminu2(r.x, u.x)) + (r.y - __vminu2(r.y, u.y));
            acc += (r.z - __vminu2(r.z, u.z)) + (r.w - __vminu2(r.w, u.w));
        }
    }
    return (int)((acc & 0xffffu) + (acc >> 16));
}

// cosine gates of one pair (warp-uniform result): PCL_GATE_* or 0.  scratch
// (kG2Scratch u16 of shared memory owned by the warp, may be null) speeds up G2.
__device__ __forceinline__ int warp_cosine_gate(const pcl_clipset &A, uint32_t a, const pcl_clipset &B, uint32_t b,
                                const Geo &g, uint32_t num, uint32_t den, int lane,
                                uint16_t *scratch = nullptr) {
    const uint64_t pa = A.pop[a], pb = B.pop[b];
    const uint64_t mn = pa < pb ? pa : pb, mx = pa < pb ? pb : pa;
    if (!((uint64_t)den * den * mn > (uint64_t)num * num * mx)) return PCL_GATE_G1_AREA;
    const int64_t um = cos_umax(pa, pb, num, den);
    const int nb2 = g.nb * g.nb;
    if (warp_g3_rejects(A.blk + (size_t)a * 2 * nb2, B.blk + (size_t)b * 2 * nb2, nb2, pa, pb, um, lane))
        return PCL_GATE_G3_DENSITY;
    const uint16_t *pra = A.prof + (size_t)a * 2 * g.N, *prb = B.prof + (size_t)b * 2 * g.N;
    bool g2;
    if (scratch) {
        switch (g.N) {
            case 64: g2 = warp_g2_rejects_smem<2>(pra, prb, g.S, um, lane, scratch); break;
            case 128: g2 = warp_g2_rejects_smem<4>(pra, prb, g.S, um, lane, scratch); break;
            case 256: g2 = warp_g2_rejects_smem<8>(pra, prb, g.S, um, lane, scratch); break;
            default: g2 = warp_g2_rejects_smem<16>(pra, prb, g.S, um, lane, scratch); break;
        }
    } else {
        g2 = warp_g2_rejects_n(pra, prb, g.N, g.S, um, lane);
    }
    if (g2) return PCL_GATE_G2_PROFILE;
    return PCL_GATE_NONE;
}

}  // namespace pcl

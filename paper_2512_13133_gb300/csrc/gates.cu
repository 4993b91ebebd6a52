// a2: lossless multi-stage pre-screening for cosine mode (Sec. 3.1 stage 1)
// and the area-sorted band join that generates candidate pairs.
//
// Every gate is an upper bound on the overlap c(s) for all shifts of the
// marker window, compared with the exact integer threshold rule of Eq. 2, so
// a rejected pair can never pass:
//   G1 area     c(s) <= min(|A|, |B|)  ->  den^2 min > num^2 max required
//   G3 density  the ones of A in a 16x16 block can only meet ones of B in the
//               block's neighbourhood: c <= sum_k min(cnt_A(k), nbr_B(k)),
//               taken both ways
//   G2 profile  c(dx, dy) <= sum_j min(r_A(j), r_B(j - dy)); the best dy
//               bounds every shift; same with column counts
// Evaluation order G1 -> G3 -> G2 (cheapest first); a rejected pair records
// the first gate that rejects it.
//
// Candidate generation: G1 passes exactly when the larger area is below
// den^2/num^2 times the smaller one, so after a counting sort of the clips by
// area every G1 survivor (i, j) lies in the band of positions
// (p, end_p) with end_p = #{clips with area <= floor((den^2 a_p - 1)/num^2)}.
// Warps take positions p from a global counter and test G3 and G2 on every
// band member with the whole warp.  A shard s of S (several GPUs sharing one
// self-join) keeps the pairs a < b with a mod S = s: its warps take the
// representatives a = s, s + S, ... and walk their two-sided band (the clips
// whose areas pass G1 with a's, found from the counting sort's bucket
// offsets), keeping the members b > a -- a partition that depends on the clip
// indices only, not on the order the counting sort gives clips of equal
// area, and each shard walks 1/S of the representatives.
#include <climits>

#include "gates.cuh"

namespace pcl {

namespace {

// position of the (r + 1)-th set bit of m, -1 if m has r set bits or fewer
__device__ __forceinline__ int nth_set_bit(unsigned m, int r) {
    if (__popc(m) <= r) return -1;
    int lo = 0, hi = 31;  // smallest p with popc(m & bits 0..p) > r
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;  // <= 30, so the mask below does not overflow
        if (__popc(m & ((2u << mid) - 1u)) > r) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// sort keys of the topological pre-screen: class * V + area, the class
// being the polygon count saturated at kTopoClasses - 1
__global__ void topo_key_kernel(const uint32_t *pop, const int32_t *esig, uint32_t n, uint32_t V, uint32_t *key) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t np = esig[(size_t)i * 8 + ES_N];
        const uint32_t cls = np < kTopoClasses - 1 ? (uint32_t)np : (uint32_t)(kTopoClasses - 1);
        key[i] = cls * V + pop[i];
    }
}

__global__ void hist_kernel(const uint32_t *pop, uint32_t n, uint32_t *hist) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(hist + pop[i], 1u);
}

// exclusive scan of v[0..m) into v (single CTA of 1024 threads)
__global__ void __launch_bounds__(1024) scan_kernel(uint32_t *v, uint32_t m) {
    __shared__ uint32_t wsum[32];
    const uint32_t per = (m + 1023) / 1024;
    const uint32_t lo = threadIdx.x * per, hi = min(m, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; ++i) s += v[i];
    // block exclusive scan of s
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t run = x - s + (wid ? wsum[wid - 1] : 0u);
    for (uint32_t i = lo; i < hi; ++i) {
        const uint32_t t = v[i];
        v[i] = run;
        run += t;
    }
}

__global__ void scatter_kernel(const uint32_t *pop, uint32_t n, const uint32_t *cum, uint32_t *fill,
                               uint32_t *order, uint32_t *spop) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t v = pop[i];
        const uint32_t pos = cum[v] + atomicAdd(fill + v, 1u);
        order[pos] = i;
        spop[pos] = v;
    }
}

// spop holds the sorted keys: the area, or with the topological pre-screen
// class * V + area (V = N^2 + 2), so that a band never leaves its class
// LP: the lane-per-member first chunk of G3 (WPL = 4, blk 16-byte aligned;
// band_lp_smem() bytes of dynamic shared memory)
template <int WPL, bool LP = false>
__global__ void __launch_bounds__(256, LP ? 6 : 8) band_join_kernel(pcl_params prm, pcl_clipset cs, const uint32_t *order,
                                                        const uint32_t *spop, const uint32_t *cum, uint32_t V,
                                                        uint32_t vmax_all, pcl_pair *out, uint64_t cap,
                                                        unsigned long long *count,
                                                        unsigned long long *local_gates,
                                                        unsigned int *next_pos, uint32_t shard,
                                                        uint32_t n_shards) {
    const Geo g = make_geo(prm);
    const int lane = threadIdx.x & 31;
    const uint32_t n = cs.n_clips;
    const int nb2 = g.nb * g.nb, words = nb2 / 2;
    const uint64_t num2 = (uint64_t)prm.cos_num * prm.cos_num, den2 = (uint64_t)prm.cos_den * prm.cos_den;
    unsigned long long kept = 0, g2 = 0, g3 = 0;
    const bool sharded = n_shards > 1;
    for (;;) {
        uint32_t p = 0;
        if (lane == 0) p = atomicAdd(next_pos, 1u);
        p = __shfl_sync(0xffffffffu, p, 0);
        // the representative: the clip at sorted position p, or with shards
        // the clip of index shard + p S
        const uint64_t ai = sharded ? (uint64_t)shard + (uint64_t)p * n_shards : p;
        if (ai >= n) break;
        const uint32_t a = sharded ? (uint32_t)ai : order[p];
        const uint32_t kp = sharded ? cs.pop[a] : spop[p];
        const uint64_t pa = kp % V;
        const uint32_t base = kp - (uint32_t)pa;  // first key of the class
        uint64_t vmax = pa == 0 ? 0 : (den2 * pa - 1) / num2;
        if (vmax > vmax_all) vmax = vmax_all;
        const uint32_t end = cum[base + vmax + 1];
        // forward band from p + 1, or the two-sided band from the smallest
        // area that passes G1 with pa (num^2 pa < den^2 pb)
        const uint32_t start = sharded ? cum[base + (pa == 0 ? 0 : (num2 * pa) / den2 + 1)] : p + 1;
        const uint32_t *cwa = reinterpret_cast<const uint32_t *>(cs.blk + (size_t)a * 2 * nb2);
        uint32_t ca[WPL], da[WPL];
#pragma unroll
        for (int c = 0; c < WPL; ++c) {
            const int t = c * 32 + lane;
            ca[c] = t < words ? cwa[t] : 0u;
            da[c] = t < words ? cwa[words + t] : 0u;
        }
        // small rasters (one word of block counts per lane: N <= 128): the
        // representative's profiles and their dilated maxima in the warp's
        // scratch for G2, which decides most band pairs there
        uint16_t *g2s = nullptr;
        if constexpr (WPL == 1) {
            extern __shared__ uint16_t g2_scratch[];
            g2s = g2_scratch + (threadIdx.x >> 5) * band_g2_warp(g.N, g.S);
            g2_rep_setup(cs.prof + (size_t)a * 2 * g.N, g.N, g.S, lane, g2s);
        }
        uint32_t *lrep = nullptr;  // LP: the representative's first-chunk words, then the member rows
        if constexpr (LP) {
            static_assert(WPL > 1, "the first chunk is 32 words");
            extern __shared__ __align__(16) uint32_t bj_lp[];
            lrep = bj_lp + (threadIdx.x >> 5) * kBjWarpWords;
            __syncwarp();  // the previous representative's words are no longer read
            lrep[lane] = ca[0];
            lrep[32 + lane] = da[0];
            __syncwarp();
        }
        if (pa == 0) {  // the band holds the other empty clips only: similar by definition
            for (uint32_t q0 = start; q0 < end; q0 += 32) {
                const uint32_t bq = q0 + lane < end ? order[q0 + lane] : 0u;
                const bool v = q0 + lane < end && (!sharded || bq > a);
                const unsigned m = __ballot_sync(0xffffffffu, v);
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(m));
                base = __shfl_sync(0xffffffffu, base, 0);
                const unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
                if (v && idx < cap) out[idx] = pcl_pair{min(a, bq), max(a, bq)};
                kept += __popc(m);
            }
            continue;
        }
        // G2 and the output for member bk once G3 keeps it
        auto after_g3 = [&](uint32_t bk, int tAk) {
            // G2 with the same threshold (tA = pa - um; never clamped in a band)
            bool g2r;
            if constexpr (WPL == 1) {
                const uint16_t *pbk = cs.prof + (size_t)bk * 2 * g.N;
                g2r = g2_rejects_small(g2s, pbk, g.N, g.S, (int64_t)pa - tAk, lane);
            } else {
                g2r = warp_g2_rejects_lite(cs.prof + (size_t)a * 2 * g.N, cs.prof + (size_t)bk * 2 * g.N, g.N,
                                           g.S, (int64_t)pa - tAk, lane);
            }
            if (g2r) {
                ++g2;
                return;
            }
            ++kept;
            if (lane == 0) {
                const unsigned long long idx = atomicAdd(count, 1ull);
                if (idx < cap) out[idx] = pcl_pair{min(a, bk), max(a, bk)};
            }
        };
        // band members 32 at a time: lane l sets up member q0 + l (index,
        // thresholds; members of a non-empty representative are non-empty),
        // then the warp tests them one after the other
        for (uint32_t q0 = start; q0 < end; q0 += 32) {
            const uint32_t q = q0 + lane;
            uint32_t b = 0;
            int tA = 0, tB = 0;  // areas are below 2^31, so are the thresholds (clamped below)
            if (q < end) {
                b = order[q];
                const uint64_t pb = spop[q] % V;
                const int64_t um = cos_umax(pa, pb, prm.cos_num, prm.cos_den);
                tA = (int)max((int64_t)pa - um, (int64_t)INT_MIN);
                tB = (int)max((int64_t)pb - um, (int64_t)INT_MIN);
            }
            int cnt = (int)min(32u, end - q0);
            if (sharded) {  // the members b > a only, moved to the low lanes in order
                const unsigned mem = __ballot_sync(0xffffffffu, q < end && b > a);
                const int src = nth_set_bit(mem, lane);  // lane of this lane's member
                const int from = src >= 0 ? src : lane;
                b = __shfl_sync(0xffffffffu, b, from);
                tA = __shfl_sync(0xffffffffu, tA, from);
                tB = __shfl_sync(0xffffffffu, tB, from);
                cnt = __popc(mem);
            }
            // the rest of the gates for member k after the pre-screen
            auto finish = [&](int k, uint32_t bk, int tAk, int tBk) {
                const uint32_t *cwb = reinterpret_cast<const uint32_t *>(cs.blk + (size_t)bk * 2 * nb2);
                if (g3_rejects_thr<WPL>(ca, da, cwb, cwb + words, words, tAk, tBk, lane)) {
                    ++g3;
                    return;
                }
                after_g3(bk, tAk);
            };
            if constexpr (LP) {
                // each lane sums its member's first chunk of both deficits
                // (A's first: on its own it rejects most band pairs); the
                // members left take the other chunks with the whole warp
                const bool mine = lane < cnt;
                uint32_t *rows = lrep + 64;
                bj_stage(rows, cs.blk, nb2, b, __ballot_sync(0xffffffffu, mine), words, lane);  // neighbourhood sums
                int DA = 0, DB = 0;
                bool rej = false;
                if (mine) {
                    DA = bj_deficit<false>(rows + 32 * lane, lane, lrep);
                    rej = DA >= tA;
                }
                const unsigned keep_a = __ballot_sync(0xffffffffu, mine && !rej);
                if (keep_a) {
                    bj_stage(rows, cs.blk, nb2, b, keep_a, 0, lane);  // block counts
                    if (mine && !rej) {
                        DB = bj_deficit<true>(rows + 32 * lane, lane, lrep + 32);
                        rej = DB >= tB;
                    }
                }
                g3 += __popc(__ballot_sync(0xffffffffu, mine && rej));
                unsigned left = __ballot_sync(0xffffffffu, mine && !rej);
                // the members left, one after the other with the whole warp; the
                // next one's second-chunk words load while the current one is tested
                uint32_t b1 = 0u, d1 = 0u;
                if (left) {
                    const uint32_t *cw = reinterpret_cast<const uint32_t *>(
                        cs.blk + (size_t)__shfl_sync(0xffffffffu, b, __ffs(left) - 1) * 2 * nb2);
                    b1 = __ldg(cw + 32 + lane);
                    d1 = __ldg(cw + words + 32 + lane);
                }
                while (left) {
                    const int k = __ffs(left) - 1;
                    left &= left - 1u;
                    const uint32_t bk = __shfl_sync(0xffffffffu, b, k);
                    const int tAk = __shfl_sync(0xffffffffu, tA, k), tBk = __shfl_sync(0xffffffffu, tB, k);
                    const int DAk = __shfl_sync(0xffffffffu, DA, k), DBk = __shfl_sync(0xffffffffu, DB, k);
                    const uint32_t cb1 = b1, cd1 = d1;
                    if (left) {
                        const uint32_t *cw = reinterpret_cast<const uint32_t *>(
                            cs.blk + (size_t)__shfl_sync(0xffffffffu, b, __ffs(left) - 1) * 2 * nb2);
                        b1 = __ldg(cw + 32 + lane);
                        d1 = __ldg(cw + words + 32 + lane);
                    }
                    const uint32_t *cwb = reinterpret_cast<const uint32_t *>(cs.blk + (size_t)bk * 2 * nb2);
                    if (g3_rest_pre<WPL>(ca, da, cwb, cwb + words, words, tAk, tBk, DAk, DBk, cb1, cd1, lane)) ++g3;
                    else after_g3(bk, tAk);
                }
                continue;
            }
            // Pre-screen two members at a time: the representative's deficit
            // over the first 64 blocks against each member (the test that
            // alone rejects most band pairs), both sums in one reduction (each
            // lane's share of one sum is at most 2 * 256, a 32-lane sum at
            // most 16384, so the two fit in 16-bit halves).  Members the
            // pre-screen keeps get the full gates, which repeat this test.
            const bool v0 = lane < words;
            int k = 0;
            for (; k + 1 < cnt; k += 2) {
                const uint32_t b0 = __shfl_sync(0xffffffffu, b, k), b1 = __shfl_sync(0xffffffffu, b, k + 1);
                const int tA0 = __shfl_sync(0xffffffffu, tA, k), tA1 = __shfl_sync(0xffffffffu, tA, k + 1);
                const uint32_t *d0p = reinterpret_cast<const uint32_t *>(cs.blk + (size_t)b0 * 2 * nb2) + words;
                const uint32_t *d1p = reinterpret_cast<const uint32_t *>(cs.blk + (size_t)b1 * 2 * nb2) + words;
                const uint32_t n0 = v0 ? __ldg(d0p + lane) : 0u, n1 = v0 ? __ldg(d1p + lane) : 0u;
                const uint32_t x0 = ca[0] - __vminu2(ca[0], n0), x1 = ca[0] - __vminu2(ca[0], n1);
                const uint32_t both = ((x0 & 0xffffu) + (x0 >> 16)) | (((x1 & 0xffffu) + (x1 >> 16)) << 16);
                const uint32_t sr = __reduce_add_sync(0xffffffffu, both);
                const bool r0 = (int)(sr & 0xffffu) >= tA0, r1 = (int)(sr >> 16) >= tA1;
                g3 += (r0 ? 1 : 0) + (r1 ? 1 : 0);
                if (!r0) finish(k, b0, tA0, __shfl_sync(0xffffffffu, tB, k));
                if (!r1) finish(k + 1, b1, tA1, __shfl_sync(0xffffffffu, tB, k + 1));
            }
            if (k < cnt)
                finish(k, __shfl_sync(0xffffffffu, b, k), __shfl_sync(0xffffffffu, tA, k),
                       __shfl_sync(0xffffffffu, tB, k));
        }
    }
    if (lane == 0) {
        if (kept) atomicAdd(local_gates + 0, kept);
        if (g2) atomicAdd(local_gates + PCL_GATE_G2_PROFILE, g2);
        if (g3) atomicAdd(local_gates + PCL_GATE_G3_DENSITY, g3);
    }
}

// add this call's gate counts to the caller's array; G1 = all pairs minus the
// pairs the band join enumerated.  With the topological pre-screen (cum of
// the class keys given, C classes of V keys) the pairs of different classes
// count as its rejections and G1 takes the rest.
__global__ void finish_gates_kernel(const unsigned long long *local, unsigned long long *gates,
                                    unsigned long long total, const uint32_t *cum, uint32_t V, uint32_t C,
                                    uint32_t n) {
    if (threadIdx.x == 0 && gates) {
        const unsigned long long seen =
            local[0] + local[PCL_GATE_G2_PROFILE] + local[PCL_GATE_G3_DENSITY];
        unsigned long long same = total;
        if (cum) {
            same = 0;
            for (uint32_t c = 0; c < C; ++c) {
                const unsigned long long k = (c + 1 < C ? cum[(c + 1) * V] : n) - cum[c * V];
                same += k * (k ? k - 1 : 0) / 2;
            }
            gates[PCL_GATE_T0_TOPO] += total - same;
        }
        gates[0] += local[0];
        gates[PCL_GATE_G1_AREA] += same - seen;
        gates[PCL_GATE_G2_PROFILE] += local[PCL_GATE_G2_PROFILE];
        gates[PCL_GATE_G3_DENSITY] += local[PCL_GATE_G3_DENSITY];
    }
}

}  // namespace

// counting sort of n clips by area: cum[v] = #clips with area < v (V entries),
// order/spop = clip indices and areas in ascending area order
cudaError_t launch_area_sort(const uint32_t *pop, uint32_t n, uint32_t V, uint32_t *cum, uint32_t *fill,
                             uint32_t *order, uint32_t *spop, int num_sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(cum, 0, 4 * (size_t)V, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(fill, 0, 4 * (size_t)V, st);
    if (e != cudaSuccess) return e;
    if (n) hist_kernel<<<num_sms * 4, 256, 0, st>>>(pop, n, cum);
    scan_kernel<<<1, 1024, 0, st>>>(cum, V);
    if (n) scatter_kernel<<<num_sms * 4, 256, 0, st>>>(pop, n, cum, fill, order, spop);
    return cudaGetLastError();
}

// workspace bytes for the band join of n clips under g (topo: the
// topological pre-screen's class keys as well)
size_t band_join_workspace(const Geo &g, uint32_t n, bool topo) {
    const size_t V = (size_t)g.N * g.N + 2;  // areas 0..N^2, plus the end slot
    const size_t Vt = V * (topo ? kTopoClasses : 1);
    return 4 * (2 * Vt + (topo ? 3 : 2) * (size_t)n) + 8 * 16 + 64;
}

// pairs i < j < n with i mod S = s: n - 1 - i for each such i
uint64_t shard_pairs(uint64_t n, uint32_t s, uint32_t S) {
    if (S <= 1) return n * (n ? n - 1 : 0) / 2;
    uint64_t t = 0;
    for (uint64_t i = s; i < n; i += S) t += n - 1 - i;
    return t;
}

cudaError_t launch_band_join(const pcl_params &prm, const pcl_clipset &cs, void *ws, size_t ws_bytes,
                             pcl_pair *out, uint64_t cap, unsigned long long *count,
                             unsigned long long *gates, int num_sms, cudaStream_t st, uint32_t shard,
                             uint32_t n_shards) {
    if (n_shards == 0 || shard >= n_shards) return cudaErrorInvalidValue;
    const Geo g = make_geo(prm);
    const uint32_t n = cs.n_clips;
    const bool topo = (prm.flags & PCL_P_TOPO_HASH) != 0;
    if (topo && (n_shards != 1 || (n && !cs.esig))) return cudaErrorInvalidValue;
    if (ws_bytes < band_join_workspace(g, n, topo)) return cudaErrorInvalidValue;
    const uint32_t V = (uint32_t)g.N * g.N + 2;
    const uint32_t C = topo ? (uint32_t)kTopoClasses : 1u, Vt = V * C;
    char *w = static_cast<char *>(ws);
    unsigned long long *local = reinterpret_cast<unsigned long long *>(w);
    unsigned int *next_pos = reinterpret_cast<unsigned int *>(w + 8 * 16);
    uint32_t *cum = reinterpret_cast<uint32_t *>(w + 8 * 16 + 64);
    uint32_t *fill = cum + Vt;
    uint32_t *order = fill + Vt;
    uint32_t *spop = order + n;
    uint32_t *key = topo ? spop + n : nullptr;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w, 0, 8 * 16 + 64 + 4 * (size_t)2 * Vt, st)) != cudaSuccess) return e;
    if (n == 0) {
        finish_gates_kernel<<<1, 32, 0, st>>>(local, gates, 0ull, nullptr, V, 1, 0);
        return cudaGetLastError();
    }
    const uint32_t *k = cs.pop;
    if (topo) {
        topo_key_kernel<<<num_sms * 4, 256, 0, st>>>(cs.pop, cs.esig, n, V, key);
        k = key;
    }
    hist_kernel<<<num_sms * 4, 256, 0, st>>>(k, n, cum);
    scan_kernel<<<1, 1024, 0, st>>>(cum, Vt);
    scatter_kernel<<<num_sms * 4, 256, 0, st>>>(k, n, cum, fill, order, spop);
    const uint32_t vall = (uint32_t)g.N * g.N;
    // the lane-per-member first chunk at 256² (4 words per lane; at 512² the
    // first 64 of 1,024 blocks decide too few pairs to pay for the staging)
    const bool lp = (reinterpret_cast<uintptr_t>(cs.blk) & 15u) == 0;  // 16-byte copies of block rows
    switch ((g.nb * g.nb / 2 + 31) / 32) {  // u32 words of block counts per lane
        case 1: band_join_kernel<1><<<num_sms * 8, 256, band_g2_smem(g.N, g.S), st>>>(prm, cs, order, spop, cum, V,
                                                                                       vall, out, cap, count,
                                                                 local, next_pos, shard, n_shards); break;
        case 4:
            if (lp) band_join_kernel<4, true><<<num_sms * 6, 256, band_lp_smem(), st>>>(prm, cs, order, spop, cum, V,
                                                                                     vall, out, cap, count, local,
                                                                                     next_pos, shard, n_shards);
            else band_join_kernel<4><<<num_sms * 8, 256, 0, st>>>(prm, cs, order, spop, cum, V, vall, out, cap, count,
                                                                  local, next_pos, shard, n_shards);
            break;
        case 16: band_join_kernel<16><<<num_sms * 8, 256, 0, st>>>(prm, cs, order, spop, cum, V, vall, out, cap,
                                                                   count, local, next_pos, shard, n_shards); break;
        default: return cudaErrorInvalidValue;
    }
    const unsigned long long total = shard_pairs(n, shard, n_shards);
    finish_gates_kernel<<<1, 32, 0, st>>>(local, gates, total, topo ? cum : nullptr, V, C, n);
    return cudaGetLastError();
}

}  // namespace pcl

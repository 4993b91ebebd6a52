// a2 for two clip sets: cosine candidates between a query set Q and a
// resident library L (Sec. 3.1 stage 1), used by the serving loop.
//
// The library is sorted by area once (launch_area_sort).  For a query of
// area a the G1 survivors are exactly the library clips with area in
// [floor(num^2 a / den^2) + 1, floor((den^2 a - 1) / num^2)], a contiguous range
// of the sorted order.  The queries of a request are sorted by area too, so
// both ends of their bands are monotone and the queries whose band meets a
// library chunk (kChunk sorted positions) are a contiguous run of them.  Work
// items are (chunk, query) pairs in chunk-major order: the warps in flight
// at any moment cover a few neighbouring chunks with all their queries, so
// each chunk's signatures come from DRAM about once per request and are
// re-read from L2 by the other queries (a band of a large library is larger
// than L2, and query-major order re-fetched it from DRAM for every query).
// Each warp tests G3 and G2 on every member of its item, as in the self-join.
#include "gates.cuh"

namespace pcl {

cudaError_t launch_area_sort(const uint32_t *, uint32_t, uint32_t, uint32_t *, uint32_t *, uint32_t *, uint32_t *,
                             int, cudaStream_t);

namespace {

constexpr uint32_t kChunk = 1024;

// per query, in area order (position i): first and end position of its band
__global__ void cross_prep_kernel(const uint32_t *qspop, uint32_t nq, const uint32_t *lib_cum, uint32_t vmax_all,
                                  uint32_t num, uint32_t den, uint32_t *beg, uint32_t *end) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const uint64_t a = qspop[q];
    const uint64_t n2 = (uint64_t)num * num, d2 = (uint64_t)den * den;
    uint64_t lo, hi;
    if (a == 0) {
        lo = 0;
        hi = 0;
    } else {
        lo = n2 * a / d2 + 1;
        hi = (d2 * a - 1) / n2;
    }
    if (hi > vmax_all) hi = vmax_all;
    // lo <= hi whenever num < den; an empty band keeps both ends monotone
    const uint32_t b = lib_cum[lo <= vmax_all + 1 ? lo : vmax_all + 1];
    const uint32_t e = lo <= hi ? lib_cum[hi + 1] : b;
    beg[q] = b;
    end[q] = e;
}

// per library chunk k: the area-order positions [qlo, qlo + cnt) of the
// queries whose band meets [k kChunk, (k + 1) kChunk) (beg and end are
// non-decreasing; a query with an empty band inside the run gets an empty item)
__global__ void cross_chunks_kernel(const uint32_t *beg, const uint32_t *end, uint32_t nq, uint32_t n_ch,
                                    uint32_t *qlo, uint32_t *cnt) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_ch) return;
    const uint32_t c0 = k * kChunk, c1 = c0 + kChunk;
    uint32_t lo = 0, hi = nq;  // first position with end > c0
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (end[mid] > c0) hi = mid;
        else lo = mid + 1;
    }
    const uint32_t a = lo;
    lo = a;
    hi = nq;  // first position with beg >= c1
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (beg[mid] >= c1) hi = mid;
        else lo = mid + 1;
    }
    qlo[k] = a;
    cnt[k] = lo - a;
}

// exclusive scan of v[0..m) into out[0..m], out[m] = total (single CTA)
__global__ void __launch_bounds__(1024) scan_items_kernel(const uint32_t *v, uint32_t m, uint32_t *out) {
    __shared__ uint32_t wsum[32];
    const uint32_t per = (m + 1023) / 1024;
    const uint32_t lo = threadIdx.x * per, hi = min(m, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; ++i) s += v[i];
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
        out[i] = run;
        run += v[i];
    }
    if (threadIdx.x == 1023) out[m] = run;
}

// WPL: u32 words of block counts per lane (the query's are held in registers).
// LP: the lane-per-member first chunk of G3, as in the self-join (WPL = 4,
// the library's blk 16-byte aligned; band_lp_smem() bytes of dynamic shared
// memory).  Without LP the minimum of blocks per SM is left unset (0): the
// compiler's own register choice, which a hint of 1 would raise.
template <int WPL, bool LP = false>
__global__ void __launch_bounds__(256, LP ? 6 : 0) cross_join_kernel(pcl_params prm, pcl_clipset Q, pcl_clipset L,
                                                         const uint32_t *lib_order, const uint32_t *lib_spop,
                                                         const uint32_t *qorder, const uint32_t *qspop,
                                                         const uint32_t *beg, const uint32_t *end,
                                                         const uint32_t *qlo, const uint32_t *item_off,
                                                         uint32_t n_ch, pcl_pair *out, uint64_t cap,
                                                         unsigned long long *count, unsigned long long *local,
                                                         unsigned int *next_item) {
    const Geo g = make_geo(prm);
    const int lane = threadIdx.x & 31;
    const uint32_t total = item_off[n_ch];
    const int nb2 = g.nb * g.nb, words = nb2 / 2;
    unsigned long long kept = 0, g2 = 0, g3 = 0;
    auto emit = [&](bool keep, uint32_t q, uint32_t b) {  // warp-aggregated
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (!m) return;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        const unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
        if (keep && idx < cap) out[idx] = pcl_pair{q, b};
    };
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(next_item, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        // chunk of item t: last k with item_off[k] <= t; then its query
        uint32_t lo = 0, hi = n_ch;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) / 2;
            if (item_off[mid] <= t) lo = mid;
            else hi = mid;
        }
        const uint32_t k = lo;
        const uint32_t i = qlo[k] + (t - item_off[k]);  // area-order position of the query
        const uint32_t q = qorder[i];
        const uint32_t p0 = max(k * kChunk, beg[i]);
        const uint32_t p1 = min(k * kChunk + kChunk, end[i]);
        if (p0 >= p1) continue;
        const uint64_t pa = qspop[i];
        if (pa == 0) {  // the band holds the empty library clips only: similar by definition
            for (uint32_t q0 = p0; q0 < p1; q0 += 32) {
                const bool v = q0 + lane < p1;
                emit(v, q, v ? lib_order[q0 + lane] : 0u);
                kept += __popc(__ballot_sync(0xffffffffu, v));
            }
            continue;
        }
        const uint32_t *cwa = reinterpret_cast<const uint32_t *>(Q.blk + (size_t)q * 2 * nb2);
        uint32_t ca[WPL], da[WPL];
#pragma unroll
        for (int c = 0; c < WPL; ++c) {
            const int w = c * 32 + lane;
            ca[c] = w < words ? cwa[w] : 0u;
            da[c] = w < words ? cwa[words + w] : 0u;
        }
        // small rasters (one word of block counts per lane: N <= 128): the
        // query's profiles and their dilated maxima in the warp's scratch for
        // G2, which decides most band pairs
        uint16_t *g2s = nullptr;
        if constexpr (WPL == 1) {
            extern __shared__ uint16_t g2_scratch[];
            g2s = g2_scratch + (threadIdx.x >> 5) * band_g2_warp(g.N, g.S);
            g2_rep_setup(Q.prof + (size_t)q * 2 * g.N, g.N, g.S, lane, g2s);
        }
        uint32_t *lrep = nullptr;  // LP: the query's first-chunk words, then the member rows
        if constexpr (LP) {
            static_assert(WPL > 1, "the first chunk is 32 words");
            extern __shared__ __align__(16) uint32_t bj_lp[];
            lrep = bj_lp + (threadIdx.x >> 5) * kBjWarpWords;
            __syncwarp();  // the previous query's words are no longer read
            lrep[lane] = ca[0];
            lrep[32 + lane] = da[0];
            __syncwarp();
        }
        // G2 and the output for library clip bk once G3 keeps it
        auto after_g3 = [&](uint32_t bk, int tAk) {
            bool g2r;
            if constexpr (WPL == 1) {
                const uint16_t *pbk = L.prof + (size_t)bk * 2 * g.N;
                g2r = g2_rejects_small(g2s, pbk, g.N, g.S, (int64_t)pa - tAk, lane);
            } else {
                g2r = warp_g2_rejects_lite(Q.prof + (size_t)q * 2 * g.N, L.prof + (size_t)bk * 2 * g.N, g.N, g.S,
                                           (int64_t)pa - tAk, lane);
            }
            if (g2r) {
                ++g2;
                return;
            }
            ++kept;
            if (lane == 0) {
                const unsigned long long idx = atomicAdd(count, 1ull);
                if (idx < cap) out[idx] = pcl_pair{q, bk};
            }
        };
        // members 32 at a time: lane l sets up member q0 + l (index, the
        // thresholds of the exact rule; G1 passes, so neither is clamped),
        // then the warp tests them one after the other
        for (uint32_t q0 = p0; q0 < p1; q0 += 32) {
            uint32_t b = 0;
            int tA = 0, tB = 0;
            if (q0 + lane < p1) {
                b = lib_order[q0 + lane];
                const uint64_t pb = lib_spop[q0 + lane];
                const int64_t um = cos_umax(pa, pb, prm.cos_num, prm.cos_den);
                tA = (int)((int64_t)pa - um);
                tB = (int)((int64_t)pb - um);
            }
            const int cnt = (int)min(32u, p1 - q0);
            if constexpr (LP) {
                // each lane sums its member's first chunk of both deficits; the
                // members left take the other chunks with the whole warp
                const bool mine = lane < cnt;
                uint32_t *rows = lrep + 64;
                bj_stage(rows, L.blk, nb2, b, __ballot_sync(0xffffffffu, mine), words, lane);  // neighbourhood sums
                int DA = 0, DB = 0;
                bool rej = false;
                if (mine) {
                    DA = bj_deficit<false>(rows + 32 * lane, lane, lrep);
                    rej = DA >= tA;
                }
                const unsigned keep_a = __ballot_sync(0xffffffffu, mine && !rej);
                if (keep_a) {
                    bj_stage(rows, L.blk, nb2, b, keep_a, 0, lane);  // block counts
                    if (mine && !rej) {
                        DB = bj_deficit<true>(rows + 32 * lane, lane, lrep + 32);
                        rej = DB >= tB;
                    }
                }
                g3 += __popc(__ballot_sync(0xffffffffu, mine && rej));
                unsigned left = __ballot_sync(0xffffffffu, mine && !rej);
                while (left) {
                    const int k = __ffs(left) - 1;
                    left &= left - 1u;
                    const uint32_t bk = __shfl_sync(0xffffffffu, b, k);
                    const int tAk = __shfl_sync(0xffffffffu, tA, k), tBk = __shfl_sync(0xffffffffu, tB, k);
                    const int DAk = __shfl_sync(0xffffffffu, DA, k), DBk = __shfl_sync(0xffffffffu, DB, k);
                    const uint32_t *cwb = reinterpret_cast<const uint32_t *>(L.blk + (size_t)bk * 2 * nb2);
                    if (g3_rest_rejects<WPL>(ca, da, cwb, cwb + words, words, tAk, tBk, DAk, DBk, lane)) ++g3;
                    else after_g3(bk, tAk);
                }
            } else {
                for (int k = 0; k < cnt; ++k) {
                    const uint32_t bk = __shfl_sync(0xffffffffu, b, k);
                    const int tAk = __shfl_sync(0xffffffffu, tA, k), tBk = __shfl_sync(0xffffffffu, tB, k);
                    const uint32_t *cwb = reinterpret_cast<const uint32_t *>(L.blk + (size_t)bk * 2 * nb2);
                    if (g3_rejects_thr<WPL>(ca, da, cwb, cwb + words, words, tAk, tBk, lane)) {
                        ++g3;
                        continue;
                    }
                    after_g3(bk, tAk);
                }
            }
        }
    }
    if (lane == 0) {
        if (kept) atomicAdd(local + 0, kept);
        if (g2) atomicAdd(local + PCL_GATE_G2_PROFILE, g2);
        if (g3) atomicAdd(local + PCL_GATE_G3_DENSITY, g3);
    }
}

__global__ void cross_finish_kernel(const unsigned long long *local, unsigned long long *gates,
                                    unsigned long long total) {
    if (threadIdx.x == 0 && gates) {
        const unsigned long long seen = local[0] + local[PCL_GATE_G2_PROFILE] + local[PCL_GATE_G3_DENSITY];
        gates[0] += local[0];
        gates[PCL_GATE_G1_AREA] += total - seen;
        gates[PCL_GATE_G2_PROFILE] += local[PCL_GATE_G2_PROFILE];
        gates[PCL_GATE_G3_DENSITY] += local[PCL_GATE_G3_DENSITY];
    }
}

}  // namespace

// workspace of the cross join for nq queries against n_lib library clips:
// 16 u64 counters + next item (64 B), the queries' area histogram and fill
// counters [2 V], their area order and sorted areas, band begins and ends
// [4 nq], per chunk the first query, the item count and the item offsets
// [3 n_ch + 1]
static uint32_t lib_chunks(uint32_t n_lib) { return (n_lib + kChunk - 1) / kChunk; }
size_t cross_join_workspace(const Geo &g, uint32_t nq, uint32_t n_lib) {
    const size_t V = (size_t)g.N * g.N + 2;
    return 8 * 16 + 64 + 4 * (2 * V + 4 * (size_t)nq + 3 * (size_t)lib_chunks(n_lib) + 1);
}

cudaError_t launch_cross_join(const pcl_params &prm, const pcl_clipset &Q, const pcl_clipset &L,
                              const uint32_t *lib_order, const uint32_t *lib_spop, const uint32_t *lib_cum,
                              void *ws, size_t ws_bytes, pcl_pair *out, uint64_t cap, unsigned long long *count,
                              unsigned long long *gates, int num_sms, cudaStream_t st) {
    const Geo g = make_geo(prm);
    const uint32_t nq = Q.n_clips, n_ch = lib_chunks(L.n_clips);
    if (ws_bytes < cross_join_workspace(g, nq, L.n_clips)) return cudaErrorInvalidValue;
    const uint32_t V = (uint32_t)g.N * g.N + 2;
    char *w = static_cast<char *>(ws);
    unsigned long long *local = reinterpret_cast<unsigned long long *>(w);
    unsigned int *next_item = reinterpret_cast<unsigned int *>(w + 8 * 16);
    uint32_t *qcum = reinterpret_cast<uint32_t *>(w + 8 * 16 + 64);
    uint32_t *qfill = qcum + V;
    uint32_t *qorder = qfill + V, *qspop = qorder + nq, *beg = qspop + nq, *endp = beg + nq;
    uint32_t *qlo = endp + nq, *cnt = qlo + n_ch, *item_off = cnt + n_ch;
    cudaError_t e = cudaMemsetAsync(w, 0, 8 * 16 + 64, st);
    if (e != cudaSuccess) return e;
    if (nq && n_ch) {
        e = launch_area_sort(Q.pop, nq, V, qcum, qfill, qorder, qspop, num_sms, st);
        if (e != cudaSuccess) return e;
        cross_prep_kernel<<<(nq + 255) / 256, 256, 0, st>>>(qspop, nq, lib_cum, (uint32_t)g.N * g.N, prm.cos_num,
                                                             prm.cos_den, beg, endp);
        cross_chunks_kernel<<<(n_ch + 255) / 256, 256, 0, st>>>(beg, endp, nq, n_ch, qlo, cnt);
        scan_items_kernel<<<1, 1024, 0, st>>>(cnt, n_ch, item_off);
        // the lane-per-member first chunk at 256² only, as in the self-join
        const bool lp = (reinterpret_cast<uintptr_t>(L.blk) & 15u) == 0;  // 16-byte copies of block rows
        switch ((g.nb * g.nb / 2 + 31) / 32) {  // u32 words of block counts per lane
            case 1: cross_join_kernel<1><<<num_sms * 8, 256, band_g2_smem(g.N, g.S), st>>>(prm, Q, L, lib_order,
                                                                      lib_spop, qorder, qspop,
                                                                      beg, endp, qlo, item_off, n_ch, out, cap,
                                                                      count, local, next_item); break;
            case 4:
                if (lp) cross_join_kernel<4, true><<<num_sms * 6, 256, band_lp_smem(), st>>>(
                    prm, Q, L, lib_order, lib_spop, qorder, qspop, beg, endp, qlo, item_off, n_ch, out, cap, count,
                    local, next_item);
                else cross_join_kernel<4><<<num_sms * 8, 256, 0, st>>>(prm, Q, L, lib_order, lib_spop, qorder, qspop,
                                                                       beg, endp, qlo, item_off, n_ch, out, cap,
                                                                       count, local, next_item);
                break;
            case 16: cross_join_kernel<16><<<num_sms * 8, 256, 0, st>>>(prm, Q, L, lib_order, lib_spop, qorder,
                                                                        qspop, beg, endp, qlo, item_off, n_ch, out,
                                                                        cap, count, local, next_item); break;
            default: return cudaErrorInvalidValue;
        }
    }
    cross_finish_kernel<<<1, 32, 0, st>>>(local, gates, (unsigned long long)nq * L.n_clips);
    return cudaGetLastError();
}

}  // namespace pcl

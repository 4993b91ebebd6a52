// a2 (edge gates) and a7: edge-displacement mode (Sec. 2.2.2) with the
// geometric Min-Max closed form of Sec. 3.2.2 (Eq. 6).
//
// Integer dbu throughout.  One thread evaluates one pair: the polygon lists
// are short (tens of rectangles) and the procedure is a handful of O(n_A n_B)
// scans with early exits, so per-thread evaluation keeps every lane busy on
// its own pair instead of idling lanes on small clips.  Partners are
// recomputed by scanning rather than stored, so no per-thread arrays are
// needed for any polygon count.
#include "edge_dev.cuh"

namespace pcl {

namespace {
using namespace edge_dev;

__device__ __forceinline__ void emit_pair(pcl_pair *out, uint64_t cap, unsigned long long *count,
                                          bool keep, uint32_t a, uint32_t b) {
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (keep) {
        const unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
        if (idx < cap) out[idx] = pcl_pair{a, b};
    }
}

constexpr int kTileI = 16;
constexpr int kQueue = 64;  // per-warp queue of pairs awaiting the full E1 check

// Self-join screen: block (bx, by) covers rows i in [kTileI bx, kTileI bx +
// kTileI) and columns j in [256 by, 256 by + 256); pairs with i < j only.
//
// Each lane owns column j and walks its rows as a small state machine: every
// iteration it may set up one new pair (empty / E2 / pre-alignment) and runs
// one occupancy-grid test of one small-side polygon.  Lanes therefore advance
// through their pairs independently instead of waiting for the slowest lane
// of every pair.  Pairs whose polygons all pass the grid test (about 0.3 % of
// random pairs) go to a per-warp queue; once 32 are queued the warp runs the
// full correspondence check on them, one pair per lane.
__global__ void __launch_bounds__(256) edge_screen_kernel(pcl_params prm, pcl_clipset cs,
                                                          pcl_pair *out, uint64_t cap,
                                                          unsigned long long *count,
                                                          unsigned long long *gates) {
    const uint32_t n = cs.n_clips;
    const uint32_t j = blockIdx.y * 256u + threadIdx.x;
    const uint32_t i0 = blockIdx.x * kTileI;
    if (i0 >= n || i0 > blockIdx.y * 256u + 255u) return;  // whole block below the diagonal
    const int W = prm.window_dbu, M = prm.marker_dbu, tol = prm.edge_tol_dbu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ int32_t es_i[kTileI][8];
    __shared__ uint32_t off_i[kTileI];
    __shared__ uint2 queue[8][kQueue];
    for (int t = threadIdx.x; t < kTileI * 8; t += blockDim.x) {
        const uint32_t i = i0 + t / 8;
        es_i[t / 8][t % 8] = i < n ? __ldg(cs.esig + (size_t)i * 8 + t % 8) : 0;
    }
    for (int t = threadIdx.x; t < kTileI; t += blockDim.x) off_i[t] = i0 + t < n ? __ldg(cs.rect_off + i0 + t) : 0;
    __syncthreads();
    const bool jv = j < n;
    int32_t eb[8];
    uint32_t ob = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) eb[k] = jv ? __ldg(cs.esig + (size_t)j * 8 + k) : 0;
    if (jv) ob = __ldg(cs.rect_off + j);
    const int4 *rects4 = reinterpret_cast<const int4 *>(cs.rects);
    const int csz = W / 64;
    const int csh = (csz & (csz - 1)) == 0 ? __ffs(csz) - 1 : -1;

    uint32_t g_e1 = 0, g_e2 = 0, kept = 0;
    int t = 0;          // next tile row to set up
    bool have = false;  // a pair is in its grid phase
    int k = 0, ns = 0, sx = 0, sy = 0;
    uint32_t cur_i = 0;
    const int4 *rs = nullptr;
    const uint16_t *ro = nullptr;
    const uint64_t *occl = nullptr;
    int qn = 0;  // queue length (warp-uniform)

    auto full_check = [&](uint2 pr, bool valid) {
        bool keep = false;
        if (valid) {
            int32_t ea[8], ebb[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                ea[q] = __ldg(cs.esig + (size_t)pr.x * 8 + q);
                ebb[q] = __ldg(cs.esig + (size_t)pr.y * 8 + q);
            }
            const uint32_t oa = __ldg(cs.rect_off + pr.x), obb = __ldg(cs.rect_off + pr.y);
            const ClipView A{rects4 + oa, ea, cs.rorder + oa, cs.occ + (size_t)pr.x * 64};
            const ClipView B{rects4 + obb, ebb, cs.rorder + obb, cs.occ + (size_t)pr.y * 64};
            const EdgeOut o = edge_eval(A, B, W, M, tol, true, true);
            if (o.gate == PCL_GATE_E1_MATCH) ++g_e1;
            else if (o.gate == PCL_GATE_E2_BBOX) ++g_e2;
            else { keep = true; ++kept; }
        }
        emit_pair(out, cap, count, keep, pr.x, pr.y);
    };

    for (;;) {
        bool push = false;
        if (!have && t < kTileI) {
            const uint32_t i = i0 + t;
            const int32_t *ea = es_i[t];
            ++t;
            if (jv && i < n && i < j) {
                const int na = ea[ES_N], nb = eb[ES_N];
                if (na == 0 || nb == 0) {
                    if (na == 0 && nb == 0) { push = true; cur_i = i; }  // kept by the full check
                    else ++g_e1;
                } else if (na == nb && !ea[ES_BORDER] && !eb[ES_BORDER] &&
                           (abs((ea[ES_HIX] - ea[ES_LOX]) - (eb[ES_HIX] - eb[ES_LOX])) > 2 * tol ||
                            abs((ea[ES_HIY] - ea[ES_LOY]) - (eb[ES_HIY] - eb[ES_LOY])) > 2 * tol)) {
                    ++g_e2;
                } else {
                    const int s0x = (ea[ES_HASX] && eb[ES_HASX])
                                        ? clampi(((ea[ES_LOX] + ea[ES_HIX]) - (eb[ES_LOX] + eb[ES_HIX])) / 2, -M, M)
                                        : 0;
                    const int s0y = (ea[ES_HASY] && eb[ES_HASY])
                                        ? clampi(((ea[ES_LOY] + ea[ES_HIY]) - (eb[ES_LOY] + eb[ES_HIY])) / 2, -M, M)
                                        : 0;
                    const bool small_is_a = na <= nb;
                    const uint32_t oa = off_i[t - 1];
                    rs = rects4 + (small_is_a ? oa : ob);
                    ro = cs.rorder + (small_is_a ? oa : ob);
                    occl = cs.occ + (size_t)(small_is_a ? j : i) * 64;
                    ns = small_is_a ? na : nb;
                    sx = small_is_a ? -s0x : s0x;
                    sy = small_is_a ? -s0y : s0y;
                    k = 0;
                    cur_i = i;
                    have = true;
                }
            }
        }
        if (have) {
            const int4 q = __ldg(rs + __ldg(ro + k));
            if (!grid_hit(occl, q.x + sx, q.y + sy, q.z + sx, q.w + sy, csz, csh)) {
                ++g_e1;
                have = false;
            } else if (++k == ns) {
                push = true;
                have = false;
            }
        }
        const unsigned pm = __ballot_sync(0xffffffffu, push);
        if (pm) {
            if (push) queue[warp][qn + __popc(pm & ((1u << lane) - 1u))] = make_uint2(cur_i, j);
            qn += __popc(pm);
            __syncwarp();
            if (qn >= 32) {
                qn -= 32;
                const uint2 pr = queue[warp][qn + lane];
                __syncwarp();
                full_check(pr, true);
            }
        }
        if (!__any_sync(0xffffffffu, have || t < kTileI)) break;
    }
    if (qn > 0) {
        const uint2 pr = lane < qn ? queue[warp][lane] : make_uint2(0u, 0u);
        __syncwarp();
        full_check(pr, lane < qn);
    }
    // gate counters: one atomic per warp and counter
    g_e1 = __reduce_add_sync(0xffffffffu, g_e1);
    g_e2 = __reduce_add_sync(0xffffffffu, g_e2);
    kept = __reduce_add_sync(0xffffffffu, kept);
    if (lane == 0 && gates) {
        if (kept) atomicAdd(gates + 0, (unsigned long long)kept);
        if (g_e1) atomicAdd(gates + PCL_GATE_E1_MATCH, (unsigned long long)g_e1);
        if (g_e2) atomicAdd(gates + PCL_GATE_E2_BBOX, (unsigned long long)g_e2);
    }
}

__global__ void __launch_bounds__(256) edge_match_kernel(pcl_params prm, pcl_clipset A, pcl_clipset B,
                                                         const pcl_pair *pairs, uint64_t n,
                                                         const unsigned long long *d_n, pcl_record *out) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d_n && *d_n < n) n = *d_n;
    if (t >= n) return;
    out[t] = edge_record(prm, A, B, pairs[t]);
}

}  // namespace

cudaError_t launch_edge_screen(const pcl_params &prm, const pcl_clipset &cs, pcl_pair *out,
                               uint64_t cap, unsigned long long *count, unsigned long long *gates,
                               cudaStream_t st) {
    const uint32_t n = cs.n_clips;
    if (n < 2) return cudaSuccess;
    dim3 grid((n + kTileI - 1) / kTileI, (n + 255) / 256);
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    edge_screen_kernel<<<grid, 256, 0, st>>>(prm, cs, out, cap, count, gates);
    return cudaGetLastError();
}

cudaError_t launch_edge_match(const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b,
                              const pcl_pair *pairs, uint64_t n, const unsigned long long *d_n, pcl_record *out,
                              cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    edge_match_kernel<<<(unsigned)blocks, 256, 0, st>>>(prm, a, b, pairs, n, d_n, out);
    return cudaGetLastError();
}

}  // namespace pcl

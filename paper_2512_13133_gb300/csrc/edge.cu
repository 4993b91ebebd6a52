// a2 (edge gates) and a7: edge-displacement mode (Sec. 2.2.2) with the
// geometric Min-Max closed form of Sec. 3.2.2 (Eq. 6), integer dbu throughout.
//
// edge_screen_kernel: the self-join screen of all pairs i < j through E2 and
// E1 (tiles of 32 row clips x 256 column clips; the cheap occupancy-grid
// tests of E1 run one pair per lane; the few survivors go to a list whose
// exact correspondence edge_check_kernel checks afterwards, one pair per
// warp).  edge_match_kernel: the Min-Max record of each listed pair, one pair
// per warp (lanes hold the polygons).
#include "edge_dev.cuh"

namespace pcl {

namespace {
using namespace edge_dev;

// the screen's list of pairs for the exact correspondence check (device
// memory; cap 0: every such pair is checked inside the screen)
struct EdgeChecks {
    int4 *list;
    uint64_t cap;
    unsigned long long *count;
};

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

// cell_of with the cell side known to be a power of two (P2) or not
template <bool P2>
__device__ __forceinline__ int cell_at(int v, int csz, int csh) {
    if constexpr (P2) return min(max(v >> csh, 0), 63);
    else return cell_of(v, csz, -1);
}

// grid_hit for a grid that may sit in shared or global memory (generic loads)
template <bool P2>
__device__ __forceinline__ bool grid_hit_any(const uint64_t *occ, int x0, int y0, int x1, int y1, int csz,
                                             int csh) {
    if (x1 <= x0 || y1 <= y0) return true;  // degenerate input: no pruning
    const int cx0 = cell_at<P2>(x0, csz, csh), cx1 = cell_at<P2>(x1 - 1, csz, csh);
    const int cy0 = cell_at<P2>(y0, csz, csh), cy1 = cell_at<P2>(y1 - 1, csz, csh);
    const uint64_t m = (~0ull >> (63 - (cx1 - cx0))) << cx0;
    uint64_t acc = 0ull;  // independent loads, no branch between them
    for (int cy = cy0; cy <= cy1; ++cy) acc |= occ[cy];
    return (acc & m) != 0ull;
}

constexpr int kColsB = 256;  // column clips per block (32 row clips: one per lane)
constexpr int kQueue = 64;   // per-warp queue capacity (grid tests, full checks)
constexpr int kGS = 65;      // stride of a staged grid in shared memory (u64, padded against bank conflicts)

// Warp-cooperative correspondence (Sec. 2.2.2 condition 1) of small list rs
// against large list rl at shift t: every small polygon has exactly one
// partner and no large polygon overlaps two small polygons.  Lanes take the
// large polygons; the result is warp-uniform and equals correspond().
// The small polygons are visited smallest first (ro: the small clip's area
// order); the result does not depend on the order.
__device__ __forceinline__ bool warp_correspond(const int4 *__restrict__ rs, const uint16_t *__restrict__ ro,
                                                int ns, const int4 *__restrict__ rl, int nl, bool small_is_a,
                                                int tx, int ty, int lane) {
    if (ns <= 64 && nl <= 64) {
        // both lists in registers, two polygons per lane at most; the large
        // list is moved by the shift once: A's polygon first and B's moved by
        // t is (s, l + t) with the small clip on side A, else (l, s + t), and
        // both overlap tests equal the plain test of s against l + t or l - t
        const bool v0 = lane < nl, v1 = lane + 32 < nl;
        const int ux = small_is_a ? tx : -tx, uy = small_is_a ? ty : -ty;
        int4 l0 = v0 ? __ldg(rl + lane) : make_int4(0, 0, 0, 0);
        int4 l1 = v1 ? __ldg(rl + lane + 32) : make_int4(0, 0, 0, 0);
        l0 = make_int4(l0.x + ux, l0.y + uy, l0.z + ux, l0.w + uy);
        l1 = make_int4(l1.x + ux, l1.y + uy, l1.z + ux, l1.w + uy);
        // small polygons in ascending area, where a missing partner is most likely
        const int4 sv0 = lane < ns ? __ldg(rs + __ldg(ro + lane)) : make_int4(0, 0, 0, 0);
        const int4 sv1 = lane + 32 < ns ? __ldg(rs + __ldg(ro + lane + 32)) : make_int4(0, 0, 0, 0);
        int c0 = 0, c1 = 0;
        if (nl <= 32) {
            for (int k = 0; k < ns; ++k) {
                const int4 sk = k < 32 ? sv0 : sv1;
                const int src = k & 31;
                const int sx0 = __shfl_sync(0xffffffffu, sk.x, src), sy0 = __shfl_sync(0xffffffffu, sk.y, src);
                const int sx1 = __shfl_sync(0xffffffffu, sk.z, src), sy1 = __shfl_sync(0xffffffffu, sk.w, src);
                const bool h0 = v0 && sx0 < l0.z && l0.x < sx1 && sy0 < l0.w && l0.y < sy1;
                const unsigned b0 = __ballot_sync(0xffffffffu, h0);
                if (b0 == 0u || (b0 & (b0 - 1u))) return false;  // not exactly one partner
                c0 += h0 ? 1 : 0;
            }
        } else {
            for (int k = 0; k < ns; ++k) {
                const int4 sk = k < 32 ? sv0 : sv1;
                const int src = k & 31;
                const int sx0 = __shfl_sync(0xffffffffu, sk.x, src), sy0 = __shfl_sync(0xffffffffu, sk.y, src);
                const int sx1 = __shfl_sync(0xffffffffu, sk.z, src), sy1 = __shfl_sync(0xffffffffu, sk.w, src);
                const bool h0 = v0 && sx0 < l0.z && l0.x < sx1 && sy0 < l0.w && l0.y < sy1;
                const bool h1 = v1 && sx0 < l1.z && l1.x < sx1 && sy0 < l1.w && l1.y < sy1;
                const unsigned b0 = __ballot_sync(0xffffffffu, h0), b1 = __ballot_sync(0xffffffffu, h1);
                if (__popc(b0) + __popc(b1) != 1) return false;
                c0 += h0 ? 1 : 0;
                c1 += h1 ? 1 : 0;
            }
        }
        return !__any_sync(0xffffffffu, c0 > 1 || c1 > 1);
    }
    for (int k = 0; k < ns; ++k) {
        const int4 s = __ldg(rs + k);
        int cnt = 0;
        for (int m0 = 0; m0 < nl && cnt < 2; m0 += 32) {
            const int m = m0 + lane;
            const bool h = m < nl && (small_is_a ? ovl(s, __ldg(rl + m), tx, ty) : ovl(__ldg(rl + m), s, tx, ty));
            cnt += __popc(__ballot_sync(0xffffffffu, h));
        }
        if (cnt != 1) return false;
    }
    for (int m0 = 0; m0 < nl; m0 += 32) {
        const int m = m0 + lane;
        int c = 0;
        if (m < nl) {
            const int4 l = __ldg(rl + m);
            for (int k = 0; k < ns && c < 2; ++k) {
                const int4 s = __ldg(rs + k);
                c += (small_is_a ? ovl(s, l, tx, ty) : ovl(l, s, tx, ty)) ? 1 : 0;
            }
        }
        if (__any_sync(0xffffffffu, c > 1)) return false;
    }
    return true;
}

// Tiles (bx, by) of 32 row clips x kColsB column clips with any pair i < j,
// column block by holding the row tiles bx < min(8 by + 8, nbx) (kColsB = 256
// = 8 row tiles), are numbered column block after column block: tile idx lies
// in column block by with cum(by) <= idx < cum(by + 1), where cum(y) =
// 4 y (y + 1) while 8 y <= nbx and grows by nbx per block after that.
static_assert(kColsB == 256, "eight row tiles per column block");
__host__ __device__ inline uint64_t screen_tiles_before(uint32_t y, uint32_t nbx) {
    const uint64_t y0 = nbx / 8;
    return y <= y0 ? 4ull * y * (y + 1) : 4ull * y0 * (y0 + 1) + (uint64_t)(y - y0) * nbx;
}
__device__ inline void screen_tile(uint32_t idx, uint32_t nbx, uint32_t &bx, uint32_t &by) {
    const uint32_t y0 = nbx / 8;
    const uint64_t c0 = 4ull * y0 * (y0 + 1);
    uint32_t y;
    if (idx < c0) {  // 4 y (y + 1) <= idx: float estimate, corrected exactly
        y = (uint32_t)((sqrtf(1.0f + (float)idx) - 1.0f) * 0.5f);
        while (4ull * (y + 1) * (y + 2) <= idx) ++y;
        while (y > 0 && 4ull * y * (y + 1) > idx) --y;
    } else {
        y = y0 + (uint32_t)((idx - c0) / nbx);
    }
    by = y;
    bx = (uint32_t)(idx - screen_tiles_before(y, nbx));
}

// Self-join screen: block (bx, by) covers row clips i = 32 bx + lane and
// column clips j in [kColsB by, kColsB by + kColsB); warp w takes the columns
// w, w + 8, ...  Pairs with i < j only.  The row clips' signatures live in
// registers and their occupancy grids in shared memory; the column clips'
// signatures are staged per block and each column's grid per warp, so every
// grid read of the first test is a shared-memory load.
//
// Phase 1 takes one column at a time for all 32 rows: empty clips, E2 and the
// pre-alignment of every pair, then the grid test of the smaller clip's
// smallest polygon, which alone rejects about three quarters of random pairs.
// Survivors with more polygons go to a per-warp queue of grid tests (polygons
// in ascending area), which runs only while it holds work for every lane, so
// lanes advance through their pairs independently without idling.  Pairs
// whose polygons all meet occupied cells (a few per thousand) go to a second
// queue, where the whole warp checks one pair at a time with ballots.
// P2: the grid's cell side W/64 is a power of two (cells by shifts).
// CROSS: rows from clip set RS and columns from CS, every (row, column) pair
// (the query x library screen of the serving loop; tiles numbered column
// block after column block, row tile fastest); otherwise RS = CS and the
// pairs i < j of the triangular tile numbering.
template <bool P2, bool CROSS, bool TOPO = false>
__global__ void __launch_bounds__(256, 4) edge_screen_kernel(pcl_params prm, pcl_clipset RS, pcl_clipset CS,
                                                          pcl_pair *out, uint64_t cap,
                                                          unsigned long long *count,
                                                          unsigned long long *gates, uint32_t shard,
                                                          uint32_t n_shards, EdgeChecks chk) {
    const pcl_clipset &RW = CROSS ? RS : CS;  // the row clips (the same set in the self-join)
    const uint32_t nr = RW.n_clips, n = CS.n_clips;  // rows, columns
    uint32_t bx, by;
    if constexpr (CROSS) {
        const uint32_t nbx = (nr + 31) / 32;
        bx = blockIdx.x % nbx;
        by = blockIdx.x / nbx;
    } else {
        screen_tile(blockIdx.x * n_shards + shard, (n + 31) / 32, bx, by);  // shard s of S: tiles s, s + S, ...
    }
    const uint32_t i0 = bx * 32u;
    const uint32_t jblk = by * (uint32_t)kColsB;
    if constexpr (CROSS) {
        if (jblk >= n || i0 >= nr) return;
    } else {
        if (jblk >= n || i0 + 1u >= min(jblk + (uint32_t)kColsB, n)) return;  // no pair i < j in the block
    }
    const int W = prm.window_dbu, M = prm.marker_dbu, tol = prm.edge_tol_dbu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ uint64_t grids[(32 + 8) * kGS];  // row clips' grids, then each warp's current column grid
    __shared__ int4 csig[kColsB][2];  // {n, flags, lox+hix, loy+hiy}, {hix-lox, hiy-loy, rect offset, 0}
    __shared__ int4 cp0[kColsB];      // smallest polygon of each column clip
    __shared__ int4 tq[8][kQueue];    // grid tests: {row | col << 8 | small_is_a << 16, sx, sy, 0}
    __shared__ int4 fq[8][kQueue];    // full checks: {row | col << 8 | small_is_a << 16, s0x, s0y, 0}
    const int4 *rrects = reinterpret_cast<const int4 *>(RW.rects), *crects = reinterpret_cast<const int4 *>(CS.rects);
    // flags: bit 0 has x edges, bit 1 has y edges, bit 2 touches the border
    auto load_sig = [&](const pcl_clipset &cl, uint32_t c, int4 &s0, int4 &s1, int4 &p0) {
        const int4 *e4 = reinterpret_cast<const int4 *>(cl.esig + (size_t)c * 8);
        const int4 lo = __ldg(e4), hi = __ldg(e4 + 1);  // {n, hasx, lox, hix}, {hasy, loy, hiy, border}
        const uint32_t off = __ldg(cl.rect_off + c);
        s0 = make_int4(lo.x, (lo.y ? 1 : 0) | (hi.x ? 2 : 0) | (hi.w ? 4 : 0), lo.z + lo.w, hi.y + hi.z);
        s1 = make_int4(lo.w - lo.z, hi.z - hi.y, (int)off, 0);
        p0 = lo.x > 0 ? __ldg(reinterpret_cast<const int4 *>(cl.rects) + off + __ldg(cl.rorder + off))
                      : make_int4(0, 0, 0, 0);
    };
    for (int c = threadIdx.x; c < kColsB; c += blockDim.x) {
        int4 s0 = make_int4(0, 0, 0, 0), s1 = s0, p0 = s0;
        if (jblk + c < n) load_sig(CS, jblk + c, s0, s1, p0);
        csig[c][0] = s0;
        csig[c][1] = s1;
        cp0[c] = p0;
    }
    for (int w = threadIdx.x; w < 32 * 64; w += blockDim.x)
        grids[(w >> 6) * kGS + (w & 63)] = i0 + (w >> 6) < nr ? __ldg(RW.occ + (size_t)i0 * 64 + w) : 0ull;
    // this lane's row clip
    const uint32_t i = i0 + lane;
    int4 a0 = make_int4(0, 0, 0, 0), a1 = a0, pa = a0;
    if (i < nr) load_sig(RW, i, a0, a1, pa);
    const int na = a0.x;
    __syncthreads();
    const int csz = W / 64;
    const int csh = (csz & (csz - 1)) == 0 ? __ffs(csz) - 1 : -1;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t *gcol = grids + (32 + warp) * kGS;  // this warp's current column grid

    uint32_t g_e1 = 0, g_e2 = 0, g_t0 = 0, kept = 0;
    int qn = 0, fn = 0;  // queue lengths (warp-uniform)
    // grid-test state of this lane
    bool h2 = false;
    int k2 = 0, ns2 = 0, sx2 = 0, sy2 = 0, e2x = 0;
    int off2 = 0;  // rectangle offset of the pair's smaller clip (its set and grid follow from e2x)

    auto run_full = [&]() {  // warp-uniform: check and emit every queued pair
        unsigned ok0 = 0u, ok1 = 0u;
        for (int q = 0; q < fn; ++q) {
            const int4 e = fq[warp][q];
            const int r = e.x & 0xff, c = (e.x >> 8) & 0xff;
            const bool sa = (e.x >> 16) & 1;
            const int offa = __shfl_sync(0xffffffffu, a1.z, r), nar = __shfl_sync(0xffffffffu, na, r);
            const int offb = csig[c][1].z, nbc = csig[c][0].x;
            // the small clip's polygons (and area order) and the large clip's
            const int4 *sr = sa ? rrects + offa : crects + offb, *lr = sa ? crects + offb : rrects + offa;
            const uint16_t *so = sa ? RW.rorder + offa : CS.rorder + offb;
            const bool ok = warp_correspond(sr, so, sa ? nar : nbc, lr, sa ? nbc : nar, sa, e.y, e.z, lane);
            if (ok) {
                if (q < 32) ok0 |= 1u << q;
                else ok1 |= 1u << (q - 32);
            }
        }
        if (lane == 0) {
            const uint32_t nk = (uint32_t)(__popc(ok0) + __popc(ok1));
            kept += nk;
            g_e1 += (uint32_t)fn - nk;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = h * 32 + lane;
            const bool mine = q < fn;
            const int4 e = mine ? fq[warp][q] : make_int4(0, 0, 0, 0);
            const bool keep = mine && (((h ? ok1 : ok0) >> lane) & 1u);
            emit_pair(out, cap, count, keep, i0 + (e.x & 0xff), jblk + ((e.x >> 8) & 0xff));
        }
        __syncwarp();
        fn = 0;
    };
    // tag: row | col << 8 | small_is_a << 16 of the pair.  The pairs go to
    // the check list while it has room, else to this warp's queue.
    auto push_full = [&](bool p, int tag, int s0x, int s0y) {
        const unsigned m = __ballot_sync(0xffffffffu, p);
        if (!m) return;
        bool here = p;
        if (chk.cap) {
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(chk.count, (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            const unsigned long long idx = base + __popc(m & lt);
            if (p && idx < chk.cap) {
                chk.list[idx] = make_int4((int)(i0 + (tag & 0xff)), (int)(jblk + ((tag >> 8) & 0xff)), s0x,
                                          s0y * 2 + ((tag >> 16) & 1));
                here = false;
            }
        }
        const unsigned mh = __ballot_sync(0xffffffffu, here);
        if (here) fq[warp][fn + __popc(mh & lt)] = make_int4(tag, s0x, s0y, 0);
        fn += __popc(mh);
        __syncwarp();
        if (fn >= 32) run_full();  // keeps fn below 32 between pushes
    };
    // one round of the grid-test queue: idle lanes take entries (pushed by any
    // lane of the warp), every lane holding a pair tests its next polygon
    auto step2 = [&]() {
        const unsigned idle = __ballot_sync(0xffffffffu, !h2);
        const int rk = __popc(idle & lt);
        const bool take = !h2 && rk < qn;
        const int4 e = take ? tq[warp][qn - 1 - rk] : make_int4(0, 0, 0, 0);
        const int r = e.x & 0xff;
        const int offa = __shfl_sync(0xffffffffu, a1.z, r), nar = __shfl_sync(0xffffffffu, na, r);
        if (take) {
            const int c = (e.x >> 8) & 0xff;
            const bool sa = (e.x >> 16) & 1;
            const int off = sa ? offa : csig[c][1].z;
            ns2 = sa ? nar : csig[c][0].x;
            off2 = off;
            sx2 = e.y;
            sy2 = e.z;
            e2x = e.x;
            k2 = 1;
            h2 = true;
        }
        qn = qn > __popc(idle) ? qn - __popc(idle) : 0;
        __syncwarp();
        bool done = false;
        if (h2) {
            const bool s2 = (e2x >> 16) & 1;
            const int4 q = __ldg((s2 ? rrects : crects) + off2 + __ldg((s2 ? RW.rorder : CS.rorder) + off2 + k2));
            const uint64_t *g2 = s2 ? CS.occ + (size_t)(jblk + ((e2x >> 8) & 0xff)) * 64 : grids + (e2x & 0xff) * kGS;
            if (!grid_hit_any<P2>(g2, q.x + sx2, q.y + sy2, q.z + sx2, q.w + sy2, csz, csh)) {
                ++g_e1;
                h2 = false;
            } else if (++k2 == ns2) {
                done = true;
                h2 = false;
            }
        }
        const bool sa = (e2x >> 16) & 1;
        push_full(done, e2x, sa ? -sx2 : sx2, sa ? -sy2 : sy2);
    };

    // columns of this warp: c = warp + 8 m; the next column's grid is fetched
    // into registers while the current one is processed
    const uint32_t jlast = min(jblk + (uint32_t)kColsB, n);  // one past the last column
    uint32_t c = warp;
    if constexpr (!CROSS)
        while (c < (uint32_t)kColsB && jblk + c <= i0) c += 8;  // columns with no row below them
    ulonglong2 gnext = make_ulonglong2(0ull, 0ull);
    if (jblk + c < jlast) gnext = __ldg(reinterpret_cast<const ulonglong2 *>(CS.occ + (size_t)(jblk + c) * 64) + lane);
    for (; jblk + c < jlast; c += 8) {
        const uint32_t j = jblk + c;
        __syncwarp();  // the previous column's grid is no longer read
        gcol[2 * lane] = gnext.x;
        gcol[2 * lane + 1] = gnext.y;
        if (j + 8 < jlast) gnext = __ldg(reinterpret_cast<const ulonglong2 *>(CS.occ + (size_t)(j + 8) * 64) + lane);
        __syncwarp();
        const int4 b0 = csig[c][0];
        const int nb = b0.x;
        bool push_t = false, push_f = false, both_empty = false;
        bool sa = false;
        int s0x = 0, s0y = 0;
        if (CROSS ? i < nr : i < j) {
            if (TOPO && topo_class(na) != topo_class(nb)) {  // lossy pre-screen: equal polygon-count classes
                ++g_t0;
            } else if (na == 0 || nb == 0) {
                if (na == 0 && nb == 0) both_empty = true;
                else ++g_e1;
            } else {
                const int4 b1 = csig[c][1];
                if (na == nb && !((a0.y | b0.y) & 4) &&
                    (abs(a1.x - b1.x) > 2 * tol || abs(a1.y - b1.y) > 2 * tol)) {
                    ++g_e2;
                } else {
                    s0x = (a0.y & b0.y & 1) ? clampi((a0.z - b0.z) / 2, -M, M) : 0;
                    s0y = (a0.y & b0.y & 2) ? clampi((a0.w - b0.w) / 2, -M, M) : 0;
                    sa = na <= nb;
                    // the smaller clip's smallest polygon in the other clip's frame
                    const int4 q = sa ? pa : cp0[c];
                    const int sx = sa ? -s0x : s0x, sy = sa ? -s0y : s0y;
                    const uint64_t *grid = sa ? gcol : grids + lane * kGS;
                    if (!grid_hit_any<P2>(grid, q.x + sx, q.y + sy, q.z + sx, q.w + sy, csz, csh)) ++g_e1;
                    else if ((sa ? na : nb) == 1) push_f = true;
                    else push_t = true;
                }
            }
        }
        const int tag = lane | (int)(c << 8) | (sa ? 1 << 16 : 0);
        const unsigned mt = __ballot_sync(0xffffffffu, push_t);
        if (push_t) tq[warp][qn + __popc(mt & lt)] = make_int4(tag, sa ? -s0x : s0x, sa ? -s0y : s0y, 0);
        qn += __popc(mt);
        push_full(push_f, tag, s0x, s0y);
        if (__any_sync(0xffffffffu, both_empty)) {  // similar by definition
            kept += both_empty ? 1u : 0u;
            emit_pair(out, cap, count, both_empty, i, j);
        }
        while (qn + __popc(__ballot_sync(0xffffffffu, h2)) >= 32) step2();
    }
    while (qn > 0 || __any_sync(0xffffffffu, h2)) step2();
    if (fn > 0) run_full();
    // gate counters: one atomic per warp and counter
    g_e1 = __reduce_add_sync(0xffffffffu, g_e1);
    g_e2 = __reduce_add_sync(0xffffffffu, g_e2);
    g_t0 = __reduce_add_sync(0xffffffffu, g_t0);
    kept = __reduce_add_sync(0xffffffffu, kept);
    if (lane == 0 && gates) {
        if (kept) atomicAdd(gates + 0, (unsigned long long)kept);
        if (g_e1) atomicAdd(gates + PCL_GATE_E1_MATCH, (unsigned long long)g_e1);
        if (g_e2) atomicAdd(gates + PCL_GATE_E2_BBOX, (unsigned long long)g_e2);
        if (g_t0) atomicAdd(gates + PCL_GATE_T0_TOPO, (unsigned long long)g_t0);
    }
}

// one pair per warp (warp_edge_record), lane 0 writes the record; warps stride
// the list (the grid is sized to the GPU, not to the list, whose length may
// only be known on the device)
__global__ void __launch_bounds__(256) edge_match_kernel(pcl_params prm, pcl_clipset A, pcl_clipset B,
                                                         const pcl_pair *pairs, uint64_t n,
                                                         const unsigned long long *d_n, pcl_record *out) {
    if (d_n && *d_n < n) n = *d_n;
    const int lane = threadIdx.x & 31;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t t = w0; t < n; t += nw) {  // warp-uniform
        const pcl_record r = warp_edge_record(prm, A, B, pairs[t], lane);
        if (lane == 0) out[t] = r;
    }
}

// The exact correspondence (Sec. 2.2.2 condition 1) of the pairs the screen
// listed: entry {i, j, tx, 2 ty + small_is_a} (i a row clip of RW, j a
// column clip of CS, (tx, ty) the shift as the screen's queue holds it).
// Warps take 32 consecutive entries at a time (grid-stride) and emit the
// pairs that pass with one atomic per batch; counters go to gates (E1 for
// the pairs that fail, [0] for the others).
template <bool CROSS>
__global__ void __launch_bounds__(256) edge_check_kernel(pcl_clipset RS, pcl_clipset CS, EdgeChecks chk,
                                                         pcl_pair *out, uint64_t cap, unsigned long long *count,
                                                         unsigned long long *gates) {
    const pcl_clipset &RW = CROSS ? RS : CS;
    const int4 *rrects = reinterpret_cast<const int4 *>(RW.rects), *crects = reinterpret_cast<const int4 *>(CS.rects);
    unsigned long long n = *chk.count;
    if (n > chk.cap) n = chk.cap;
    const int lane = threadIdx.x & 31;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long kept = 0, e1 = 0;
    for (uint64_t t0 = w0 * 32; t0 < n; t0 += nw * 32) {  // warp-uniform
        const int m = (int)(n - t0 < 32 ? n - t0 : 32);
        const int4 mine = lane < m ? chk.list[t0 + lane] : make_int4(0, 0, 0, 0);
        unsigned ok = 0u;
        for (int q = 0; q < m; ++q) {
            const uint32_t i = (uint32_t)__shfl_sync(0xffffffffu, mine.x, q);
            const uint32_t j = (uint32_t)__shfl_sync(0xffffffffu, mine.y, q);
            const int tx = __shfl_sync(0xffffffffu, mine.z, q), tw = __shfl_sync(0xffffffffu, mine.w, q);
            const bool sa = tw & 1;
            const int ty = tw >> 1;
            const int offa = (int)__ldg(RW.rect_off + i), na = __ldg(RW.esig + (size_t)i * 8);
            const int offb = (int)__ldg(CS.rect_off + j), nb = __ldg(CS.esig + (size_t)j * 8);
            const int4 *sr = sa ? rrects + offa : crects + offb, *lr = sa ? crects + offb : rrects + offa;
            const uint16_t *so = sa ? RW.rorder + offa : CS.rorder + offb;
            if (warp_correspond(sr, so, sa ? na : nb, lr, sa ? nb : na, sa, tx, ty, lane)) ok |= 1u << q;
        }
        const bool keep = (ok >> lane) & 1u;
        emit_pair(out, cap, count, keep, (uint32_t)mine.x, (uint32_t)mine.y);
        kept += (unsigned long long)__popc(ok);
        e1 += (unsigned long long)(m - __popc(ok));
    }
    if (lane == 0 && gates) {
        if (kept) atomicAdd(gates + 0, kept);
        if (e1) atomicAdd(gates + PCL_GATE_E1_MATCH, e1);
    }
}

}  // namespace

// bytes of the check list for a screen of `pairs` pairs: a count, then
// entries for one pair in 256 (at least 65,536 and at most 2^24 entries);
// pairs past the list are checked inside the screen
uint64_t edge_checks_capacity(uint64_t pairs) {
    const uint64_t c = pairs / 256;
    return c < (1ull << 16) ? (1ull << 16) : c > (1ull << 24) ? (1ull << 24) : c;
}
size_t edge_checks_workspace(uint64_t pairs) { return 16 + 16 * (size_t)edge_checks_capacity(pairs); }

// the check list of a screen of `pairs` pairs at the start of the workspace
// (none if the workspace is missing or smaller than edge_checks_workspace)
static EdgeChecks edge_checks(void *ws, size_t ws_bytes, uint64_t pairs) {
    EdgeChecks c{nullptr, 0, nullptr};
    if (ws && ws_bytes >= edge_checks_workspace(pairs)) {
        c.count = static_cast<unsigned long long *>(ws);
        c.list = reinterpret_cast<int4 *>(static_cast<char *>(ws) + 16);
        c.cap = edge_checks_capacity(pairs);
    }
    return c;
}

// shard s of S (several GPUs sharing one self-join) screens the tiles
// s, s + S, s + 2S, ... of the 1-D tile numbering: a partition by clip index
uint64_t edge_screen_tiles(uint32_t n) {
    if (n < 2) return 0;
    return screen_tiles_before((n + kColsB - 1) / kColsB, (n + 31) / 32);
}

cudaError_t launch_edge_screen(const pcl_params &prm, const pcl_clipset &cs, pcl_pair *out,
                               uint64_t cap, unsigned long long *count, unsigned long long *gates,
                               cudaStream_t st, uint32_t shard, uint32_t n_shards, void *ws, size_t ws_bytes,
                               int num_sms) {
    if (n_shards == 0 || shard >= n_shards) return cudaErrorInvalidValue;
    // only the tiles that hold pairs i < j (about half of them)
    const uint64_t tiles = edge_screen_tiles(cs.n_clips);
    if (tiles > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    if (tiles <= shard) return cudaSuccess;
    const unsigned grid = (unsigned)((tiles - shard + n_shards - 1) / n_shards);
    const int csz = prm.window_dbu / 64;
    const bool p2 = (csz & (csz - 1)) == 0, topo = (prm.flags & PCL_P_TOPO_HASH) != 0;
    const uint64_t n = cs.n_clips;
    const EdgeChecks chk = edge_checks(ws, ws_bytes, n * (n - (n > 0)) / 2 / n_shards);
    if (chk.cap) {
        const cudaError_t e = cudaMemsetAsync(chk.count, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    if (topo && p2)
        edge_screen_kernel<true, false, true><<<grid, 256, 0, st>>>(prm, cs, cs, out, cap, count, gates, shard,
                                                                    n_shards, chk);
    else if (topo)
        edge_screen_kernel<false, false, true><<<grid, 256, 0, st>>>(prm, cs, cs, out, cap, count, gates, shard,
                                                                     n_shards, chk);
    else if (p2)
        edge_screen_kernel<true, false><<<grid, 256, 0, st>>>(prm, cs, cs, out, cap, count, gates, shard, n_shards,
                                                              chk);
    else
        edge_screen_kernel<false, false><<<grid, 256, 0, st>>>(prm, cs, cs, out, cap, count, gates, shard,
                                                               n_shards, chk);
    if (chk.cap) edge_check_kernel<false><<<num_sms * 8, 256, 0, st>>>(cs, cs, chk, out, cap, count, gates);
    return cudaGetLastError();
}

// query x library screen (serving): every (q, l) pair through E2 and E1, the
// survivors written as (q, l); tiles of 32 queries x 256 library clips.  With
// no workspace (ws NULL: the server's slots) every pair is checked inside the
// screen.
cudaError_t launch_edge_screen_cross(const pcl_params &prm, const pcl_clipset &q, const pcl_clipset &lib,
                                     pcl_pair *out, uint64_t cap, unsigned long long *count,
                                     unsigned long long *gates, cudaStream_t st, void *ws, size_t ws_bytes,
                                     int num_sms) {
    if (q.n_clips == 0 || lib.n_clips == 0) return cudaSuccess;
    const uint64_t tiles = (uint64_t)((q.n_clips + 31) / 32) * ((lib.n_clips + kColsB - 1) / kColsB);
    if (tiles > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    const int csz = prm.window_dbu / 64;
    const EdgeChecks chk = edge_checks(ws, ws_bytes, (uint64_t)q.n_clips * lib.n_clips);
    if (chk.cap) {
        const cudaError_t e = cudaMemsetAsync(chk.count, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    if ((csz & (csz - 1)) == 0)
        edge_screen_kernel<true, true><<<(unsigned)tiles, 256, 0, st>>>(prm, q, lib, out, cap, count, gates, 0, 1,
                                                                        chk);
    else
        edge_screen_kernel<false, true><<<(unsigned)tiles, 256, 0, st>>>(prm, q, lib, out, cap, count, gates, 0, 1,
                                                                         chk);
    if (chk.cap) edge_check_kernel<true><<<num_sms * 8, 256, 0, st>>>(q, lib, chk, out, cap, count, gates);
    return cudaGetLastError();
}

cudaError_t launch_edge_match(const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b,
                              const pcl_pair *pairs, uint64_t n, const unsigned long long *d_n, pcl_record *out,
                              int num_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint64_t need = (n + 7) / 8;  // 8 warps per block, one pair per warp
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_match_kernel, 256, 0);
    if (e != cudaSuccess) return e;
    const uint64_t cap = (uint64_t)num_sms * (uint64_t)(per_sm > 0 ? per_sm : 1);  // resident blocks
    edge_match_kernel<<<(unsigned)(need < cap ? need : cap), 256, 0, st>>>(prm, a, b, pairs, n, d_n, out);
    return cudaGetLastError();
}

}  // namespace pcl

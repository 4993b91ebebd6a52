// Device code of the edge-displacement mode (Sec. 2.2.2; geometric Min-Max of
// Sec. 3.2.2, Eq. 6), shared by the edge kernels and the mixed-batch kernel.
#pragma once

#include <climits>

#include "common.cuh"

namespace pcl {
namespace edge_dev {


struct EdgeOut {
    int gate;      // PCL_GATE_* (0: passed the gates)
    int tx, ty;    // translation applied to B (dbu)
    int E;         // max(E_x, E_y)
    bool verified; // correspondence unchanged at T
    bool pass;
    bool empty;
};

__device__ __forceinline__ bool ovl(const int4 a, const int4 b, int tx, int ty) {
    return a.x < b.z + tx && b.x + tx < a.z && a.y < b.w + ty && b.y + ty < a.w;
}

// partner of small-side polygon k at shift (tx, ty): index in the large list,
// -1 if none, -2 if more than one.
__device__ __forceinline__ int partner(const int4 *__restrict__ rs, const int4 *__restrict__ rl, int nl,
                                       bool small_is_a, int k, int tx, int ty) {
    const int4 s = __ldg(rs + k);
    int who = -1;
    for (int m = 0; m < nl; ++m) {
        const int4 l = __ldg(rl + m);
        const bool hit = small_is_a ? ovl(s, l, tx, ty) : ovl(l, s, tx, ty);
        if (hit) {
            if (who >= 0) return -2;
            who = m;
        }
    }
    return who;
}

// correspondence (Sec. 2.2.2 condition 1) at shift t, with injectivity
__device__ inline bool correspond(const int4 *rs, int ns, const int4 *rl, int nl, bool small_is_a, int tx,
                           int ty) {
    for (int k = 0; k < ns; ++k)
        if (partner(rs, rl, nl, small_is_a, k, tx, ty) < 0) return false;
    // every small polygon has exactly one partner; the map is injective iff no
    // large polygon overlaps two small polygons
    for (int m = 0; m < nl; ++m) {
        const int4 l = __ldg(rl + m);
        int cnt = 0;
        for (int k = 0; k < ns && cnt < 2; ++k) {
            const int4 s = __ldg(rs + k);
            cnt += (small_is_a ? ovl(s, l, tx, ty) : ovl(l, s, tx, ty)) ? 1 : 0;
        }
        if (cnt > 1) return false;
    }
    return true;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// grid cell of coordinate v: floor(v / csz) clamped to the 64 cells; csh >= 0
// is log2(csz) when csz is a power of two (arithmetic shift = floor division)
__device__ __forceinline__ int cell_of(int v, int csz, int csh) {
    const int q = csh >= 0 ? (v >> csh) : (v >= 0 ? v / csz : -((-v + csz - 1) / csz));
    return min(max(q, 0), 63);
}

// Does rectangle [x0,x1) x [y0,y1) (in the frame of the clip owning occ) meet
// a marked cell of its occupancy grid?  Positive-area overlap with any of the
// clip's rectangles implies a shared marked cell, so "false" proves that the
// rectangle overlaps none of them.
__device__ __forceinline__ bool grid_hit(const uint64_t *__restrict__ occ, int x0, int y0, int x1, int y1,
                                         int csz, int csh) {
    if (x1 <= x0 || y1 <= y0) return true;  // degenerate input: no pruning
    const int cx0 = cell_of(x0, csz, csh), cx1 = cell_of(x1 - 1, csz, csh);
    const int cy0 = cell_of(y0, csz, csh), cy1 = cell_of(y1 - 1, csz, csh);
    const uint64_t m = (~0ull >> (63 - (cx1 - cx0))) << cx0;
    for (int cy = cy0; cy <= cy1; ++cy)
        if (__ldg(occ + cy) & m) return true;
    return false;
}

struct ClipView {
    const int4 *r;       // rectangles
    const int32_t *e;    // edge signature
    const uint16_t *ro;  // rectangles by ascending area
    const uint64_t *occ; // occupancy grid
};

// Gates E2 and E1 and, unless screen_only, the full Min-Max procedure.
__device__ inline EdgeOut edge_eval(const ClipView &A, const ClipView &B, int W, int M, int tol, bool gates,
                             bool screen_only) {
    const int4 *ra = A.r, *rb = B.r;
    const int32_t *ea = A.e, *eb = B.e;
    EdgeOut o{};
    const int na = ea[ES_N], nb = eb[ES_N];
    if (na == 0 && nb == 0) {
        o.empty = true;
        o.pass = true;
        o.verified = true;
        return o;
    }
    if (na == 0 || nb == 0) {
        o.gate = PCL_GATE_E1_MATCH;
        return o;
    }
    const int lxa = ea[ES_LOX], uxa = ea[ES_HIX], lya = ea[ES_LOY], uya = ea[ES_HIY];
    const int lxb = eb[ES_LOX], uxb = eb[ES_HIX], lyb = eb[ES_LOY], uyb = eb[ES_HIY];
    if (gates && na == nb && !ea[ES_BORDER] && !eb[ES_BORDER]) {
        // E2: with a bijection and no border edges every displacement lies in
        // [T - tol, T + tol], so the bbox sizes differ by at most 2 tol
        if (abs((uxa - lxa) - (uxb - lxb)) > 2 * tol || abs((uya - lya) - (uyb - lyb)) > 2 * tol) {
            o.gate = PCL_GATE_E2_BBOX;
            return o;
        }
    }
    // pre-alignment: difference of the bbox centres (doubled centres halved,
    // truncated toward zero), clamped to the marker window
    const int s0x = (ea[ES_HASX] && eb[ES_HASX]) ? clampi(((lxa + uxa) - (lxb + uxb)) / 2, -M, M) : 0;
    const int s0y = (ea[ES_HASY] && eb[ES_HASY]) ? clampi(((lya + uya) - (lyb + uyb)) / 2, -M, M) : 0;
    const bool small_is_a = na <= nb;
    const int4 *rs = small_is_a ? ra : rb;
    const int4 *rl = small_is_a ? rb : ra;
    const int ns = small_is_a ? na : nb, nl = small_is_a ? nb : na;
    o.tx = s0x;
    o.ty = s0y;
    // occupancy pre-check of E1, smallest polygons first (most likely to meet
    // nothing): a small polygon over empty cells of the other clip has no partner
    {
        const uint16_t *ro = small_is_a ? A.ro : B.ro;
        const uint64_t *occ_l = small_is_a ? B.occ : A.occ;
        const int csz = W / 64;
        const int csh = (csz & (csz - 1)) == 0 ? __ffs(csz) - 1 : -1;
        // small polygon in the large clip's frame: a - t (small is A) or b + t
        const int sx = small_is_a ? -s0x : s0x, sy = small_is_a ? -s0y : s0y;
        for (int k = 0; k < ns; ++k) {
            const int4 q = __ldg(rs + __ldg(ro + k));
            if (!grid_hit(occ_l, q.x + sx, q.y + sy, q.z + sx, q.w + sy, csz, csh)) {
                o.gate = PCL_GATE_E1_MATCH;
                return o;
            }
        }
    }
    if (!correspond(rs, ns, rl, nl, small_is_a, s0x, s0y)) {
        o.gate = PCL_GATE_E1_MATCH;
        return o;
    }
    if (screen_only) return o;
    // displacements d = e_A - e_B of matched edges off the window border
    int cx = 0, cy = 0, dminx = INT_MAX, dmaxx = INT_MIN, dminy = INT_MAX, dmaxy = INT_MIN;
    for (int k = 0; k < ns; ++k) {
        const int m = partner(rs, rl, nl, small_is_a, k, s0x, s0y);
        const int4 pa = __ldg(small_is_a ? ra + k : ra + m);
        const int4 pb = __ldg(small_is_a ? rb + m : rb + k);
        if (pa.x != 0 && pb.x != 0) { const int d = pa.x - pb.x; dminx = min(dminx, d); dmaxx = max(dmaxx, d); cx = 1; }
        if (pa.z != W && pb.z != W) { const int d = pa.z - pb.z; dminx = min(dminx, d); dmaxx = max(dmaxx, d); cx = 1; }
        if (pa.y != 0 && pb.y != 0) { const int d = pa.y - pb.y; dminy = min(dminy, d); dmaxy = max(dmaxy, d); cy = 1; }
        if (pa.w != W && pb.w != W) { const int d = pa.w - pb.w; dminy = min(dminy, d); dmaxy = max(dmaxy, d); cy = 1; }
    }
    // Eq. 6 per separable axis: midpoint (trunc toward zero), clamped
    const int Tx = cx ? clampi((dminx + dmaxx) / 2, -M, M) : s0x;
    const int Ty = cy ? clampi((dminy + dmaxy) / 2, -M, M) : s0y;
    const int Ex = cx ? max(Tx - dminx, dmaxx - Tx) : 0;
    const int Ey = cy ? max(Ty - dminy, dmaxy - Ty) : 0;
    // the correspondence must hold at T with the same partners
    bool ok = true;
    for (int k = 0; k < ns && ok; ++k) {
        const int m0 = partner(rs, rl, nl, small_is_a, k, s0x, s0y);
        const int m1 = partner(rs, rl, nl, small_is_a, k, Tx, Ty);
        ok = (m0 == m1);
    }
    o.tx = Tx;
    o.ty = Ty;
    o.E = max(Ex, Ey);
    o.verified = ok;
    o.pass = ok && Ex <= tol && Ey <= tol;
    return o;
}


// edge_eval for one pair per warp (the result is the same, in every lane):
// lanes hold the polygons of both clips (at most 64 per clip, otherwise every
// lane runs edge_eval); the small clip's polygons are broadcast one at a time
// and ballots over the large clip's give each one's partner.  Partners,
// displacement extremes and the re-check at T do not depend on the order in
// which the small polygons are visited.
__device__ inline EdgeOut warp_edge_eval(const ClipView &A, const ClipView &B, int W, int M, int tol, bool gates,
                                         int lane) {
    const int32_t *ea = A.e, *eb = B.e;
    const int na = ea[ES_N], nb = eb[ES_N];
    if (na > 64 || nb > 64) return edge_eval(A, B, W, M, tol, gates, false);
    EdgeOut o{};
    if (na == 0 && nb == 0) {
        o.empty = true;
        o.pass = true;
        o.verified = true;
        return o;
    }
    if (na == 0 || nb == 0) {
        o.gate = PCL_GATE_E1_MATCH;
        return o;
    }
    const int lxa = ea[ES_LOX], uxa = ea[ES_HIX], lya = ea[ES_LOY], uya = ea[ES_HIY];
    const int lxb = eb[ES_LOX], uxb = eb[ES_HIX], lyb = eb[ES_LOY], uyb = eb[ES_HIY];
    if (gates && na == nb && !ea[ES_BORDER] && !eb[ES_BORDER]) {
        if (abs((uxa - lxa) - (uxb - lxb)) > 2 * tol || abs((uya - lya) - (uyb - lyb)) > 2 * tol) {
            o.gate = PCL_GATE_E2_BBOX;
            return o;
        }
    }
    const int s0x = (ea[ES_HASX] && eb[ES_HASX]) ? clampi(((lxa + uxa) - (lxb + uxb)) / 2, -M, M) : 0;
    const int s0y = (ea[ES_HASY] && eb[ES_HASY]) ? clampi(((lya + uya) - (lyb + uyb)) / 2, -M, M) : 0;
    const bool small_is_a = na <= nb;
    const int4 *rs = small_is_a ? A.r : B.r;
    const int4 *rl = small_is_a ? B.r : A.r;
    const int ns = small_is_a ? na : nb, nl = small_is_a ? nb : na;
    o.tx = s0x;
    o.ty = s0y;
    const unsigned full = 0xffffffffu;
    // the small polygons, lane k holding k and k + 32
    const bool w0 = lane < ns, w1 = lane + 32 < ns;
    const int4 sv0 = w0 ? __ldg(rs + lane) : make_int4(0, 0, 0, 0);
    const int4 sv1 = w1 ? __ldg(rs + lane + 32) : make_int4(0, 0, 0, 0);
    if (gates) {  // occupancy pre-check of E1
        const uint64_t *occ_l = small_is_a ? B.occ : A.occ;
        const int csz = W / 64;
        const int csh = (csz & (csz - 1)) == 0 ? __ffs(csz) - 1 : -1;
        const int sx = small_is_a ? -s0x : s0x, sy = small_is_a ? -s0y : s0y;
        bool miss = w0 && !grid_hit(occ_l, sv0.x + sx, sv0.y + sy, sv0.z + sx, sv0.w + sy, csz, csh);
        miss = miss || (w1 && !grid_hit(occ_l, sv1.x + sx, sv1.y + sy, sv1.z + sx, sv1.w + sy, csz, csh));
        if (__any_sync(full, miss)) {
            o.gate = PCL_GATE_E1_MATCH;
            return o;
        }
    }
    // the large polygons, lane m holding m and m + 32; an overlap of A's
    // polygon with B's moved by t is the plain overlap of the small polygon
    // with the large one moved by u = t (small on side A) or -t
    const bool v0 = lane < nl, v1 = lane + 32 < nl;
    const int4 lv0 = v0 ? __ldg(rl + lane) : make_int4(0, 0, 0, 0);
    const int4 lv1 = v1 ? __ldg(rl + lane + 32) : make_int4(0, 0, 0, 0);
    // partner of small polygon k with the large list moved by (ux, uy): its
    // index, -1 if none, -2 if several
    auto partner_at = [&](int k, int ux, int uy) {
        const int4 sk = k < 32 ? sv0 : sv1;
        const int src = k & 31;
        const int x0 = __shfl_sync(full, sk.x, src), y0 = __shfl_sync(full, sk.y, src);
        const int x1 = __shfl_sync(full, sk.z, src), y1 = __shfl_sync(full, sk.w, src);
        const bool h0 = v0 && x0 < lv0.z + ux && lv0.x + ux < x1 && y0 < lv0.w + uy && lv0.y + uy < y1;
        const bool h1 = v1 && x0 < lv1.z + ux && lv1.x + ux < x1 && y0 < lv1.w + uy && lv1.y + uy < y1;
        const unsigned b0 = __ballot_sync(full, h0), b1 = __ballot_sync(full, h1);
        const int c = __popc(b0) + __popc(b1);
        return c == 0 ? -1 : (c > 1 ? -2 : (b0 ? __ffs(b0) - 1 : 32 + __ffs(b1) - 1));
    };
    // correspondence at s0 (Sec. 2.2.2 condition 1), with injectivity
    const int u0x = small_is_a ? s0x : -s0x, u0y = small_is_a ? s0y : -s0y;
    int mk0 = -1, mk1 = -1;  // partners of this lane's small polygons
    for (int k = 0; k < ns; ++k) {
        const int m = partner_at(k, u0x, u0y);
        if (m < 0) {
            o.gate = PCL_GATE_E1_MATCH;
            return o;
        }
        if (lane == (k & 31)) {
            if (k < 32) mk0 = m;
            else mk1 = m;
        }
    }
    // injectivity: no large polygon is the partner of two small polygons
    {
        int cnt0 = 0, cnt1 = 0;  // small polygons partnered with large polygons lane, lane + 32
        for (int k = 0; k < ns; ++k) {
            const int m = __shfl_sync(full, k < 32 ? mk0 : mk1, k & 31);
            cnt0 += (m == lane) ? 1 : 0;
            cnt1 += (m == lane + 32) ? 1 : 0;
        }
        if (__any_sync(full, cnt0 > 1 || cnt1 > 1)) {
            o.gate = PCL_GATE_E1_MATCH;
            return o;
        }
    }
    // displacements d = e_A - e_B of matched edges off the window border
    int cx = 0, cy = 0, dminx = INT_MAX, dmaxx = INT_MIN, dminy = INT_MAX, dmaxy = INT_MIN;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (h ? w1 : w0) {
            const int4 sp = h ? sv1 : sv0;
            const int4 lp = __ldg(rl + (h ? mk1 : mk0));
            const int4 pa = small_is_a ? sp : lp, pb = small_is_a ? lp : sp;
            if (pa.x != 0 && pb.x != 0) { const int d = pa.x - pb.x; dminx = min(dminx, d); dmaxx = max(dmaxx, d); cx = 1; }
            if (pa.z != W && pb.z != W) { const int d = pa.z - pb.z; dminx = min(dminx, d); dmaxx = max(dmaxx, d); cx = 1; }
            if (pa.y != 0 && pb.y != 0) { const int d = pa.y - pb.y; dminy = min(dminy, d); dmaxy = max(dmaxy, d); cy = 1; }
            if (pa.w != W && pb.w != W) { const int d = pa.w - pb.w; dminy = min(dminy, d); dmaxy = max(dmaxy, d); cy = 1; }
        }
    }
    cx = __reduce_or_sync(full, (unsigned)cx);
    cy = __reduce_or_sync(full, (unsigned)cy);
    dminx = __reduce_min_sync(full, dminx);
    dmaxx = __reduce_max_sync(full, dmaxx);
    dminy = __reduce_min_sync(full, dminy);
    dmaxy = __reduce_max_sync(full, dmaxy);
    // Eq. 6 per separable axis: midpoint (trunc toward zero), clamped
    const int Tx = cx ? clampi((dminx + dmaxx) / 2, -M, M) : s0x;
    const int Ty = cy ? clampi((dminy + dmaxy) / 2, -M, M) : s0y;
    const int Ex = cx ? max(Tx - dminx, dmaxx - Tx) : 0;
    const int Ey = cy ? max(Ty - dminy, dmaxy - Ty) : 0;
    // the correspondence must hold at T with the same partners
    const int uTx = small_is_a ? Tx : -Tx, uTy = small_is_a ? Ty : -Ty;
    bool ok = true;
    for (int k = 0; k < ns && ok; ++k) {
        const int m0 = __shfl_sync(full, k < 32 ? mk0 : mk1, k & 31);
        ok = partner_at(k, uTx, uTy) == m0;
    }
    o.tx = Tx;
    o.ty = Ty;
    o.E = max(Ex, Ey);
    o.verified = ok;
    o.pass = ok && Ex <= tol && Ey <= tol;
    return o;
}

// The gates of the edge-mode record for one pair in one thread (empty clips,
// E2, the occupancy pre-check of E1): true when the pair passes them and needs
// the rest of the procedure (then *rec is not set); otherwise *rec is the
// record warp_edge_record would write.
__device__ inline bool edge_gate_record(const pcl_params &prm, const pcl_clipset &A, const pcl_clipset &B,
                                        pcl_pair pr, pcl_record *rec) {
    pcl_record r{};
    r.a = pr.a;
    r.b = pr.b;
    r.mode = PCL_MODE_EDGE;
    if (pr.a >= A.n_clips || pr.b >= B.n_clips) {
        r.flags = PCL_GATE_BAD_INDEX;
        *rec = r;
        return false;
    }
    const int4 *e4a = reinterpret_cast<const int4 *>(A.esig + (size_t)pr.a * 8);
    const int4 *e4b = reinterpret_cast<const int4 *>(B.esig + (size_t)pr.b * 8);
    const int4 alo = __ldg(e4a), ahi = __ldg(e4a + 1), blo = __ldg(e4b), bhi = __ldg(e4b + 1);
    // {n, hasx, lox, hix}, {hasy, loy, hiy, border}
    const int na = alo.x, nb = blo.x;
    if (na == 0 && nb == 0) {
        r.flags = PCL_F_EMPTY;
        r.pass = 1;
        *rec = r;
        return false;
    }
    if (na == 0 || nb == 0) {
        r.flags = PCL_GATE_E1_MATCH;
        *rec = r;
        return false;
    }
    if (prm.flags & PCL_P_NO_GATES) return true;
    const int W = prm.window_dbu, M = prm.marker_dbu, tol = prm.edge_tol_dbu;
    if (na == nb && !ahi.w && !bhi.w &&
        (abs((alo.w - alo.z) - (blo.w - blo.z)) > 2 * tol || abs((ahi.z - ahi.y) - (bhi.z - bhi.y)) > 2 * tol)) {
        r.flags = PCL_GATE_E2_BBOX;
        *rec = r;
        return false;
    }
    const int s0x = (alo.y && blo.y) ? clampi(((alo.z + alo.w) - (blo.z + blo.w)) / 2, -M, M) : 0;
    const int s0y = (ahi.x && bhi.x) ? clampi(((ahi.y + ahi.z) - (bhi.y + bhi.z)) / 2, -M, M) : 0;
    const bool small_is_a = na <= nb;
    const uint32_t oa = __ldg(A.rect_off + pr.a), ob = __ldg(B.rect_off + pr.b);
    const int4 *rs = reinterpret_cast<const int4 *>(small_is_a ? A.rects : B.rects) + (small_is_a ? oa : ob);
    const uint16_t *ro = (small_is_a ? A.rorder : B.rorder) + (small_is_a ? oa : ob);
    const uint64_t *occ_l = small_is_a ? B.occ + (size_t)pr.b * 64 : A.occ + (size_t)pr.a * 64;
    const int ns = small_is_a ? na : nb;
    const int csz = W / 64;
    const int csh = (csz & (csz - 1)) == 0 ? __ffs(csz) - 1 : -1;
    const int sx = small_is_a ? -s0x : s0x, sy = small_is_a ? -s0y : s0y;
    for (int k = 0; k < ns; ++k) {
        const int4 q = __ldg(rs + __ldg(ro + k));
        if (!grid_hit(occ_l, q.x + sx, q.y + sy, q.z + sx, q.w + sy, csz, csh)) {
            r.flags = PCL_GATE_E1_MATCH;
            r.dx_dbu = s0x;
            r.dy_dbu = s0y;
            *rec = r;
            return false;
        }
    }
    return true;
}

// One edge-mode record for pair pr (bounds-checked), computed by a whole warp
// (every lane gets the record)
__device__ __forceinline__ pcl_record warp_edge_record(const pcl_params &prm, const pcl_clipset &A,
                                                       const pcl_clipset &B, pcl_pair pr, int lane) {
    pcl_record r{};
    r.a = pr.a;
    r.b = pr.b;
    r.mode = PCL_MODE_EDGE;
    if (pr.a >= A.n_clips || pr.b >= B.n_clips) {
        r.flags = PCL_GATE_BAD_INDEX;
        return r;
    }
    int32_t ea[8], eb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        ea[k] = __ldg(A.esig + (size_t)pr.a * 8 + k);
        eb[k] = __ldg(B.esig + (size_t)pr.b * 8 + k);
    }
    const uint32_t oa = __ldg(A.rect_off + pr.a), ob = __ldg(B.rect_off + pr.b);
    const ClipView va{reinterpret_cast<const int4 *>(A.rects) + oa, ea, A.rorder + oa, A.occ + (size_t)pr.a * 64};
    const ClipView vb{reinterpret_cast<const int4 *>(B.rects) + ob, eb, B.rorder + ob, B.occ + (size_t)pr.b * 64};
    const bool gates = !(prm.flags & PCL_P_NO_GATES);
    const EdgeOut o = warp_edge_eval(va, vb, prm.window_dbu, prm.marker_dbu, prm.edge_tol_dbu, gates, lane);
    r.dx_dbu = o.tx;
    r.dy_dbu = o.ty;
    if (o.empty) {
        r.flags = PCL_F_EMPTY;
        r.pass = 1;
    } else if (o.gate) {
        r.flags = (uint16_t)o.gate;
    } else {
        r.flags = PCL_F_ALIGNED | (o.verified ? 0 : PCL_F_EDGE_VERIFY_FAIL);
        r.score = (uint32_t)o.E;
        r.sim = (float)o.E;
        r.pass = o.pass ? 1 : 0;
    }
    return r;
}

}  // namespace edge_dev
}  // namespace pcl

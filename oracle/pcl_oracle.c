/*
 * CPU ORACLE -- test infrastructure only.
 *
 * A plain, slow, obviously-correct statement of what the GPU path computes.
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this file.  It shares no code, header, table or helper with the
 * CUDA library; the only common module is the seeded rectangle generator.
 *
 * Every function cites the passage of the paper it follows (section and
 * equation numbers of "An Optimal Alignment-Driven Iterative Closed-Loop
 * Convergence Framework for High-Performance Ultra-Large Scale Layout Pattern
 * Clustering").  Where the paper is silent the reading taken is stated inline.
 *
 * Conventions
 *   clip      W x W dbu window, rectangles (x0, y0, x1, y1), window-relative.
 *   raster    N = W / p pixels per side; pixel (i, j) -> x index i, y index j.
 *   shift     s = (dx, dy) in pixels applied to the member B:
 *               c(s) = sum_x A(x) * B(x - s)            (linear, B = 0 outside)
 *             reported in dbu as s * p.
 *   window    |dx|, |dy| <= S = M / p (M = marker half-width in dbu).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- records */

enum {
    ORC_MODE_COSINE = 1,
    ORC_MODE_EDGE = 2,
    ORC_MODE_COSINE_XYSEP = 3,  /* cosine mode, shift by interval competition */
    ORC_MODE_COSINE_HALO = 4,   /* cosine mode, member window re-extracted at each shift */
};

/* gate / outcome codes (low 4 bits of flags) */
enum {
    ORC_GATE_NONE = 0,
    ORC_GATE_G1_AREA = 1,
    ORC_GATE_G2_PROFILE = 2,
    ORC_GATE_G3_DENSITY = 3,
    ORC_GATE_E1_MATCH = 4,
    ORC_GATE_E2_BBOX = 5,
    ORC_GATE_T0_TOPO = 6,  /* lossy pre-screen: different topological classes */
};
enum {
    ORC_F_NEAR_BAND = 1u << 4,
    ORC_F_EMPTY = 1u << 8,
    ORC_F_ALIGNED = 1u << 9,
    ORC_F_EDGE_VERIFY_FAIL = 1u << 7,
};

typedef struct orc_rec {
    uint32_t a, b;
    int32_t dx_dbu, dy_dbu;   /* best shift applied to b, dbu */
    double sim;               /* cosine: c_best / sqrt(pop_A pop_B); edge: max(Ex, Ey) */
    int64_t score;            /* cosine: c* (overlap pixels); edge: max(Ex, Ey) */
    uint32_t flags;
    int32_t pass;
    int32_t mode;
    int32_t pad;
} orc_rec;

typedef struct orc_params {
    int32_t pitch_dbu;
    int32_t window_dbu;
    int32_t marker_dbu;
    uint32_t cos_num, cos_den;  /* T = num / den */
    int32_t edge_tol_dbu;
    int32_t use_gates;          /* 0: evaluate every pair by brute force */
    int32_t use_topo;           /* candidate screens: lossy topological pre-screen first */
} orc_params;

/* ---------------------------------------------------------------- clip set */

typedef struct orc_set {
    int W, p, N, nw, S, M;
    int nb;        /* density blocks per side (16 px blocks) */
    int rb;        /* block radius covering S pixels: ceil(S / 16) */
    int n;
    uint8_t *img;   /* n * N * N, [j][i] */
    uint64_t *wd;   /* n * N * nw, oracle's own packing: bit i%64 of word i/64 */
    int64_t *pop;
    int32_t *rows;  /* n * N: ones in row j */
    int32_t *cols;  /* n * N: ones in column i */
    int32_t *blk;   /* n * nb * nb: ones in 16x16 block */
    int32_t *dil;   /* n * nb * nb: ones in the (2rb+1)^2 block neighbourhood */
    uint32_t *roff; /* n + 1 */
    int32_t *rects; /* 4 * roff[n] */
    uint8_t *himg;  /* n * (N + 2S)^2 or NULL: rasters of [-M, W + M)^2, see orc_set_add_halo */
} orc_set;

/*
 * Rasterisation (Sec. 2.2.1 step 1, "convert the vector-based patterns into
 * bitmap images").  Reading: a pixel is 1 iff its centre (p*i + p/2,
 * p*j + p/2) lies in some rectangle, half-open in x and y; overlapping
 * rectangles union.  Evaluated in doubled coordinates so that odd pitches stay
 * integer.
 */
void orc_rasterize(int W, int p, const int32_t *rects, int n, uint8_t *img) {
    int N = W / p;
    for (int j = 0; j < N; ++j) {
        for (int i = 0; i < N; ++i) {
            int64_t X2 = 2LL * p * i + p, Y2 = 2LL * p * j + p;
            uint8_t v = 0;
            for (int r = 0; r < n; ++r) {
                const int32_t *q = rects + 4 * r;
                if (2LL * q[0] <= X2 && X2 < 2LL * q[2] && 2LL * q[1] <= Y2 && Y2 < 2LL * q[3]) v = 1;
            }
            img[(size_t)j * N + i] = v;
        }
    }
}

static void pack_rows(const uint8_t *img, int N, uint64_t *wd) {
    int nw = (N + 63) / 64;
    memset(wd, 0, sizeof(uint64_t) * (size_t)N * nw);
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i)
            if (img[(size_t)j * N + i]) wd[(size_t)j * nw + i / 64] |= 1ull << (i % 64);
}

/*
 * c(dx, dy) = sum_x A(x) B(x - s), pixel loop (Eq. 2 numerator, pixel domain).
 * Used on tiny clips to pin the word version below.
 */
int64_t orc_corr_pixel(const uint8_t *A, const uint8_t *B, int N, int dx, int dy) {
    int64_t c = 0;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            int bi = i - dx, bj = j - dy;
            if (bi < 0 || bi >= N || bj < 0 || bj >= N) continue;
            c += (int64_t)A[(size_t)j * N + i] * B[(size_t)bj * N + bi];
        }
    return c;
}

static uint64_t get_word(const uint64_t *row, int nw, int64_t k) {
    return (k >= 0 && k < nw) ? row[k] : 0ull;
}

/* word w of `row` moved toward larger x by dx pixels: bit t of the result is
   pixel 64*w + t - dx of the row */
static uint64_t shifted_word(const uint64_t *row, int nw, int w, int dx) {
    int64_t base = 64LL * w - dx;
    int64_t wi = base >= 0 ? base / 64 : -((-base + 63) / 64);
    int off = (int)(base - 64 * wi);
    uint64_t lo = get_word(row, nw, wi), hi = get_word(row, nw, wi + 1);
    return off ? ((lo >> off) | (hi << (64 - off))) : lo;
}

/* the same sum through AND + popcount on packed words */
static int64_t corr_words(const uint64_t *A, const uint64_t *B, int N, int nw, int dx, int dy) {
    int64_t c = 0;
    for (int j = 0; j < N; ++j) {
        int bj = j - dy;
        if (bj < 0 || bj >= N) continue;
        const uint64_t *ra = A + (size_t)j * nw, *rb = B + (size_t)bj * nw;
        for (int w = 0; w < nw; ++w) c += __builtin_popcountll(ra[w] & shifted_word(rb, nw, w, dx));
    }
    return c;
}

int64_t orc_corr_words_img(const uint8_t *A, const uint8_t *B, int N, int dx, int dy) {
    int nw = (N + 63) / 64;
    uint64_t *wa = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N * nw);
    uint64_t *wb = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N * nw);
    pack_rows(A, N, wa);
    pack_rows(B, N, wb);
    int64_t c = corr_words(wa, wb, N, nw, dx, dy);
    free(wa);
    free(wb);
    return c;
}

void orc_set_free(orc_set *s) {
    if (!s) return;
    free(s->img); free(s->wd); free(s->pop); free(s->rows); free(s->cols);
    free(s->blk); free(s->dil); free(s->roff); free(s->rects); free(s->himg);
    free(s);
}

/*
 * Prepare a clip set: rasters and the signatures the lossless gates read.
 * Signatures: |A| (ones), row counts r(j), column counts q(i), 16x16 block
 * counts and their (2*rb+1)^2 neighbourhood sums (rb = ceil(S/16)).
 */
/* raster = 0 builds a geometry-only set (rectangles, no images or
   signatures): enough for the edge procedure, which reads rectangles only */
orc_set *orc_set_create_ex(int W, int p, int M, const uint32_t *roff, const int32_t *rects, int n,
                           int raster) {
    if (p <= 0 || W % p != 0 || M % p != 0) return NULL;
    orc_set *s = (orc_set *)calloc(1, sizeof(orc_set));
    s->W = W; s->p = p; s->N = W / p; s->nw = (s->N + 63) / 64;
    s->M = M; s->S = M / p; s->n = n;
    s->nb = (s->N + 15) / 16;
    s->rb = (s->S + 15) / 16;
    if (!raster) {
        s->roff = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
        memcpy(s->roff, roff, sizeof(uint32_t) * ((size_t)n + 1));
        s->rects = (int32_t *)malloc(sizeof(int32_t) * (4 * (size_t)roff[n] + 1));
        memcpy(s->rects, rects, sizeof(int32_t) * 4 * (size_t)roff[n]);
        return s;
    }
    int N = s->N, nw = s->nw, nb = s->nb;
    s->img = (uint8_t *)malloc((size_t)n * N * N + 1);
    s->wd = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n * N * nw + 1));
    s->pop = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    s->rows = (int32_t *)calloc((size_t)n * N + 1, sizeof(int32_t));
    s->cols = (int32_t *)calloc((size_t)n * N + 1, sizeof(int32_t));
    s->blk = (int32_t *)calloc((size_t)n * nb * nb + 1, sizeof(int32_t));
    s->dil = (int32_t *)calloc((size_t)n * nb * nb + 1, sizeof(int32_t));
    s->roff = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    memcpy(s->roff, roff, sizeof(uint32_t) * ((size_t)n + 1));
    s->rects = (int32_t *)malloc(sizeof(int32_t) * (4 * (size_t)roff[n] + 1));
    memcpy(s->rects, rects, sizeof(int32_t) * 4 * (size_t)roff[n]);
    for (int c = 0; c < n; ++c) {
        uint8_t *im = s->img + (size_t)c * N * N;
        orc_rasterize(W, p, s->rects + 4 * (size_t)roff[c], (int)(roff[c + 1] - roff[c]), im);
        pack_rows(im, N, s->wd + (size_t)c * N * nw);
        int32_t *rw = s->rows + (size_t)c * N, *cl = s->cols + (size_t)c * N;
        int32_t *bk = s->blk + (size_t)c * nb * nb, *dl = s->dil + (size_t)c * nb * nb;
        int64_t pop = 0;
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i)
                if (im[(size_t)j * N + i]) {
                    ++pop; ++rw[j]; ++cl[i]; ++bk[(j / 16) * nb + i / 16];
                }
        s->pop[c] = pop;
        for (int by = 0; by < nb; ++by)
            for (int bx = 0; bx < nb; ++bx) {
                int32_t t = 0;
                for (int oy = -s->rb; oy <= s->rb; ++oy)
                    for (int ox = -s->rb; ox <= s->rb; ++ox) {
                        int yy = by + oy, xx = bx + ox;
                        if (yy >= 0 && yy < nb && xx >= 0 && xx < nb) t += bk[yy * nb + xx];
                    }
                dl[by * nb + bx] = t;
            }
    }
    return s;
}

orc_set *orc_set_create(int W, int p, int M, const uint32_t *roff, const int32_t *rects, int n) {
    return orc_set_create_ex(W, p, M, roff, rects, n, 1);
}

int orc_set_N(const orc_set *s) { return s->N; }
int64_t orc_set_pop(const orc_set *s, int c) { return s->pop[c]; }
void orc_set_image(const orc_set *s, int c, uint8_t *out) {
    memcpy(out, s->img + (size_t)c * s->N * s->N, (size_t)s->N * s->N);
}
void orc_set_sig(const orc_set *s, int c, int32_t *rows, int32_t *cols, int32_t *blk, int32_t *dil) {
    int N = s->N, nb = s->nb;
    memcpy(rows, s->rows + (size_t)c * N, sizeof(int32_t) * N);
    memcpy(cols, s->cols + (size_t)c * N, sizeof(int32_t) * N);
    memcpy(blk, s->blk + (size_t)c * nb * nb, sizeof(int32_t) * nb * nb);
    memcpy(dil, s->dil + (size_t)c * nb * nb, sizeof(int32_t) * nb * nb);
}

/* ---------------------------------------------------------------- cosine */

/* Cosine threshold test of Eq. 2 with strict ">" in exact integers:
   c / sqrt(|A||B|) > num/den  <=>  c > 0 and den^2 c^2 > num^2 |A| |B|. */
static int cos_exceeds(int64_t c, int64_t pa, int64_t pb, uint32_t num, uint32_t den) {
    if (c <= 0) return 0;
    __int128 lhs = (__int128)den * den * c * c;
    __int128 rhs = (__int128)num * num * pa * pb;
    return lhs > rhs;
}

int orc_cos_exceeds(int64_t c, int64_t pa, int64_t pb, uint32_t num, uint32_t den) {
    return cos_exceeds(c, pa, pb, num, den);
}

/* G1 (area): c* <= min(|A|,|B|) bounds the cosine by sqrt(min/max). */
static int gate_g1(int64_t pa, int64_t pb, uint32_t num, uint32_t den) {
    int64_t mn = pa < pb ? pa : pb, mx = pa < pb ? pb : pa;
    return (__int128)den * den * mn > (__int128)num * num * mx;
}

/* G3 (density): for any |s| <= S the ones of A in block k can only meet ones
   of B inside the block neighbourhood; bound taken both ways, minimum kept. */
static int64_t bound_g3(const orc_set *s, int a, int b) {
    int nb2 = s->nb * s->nb;
    const int32_t *ba = s->blk + (size_t)a * nb2, *bb = s->blk + (size_t)b * nb2;
    const int32_t *da = s->dil + (size_t)a * nb2, *db = s->dil + (size_t)b * nb2;
    int64_t u1 = 0, u2 = 0;
    for (int k = 0; k < nb2; ++k) {
        u1 += ba[k] < db[k] ? ba[k] : db[k];
        u2 += bb[k] < da[k] ? bb[k] : da[k];
    }
    return u1 < u2 ? u1 : u2;
}

/* G2 (projection profiles): row j of A overlaps row j - dy of B in at most
   min(r_A(j), r_B(j - dy)) pixels; the best dy bounds every shift.  Same for
   columns; the smaller of the two bounds is kept. */
static int64_t bound_g2(const orc_set *s, int a, int b) {
    int N = s->N, S = s->S;
    const int32_t *ra = s->rows + (size_t)a * N, *rb = s->rows + (size_t)b * N;
    const int32_t *qa = s->cols + (size_t)a * N, *qb = s->cols + (size_t)b * N;
    int64_t ur = 0, uc = 0;
    for (int d = -S; d <= S; ++d) {
        int64_t tr = 0, tc = 0;
        for (int j = 0; j < N; ++j) {
            int k = j - d;
            if (k < 0 || k >= N) continue;
            tr += ra[j] < rb[k] ? ra[j] : rb[k];
            tc += qa[j] < qb[k] ? qa[j] : qb[k];
        }
        if (tr > ur) ur = tr;
        if (tc > uc) uc = tc;
    }
    return ur < uc ? ur : uc;
}

/* the three cosine upper bounds on c(s) for |s| <= S: out = {G1, G2, G3} */
void orc_gate_bounds(const orc_set *s, int a, int b, int64_t *out) {
    out[0] = s->pop[a] < s->pop[b] ? s->pop[a] : s->pop[b];
    out[1] = bound_g2(s, a, b);
    out[2] = bound_g3(s, a, b);
}

/* cosine gates in evaluation order G1, G3, G2; returns the rejecting gate */
static int cosine_gate(const orc_set *s, int a, int b, const orc_params *P) {
    int64_t pa = s->pop[a], pb = s->pop[b];
    if (!gate_g1(pa, pb, P->cos_num, P->cos_den)) return ORC_GATE_G1_AREA;
    int64_t u3 = bound_g3(s, a, b);
    if (!cos_exceeds(u3, pa, pb, P->cos_num, P->cos_den)) return ORC_GATE_G3_DENSITY;
    int64_t u2 = bound_g2(s, a, b);
    if (!cos_exceeds(u2, pa, pb, P->cos_num, P->cos_den)) return ORC_GATE_G2_PROFILE;
    return ORC_GATE_NONE;
}

/* lexicographic order of candidate shifts: larger overlap first, then
   smaller |dx|+|dy|, then smaller dy, then smaller dx.  Returns 1 if
   (c1, dx1, dy1) comes before (c2, dx2, dy2). */
static int shift_before(int64_t c1, int dx1, int dy1, int64_t c2, int dx2, int dy2) {
    if (c1 != c2) return c1 > c2;
    int l1 = abs(dx1) + abs(dy1), l2 = abs(dx2) + abs(dy2);
    if (l1 != l2) return l1 < l2;
    if (dy1 != dy2) return dy1 < dy2;
    return dx1 < dx2;
}

/*
 * Cosine-mode pair test (Sec. 2.2.1, Eq. 2; optimal alignment of Sec. 3.2).
 * The DCT feature vectors of Sec. 2.2.1 step 2 are read as the full
 * orthonormal 2-D DCT-II, so by Parseval the cosine of the coefficient
 * vectors equals the cosine of the pixel vectors; the norms are the full
 * (unshifted) norms.  The optimal shift is found by brute force over every
 * pixel-grid shift of the marker window: s* = argmax c(s) with the tie order
 * of shift_before().  Both clips empty: similar by reading (sim 1, pass).
 */
void orc_cosine_pair(const orc_set *s, int a, int b, const orc_params *P, orc_rec *out) {
    memset(out, 0, sizeof(*out));
    out->a = (uint32_t)a; out->b = (uint32_t)b; out->mode = ORC_MODE_COSINE;
    int64_t pa = s->pop[a], pb = s->pop[b];
    if (pa == 0 && pb == 0) {
        out->sim = 1.0; out->pass = 1; out->flags = ORC_F_EMPTY;
        return;
    }
    if (P->use_gates) {
        int g = cosine_gate(s, a, b, P);
        if (g != ORC_GATE_NONE) { out->flags = (uint32_t)g; return; }
    }
    int N = s->N, nw = s->nw, S = s->S;
    const uint64_t *A = s->wd + (size_t)a * N * nw, *B = s->wd + (size_t)b * N * nw;
    int64_t bc = -1;
    int bdx = 0, bdy = 0;
    for (int dy = -S; dy <= S; ++dy)
        for (int dx = -S; dx <= S; ++dx) {
            int64_t c = corr_words(A, B, N, nw, dx, dy);
            if (bc < 0 || shift_before(c, dx, dy, bc, bdx, bdy)) { bc = c; bdx = dx; bdy = dy; }
        }
    out->dx_dbu = bdx * s->p;
    out->dy_dbu = bdy * s->p;
    out->score = bc;
    /* a zero vector has cosine 0 with anything (one clip empty) */
    out->sim = (pa > 0 && pb > 0) ? (double)bc / sqrt((double)pa * (double)pb) : 0.0;
    out->pass = cos_exceeds(bc, pa, pb, P->cos_num, P->cos_den);
    out->flags = ORC_F_ALIGNED;
}

/* full correlation surface over the marker window, [dy+S][dx+S] */
void orc_corr_window(const orc_set *s, int a, int b, int64_t *out) {
    int N = s->N, nw = s->nw, S = s->S, K = 2 * S + 1;
    const uint64_t *A = s->wd + (size_t)a * N * nw, *B = s->wd + (size_t)b * N * nw;
    for (int dy = -S; dy <= S; ++dy)
        for (int dx = -S; dx <= S; ++dx)
            out[(dy + S) * K + (dx + S)] = corr_words(A, B, N, nw, dx, dy);
}

/* ---------------------------------------------------------------- edge mode */

typedef struct { int32_t x0, y0, x1, y1; } orc_rect;

static const orc_rect *clip_rects(const orc_set *s, int c, int *n) {
    *n = (int)(s->roff[c + 1] - s->roff[c]);
    return (const orc_rect *)(s->rects + 4 * (size_t)s->roff[c]);
}

/* positive-area overlap of rectangle a with rectangle b translated by t */
static int overlaps(const orc_rect *a, const orc_rect *b, int tx, int ty) {
    return a->x0 < b->x1 + tx && b->x0 + tx < a->x1 && a->y0 < b->y1 + ty && b->y0 + ty < a->y1;
}

/* bbox over the edges that do not lie on the window border (border edges are
   cuts made by the window, not layout edges) -- reading, paper silent */
static void edge_bbox(const orc_rect *r, int n, int W, int *has_x, int *lx, int *hx, int *has_y,
                      int *ly, int *hy) {
    *has_x = *has_y = 0;
    *lx = *ly = 0; *hx = *hy = 0;
    for (int i = 0; i < n; ++i) {
        int vx[2] = {r[i].x0, r[i].x1}, vy[2] = {r[i].y0, r[i].y1};
        int okx[2] = {r[i].x0 != 0, r[i].x1 != W}, oky[2] = {r[i].y0 != 0, r[i].y1 != W};
        for (int k = 0; k < 2; ++k) {
            if (okx[k]) {
                if (!*has_x) { *lx = *hx = vx[k]; *has_x = 1; }
                if (vx[k] < *lx) *lx = vx[k];
                if (vx[k] > *hx) *hx = vx[k];
            }
            if (oky[k]) {
                if (!*has_y) { *ly = *hy = vy[k]; *has_y = 1; }
                if (vy[k] < *ly) *ly = vy[k];
                if (vy[k] > *hy) *hy = vy[k];
            }
        }
    }
}

static int touches_border(const orc_rect *r, int n, int W) {
    for (int i = 0; i < n; ++i)
        if (r[i].x0 == 0 || r[i].y0 == 0 || r[i].x1 == W || r[i].y1 == W) return 1;
    return 0;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/*
 * Polygon correspondence (Sec. 2.2.2 condition 1): each polygon of the clip
 * with fewer polygons (A when the counts tie) overlaps exactly one polygon of
 * the other clip, B being translated by t.  Reading: the map must also be
 * injective.  match[k] receives the partner of small-side polygon k.
 * Returns 1 when the correspondence holds.
 */
static int correspond(const orc_rect *ra, int na, const orc_rect *rb, int nb, int tx, int ty,
                      int *match) {
    int small_is_a = na <= nb;
    int ns = small_is_a ? na : nb, nl = small_is_a ? nb : na;
    for (int k = 0; k < ns; ++k) {
        int cnt = 0, who = -1;
        for (int m = 0; m < nl; ++m) {
            int hit = small_is_a ? overlaps(&ra[k], &rb[m], tx, ty) : overlaps(&ra[m], &rb[k], tx, ty);
            if (hit) { ++cnt; who = m; }
        }
        if (cnt != 1) return 0;
        match[k] = who;
    }
    for (int k = 0; k < ns; ++k)
        for (int k2 = k + 1; k2 < ns; ++k2)
            if (match[k] == match[k2]) return 0;
    return 1;
}

/*
 * Edge-displacement pair test (Sec. 2.2.2; Geometric Min-Max of Sec. 3.2.2,
 * Eq. 6).  Integer dbu throughout.  Steps:
 *  0. both clips empty -> pass; exactly one empty -> no correspondence (E1).
 *  E2 (gate, lossless): equal polygon counts and no border edge in either
 *     clip -> the bbox width and height may differ by at most 2*tol.
 *  1. pre-alignment s0 = trunc((centre_A - centre_B)) per axis from the
 *     non-border-edge bboxes (doubled centres halved, truncated toward zero),
 *     clamped to +/-M; 0 on an axis that lacks such edges in either clip.
 *  2. correspondence at s0 (E1 on failure).
 *  3. displacements d = e_A - e_B of every matched edge pair whose two edges
 *     are off the window border; d_min, d_max per axis.
 *  4. closed form of Eq. 6 per separable axis: T = trunc((d_min + d_max)/2)
 *     clamped to +/-M, E = max(T - d_min, d_max - T); an axis without
 *     displacements keeps T = s0 and E = 0.
 *  5. the correspondence must still hold at T, with the same partners.
 *  6. pass iff step 5 holds and E_x, E_y <= tol (condition 2, "not exceed").
 */
void orc_edge_pair(const orc_set *s, int a, int b, const orc_params *P, orc_rec *out) {
    memset(out, 0, sizeof(*out));
    out->a = (uint32_t)a; out->b = (uint32_t)b; out->mode = ORC_MODE_EDGE;
    int na, nb;
    const orc_rect *ra = clip_rects(s, a, &na), *rb = clip_rects(s, b, &nb);
    int W = s->W, M = P->marker_dbu, tol = P->edge_tol_dbu;
    if (na == 0 && nb == 0) { out->pass = 1; out->flags = ORC_F_EMPTY; return; }
    if (na == 0 || nb == 0) { out->flags = ORC_GATE_E1_MATCH; return; }
    int hxa, lxa, uxa, hya, lya, uya, hxb, lxb, uxb, hyb, lyb, uyb;
    edge_bbox(ra, na, W, &hxa, &lxa, &uxa, &hya, &lya, &uya);
    edge_bbox(rb, nb, W, &hxb, &lxb, &uxb, &hyb, &lyb, &uyb);
    if (P->use_gates && na == nb && !touches_border(ra, na, W) && !touches_border(rb, nb, W)) {
        int wa = uxa - lxa, wb = uxb - lxb, ha = uya - lya, hb = uyb - lyb;
        if (abs(wa - wb) > 2 * tol || abs(ha - hb) > 2 * tol) { out->flags = ORC_GATE_E2_BBOX; return; }
    }
    int s0x = (hxa && hxb) ? clampi(((lxa + uxa) - (lxb + uxb)) / 2, -M, M) : 0;
    int s0y = (hya && hyb) ? clampi(((lya + uya) - (lyb + uyb)) / 2, -M, M) : 0;
    int ns = na <= nb ? na : nb;
    int *match = (int *)malloc(sizeof(int) * (size_t)(ns + 1));
    int *match2 = (int *)malloc(sizeof(int) * (size_t)(ns + 1));
    if (!correspond(ra, na, rb, nb, s0x, s0y, match)) {
        out->flags = ORC_GATE_E1_MATCH;
        out->dx_dbu = s0x; out->dy_dbu = s0y;
        free(match); free(match2);
        return;
    }
    int small_is_a = na <= nb;
    int cx = 0, cy = 0, dminx = 0, dmaxx = 0, dminy = 0, dmaxy = 0;
    for (int k = 0; k < ns; ++k) {
        const orc_rect *pa = small_is_a ? &ra[k] : &ra[match[k]];
        const orc_rect *pb = small_is_a ? &rb[match[k]] : &rb[k];
        int dx[2] = {pa->x0 - pb->x0, pa->x1 - pb->x1};
        int okx[2] = {pa->x0 != 0 && pb->x0 != 0, pa->x1 != W && pb->x1 != W};
        int dy[2] = {pa->y0 - pb->y0, pa->y1 - pb->y1};
        int oky[2] = {pa->y0 != 0 && pb->y0 != 0, pa->y1 != W && pb->y1 != W};
        for (int e = 0; e < 2; ++e) {
            if (okx[e]) {
                if (!cx || dx[e] < dminx) dminx = dx[e];
                if (!cx || dx[e] > dmaxx) dmaxx = dx[e];
                cx = 1;
            }
            if (oky[e]) {
                if (!cy || dy[e] < dminy) dminy = dy[e];
                if (!cy || dy[e] > dmaxy) dmaxy = dy[e];
                cy = 1;
            }
        }
    }
    int Tx = cx ? clampi((dminx + dmaxx) / 2, -M, M) : s0x;
    int Ty = cy ? clampi((dminy + dmaxy) / 2, -M, M) : s0y;
    int Ex = cx ? ((Tx - dminx) > (dmaxx - Tx) ? (Tx - dminx) : (dmaxx - Tx)) : 0;
    int Ey = cy ? ((Ty - dminy) > (dmaxy - Ty) ? (Ty - dminy) : (dmaxy - Ty)) : 0;
    int ok = correspond(ra, na, rb, nb, Tx, Ty, match2);
    for (int k = 0; ok && k < ns; ++k)
        if (match2[k] != match[k]) ok = 0;
    int E = Ex > Ey ? Ex : Ey;
    out->dx_dbu = Tx; out->dy_dbu = Ty;
    out->score = E;
    out->sim = (double)E;
    out->flags = ORC_F_ALIGNED | (ok ? 0u : ORC_F_EDGE_VERIFY_FAIL);
    out->pass = ok && Ex <= tol && Ey <= tol;
    free(match); free(match2);
}

/*
 * Brute-force check of the closed form (Sec. 3.2.2: "any deviation from this
 * midpoint would inevitably increase the error"): for displacements d[0..n),
 * scan every integer T in [-M, M] and return min_T max_i |d_i - T|; the
 * smallest and largest minimisers are written to tlo/thi.
 */
int orc_minmax_scan(const int32_t *d, int n, int M, int *tlo, int *thi) {
    int best = -1;
    *tlo = *thi = 0;
    for (int T = -M; T <= M; ++T) {
        int e = 0;
        for (int i = 0; i < n; ++i) {
            int v = abs(d[i] - T);
            if (v > e) e = v;
        }
        if (best < 0 || e < best) { best = e; *tlo = *thi = T; }
        else if (e == best) *thi = T;
    }
    return best;
}

/* the closed form alone (Eq. 6, per axis), same integer reading as above */
void orc_minmax_closed(const int32_t *d, int n, int M, int *T, int *E) {
    int dmin = d[0], dmax = d[0];
    for (int i = 1; i < n; ++i) {
        if (d[i] < dmin) dmin = d[i];
        if (d[i] > dmax) dmax = d[i];
    }
    *T = clampi((dmin + dmax) / 2, -M, M);
    *E = (*T - dmin) > (dmax - *T) ? (*T - dmin) : (dmax - *T);
}

/*
 * Cosine mode with the shift of the XY-separation interval competition
 * (Sec. 3.2.1 (2), the geometric alternative to phase correlation), written
 * from its four steps with the readings below (the paper states only the
 * steps):
 *  0. both clips empty -> pass (sim 1); the cosine gates first when enabled.
 *  1. polygon pairs: pre-alignment s0 as in edge mode (doubled centres of the
 *     non-border-edge bboxes, truncated, clamped to +/-M; 0 on an axis that
 *     lacks such edges in either clip); each polygon k of the clip with fewer
 *     polygons (A on a tie) pairs with its partner m when exactly one polygon
 *     of the other clip overlaps it at s0 (no pair otherwise).
 *     Allowable interval of a pair on an axis: [d_min, d_max] over the
 *     displacements d = e_A - e_B of its two edges on that axis, edges on the
 *     window border in either clip excluded (no interval if both are).
 *  2. interval quality Q = d_max - d_min.
 *  3. axis winner: the pair with the smallest Q; ties go to the smaller k.
 *  4. T = trunc((d_min + d_max) / 2) of the winner, clamped to +/-M; an axis
 *     without any interval keeps T = s0.
 * The dbu shift becomes the raster shift s = T / p rounded half away from
 * zero and clamped to +/-S; the record holds c(s) (exact overlap), sim and
 * the integer decision of Eq. 2 at that shift.  Since c(s) <= c(s*), this
 * engine can only lose passes of the exact argmax, never add any.
 */
static int round_div_away(int v, int p) { return v >= 0 ? (v + p / 2) / p : -((-v + p / 2) / p); }

void orc_xysep_pair(const orc_set *s, int a, int b, const orc_params *P, orc_rec *out) {
    memset(out, 0, sizeof(*out));
    out->a = (uint32_t)a; out->b = (uint32_t)b; out->mode = ORC_MODE_COSINE;
    int64_t pa = s->pop[a], pb = s->pop[b];
    if (pa == 0 && pb == 0) {
        out->sim = 1.0; out->pass = 1; out->flags = ORC_F_EMPTY;
        return;
    }
    if (P->use_gates) {
        int g = cosine_gate(s, a, b, P);
        if (g != ORC_GATE_NONE) { out->flags = (uint32_t)g; return; }
    }
    int na, nb;
    const orc_rect *ra = clip_rects(s, a, &na), *rb = clip_rects(s, b, &nb);
    int W = s->W, M = P->marker_dbu;
    int hxa, lxa, uxa, hya, lya, uya, hxb, lxb, uxb, hyb, lyb, uyb;
    edge_bbox(ra, na, W, &hxa, &lxa, &uxa, &hya, &lya, &uya);
    edge_bbox(rb, nb, W, &hxb, &lxb, &uxb, &hyb, &lyb, &uyb);
    int s0x = (hxa && hxb) ? clampi(((lxa + uxa) - (lxb + uxb)) / 2, -M, M) : 0;
    int s0y = (hya && hyb) ? clampi(((lya + uya) - (lyb + uyb)) / 2, -M, M) : 0;
    int small_is_a = na <= nb;
    int ns = small_is_a ? na : nb, nl = small_is_a ? nb : na;
    /* best interval per axis: quality, d_min + d_max */
    int qx = -1, sx = 0, qy = -1, sy = 0;
    for (int k = 0; k < ns; ++k) {
        int cnt = 0, m = -1;
        for (int j = 0; j < nl; ++j) {
            int hit = small_is_a ? overlaps(&ra[k], &rb[j], s0x, s0y) : overlaps(&ra[j], &rb[k], s0x, s0y);
            if (hit) { ++cnt; m = j; }
        }
        if (cnt != 1) continue;
        const orc_rect *p_a = small_is_a ? &ra[k] : &ra[m];
        const orc_rect *p_b = small_is_a ? &rb[m] : &rb[k];
        int dx[2] = {p_a->x0 - p_b->x0, p_a->x1 - p_b->x1};
        int okx[2] = {p_a->x0 != 0 && p_b->x0 != 0, p_a->x1 != W && p_b->x1 != W};
        int dy[2] = {p_a->y0 - p_b->y0, p_a->y1 - p_b->y1};
        int oky[2] = {p_a->y0 != 0 && p_b->y0 != 0, p_a->y1 != W && p_b->y1 != W};
        int has = 0, lo = 0, hi = 0;
        for (int e = 0; e < 2; ++e)
            if (okx[e]) {
                if (!has || dx[e] < lo) lo = dx[e];
                if (!has || dx[e] > hi) hi = dx[e];
                has = 1;
            }
        if (has && (qx < 0 || hi - lo < qx)) { qx = hi - lo; sx = lo + hi; }
        has = 0;
        for (int e = 0; e < 2; ++e)
            if (oky[e]) {
                if (!has || dy[e] < lo) lo = dy[e];
                if (!has || dy[e] > hi) hi = dy[e];
                has = 1;
            }
        if (has && (qy < 0 || hi - lo < qy)) { qy = hi - lo; sy = lo + hi; }
    }
    int Tx = qx >= 0 ? clampi(sx / 2, -M, M) : s0x;
    int Ty = qy >= 0 ? clampi(sy / 2, -M, M) : s0y;
    int S = s->S, p = s->p;
    int dxp = clampi(round_div_away(Tx, p), -S, S), dyp = clampi(round_div_away(Ty, p), -S, S);
    int N = s->N, nw = s->nw;
    const uint64_t *A = s->wd + (size_t)a * N * nw, *B = s->wd + (size_t)b * N * nw;
    int64_t c = corr_words(A, B, N, nw, dxp, dyp);
    out->dx_dbu = dxp * p;
    out->dy_dbu = dyp * p;
    out->score = c;
    out->sim = (pa > 0 && pb > 0) ? (double)c / sqrt((double)pa * (double)pb) : 0.0;
    out->pass = cos_exceeds(c, pa, pb, P->cos_num, P->cos_den);
    out->flags = ORC_F_ALIGNED;
}

/* edge gates alone (E2 then E1 correspondence at s0); returns rejecting gate */
static int edge_gate(const orc_set *s, int a, int b, const orc_params *P) {
    orc_rec r;
    orc_params q = *P;
    q.use_gates = 1;
    orc_edge_pair(s, a, b, &q, &r);
    uint32_t g = r.flags & 15u;
    return (g == ORC_GATE_E1_MATCH || g == ORC_GATE_E2_BBOX) ? (int)g : ORC_GATE_NONE;
}

/* ---------------------------------------------------------------- batches */

void orc_halo_pair(const orc_set *s, int a, int b, const orc_params *P, orc_rec *out);

typedef struct {
    const orc_set *s;
    const orc_params *P;
    int mode;
    const uint32_t *pairs;  /* 2 * n */
    size_t n;
    orc_rec *out;
    size_t next;
    pthread_mutex_t mu;
} match_job;

static void *match_worker(void *arg) {
    match_job *j = (match_job *)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        size_t lo = j->next;
        j->next += 64;
        pthread_mutex_unlock(&j->mu);
        if (lo >= j->n) break;
        size_t hi = lo + 64 < j->n ? lo + 64 : j->n;
        for (size_t i = lo; i < hi; ++i) {
            int a = (int)j->pairs[2 * i], b = (int)j->pairs[2 * i + 1];
            if (j->mode == ORC_MODE_COSINE) orc_cosine_pair(j->s, a, b, j->P, &j->out[i]);
            else if (j->mode == ORC_MODE_COSINE_XYSEP) orc_xysep_pair(j->s, a, b, j->P, &j->out[i]);
            else if (j->mode == ORC_MODE_COSINE_HALO) orc_halo_pair(j->s, a, b, j->P, &j->out[i]);
            else orc_edge_pair(j->s, a, b, j->P, &j->out[i]);
        }
    }
    return NULL;
}

/* one record per listed pair, in list order, on `threads` host threads */
void orc_match(const orc_set *s, const orc_params *P, int mode, const uint32_t *pairs, size_t n,
               orc_rec *out, int threads) {
    match_job j = {s, P, mode, pairs, n, out, 0, PTHREAD_MUTEX_INITIALIZER};
    if (threads < 1) threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, match_worker, &j);
    for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
    free(th);
}

typedef struct {
    const orc_set *s;
    const orc_params *P;
    int mode;
    int next;
    pthread_mutex_t mu;
    uint8_t *keep;     /* n*(n-1)/2 flags in (i<j) row order */
    uint64_t counts[16];
} cand_job;

/*
 * Topological class of a clip for the lossy pre-screen (Sec. 3.1 stage 1
 * names topological hashing): its polygon count, saturated at 63.  Reading:
 * each rectangle is a polygon (as in edge mode), and a count is what small
 * edge moves that keep polygons apart leave unchanged.  A pair of different
 * classes is screened out before any exact test.
 */
static int topo_class_of(const orc_set *s, int c) {
    int n = (int)(s->roff[c + 1] - s->roff[c]);
    return n < 63 ? n : 63;
}

static size_t tri_index(int n, int i, int j) {  /* i < j */
    return (size_t)i * (size_t)(2 * n - i - 1) / 2 + (size_t)(j - i - 1);
}

static void *cand_worker(void *arg) {
    cand_job *c = (cand_job *)arg;
    uint64_t local[16] = {0};
    int n = c->s->n;
    for (;;) {
        pthread_mutex_lock(&c->mu);
        int i = c->next++;
        pthread_mutex_unlock(&c->mu);
        if (i >= n) break;
        for (int j = i + 1; j < n; ++j) {
            int g;
            if (c->P->use_topo && topo_class_of(c->s, i) != topo_class_of(c->s, j)) {
                g = ORC_GATE_T0_TOPO;
            } else if (c->mode == ORC_MODE_COSINE) {
                if (c->s->pop[i] == 0 && c->s->pop[j] == 0) g = ORC_GATE_NONE;
                else g = cosine_gate(c->s, i, j, c->P);
            } else {
                g = edge_gate(c->s, i, j, c->P);
            }
            local[g]++;
            c->keep[tri_index(n, i, j)] = (uint8_t)(g == ORC_GATE_NONE);
        }
    }
    pthread_mutex_lock(&c->mu);
    for (int k = 0; k < 16; ++k) c->counts[k] += local[k];
    pthread_mutex_unlock(&c->mu);
    return NULL;
}

/*
 * Self-join candidate generation by exhaustive gate evaluation over all
 * i < j (the lossless multi-stage pre-screening of Sec. 3.1 stage 1, without
 * any join acceleration).  Survivors are written as (i, j) pairs in row
 * order; returns their count (or the required count if cap is too small).
 * gate_counts[g] counts pairs rejected by gate g (index 0 = survivors).
 */
int64_t orc_candidates(const orc_set *s, const orc_params *P, int mode, uint32_t *pairs,
                       int64_t cap, uint64_t *gate_counts, int threads) {
    int n = s->n;
    size_t tot = (size_t)n * (size_t)(n > 0 ? n - 1 : 0) / 2;
    cand_job c;
    memset(&c, 0, sizeof(c));
    c.s = s; c.P = P; c.mode = mode;
    pthread_mutex_init(&c.mu, NULL);
    c.keep = (uint8_t *)calloc(tot + 1, 1);
    if (threads < 1) threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, cand_worker, &c);
    for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
    free(th);
    int64_t m = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (c.keep[tri_index(n, i, j)]) {
                if (m < cap) { pairs[2 * m] = (uint32_t)i; pairs[2 * m + 1] = (uint32_t)j; }
                ++m;
            }
    for (int k = 0; k < 16; ++k) gate_counts[k] = c.counts[k];
    free(c.keep);
    pthread_mutex_destroy(&c.mu);
    return m;
}

/*
 * Two-set candidate generation by exhaustive gate evaluation: the set holds
 * the clips of A (indices 0 .. n_a-1) followed by those of B, and every pair
 * (i, n_a + j) goes through the same gates as in the self-join (Sec. 3.1
 * stage 1; Sec. 2.3 makes every pair of patterns a candidate).  Survivors
 * are written as (i, j), j relative to B, in row order; returns their count
 * (or the required count if cap is too small).
 */
typedef struct {
    const orc_set *s;
    const orc_params *P;
    int mode, n_a;
    int next;
    pthread_mutex_t mu;
    uint8_t *keep;     /* n_a * n_b flags, row i then column j */
    uint64_t counts[16];
} cand_ab_job;

static void *cand_ab_worker(void *arg) {
    cand_ab_job *c = (cand_ab_job *)arg;
    uint64_t local[16] = {0};
    int n = c->s->n, na = c->n_a, nb = n - na;
    for (;;) {
        pthread_mutex_lock(&c->mu);
        int i = c->next++;
        pthread_mutex_unlock(&c->mu);
        if (i >= na) break;
        for (int j = 0; j < nb; ++j) {
            int b = na + j, g;
            if (c->mode == ORC_MODE_COSINE) {
                if (c->s->pop[i] == 0 && c->s->pop[b] == 0) g = ORC_GATE_NONE;
                else g = cosine_gate(c->s, i, b, c->P);
            } else {
                g = edge_gate(c->s, i, b, c->P);
            }
            local[g]++;
            c->keep[(size_t)i * nb + j] = (uint8_t)(g == ORC_GATE_NONE);
        }
    }
    pthread_mutex_lock(&c->mu);
    for (int k = 0; k < 16; ++k) c->counts[k] += local[k];
    pthread_mutex_unlock(&c->mu);
    return NULL;
}

int64_t orc_candidates_ab(const orc_set *s, const orc_params *P, int mode, int n_a, uint32_t *pairs,
                          int64_t cap, uint64_t *gate_counts, int threads) {
    int nb = s->n - n_a;
    if (n_a < 0 || nb < 0) return -1;
    cand_ab_job c;
    memset(&c, 0, sizeof(c));
    c.s = s; c.P = P; c.mode = mode; c.n_a = n_a;
    pthread_mutex_init(&c.mu, NULL);
    c.keep = (uint8_t *)calloc((size_t)n_a * nb + 1, 1);
    if (threads < 1) threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, cand_ab_worker, &c);
    for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
    free(th);
    int64_t m = 0;
    for (int i = 0; i < n_a; ++i)
        for (int j = 0; j < nb; ++j)
            if (c.keep[(size_t)i * nb + j]) {
                if (m < cap) { pairs[2 * m] = (uint32_t)i; pairs[2 * m + 1] = (uint32_t)j; }
                ++m;
            }
    for (int k = 0; k < 16; ++k) gate_counts[k] = c.counts[k];
    free(c.keep);
    pthread_mutex_destroy(&c.mu);
    return m;
}


/* ---------------------------------------------------------- re-extraction */

/*
 * Halo rasters for re-extraction (Sec. 2.1: a pattern is the layout cut out
 * around its centre, and the centre may lie anywhere in the marker region).
 * Reading: each clip carries its rectangles over [-M, W + M)^2, and its halo
 * raster samples that region at the pixel centres p*i + p/2 for
 * i in [-S, N + S); pixel i is stored at index i + S.  Computed by the
 * rasteriser above on the rectangles moved by +M in a window of W + 2M.
 */
void orc_set_add_halo(orc_set *s) {
    int NH = s->N + 2 * s->S, M = s->M;
    free(s->himg);
    s->himg = (uint8_t *)malloc((size_t)s->n * NH * NH + 1);
    int32_t *tmp = NULL;
    size_t cap = 0;
    for (int c = 0; c < s->n; ++c) {
        int k = (int)(s->roff[c + 1] - s->roff[c]);
        if ((size_t)k > cap) {
            cap = (size_t)k;
            tmp = (int32_t *)realloc(tmp, sizeof(int32_t) * 4 * cap);
        }
        const int32_t *r = s->rects + 4 * (size_t)s->roff[c];
        for (int q = 0; q < 4 * k; ++q) tmp[q] = r[q] + M;
        orc_rasterize(s->W + 2 * M, s->p, tmp, k, s->himg + (size_t)c * NH * NH);
    }
    free(tmp);
}

/* c(s) and the moved window's pixel count n_B(s) for one shift, pixel loops:
   the member's window moved by s holds B's halo pixels x - s, x in [0, N)^2 */
static void halo_shift(const orc_set *s, const uint8_t *A, const uint8_t *Bh, int dx, int dy, int64_t *c,
                       int64_t *nb) {
    int N = s->N, S = s->S, NH = N + 2 * S;
    int64_t cc = 0, nn = 0;
    for (int y = 0; y < N; ++y)
        for (int x = 0; x < N; ++x) {
            int v = Bh[(size_t)(y - dy + S) * NH + (x - dx + S)];
            nn += v;
            cc += v & A[(size_t)y * N + x];
        }
    *c = cc;
    *nb = nn;
}

/* the window of c(s) and n_B(s), indexed [dy + S][dx + S] */
void orc_halo_window(const orc_set *s, int a, int b, int64_t *c_out, int64_t *n_out) {
    int N = s->N, S = s->S, K = 2 * S + 1, NH = N + 2 * S;
    const uint8_t *A = s->img + (size_t)a * N * N, *Bh = s->himg + (size_t)b * NH * NH;
    for (int dy = -S; dy <= S; ++dy)
        for (int dx = -S; dx <= S; ++dx)
            halo_shift(s, A, Bh, dx, dy, c_out + (size_t)(dy + S) * K + (dx + S), n_out + (size_t)(dy + S) * K + (dx + S));
}

/* cosine at a shift as the exact rational num/den of its square:
   both windows empty -> 1, exactly one empty -> 0, else c^2 / (|A| n_B) */
static void halo_sim2(int64_t c, int64_t pa, int64_t nb, unsigned __int128 *num, unsigned __int128 *den) {
    if (pa == 0 || nb == 0) {
        *num = (pa == 0 && nb == 0) ? 1 : 0;
        *den = 1;
    } else {
        *num = (unsigned __int128)c * (unsigned __int128)c;
        *den = (unsigned __int128)pa * (unsigned __int128)nb;
    }
}

/*
 * Cosine pair test with re-extraction (Sec. 2.1 and Eq. 2): the
 * representative A keeps its window, the member's window moves with the
 * shift s, |dx|, |dy| <= S, so content from B's halo enters it, and its norm
 * is the pixel count n_B(s) of the moved window.  sim(s) = c(s) /
 * sqrt(|A| n_B(s)); the best shift maximises sim (exact rational
 * comparison; ties: smaller |dx| + |dy|, then dy, then dx); pass iff
 * c* > 0 and den^2 c*^2 > num^2 |A| n_B(s*), or both windows are empty at
 * s*.  No gates (the lossless bounds assume fixed norms).  The record's pad
 * holds n_B(s*).  Needs orc_set_add_halo.
 */
void orc_halo_pair(const orc_set *s, int a, int b, const orc_params *P, orc_rec *out) {
    memset(out, 0, sizeof(*out));
    out->a = (uint32_t)a; out->b = (uint32_t)b; out->mode = ORC_MODE_COSINE;
    int N = s->N, S = s->S, NH = N + 2 * S;
    const uint8_t *A = s->img + (size_t)a * N * N, *Bh = s->himg + (size_t)b * NH * NH;
    int64_t pa = s->pop[a];
    int have = 0, bdx = 0, bdy = 0;
    int64_t bc = 0, bn = 0;
    unsigned __int128 bnum = 0, bden = 1;
    for (int dy = -S; dy <= S; ++dy)
        for (int dx = -S; dx <= S; ++dx) {
            int64_t c, nb;
            halo_shift(s, A, Bh, dx, dy, &c, &nb);
            unsigned __int128 num, den;
            halo_sim2(c, pa, nb, &num, &den);
            int take = 0;
            if (!have) take = 1;
            else {
                unsigned __int128 l = num * bden, r = bnum * den;
                if (l != r) take = l > r;
                else {
                    int l1 = abs(dx) + abs(dy), l2 = abs(bdx) + abs(bdy);
                    if (l1 != l2) take = l1 < l2;
                    else if (dy != bdy) take = dy < bdy;
                    else take = dx < bdx;
                }
            }
            if (take) {
                have = 1; bdx = dx; bdy = dy; bc = c; bn = nb; bnum = num; bden = den;
            }
        }
    out->dx_dbu = bdx * s->p;
    out->dy_dbu = bdy * s->p;
    out->score = bc;
    out->pad = (int32_t)bn;
    out->flags = ORC_F_ALIGNED;
    if (pa == 0 && bn == 0) {
        out->sim = 1.0;
        out->pass = 1;
        out->flags |= ORC_F_EMPTY;
    } else if (pa == 0 || bn == 0) {
        out->sim = 0.0;
    } else {
        out->sim = (double)bc / sqrt((double)pa * (double)bn);
        unsigned __int128 l = (unsigned __int128)P->cos_den * P->cos_den * (unsigned __int128)bc * (unsigned __int128)bc;
        unsigned __int128 r = (unsigned __int128)P->cos_num * P->cos_num * (unsigned __int128)pa * (unsigned __int128)bn;
        out->pass = bc > 0 && l > r;
    }
}

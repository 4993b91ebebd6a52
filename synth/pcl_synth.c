/*
 * Seeded synthetic Manhattan clip generator.
 *
 * This file only places rectangles: it holds none of the similarity
 * arithmetic (no rasterisation, no correlation, no shifts, no gates).  It is
 * the one module that both the CPU oracle and the CUDA path consume, so that
 * both see identical inputs.
 *
 * Workload shape (stands in for the contest benchmark of the paper, Sec. 4.1,
 * which is not available): a clip is a W x W dbu window of axis-aligned
 * rectangles with integer dbu coordinates (design layer of Sec. 2.1).
 *   - seed clips: R ~ U{min_rects..max_rects} rectangles, sides on a `grid`
 *     dbu grid in [min_side, max_side], positions on the same grid, placed
 *     without overlap and at least `spacing` dbu apart, on the extended region
 *     [-margin, W + margin)^2, then cut to the window [0, W)^2 (or, with a
 *     halo h, to [-h, W + h)^2: the clip then carries the layout around its
 *     window);
 *   - perturbed copies: a uniformly drawn seed, every rectangle edge moved by
 *     U{-jitter..jitter} dbu, the whole clip moved by U{-shift..shift} dbu per
 *     axis, then cut to the window;
 *   - independent clips: fresh seeds that no copy refers to.
 * The clip order is a seeded permutation of (seeds, copies, independents).
 *
 * Randomness: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), one stream per generated clip derived from
 * (cfg seed, role, index).  Integer-only, so x86 and Arm produce identical
 * bytes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct pcl_synth_cfg {
    uint64_t seed;
    uint32_t n_clips;     /* total clips */
    uint32_t n_seeds;     /* seed clips (appear themselves, and are copied) */
    uint32_t n_copies;    /* perturbed copies of seeds */
    int32_t window_dbu;   /* W */
    int32_t margin_dbu;   /* extended generation region margin (marker half-width) */
    int32_t min_rects, max_rects;
    int32_t min_side, max_side, grid;
    int32_t spacing;      /* minimum gap between rectangles of one seed */
    int32_t edge_jitter;  /* per-edge perturbation of copies, +/- dbu */
    int32_t shift_max;    /* whole-clip perturbation of copies, +/- dbu */
    int32_t halo_dbu;     /* rectangles are cut to [-halo, W + halo)^2 (0: to the window) */
} pcl_synth_cfg;

static uint64_t sm64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* uniform integer in [lo, hi] (inclusive); modulo bias is below 2^-40 here */
static int64_t uni(uint64_t *s, int64_t lo, int64_t hi) {
    uint64_t span = (uint64_t)(hi - lo + 1);
    return lo + (int64_t)(sm64(s) % span);
}

static uint64_t stream_of(uint64_t seed, uint64_t role, uint64_t idx) {
    uint64_t s = seed ^ (role * 0xD1B54A32D192ED03ull);
    uint64_t a = sm64(&s);
    s = a ^ (idx * 0x8CB92BA72F3D8DD7ull);
    (void)sm64(&s);
    return s;
}

typedef struct { int32_t x0, y0, x1, y1; } rect_t;

static int floor_div(int a, int b) { /* b > 0 */
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
static int ceil_div(int a, int b) { return -floor_div(-a, b); }

/* rectangles of one seed on the extended region; returns count */
static int gen_seed(const pcl_synth_cfg *c, uint64_t st, rect_t *out, int cap) {
    int target = (int)uni(&st, c->min_rects, c->max_rects);
    if (target > cap) target = cap;
    int n = 0;
    int lo = -c->margin_dbu, hi = c->window_dbu + c->margin_dbu;
    int gmin = (c->min_side + c->grid - 1) / c->grid, gmax = c->max_side / c->grid;
    int tries = 0, max_tries = 400 * (target + 1);
    while (n < target && tries < max_tries) {
        ++tries;
        int w = c->grid * (int)uni(&st, gmin, gmax);
        int h = c->grid * (int)uni(&st, gmin, gmax);
        /* grid positions k*grid with lo <= k*grid and k*grid + side <= hi */
        int kx0 = ceil_div(lo, c->grid), ky0 = kx0;
        int kx1 = floor_div(hi - w, c->grid);
        int ky1 = floor_div(hi - h, c->grid);
        if (kx1 < kx0 || ky1 < ky0) continue;
        rect_t r;
        r.x0 = c->grid * (int)uni(&st, kx0, kx1);
        r.y0 = c->grid * (int)uni(&st, ky0, ky1);
        r.x1 = r.x0 + w;
        r.y1 = r.y0 + h;
        int ok = 1;
        for (int i = 0; i < n && ok; ++i) {
            const rect_t *q = &out[i];
            int apart = (r.x1 + c->spacing <= q->x0) || (q->x1 + c->spacing <= r.x0) ||
                        (r.y1 + c->spacing <= q->y0) || (q->y1 + c->spacing <= r.y0);
            if (!apart) ok = 0;
        }
        if (ok) out[n++] = r;
    }
    return n;
}

/* cut to [lo, hi)^2 and append non-empty rectangles; returns appended count */
static int cut_append(const rect_t *in, int n, int lo, int hi, int32_t *dst) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        int x0 = in[i].x0 < lo ? lo : in[i].x0;
        int y0 = in[i].y0 < lo ? lo : in[i].y0;
        int x1 = in[i].x1 > hi ? hi : in[i].x1;
        int y1 = in[i].y1 > hi ? hi : in[i].y1;
        if (x0 < x1 && y0 < y1) {
            dst[4 * m + 0] = x0; dst[4 * m + 1] = y0;
            dst[4 * m + 2] = x1; dst[4 * m + 3] = y1;
            ++m;
        }
    }
    return m;
}

/*
 * Generate cfg->n_clips clips.
 *   rect_off  [n_clips + 1]  out: clip i owns rects[rect_off[i] .. rect_off[i+1])
 *   rects     [4 * rect_cap] out: x0, y0, x1, y1 (window-relative dbu)
 *   label     [n_clips]      out: seed index the clip derives from, or -1
 * Returns the total rectangle count, or -1 if rect_cap is too small / the
 * configuration is invalid.
 */
int64_t pcl_synth_generate(const pcl_synth_cfg *cfg, uint32_t *rect_off, int32_t *rects,
                           int64_t rect_cap, int32_t *label) {
    const pcl_synth_cfg *c = cfg;
    if (c->n_seeds + c->n_copies > c->n_clips) return -1;
    if (c->n_copies > 0 && c->n_seeds == 0) return -1;
    if (c->grid <= 0 || c->min_side <= 0 || c->max_side < c->min_side) return -1;
    if (c->min_rects < 0 || c->max_rects < c->min_rects) return -1;
    int cap = c->max_rects;
    rect_t *seedbuf = (rect_t *)malloc(sizeof(rect_t) * (size_t)cap * (c->n_seeds ? c->n_seeds : 1));
    int *seedn = (int *)malloc(sizeof(int) * (c->n_seeds ? c->n_seeds : 1));
    rect_t *tmp = (rect_t *)malloc(sizeof(rect_t) * (size_t)(cap > 0 ? cap : 1));
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * (c->n_clips ? c->n_clips : 1));
    if (!seedbuf || !seedn || !tmp || !perm) {
        free(seedbuf); free(seedn); free(tmp); free(perm);
        return -1;
    }
    for (uint32_t s = 0; s < c->n_seeds; ++s)
        seedn[s] = gen_seed(c, stream_of(c->seed, 1, s), seedbuf + (size_t)s * cap, cap);

    /* seeded permutation of generation slots -> output positions */
    for (uint32_t i = 0; i < c->n_clips; ++i) perm[i] = i;
    {
        uint64_t st = stream_of(c->seed, 4, 0);
        for (uint32_t i = c->n_clips; i > 1; --i) {
            uint32_t j = (uint32_t)uni(&st, 0, i - 1);
            uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
        }
    }
    /* slot k (generation order) is written at output position perm[k]; emit
       in output order by inverting the permutation */
    uint32_t *inv = (uint32_t *)malloc(sizeof(uint32_t) * (c->n_clips ? c->n_clips : 1));
    if (!inv) { free(seedbuf); free(seedn); free(tmp); free(perm); return -1; }
    for (uint32_t k = 0; k < c->n_clips; ++k) inv[perm[k]] = k;

    int64_t total = 0;
    const int lo = -c->halo_dbu, hi = c->window_dbu + c->halo_dbu;
    for (uint32_t pos = 0; pos < c->n_clips; ++pos) {
        uint32_t k = inv[pos];
        rect_off[pos] = (uint32_t)total;
        if (total + cap > rect_cap) { total = -1; break; }
        int m = 0;
        if (k < c->n_seeds) {
            m = cut_append(seedbuf + (size_t)k * cap, seedn[k], lo, hi, rects + 4 * total);
            label[pos] = (int32_t)k;
        } else if (k < c->n_seeds + c->n_copies) {
            uint64_t st = stream_of(c->seed, 2, k);
            uint32_t s = (uint32_t)uni(&st, 0, c->n_seeds - 1);
            const rect_t *src = seedbuf + (size_t)s * cap;
            int n = seedn[s];
            int tx = (int)uni(&st, -c->shift_max, c->shift_max);
            int ty = (int)uni(&st, -c->shift_max, c->shift_max);
            for (int i = 0; i < n; ++i) {
                rect_t r = src[i];
                r.x0 += (int)uni(&st, -c->edge_jitter, c->edge_jitter);
                r.x1 += (int)uni(&st, -c->edge_jitter, c->edge_jitter);
                r.y0 += (int)uni(&st, -c->edge_jitter, c->edge_jitter);
                r.y1 += (int)uni(&st, -c->edge_jitter, c->edge_jitter);
                if (r.x1 <= r.x0) r.x1 = r.x0 + 1;
                if (r.y1 <= r.y0) r.y1 = r.y0 + 1;
                r.x0 += tx; r.x1 += tx; r.y0 += ty; r.y1 += ty;
                tmp[i] = r;
            }
            m = cut_append(tmp, n, lo, hi, rects + 4 * total);
            label[pos] = (int32_t)s;
        } else {
            int n = gen_seed(c, stream_of(c->seed, 3, k), tmp, cap);
            m = cut_append(tmp, n, lo, hi, rects + 4 * total);
            label[pos] = -1;
        }
        total += m;
    }
    if (total >= 0) rect_off[c->n_clips] = (uint32_t)total;
    free(seedbuf); free(seedn); free(tmp); free(perm); free(inv);
    return total;
}

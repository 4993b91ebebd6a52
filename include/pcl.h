/*
 * pcl.h -- C ABI of the GB300 pairwise optimal-alignment similarity library.
 *
 * The library implements the data-parallel hot path of the layout-pattern
 * clustering method of "An Optimal Alignment-Driven Iterative Closed-Loop
 * Convergence Framework for High-Performance Ultra-Large Scale Layout Pattern
 * Clustering" (arXiv 2512.13133): rasterisation of Manhattan clips
 * (Sec. 2.2.1), the multi-stage lossless pre-screening (Sec. 3.1 stage 1),
 * FFT phase correlation with the cosine test at the optimal shift
 * (Sec. 3.2.1, Eqs. 2-5), the geometric Min-Max edge-displacement alignment
 * (Sec. 3.2.2, Eq. 6), and the surprisal lazy-greedy set cover with the
 * coarse-to-fine loop as host code (Sec. 3.3, Eqs. 7-9; Sec. 3.1 stages 2-4).
 *
 * Conventions shared by every call
 *  - Every call returns pcl_status; no C++ exception crosses the ABI.
 *    pcl_last_error(ctx) gives a message owned by the context.
 *  - "d_" pointers are device pointers (any allocator: cudaMalloc, PyTorch,
 *    ...), "h_" pointers are host pointers.  The caller owns every buffer it
 *    passes and keeps it alive until the stream has passed the call.
 *  - Device work is enqueued on the caller's stream and is asynchronous;
 *    results are valid once the stream has reached the call.  Calls that
 *    return counts write them to device memory for the same reason.
 *  - A context is used by one host thread at a time.
 *  - Geometry is integer dbu.  A clip is a W x W window; its rectangles
 *    (x0, y0, x1, y1) are window-relative with x0 < x1, y0 < y1 (results for
 *    a clip holding a degenerate rectangle are unspecified; no call faults on
 *    one).  Manhattan polygons enter as rectangle decompositions.
 *  - Raster: N = W / p pixels per side; pixel (i, j) is 1 iff its centre
 *    (p*i + p/2, p*j + p/2) lies in some rectangle (half-open), i.e. the
 *    union of the rectangles sampled at pixel centres.
 *  - Shift: s = (dx, dy) moves the member B onto the representative A;
 *    c(s) = sum_x A(x) B(x - s) counts overlapping pixels (B is zero outside
 *    its window).  Shifts are searched over the marker window
 *    |dx|, |dy| <= S = M / p and reported in dbu.
 */
#ifndef PCL_H
#define PCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pcl_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum pcl_status {
    PCL_OK = 0,
    PCL_ERR_INVALID = 1,     /* bad argument or parameter combination */
    PCL_ERR_OOM = 2,         /* a library-owned allocation failed */
    PCL_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    PCL_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out */
    PCL_ERR_BUSY = 5,        /* output capacity too small / not admitted */
    PCL_ERR_UNSUPPORTED = 6  /* valid request outside what the kernels cover */
} pcl_status;

enum { PCL_MODE_COSINE = 1, PCL_MODE_EDGE = 2 };
/* cosine engines: FFT phase correlation (Sec. 3.2.1), or the direct windowed
   correlation on tensor cores with FP16 (TC_DIRECT) or E4M3 (TC_DIRECT_FP8)
   0/1 operands and FP32 accumulation -- both exact for 0/1 pixels */
enum {
    PCL_ENGINE_FFT_PCM = 0,
    PCL_ENGINE_TC_DIRECT = 1,      /* tensor cores, FP16 operands */
    PCL_ENGINE_TC_DIRECT_FP8 = 2,  /* tensor cores, E4M3 operands */
    PCL_ENGINE_XYSEP = 3,
    PCL_ENGINE_TC_DIRECT_BF16 = 4, /* tensor cores, BF16 operands */
    PCL_ENGINE_EXACT_SCAN = 5      /* bound-pruned popcount scan of the window (N = 128, 256, 512) */
};
enum { PCL_SHIFT_EXACT_ARGMAX = 0, PCL_SHIFT_PCM_PEAK = 1 };

/* pcl_params.flags */
enum {
    PCL_P_NO_GATES = 1u << 0, /* match every listed pair without the lossless gates */
    PCL_P_NO_PCM = 1u << 1,   /* FFT engine: skip the phase-correlation surface */
    PCL_P_TOPO_HASH = 1u << 2 /* self-join candidates: lossy topological pre-screen (see pcl_candidates) */
};

/*
 * Method parameters (Sec. 2: pattern window, marker region, cosine threshold
 * T_cos of Eq. 2, edge tolerance T_edge of Sec. 2.2.2).
 *   pitch_dbu    raster pitch p (dbu per pixel)
 *   window_dbu   W, a multiple of p with N = W/p in {64, 128, 256, 512}
 *   marker_dbu   M, shift half-range, a multiple of p; S = M/p <= N/16 for
 *                the cosine engines (edge mode accepts any M >= 0)
 *   cos_num/den  T_cos = num/den as an exact rational, 0 < num < den <= 65535
 *   edge_tol_dbu T_edge >= 0 ("must not exceed")
 *   cos_engine   PCL_ENGINE_*; shift_rule PCL_SHIFT_*
 *   near_band    |sim - T| below which the cosine is re-evaluated in FP64
 *   flags        PCL_P_*
 */
typedef struct pcl_params {
    int32_t pitch_dbu;
    int32_t window_dbu;
    int32_t marker_dbu;
    uint32_t cos_num;
    uint32_t cos_den;
    int32_t edge_tol_dbu;
    uint32_t cos_engine;
    uint32_t shift_rule;
    float near_band;
    uint32_t flags;
} pcl_params;

typedef struct pcl_pair {
    uint32_t a, b; /* representative index (set A), member index (set B) */
} pcl_pair;

/* record flags: low 4 bits = rejecting gate (0 = none) */
enum {
    PCL_GATE_NONE = 0,
    PCL_GATE_G1_AREA = 1,     /* sqrt(min|A|,|B| / max) <= T */
    PCL_GATE_G2_PROFILE = 2,  /* row/column projection bound */
    PCL_GATE_G3_DENSITY = 3,  /* 16x16 block-density bound */
    PCL_GATE_E1_MATCH = 4,    /* no polygon correspondence at the pre-alignment */
    PCL_GATE_E2_BBOX = 5,     /* bbox size differs by more than 2*tol */
    PCL_GATE_T0_TOPO = 6,     /* topological classes differ (lossy pre-screen, PCL_P_TOPO_HASH) */
    PCL_GATE_UNSUPPORTED = 14, /* size class outside the engine's range (no work done) */
    PCL_GATE_BAD_INDEX = 15,  /* pair index outside its clip set (no work done) */
    PCL_F_NEAR_BAND = 1u << 4,
    PCL_F_FFT_GUARD = 1u << 5,   /* FFT residual too large: exact scan used */
    PCL_F_PCM_AGREES = 1u << 6,  /* phase-correlation peak == exact argmax */
    PCL_F_EDGE_VERIFY_FAIL = 1u << 7,
    PCL_F_EMPTY = 1u << 8,       /* both clips empty: similar by definition */
    PCL_F_ALIGNED = 1u << 9      /* the pair reached the alignment engine */
};

/*
 * One record per matched pair (40 bytes).
 *   cosine: dx/dy = best shift (dbu) applied to b, sim = c_best / sqrt(|A||B|) (FP32,
 *           FP64-evaluated inside the near band), score = c_best (overlap pixels),
 *           pcm_dx/dy = phase-correlation peak (dbu)
 *   edge:   dx/dy = Min-Max translation T (dbu), sim = score = max(E_x, E_y)
 *   pass:   the exact decision (integer rule), mode: PCL_MODE_*
 */
typedef struct pcl_record {
    uint32_t a, b;
    int32_t dx_dbu, dy_dbu;
    float sim;
    uint32_t score;
    int32_t pcm_dx_dbu, pcm_dy_dbu;
    uint16_t flags;
    uint8_t pass;
    uint8_t mode;
    uint32_t reserved;
} pcl_record;

/*
 * A clip set: the caller allocates every buffer (device memory, sizes from
 * pcl_clipset_sizes) and fills rect_off/rects; the library fills the rest.
 * rects, bits, esig and occ must start on 16-byte boundaries (cudaMalloc and
 * PyTorch allocations do); calls taking a clip set return PCL_ERR_INVALID
 * otherwise.
 *   rect_off [n+1] u32   clip i owns rects[4*rect_off[i] .. 4*rect_off[i+1])
 *   rects    [4R]  i32   x0, y0, x1, y1 (window-relative dbu)
 *   bits     [n][N][N/64] u64   raster rows; bit t of word w = pixel 64w+t
 *   pop      [n] u32     |A| (ones of the raster)
 *   prof     [n][2N] u16 row counts r(j), then column counts q(i)
 *   blk      [n][2*nb*nb] u16  16x16 block counts, then their neighbourhood
 *                        sums over (2*ceil(S/16)+1)^2 blocks (nb = N/16);
 *                        block (by, bx) at position ((by%4)*4 + bx%4) * q*q
 *                        + (by/4)*q + bx/4, q = nb/4 (spread blocks first)
 *   esig     [n][8] i32  edge signature: n_rects, has_x, lo_x, hi_x, has_y,
 *                        lo_y, hi_y, touches_border (non-border edges only)
 *   occ      [n][64] u64 64 x 64 occupancy grid of the rectangles (cell side
 *                        W/64 dbu; bit cx of row cy set iff some rectangle's
 *                        interior meets the cell), for the edge screen
 *   rorder   [R] u16     per clip, local rectangle indices by ascending area
 *                        (ties by index), parallel to rects
 *   spec     [n][L][Ls] float2 or NULL   cached R2C spectrum of the raster
 *                        zero-padded to L = 9N/8 (rows ky, columns kx < L/2+1)
 *   spec_state [n] u8 or NULL            1 once spec[i] holds the spectrum
 */
typedef struct pcl_clipset {
    uint32_t n_clips;
    uint32_t reserved;
    const uint32_t *rect_off;
    const int32_t *rects;
    uint64_t *bits;
    uint32_t *pop;
    uint16_t *prof;
    uint16_t *blk;
    int32_t *esig;
    uint64_t *occ;
    uint16_t *rorder;
    void *spec;
    uint8_t *spec_state;
} pcl_clipset;

/* bytes of each clip-set buffer for n clips holding R rectangles in total
   (spec may be sized 0 by the caller when the cosine FFT engine is not used) */
typedef struct pcl_clipset_sizes {
    uint64_t bits, pop, prof, blk, esig, occ, rorder, spec, spec_state;
    int32_t N, S, L, Ls; /* raster side, shift half-range, FFT side, FFT row stride */
} pcl_clipset_sizes;

typedef struct pcl_ctx pcl_ctx;

/* ---- context ----------------------------------------------------------- */

/* Create a context bound to CUDA device `device` (made current on every
   call).  Errors: PCL_ERR_INVALID (NULL out / no such device). */
pcl_status pcl_create(pcl_ctx **out, int device);
/* Destroy; frees the context's grow-only device workspace.  NULL is a no-op. */
void pcl_destroy(pcl_ctx *ctx);
/* Message of the last failed call on ctx ("" if none); owned by ctx. */
const char *pcl_last_error(const pcl_ctx *ctx);
const char *pcl_status_string(pcl_status s);

/* Check a parameter block (rules listed at pcl_params). */
pcl_status pcl_params_validate(const pcl_params *P);

/* Buffer sizes of a clip set of n clips with R rectangles under P.
   Errors: PCL_ERR_INVALID. */
pcl_status pcl_clipset_sizes_get(const pcl_params *P, uint32_t n_clips, uint64_t n_rects,
                                 pcl_clipset_sizes *out);

/* ---- a1: rasterisation + signatures (Sec. 2.2.1 step 1) --------------------
   Fills bits, pop, prof, blk, esig, occ, rorder of every clip from
   rect_off/rects and clears spec_state.  One CTA per clip.  Errors: PCL_ERR_INVALID (params or
   NULL buffer), PCL_ERR_CUDA (launch). */
pcl_status pcl_rasterize(pcl_ctx *ctx, const pcl_params *P, pcl_clipset *cs, pcl_stream stream);

/* ---- a3: forward FFT cache (Sec. 3.2.1, Eq. 3) ---------------------------
   Computes spec[i] for every clip i with spec_state[i] == 0 (or, with
   d_list != NULL, for the n_list listed clips) and sets spec_state[i] = 1.
   Requires cs->spec and cs->spec_state.  Errors: PCL_ERR_INVALID,
   PCL_ERR_UNSUPPORTED (S > N/16), PCL_ERR_CUDA. */
pcl_status pcl_spectra(pcl_ctx *ctx, const pcl_params *P, pcl_clipset *cs, const uint32_t *d_list,
                       uint32_t n_list, pcl_stream stream);

/* ---- a2: lossless pre-screening + candidate generation (Sec. 3.1 stage 1) --
   Emits every pair that no gate of `mode` rejects (Sec. 2.3: every pair of
   patterns is a candidate before the screening).
   b == NULL: self-join of a, pairs (i, j) with i < j.
   b != NULL: every pair (i, j) of clip i of a and clip j of b (a query set
     against a library, say); a and b are clip sets of the same parameters P.
   COSINE: area-sorted band join (exactly the G1 survivors: a contiguous band
   of the other set's area order), then G3 density and G2 profile bounds.
   EDGE: every pair, E2 bbox then E1 correspondence at the pre-alignment
   (each polygon of the smaller clip, smallest first, is first checked
   against the other clip's occupancy grid: no occupied cell under it means
   no overlap, so E1 fails without scanning rectangles); tiles of 32 clips
   of a x 256 clips of b (or of a, for the self-join).  Pairs are written to
   d_out[0 .. min(count, cap)) in unspecified order; *d_count (u64, device)
   receives the survivor count, which may exceed cap (then re-run with a
   larger buffer).  d_gate_counts (u64[16], device, may be NULL) is
   incremented: [0] survivors, [g] pairs rejected by gate g (their sum is
   the number of pairs screened).  COSINE uses the context workspace (two
   sets: about 16 (N^2 + 2) + 16 |a| + 8 |b| bytes for the area orders of
   both sets and the bands of a's clips).  EDGE uses it for the list of pairs
   whose polygons all meet occupied cells, which a second kernel checks for
   the exact correspondence: 16 bytes per entry, one entry per 256 pairs
   screened, at least 65,536 and at most 2^24 entries (pairs past the list
   are checked inside the screen).  Calls that use the context workspace run
   in stream order on one stream at a time.
   With P->flags & PCL_P_TOPO_HASH (self-join only) a lossy topological
   pre-screen runs first (Sec. 3.1 stage 1 filters with topological hashing
   before the exact tests): a pair is kept only if both clips have the same
   class, the polygon count saturated at 63 (the number of connected pieces,
   which edge moves that keep the polygons apart do not change); rejected
   pairs count under PCL_GATE_T0_TOPO.  Cosine sorts the clips by (class,
   area) so that each band stays inside its class (workspace 64 times the
   area histogram); edge mode checks the classes first in the screen's
   lockstep test.  Pairs of different polygon counts that would pass are
   lost: the recall is a measured quantity, not a guarantee.
   Errors: PCL_ERR_INVALID, PCL_ERR_UNSUPPORTED (COSINE with S > N/16; the
   topological pre-screen with b != NULL), PCL_ERR_OOM (workspace),
   PCL_ERR_CUDA. */
pcl_status pcl_candidates(pcl_ctx *ctx, const pcl_params *P, uint32_t mode, const pcl_clipset *a,
                          const pcl_clipset *b, pcl_pair *d_out, uint64_t cap, uint64_t *d_count,
                          uint64_t *d_gate_counts, pcl_stream stream);

/* One shard of the self-join of pcl_candidates, for n_shards GPUs (or calls)
   sharing one clip set: shard s of S (0 <= s < S) screens a fixed subset of
   the pairs, the S subsets are disjoint and their union is every pair, so
   the union of the shards' outputs is exactly pcl_candidates' output and the
   shards' gate counts sum to its counts.  The subsets depend on clip indices
   only (every caller holds the whole clip set, in the same order):
     COSINE  pairs a < b with a mod S = s (the band join walks the
             two-sided area band of the representatives a = s, s + S, ...
             only, keeping the members b > a; the G1 count is the shard's
             pair count minus the pairs it enumerated);
     EDGE    the tiles s, s + S, s + 2S, ... of the screen's tile numbering
             (32 row clips i x 256 column clips j with i < j, numbered column
             block after column block: column block y holds row tiles
             0 .. min(8y + 8, ceil(n/32)) - 1 and starts at tile 4y(y + 1)
             while 8y <= ceil(n/32), then grows by ceil(n/32) per block).
   pcl_candidates is shard 0 of 1.  Errors: those of pcl_candidates, and
   PCL_ERR_INVALID when s >= S or S = 0, PCL_ERR_UNSUPPORTED for the
   topological pre-screen with S > 1. */
pcl_status pcl_candidates_shard(pcl_ctx *ctx, const pcl_params *P, uint32_t mode, const pcl_clipset *cs,
                                uint32_t shard, uint32_t n_shards, pcl_pair *d_out, uint64_t cap, uint64_t *d_count,
                                uint64_t *d_gate_counts, pcl_stream stream);

/* Cosine candidate generation without any device allocation (the paper has
   no counterpart; this serves callers that cannot allocate device memory,
   e.g. when another allocator owns the device's memory under a fixed budget,
   or in a service loop where cudaMalloc/cudaFree would synchronise the device
   mid-request).  Same results and arguments as pcl_candidates with
   mode = PCL_MODE_COSINE, but the scratch (area histogram, sorted order) is a
   fixed 8 MiB array in the library's device memory instead of the context
   workspace: 8 (N^2 + 2) + 8 n + 192 bytes must fit, otherwise
   PCL_ERR_INVALID with the required size in pcl_last_error.  The first call
   on a device looks up the array's device address (cudaGetSymbolAddress);
   make that first call before any stream capture.  All calls share the one
   array: calls whose work overlaps on the GPU (other streams, other host
   threads) race on it and must be serialised by the caller.
   Errors: PCL_ERR_INVALID, PCL_ERR_UNSUPPORTED (S > N/16), PCL_ERR_CUDA. */
pcl_status pcl_candidates_cosine_noalloc(pcl_ctx *ctx, const pcl_params *P, const pcl_clipset *cs,
                                         pcl_pair *d_out, uint64_t cap, uint64_t *d_count,
                                         uint64_t *d_gate_counts, pcl_stream stream);

/* ---- a4-a7: alignment + decision for listed pairs ------------------------
   One record per pair, in list order, pair (a, b) = (clip a of set A, clip b
   of set B).  Gates of the mode run first unless PCL_P_NO_GATES.
   COSINE (Sec. 3.2.1 + Eq. 2): cross-power spectrum of the cached spectra,
   one packed inverse FFT pruned to the marker window giving the phase-
   correlation surface (Eq. 5) and the correlation c(s); exact integer argmax
   with the tie order (-c, |dx|+|dy|, dy, dx); c_best verified by popcount;
   decision den^2 c_best^2 > num^2 |A||B|.  Spectra of referenced clips are
   computed first when missing (spec_state == 0).  512^2 rasters (S <= 32)
   hold no spectra: after the gates their pairs take an exact window scan
   with popcounts in shared memory (pcm fields 0, spectra not read), which
   requires shift_rule = EXACT_ARGMAX (else PCL_ERR_UNSUPPORTED).  The scan
   skips the groups of shifts whose projection-profile bound (the bound of
   gate G2: c(dx, dy) <= min(sum_y min(r_A(y), r_B(y - dy)), the same over
   the columns)) is below an overlap it has already counted, so the argmax
   and its ties are those of the full scan; pcl_stats_get reports how much of
   the window was counted.  cos_engine = PCL_ENGINE_EXACT_SCAN takes the same
   scan at 128^2 and 256^2 (S <= N/16; no spectra: spec/spec_state may be
   NULL, EXACT_ARGMAX only).
   With cos_engine = PCL_ENGINE_TC_DIRECT (FP16 operands),
   PCL_ENGINE_TC_DIRECT_BF16 (BF16 operands) or PCL_ENGINE_TC_DIRECT_FP8
   (E4M3 operands) the overlaps of every shift come
   from the tensor cores instead (a direct windowed correlation, exact for 0/1
   pixels; the L-shaped edge of the window, the row dy = S and the column
   dx = S, is counted with popcounts): pairs are grouped by representative
   (a list sorted by a, b runs fastest), no phase-correlation surface is formed
   (pcm fields 0), and the engine covers N = 64, 128 and 256 with any
   S <= N/16 (the kernel of each size correlates the window S = N/16 and the
   argmax keeps the marker's shifts) and shift_rule = EXACT_ARGMAX (else
   PCL_ERR_UNSUPPORTED).  A
   device-side wait that runs out is reported by pcl_device_error.
   With cos_engine = PCL_ENGINE_XYSEP the shift is not searched but
   synthesised by the XY-separation interval competition of Sec. 3.2.1 (2):
   polygon pairs from the pre-alignment of EDGE mode (each polygon of the
   clip with fewer polygons with its unique overlapping partner), per axis the
   pair whose edge displacements span the narrowest interval, T = its
   truncated midpoint clamped to +/-M, rounded half away from zero to the
   pixel grid; the record holds the exact overlap at that shift and the
   decision of Eq. 2 there (so it can only miss passes of the exact argmax;
   pcm fields 0; shift_rule is ignored).  Any N and S; needs esig, occ and
   rorder like EDGE mode, no spectra.  One warp per pair.
   EDGE (Sec. 2.2.2 + Eq. 6): pre-alignment, correspondence, per-axis
   d_min/d_max of matched non-border edges, T = trunc((d_min+d_max)/2)
   clamped to +/-M, E = max(T - d_min, d_max - T), re-check at T,
   pass iff E_x, E_y <= tol.
   d_n (u64, device, may be NULL): when given, only the first min(n, *d_n)
   pairs are processed, so a candidate list can be matched without reading
   its length back to the host; records past that count are not written.
   Errors: PCL_ERR_INVALID, PCL_ERR_UNSUPPORTED, PCL_ERR_CUDA. */
pcl_status pcl_match_pairs(pcl_ctx *ctx, const pcl_params *P, uint32_t mode, pcl_clipset *a,
                           pcl_clipset *b, const pcl_pair *d_pairs, uint64_t n, const uint64_t *d_n,
                           pcl_record *d_out, pcl_stream stream);

/* Limit of each bounded device-side wait of the kernels launched through ctx
   from now on, in nanoseconds (0 = the default of one second).  Only the
   tensor-core engine waits on the device (its warps hand buffers over
   through shared-memory barriers); a wait that runs out makes the kernel
   give up its work, wait (always up to one second) for the tensor-core
   operations it has in flight, release its tensor memory and return, and
   is reported by pcl_device_error (pcl_match_pairs) or as a completion
   status PCL_ERR_TIMEOUT (serving).  A limit shorter than the engine's
   normal hand-over times makes every such launch time out: tests use that
   to exercise the time-out path without any fault.  Errors:
   PCL_ERR_INVALID (NULL ctx). */
pcl_status pcl_set_wait_limit(pcl_ctx *ctx, uint64_t ns);

/* Work counters of the kernels launched through ctx since it was created or
   last reset, read synchronously (waits for the device): out[0] = the
   (dy, 8 consecutive dx) groups of shifts the exact window scan counted,
   out[1] = the groups in the windows of the pairs it aligned
   (pcl_match_pairs and serving; not the mixed batch); out[2], out[3] = the
   same for the re-extraction pair kernel (pcl_match_halo).  out[0] / out[1]
   is the fraction of the definition's work the bounds left.  reset != 0
   zeroes the counters after reading them.  out: host array of 4.  Errors:
   PCL_ERR_INVALID (NULL ctx or out), PCL_ERR_CUDA. */
pcl_status pcl_stats_get(pcl_ctx *ctx, uint64_t *out, int reset);

/* ---- NEXT: cosine with re-extraction of the member's window --------------
   Sec. 2.1 extracts a pattern as the layout around its centre, and that
   centre may lie anywhere in the marker region; read as: each clip carries
   its rectangles over [-M, W + M)^2 (the layout around its window, a halo
   of M; rectangles may extend past the window), and at the shift s the
   member's window moves with the shift, so content from the halo enters it
   and its norm is the pixel count n_B(s) of the moved window:
     c(s) = sum_x A(x) Bh(x - s), n_B(s) = sum_x Bh(x - s), x in [0, N)^2,
     sim(s) = c(s) / sqrt(|A| n_B(s))  (Eq. 2 at every shift).
   The best shift maximises sim (compared exactly as c1^2 n2 vs c2^2 n1;
   ties: smaller |dx| + |dy|, then dy, then dx); pass iff c* > 0 and
   den^2 c*^2 > num^2 |A| n_B(s*) (both windows empty: sim 1, pass).  Needs
   S <= 32 and S <= N/2.
   pcl_halo_sizes_get: bytes of the halo rasters ([n][N + 2S][ceil((N +
   2S) / 64)] u64: row j + S, bit i + S holds the pixel of centre (p i +
   p/2, p j + p/2), i, j in [-S, N + S)) and of the moved-window pixel
   counts with the pair kernel's bounds ([n][(2S + 1)^2 + 2 (N + 2S)] u32:
   n_B at index (dy + S)(2S + 1) + dx + S, then per halo row the most ones it
   has in the columns of a moved window, then per halo column the most ones
   it has in the rows of a moved window).
   pcl_rasterize_halo: fills both for every clip of cs from its rectangles
   (one CTA per clip); the window rasters of cs are not touched.
   pcl_match_halo: one record per pair (a = clip of set a, rasterised by
   pcl_rasterize; b = clip of set b with the halo buffers above), in list
   order: dx/dy the best shift (dbu), score c(s*), sim (FP32, FP64 inside
   the near band), pass, reserved = n_B(s*), flags ALIGNED (| EMPTY); no
   gates run (the lossless bounds assume fixed norms) and pcm fields are 0.
   One CTA per pair with both rasters in shared memory; groups of shifts
   are counted best first and skipped when min(row bound, column bound)^2
   n_best < c_best^2 n_B(s) for each of their shifts (a's profiles against
   b's bounds above), which leaves the chosen shift unchanged
   (pcl_stats_get reports the share counted); d_n as in pcl_match_pairs.  Errors: PCL_ERR_INVALID, PCL_ERR_UNSUPPORTED,
   PCL_ERR_CUDA. */
pcl_status pcl_halo_sizes_get(const pcl_params *P, uint32_t n_clips, uint64_t *hbits_bytes, uint64_t *norms_bytes);
pcl_status pcl_rasterize_halo(pcl_ctx *ctx, const pcl_params *P, const pcl_clipset *cs, uint64_t *d_hbits,
                              uint32_t *d_norms, pcl_stream stream);
pcl_status pcl_match_halo(pcl_ctx *ctx, const pcl_params *P, const pcl_clipset *a, const pcl_clipset *b,
                          const uint64_t *d_hbits_b, const uint32_t *d_norms_b, const pcl_pair *d_pairs, uint64_t n,
                          const uint64_t *d_n, pcl_record *d_out, pcl_stream stream);

/* Synchronises the device and reports (then clears) the context's device
   error word: PCL_ERR_TIMEOUT if a kernel's bounded wait ran out (its records
   are then incomplete), PCL_OK otherwise; *flag (may be NULL) gets the word. */
pcl_status pcl_device_error(pcl_ctx *ctx, int *flag);

/* Passing pairs of d_rec[0..min(n, *d_n)) as (a, b), order unspecified
   (d_n as in pcl_match_pairs, may be NULL); *d_count (u64, device) receives
   the count (may exceed cap).  Errors: PCL_ERR_INVALID, PCL_ERR_CUDA. */
pcl_status pcl_compact_pass(pcl_ctx *ctx, const pcl_record *d_rec, uint64_t n, const uint64_t *d_n,
                            pcl_pair *d_out, uint64_t cap, uint64_t *d_count, pcl_stream stream);

/* ---- a9: mixed batches in one persistent launch ---------------------------
   One work item per pair: clip indices within the clip set of size class
   `cls`, and the mode.  The list holds every PCL_MODE_COSINE item first
   (n_cosine of them), then the PCL_MODE_EDGE items. */
typedef struct pcl_work {
    uint32_t a, b;
    uint16_t cls;
    uint16_t mode;
} pcl_work;

/* Launch parameters picked by the autotuner: fft_radix 2 or 4 (register DFT
   of the FFT engine), ctas_per_sm (persistent CTAs per SM, 0 = as many as
   fit), items_per_warp (cosine items each warp claims and gates per round,
   1..64, 0 = 16: a CTA's round aligns the survivors of its 10 warps' claims,
   so this sets the pairs per CTA per round). */
typedef struct pcl_tuning {
    uint32_t fft_radix;
    uint32_t ctas_per_sm;
    uint32_t items_per_warp;
} pcl_tuning;

/* One record per work item, in list order, for n_classes (1..4) size classes
   (params[c], sets[c]; a class's set serves as both sides of its pairs).
   Spectra of referenced clips are computed first when missing; then a single
   persistent kernel gates the cosine items a warp at a time, aligns the
   survivors with the FFT engine of their class, and evaluates the edge items
   one per thread.  Cosine items of a 512^2 class (S <= 32) take the exact
   window scan of pcl_match_pairs instead of the FFT, so such a class needs
   no spec buffers (spec and spec_state may be NULL); with a shift_rule other
   than EXACT_ARGMAX, and in any other class with N > 256 or S > N/16, cosine
   items get flags = PCL_GATE_UNSUPPORTED.  Uses 8 bytes of the context workspace.
   Errors: PCL_ERR_INVALID, PCL_ERR_OOM, PCL_ERR_CUDA. */
pcl_status pcl_match_mixed(pcl_ctx *ctx, const pcl_params *params, pcl_clipset *sets, uint32_t n_classes,
                           const pcl_work *d_work, uint64_t n_cosine, uint64_t n, pcl_record *d_out,
                           const pcl_tuning *tune, pcl_stream stream);

/* ---- a10: serving loop ----------------------------------------------------
   Resident representative libraries, one per raster size class, and
   continuously batched query requests (cfg mode COSINE: per class the engine
   its parameters name, PCL_ENGINE_FFT_PCM, PCL_ENGINE_TC_DIRECT(_BF16,
   _FP8) or PCL_ENGINE_EXACT_SCAN (from 128^2 px), and for a 512^2 px class
   the exact window scan of pcl_match_pairs;
   EDGE: the Min-Max procedure).  pcl_server_create_classes takes n_classes
   (1..16) parameter blocks and libraries (class c: params[c], libraries[c]);
   pcl_server_create is the one-class form.  For COSINE each library must be
   rasterised (bits, pop, prof, blk) and is sorted by area at creation; with
   the FFT engine its spectra are computed too (spec/spec_state required),
   while the tensor-core engine and the exact scan read the rasters only
   (spec may be NULL: ~10.6 KB per 256^2 clip instead of ~350 KB, so
   2,000,000 library clips fit in ~21 GB).  An EDGE library needs its rasters
   and edge signatures only (esig, occ, rorder).  The server then allocates
   max_inflight request slots (one stream each, pinned staging) and one
   device arena of mem_budget bytes, shared by all classes.
   pcl_server_submit_class admits a request of n_clips query clips of size
   class `cls` (host rectangles h_rects indexed by h_rect_off, clip i owning
   rectangles h_rect_off[i] .. h_rect_off[i+1]; copied before return) when
   a slot is free and its device footprint (its clip set, candidate/record
   buffers of cand_per_query entries per clip) fits in the arena, else
   returns PCL_ERR_BUSY at once (resubmit after a poll/release); requests of
   every class compete for the same slots and memory.  pcl_server_submit is
   class 0.  A request then runs asynchronously on its stream:
   rasterisation, query x library band join with the G1/G3/G2 gates, and the
   class's engine (FFT: spectra of the referenced query clips and phase
   correlation; tensor cores: the candidates grouped by query clip through
   the direct correlation, its workspace of 20 bytes per candidate slot
   sharing the band join's; 512^2 px: the exact scan), pass compaction and
   the copies back (EDGE: every query x library pair through E2 and E1 in the
   tiled screen of pcl_candidates -- 32 query clips x 256 library clips per
   tile -- then the Min-Max record of each survivor by a whole warp).
   pcl_server_poll returns finished requests: the pass pairs as (query
   index, library index), and one pcl_record per candidate that reached the
   engine (a = query index, b = library index; shift, similarity, overlap,
   flags and decision, in unspecified order), both in server-owned host
   memory valid until pcl_server_release frees the request's slot and arena
   region.  A request whose candidates exceeded its capacity completes with
   PCL_ERR_BUSY (records and passes cover the first cap candidates), one
   whose tensor-core wait ran out (records not valid) with PCL_ERR_TIMEOUT.
   Timestamps are steady-clock nanoseconds: submit, and device completion as
   stamped by a host callback on the request's stream.  One host thread at a
   time per server.  Errors: PCL_ERR_INVALID, PCL_ERR_UNSUPPORTED (COSINE
   with S > N/16; the FFT engine with N > 256; the tensor-core engine with
   N = 512; a shift rule other than
   EXACT_ARGMAX for the tensor-core engine or a 512^2 px class; any other
   cosine engine), PCL_ERR_OOM, PCL_ERR_CUDA, PCL_ERR_BUSY (not admitted). */
typedef struct pcl_server pcl_server;

typedef struct pcl_server_cfg {
    uint32_t max_inflight;     /* request slots, 1..64 */
    uint32_t max_query_clips;  /* clips per request */
    uint64_t max_query_rects;  /* rectangles per request */
    uint32_t cand_per_query;   /* candidate capacity per query clip */
    uint32_t pass_copy;        /* passes and records copied back without a second copy */
    uint64_t mem_budget;       /* device bytes for in-flight requests */
    uint32_t mode;             /* PCL_MODE_COSINE (or 0) or PCL_MODE_EDGE */
    uint32_t reserved;
} pcl_server_cfg;

typedef struct pcl_completion {
    uint64_t request_id;
    int32_t status;        /* PCL_OK, PCL_ERR_BUSY (candidate capacity exceeded) or PCL_ERR_TIMEOUT */
    uint32_t n_queries;
    uint64_t n_candidates; /* pairs that reached the alignment engine */
    uint64_t n_pass;
    const pcl_pair *pass;  /* (query, library) pairs, valid until pcl_server_release */
    int64_t t_submit_ns, t_done_ns;
    uint32_t size_class;   /* the class the request was submitted to */
    uint32_t reserved;
    uint64_t n_records;    /* min(n_candidates, capacity) */
    const pcl_record *records; /* one per candidate, valid until pcl_server_release */
} pcl_completion;

pcl_status pcl_server_create_classes(pcl_ctx *ctx, const pcl_params *params, const pcl_clipset *libraries,
                                     uint32_t n_classes, const pcl_server_cfg *cfg, pcl_server **out);
pcl_status pcl_server_create(pcl_ctx *ctx, const pcl_params *P, const pcl_clipset *library,
                             const pcl_server_cfg *cfg, pcl_server **out);
pcl_status pcl_server_submit_class(pcl_server *srv, uint32_t cls, const uint32_t *h_rect_off,
                                   const int32_t *h_rects, uint32_t n_clips, uint64_t request_id);
pcl_status pcl_server_submit(pcl_server *srv, const uint32_t *h_rect_off, const int32_t *h_rects,
                             uint32_t n_clips, uint64_t request_id);
pcl_status pcl_server_poll(pcl_server *srv, pcl_completion *out, uint32_t cap, uint32_t *n_out);
pcl_status pcl_server_release(pcl_server *srv, uint64_t request_id);
/* requests holding a slot, and free arena bytes (admission state) */
pcl_status pcl_server_stats(pcl_server *srv, uint32_t *inflight, uint64_t *free_bytes);
/* waits for in-flight work, frees the slots, arena and library indexes */
void pcl_server_destroy(pcl_server *srv);

/* ---- a11 on the GPU: degrees and surprisal of the pass graph --------------
   For the undirected graph d_edges[0..min(n_edges, *d_n)) on n_nodes nodes
   (device pairs; d_n as in pcl_match_pairs, may be NULL): d_degree[i] (u32)
   = edges at node i, d_weight[i] (u64) = S_i = floor(2^32 / (1 + deg(i)))
   (Sec. 3.3.1, Eqs. 7-8, 32-bit fixed point), d_score[j] (u64) = S_j + sum
   of S_k over the neighbours k of j (Eq. 9 with every node uncovered: the
   scores the lazy greedy of pcl_setcover starts from).  Each listed edge
   counts once per endpoint; edges with an endpoint >= n_nodes or with
   a == b are ignored.  Integer atomics: exact and order independent.
   Errors: PCL_ERR_INVALID (NULL buffer), PCL_ERR_CUDA. */
pcl_status pcl_surprisal(pcl_ctx *ctx, const pcl_pair *d_edges, uint64_t n_edges, const uint64_t *d_n,
                         uint32_t n_nodes, uint32_t *d_degree, uint64_t *d_weight, uint64_t *d_score,
                         pcl_stream stream);

/* ---- a11: host set cover + coarse-to-fine loop (Sec. 3.3, Sec. 3.1) -------
   Surprisal lazy greedy over the undirected graph h_edges[0..n_edges) on
   n_nodes nodes: f_i = 1 + deg(i), S_i = floor(2^32 / f_i), Score_j =
   S_j + sum of S_k over uncovered neighbours (Eqs. 7-9); candidates are the
   uncovered nodes; ties: higher score, then lower index.  h_order receives
   the selected representatives in selection order (*n_selected of them),
   h_rep_of[i] the representative that first covered i.  Pure host code.
   Errors: PCL_ERR_INVALID (edge index out of range / NULL). */
pcl_status pcl_setcover(const pcl_pair *h_edges, uint64_t n_edges, uint32_t n_nodes,
                        uint32_t *h_rep_of, uint32_t *h_order, uint32_t *n_selected);

/* Coarse-to-fine loop over candidate pairs h_pairs[0..m) with per-pair
   strict and relaxed decisions (u8 0/1): each round runs the set cover on
   the relaxed graph of the remaining clips, accepts members that pass the
   strict test against their representative, lets orphans try the
   representatives so far in index order, and re-injects the rest.  Ends
   when every clip is assigned.  h_rep_of[n_nodes] out; *n_clusters,
   *n_rounds out.  Pure host code.  Errors: PCL_ERR_INVALID. */
pcl_status pcl_cluster_loop(const pcl_pair *h_pairs, const uint8_t *h_strict,
                            const uint8_t *h_relaxed, uint64_t m, uint32_t n_nodes,
                            uint32_t *h_rep_of, uint32_t *n_clusters, uint32_t *n_rounds);

#ifdef __cplusplus
}
#endif

#endif /* PCL_H */

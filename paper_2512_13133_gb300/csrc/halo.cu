// Cosine matching with re-extraction of the member's window (Sec. 2.1: a
// pattern is the layout cut out around its centre, and the centre may lie
// anywhere in the marker region; Eq. 2 at every shift).
//
// Each clip carries its rectangles over [-M, W + M)^2.  Its halo raster
// samples that region at the pixel centres p i + p/2, i in [-S, N + S): row
// j + S, bit i + S of a row of NWH = ceil((N + 2S) / 64) words.  For the
// shift s the member's window moved by s holds the halo pixels x - s,
// x in [0, N)^2, so
//   c(s)   = sum_x A(x) Bh(x - s)         (A: the representative's window)
//   n_B(s) = sum_x Bh(x - s)              (pixels of the moved window)
//   sim(s) = c(s) / sqrt(|A| n_B(s)).
// n_B depends on the member alone: halo_raster_kernel tabulates it for every
// shift once per clip (the window sums of the halo raster, as a summed-area
// table would give them), beside the halo raster itself.  halo_pair_kernel
// counts c(s) for every shift by AND + popcount with both rasters staged in
// shared memory and keeps the shift of largest sim, compared exactly as
// c1^2 n2 vs c2^2 n1 (|A| is common; products < 2^55 up to 512^2 px), ties by
// smaller |dx| + |dy|, then dy, then dx; the decision is Eq. 2's exact rule
// with n_B(s*) for |B|.  No lossless gates here: they bound c against fixed
// norms.
#include "common.cuh"
#include "ctx.h"

using pcl::cos_exceeds;
using pcl::Geo;
using pcl::make_geo;

namespace {

constexpr int kThreads = 256;

__host__ __device__ inline int halo_side(int N, int S) { return N + 2 * S; }
__host__ __device__ inline int halo_words(int N, int S) { return (N + 2 * S + 63) / 64; }
// u32 per clip in the norms buffer: n_B(s) for the K^2 shifts, then the row
// bounds hrow[NH] and the column bounds hcol[NH] of the pair kernel's pruning
__host__ __device__ inline int norms_stride(int N, int S) { return (2 * S + 1) * (2 * S + 1) + 2 * halo_side(N, S); }

// shared-memory row strides in 64-bit words, odd so that the 16 lanes of a
// half-warp reading 16 consecutive rows hit 16 different bank pairs: A's rows
// (NW words) and the halo rows (NWH words and a zero word)
__host__ __device__ inline int a_stride(int NW) { return NW | 1; }
__host__ __device__ inline int h_stride(int NWH) { return (NWH + 1) | 1; }

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int ceil_div(int a, int b) { return -floor_div(-a, b); }

// one CTA per clip: halo raster rows, then the window sums n_B(s)
__global__ void __launch_bounds__(kThreads) halo_raster_kernel(pcl_params prm, pcl_clipset cs, uint64_t *hbits,
                                                               uint32_t *norms) {
    const Geo g = make_geo(prm);
    const int N = g.N, S = g.S, p = g.p, NH = halo_side(N, S), NWH = halo_words(N, S), K = 2 * S + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *rows = reinterpret_cast<uint64_t *>(smem);                     // [NH][NWH]
    uint16_t *cnt = reinterpret_cast<uint16_t *>(rows + (size_t)NH * NWH);   // [NH][K]
    const uint32_t c = blockIdx.x;
    const int32_t *r = cs.rects + 4 * (size_t)cs.rect_off[c];
    const int nr = (int)(cs.rect_off[c + 1] - cs.rect_off[c]);
    // row t = j + S has its pixel centres at y = p j + p/2 (doubled: 2 p j + p)
    for (int t = threadIdx.x; t < NH; t += blockDim.x) {
        uint64_t w[9];
        for (int k = 0; k < NWH; ++k) w[k] = 0ull;
        const int Y2 = 2 * p * (t - S) + p;
        for (int q = 0; q < nr; ++q) {
            const int x0 = r[4 * q], y0 = r[4 * q + 1], x1 = r[4 * q + 2], y1 = r[4 * q + 3];
            if (!(2 * y0 <= Y2 && Y2 < 2 * y1)) continue;
            // columns i with 2 x0 <= 2 p i + p < 2 x1, as halo bits i + S
            int b0 = ceil_div(2 * x0 - p, 2 * p) + S, b1 = ceil_div(2 * x1 - p, 2 * p) + S;
            b0 = b0 < 0 ? 0 : b0;
            b1 = b1 > NH ? NH : b1;
            for (int k = 0; k < NWH; ++k) {
                const int lo = max(b0, 64 * k), hi = min(b1, 64 * k + 64);
                if (lo >= hi) continue;
                const int n = hi - lo, o = lo - 64 * k;
                w[k] |= (n == 64 ? ~0ull : ((1ull << n) - 1ull)) << o;
            }
        }
        for (int k = 0; k < NWH; ++k) {
            rows[(size_t)t * NWH + k] = w[k];
            hbits[((size_t)c * NH + t) * NWH + k] = w[k];
        }
    }
    __syncthreads();
    // cnt[t][dx + S]: bits of halo row t at positions [S - dx, S - dx + N)
    for (int task = threadIdx.x; task < NH * K; task += blockDim.x) {
        const int t = task / K, dx = task % K - S;
        const int lo = S - dx, hi = lo + N;
        uint32_t n = 0;
        for (int k = lo >> 6; k <= (hi - 1) >> 6; ++k) {
            uint64_t m = ~0ull;
            if (64 * k < lo) m &= ~0ull << (lo - 64 * k);
            if (64 * k + 64 > hi) m &= (hi - 64 * k) >= 64 ? ~0ull : ((1ull << (hi - 64 * k)) - 1ull);
            n += (uint32_t)__popcll(rows[(size_t)t * NWH + k] & m);
        }
        cnt[(size_t)t * K + dx + S] = (uint16_t)n;
    }
    __syncthreads();
    // n_B(dx, dy) = sum over window rows y of cnt[y - dy + S][dx]
    uint32_t *nrm = norms + (size_t)c * norms_stride(N, S);
    for (int task = threadIdx.x; task < K * K; task += blockDim.x) {
        const int dy = task / K - S, kx = task % K;
        uint32_t s = 0;
        for (int y = 0; y < N; ++y) s += cnt[(size_t)(y - dy + S) * K + kx];
        nrm[task] = s;
    }
    // bounds for the pair kernel: hrow[t] = the most ones halo row t has in
    // the N columns of a moved window (max over dx), hcol[x] = the most ones
    // halo column x has in the N rows of a moved window (max over dy: rows
    // [t0, t0 + N), t0 = S - dy = 0 .. 2S, a sliding sum)
    for (int t = threadIdx.x; t < NH; t += blockDim.x) {
        uint32_t m = 0;
        for (int k = 0; k < K; ++k) m = max(m, (uint32_t)cnt[(size_t)t * K + k]);
        nrm[K * K + t] = m;
    }
    for (int x = threadIdx.x; x < NH; x += blockDim.x) {
        const int w = x >> 6, b = x & 63;
        uint32_t win = 0;
        for (int t = 0; t < N; ++t) win += (uint32_t)((rows[(size_t)t * NWH + w] >> b) & 1ull);
        uint32_t m = win;
        for (int t0 = 1; t0 <= 2 * S; ++t0) {
            win += (uint32_t)((rows[(size_t)(t0 + N - 1) * NWH + w] >> b) & 1ull);
            win -= (uint32_t)((rows[(size_t)(t0 - 1) * NWH + w] >> b) & 1ull);
            m = max(m, win);
        }
        nrm[K * K + NH + x] = m;
    }
}

// c for 8 shifts of one row pair: A's 32-bit word w against halo bits
// [32 (w + QQ) + r, +32), r = rb + u
template <int NW32, int QQ>
__device__ __forceinline__ void halo_row_counts(const uint32_t (&a)[NW32], const uint32_t (&h)[NW32 + 4], int rb,
                                                uint32_t (&cnt)[8]) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int r = rb + u;
        uint32_t x[NW32];
#pragma unroll
        for (int w = 0; w < NW32; ++w) x[w] = a[w] & __funnelshift_r(h[w + QQ], h[w + QQ + 1], r);
        cnt[u] += pcl::popc_sum<NW32>(x);
    }
}

// sim(c1, n1) > sim(c2, n2), with |A| = pa common to both
__device__ __forceinline__ int sim_cmp(uint32_t c1, uint32_t n1, uint32_t c2, uint32_t n2, uint64_t pa) {
    uint64_t a1, d1, a2, d2;
    if (pa == 0 || n1 == 0) {
        a1 = (pa == 0 && n1 == 0) ? 1u : 0u;
        d1 = 1;
    } else {
        a1 = (uint64_t)c1 * c1;
        d1 = n1;
    }
    if (pa == 0 || n2 == 0) {
        a2 = (pa == 0 && n2 == 0) ? 1u : 0u;
        d2 = 1;
    } else {
        a2 = (uint64_t)c2 * c2;
        d2 = n2;
    }
    const uint64_t l = a1 * d2, r = a2 * d1;
    return l > r ? 1 : (l < r ? -1 : 0);
}

struct Best {
    uint32_t c, n;
    int dx, dy;
    bool valid;
};

// b1 before b2 in the order (-sim, |dx| + |dy|, dy, dx)
__device__ __forceinline__ bool before(const Best &b1, const Best &b2, uint64_t pa) {
    if (!b2.valid) return b1.valid;
    if (!b1.valid) return false;
    const int s = sim_cmp(b1.c, b1.n, b2.c, b2.n, pa);
    if (s) return s > 0;
    const int l1 = abs(b1.dx) + abs(b1.dy), l2 = abs(b2.dx) + abs(b2.dy);
    if (l1 != l2) return l1 < l2;
    if (b1.dy != b2.dy) return b1.dy < b2.dy;
    return b1.dx < b2.dx;
}

// one CTA per pair (CTAs stride the list)
template <int NW>
__global__ void __launch_bounds__(kThreads, NW >= 8 ? 2 : 4) halo_pair_kernel(pcl_params prm, pcl_clipset A, pcl_clipset B,
                                                             const uint64_t *__restrict__ hbits,
                                                             const uint32_t *__restrict__ norms, const pcl_pair *pairs,
                                                             uint64_t npairs, const unsigned long long *d_n,
                                                             pcl_record *out, unsigned long long *stats) {
    constexpr int N = 64 * NW;
    const Geo g = make_geo(prm);
    const int S = g.S, NH = halo_side(N, S), NWH = halo_words(N, S), K = 2 * S + 1, KK = K * K;
    const int RW = NWH + 1;  // halo row words read: NWH and one zero word of padding
    const int SA = a_stride(NW), SH = h_stride(NWH);  // row strides in shared memory
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sa = reinterpret_cast<uint64_t *>(smem);          // [N][SA]
    uint64_t *sh = sa + (size_t)N * SA;                         // [NH][SH]
    uint32_t *sn = reinterpret_cast<uint32_t *>(sh + (size_t)NH * SH);  // [K*K]
    Best *wb = reinterpret_cast<Best *>(sn + ((KK + 3) & ~3));  // [warps]
    unsigned long long *order = reinterpret_cast<unsigned long long *>(wb + kThreads / 32);  // [1024] sort keys
    unsigned long long *bestcn = order + 1024;                  // best (c << 32 | n) so far
    uint32_t *hbd = reinterpret_cast<uint32_t *>(bestcn + 1);   // [2 NH]: hrow, hcol of B
    uint32_t *rhb = hbd + 2 * NH, *chb = rhb + K;               // [K] Rh(dy), [K] Ch(dx)
    uint32_t *ntasks_done = chb + K;                            // [1]
    uint16_t *prA = reinterpret_cast<uint16_t *>(ntasks_done + 1);  // [2N]: A's row, column counts
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (d_n && *d_n < npairs) npairs = *d_n;
    for (uint64_t pid = blockIdx.x; pid < npairs; pid += gridDim.x) {
        const pcl_pair pr = pairs[pid];
        pcl_record rec{};
        rec.a = pr.a;
        rec.b = pr.b;
        rec.mode = PCL_MODE_COSINE;
        if (pr.a >= A.n_clips || pr.b >= B.n_clips) {
            if (threadIdx.x == 0) {
                rec.flags = PCL_GATE_BAD_INDEX;
                out[pid] = rec;
            }
            continue;
        }
        __syncthreads();  // the previous pair's buffers are no longer read
        const uint64_t *ga = A.bits + (size_t)pr.a * N * NW;
        const uint64_t *gh = hbits + (size_t)pr.b * NH * NWH;
        for (int t = threadIdx.x; t < N * NW; t += blockDim.x) sa[(t / NW) * SA + t % NW] = __ldg(ga + t);
        for (int t = threadIdx.x; t < NH * RW; t += blockDim.x) {
            const int row = t / RW, k = t % RW;
            sh[row * SH + k] = k < NWH ? __ldg(gh + (size_t)row * NWH + k) : 0ull;
        }
        const uint32_t *gn = norms + (size_t)pr.b * norms_stride(N, S);
        for (int t = threadIdx.x; t < KK; t += blockDim.x) sn[t] = __ldg(gn + t);
        for (int t = threadIdx.x; t < 2 * NH; t += blockDim.x) hbd[t] = __ldg(gn + KK + t);
        for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) prA[t] = __ldg(A.prof + (size_t)pr.a * 2 * N + t);
        if (threadIdx.x == 0) {
            *bestcn = 0ull;
            *ntasks_done = 0u;
        }
        __syncthreads();
        const uint64_t pa = A.pop[pr.a];
        // Upper bounds of c(s): A's row y meets halo row y - dy + S in at most
        // min(r_A(y), hrow) ones, so c(dx, dy) <= Rh(dy) = sum_y min(r_A(y),
        // hrow(y - dy + S)), and c(dx, dy) <= Ch(dx) over the columns; with the
        // moved-window count n_B(s), sim(s) <= min(Rh, Ch) / sqrt(|A| n_B(s)).
        for (int v = warp; v < 2 * K; v += nwarps) {
            const bool col = v >= K;
            const int d = (col ? v - K : v) - S;
            const uint16_t *pa_ = prA + (col ? N : 0);
            const uint32_t *hb_ = hbd + (col ? NH : 0);
            uint32_t sum = 0;
            for (int y = lane; y < N; y += 32) sum += min((uint32_t)pa_[y], hb_[y - d + S]);
            sum = __reduce_add_sync(0xffffffffu, sum);
            if (lane == 0) (col ? chb : rhb)[d + S] = sum;
        }
        __syncthreads();
        Best best{0, 0, 0, 0, false};
        // warp task: (dy, 8 consecutive sd = S - dx starting at a multiple of
        // 8); lanes take rows y and count the 8 shifts from registers as
        // 32-bit words: A's word w lines up with halo bits [32 w + sd, +32),
        // which start in halo word w + sd / 32, the same word for the 8
        // shifts of a task
        const int nch = (2 * S) / 8 + 1, ntask = K * nch;
        // a task can be skipped when every shift's bound is below the best
        // similarity found so far, (cb, nb): U^2 nb < cb^2 n_B(s), exactly in
        // integers (U^2 n < 2^54 up to 512^2); not for an empty A (sim 1
        // for an empty window)
        auto prunable = [&](int task, uint32_t cb, uint32_t nb) -> bool {
            if (pa == 0 || cb == 0) return false;
            const int dy = task / nch - S, sd0 = (task % nch) * 8;
            for (int u = 0; u < 8; ++u) {
                const int sd = sd0 + u;
                if (sd > 2 * S) break;
                const int dx = S - sd;
                const uint32_t n = sn[(dy + S) * K + dx + S];
                if (n == 0) continue;  // c = 0 there: sim 0 < the best
                const uint64_t U = min(rhb[dy + S], chb[dx + S]);
                if (U * U * nb >= (uint64_t)cb * cb * n) return false;
            }
            return true;
        };
        auto eval_task = [&](int task) {
            const int dy = task / nch - S, sd0 = (task % nch) * 8;
            const int qq = sd0 >> 5, rb = sd0 & 31;  // sd = 32 qq + rb + u, rb + u <= 31
            uint32_t cnt[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) cnt[u] = 0;
            for (int y = lane; y < N; y += 32) {
                // A's row and the halo row into registers once (RW = NW + 2
                // words for 1 <= S <= 32, NW + 1 for S = 0)
                const uint64_t *ra = sa + (size_t)y * SA;
                const uint64_t *rh = sh + (size_t)(y - dy + S) * SH;
                uint32_t a[2 * NW], h[2 * NW + 4];
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const uint64_t v = ra[w];
                    a[2 * w] = (uint32_t)v;
                    a[2 * w + 1] = (uint32_t)(v >> 32);
                }
#pragma unroll
                for (int k = 0; k < NW + 2; ++k) {
                    const uint64_t v = k < RW ? rh[k] : 0ull;
                    h[2 * k] = (uint32_t)v;
                    h[2 * k + 1] = (uint32_t)(v >> 32);
                }
                if (qq == 0) halo_row_counts<2 * NW, 0>(a, h, rb, cnt);
                else if (qq == 1) halo_row_counts<2 * NW, 1>(a, h, rb, cnt);
                else halo_row_counts<2 * NW, 2>(a, h, rb, cnt);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int sd = sd0 + u, dx = S - sd;
                const uint32_t c = __reduce_add_sync(0xffffffffu, cnt[u]);
                if (sd <= 2 * S) {
                    const Best cand{c, sn[(dy + S) * K + dx + S], dx, dy, true};
                    if (before(cand, best, pa)) best = cand;
                }
            }
        };
        // best first: tasks sorted by their largest bound of U^2 / n_B (float
        // keys, descending; ties by task index), bitonic sort in shared memory;
        // the keys only order the work, the skip test above is exact
        int nsort = 32;
        while (nsort < ntask) nsort <<= 1;
        for (int t = threadIdx.x; t < nsort; t += blockDim.x) {
            unsigned long long key = 0ull;
            if (t < ntask) {
                const int dy = t / nch - S, sd0 = (t % nch) * 8;
                float kb = 0.0f;
                for (int u = 0; u < 8 && sd0 + u <= 2 * S; ++u) {
                    const int dx = S - (sd0 + u);
                    const uint32_t n = sn[(dy + S) * K + dx + S];
                    const float U = (float)min(rhb[dy + S], chb[dx + S]);
                    if (n) kb = fmaxf(kb, U * U / (float)n);
                }
                key = ((unsigned long long)__float_as_uint(kb) << 32) | (0xffffffffu - (uint32_t)t);
            }
            order[t] = key;
        }
        __syncthreads();
        for (int k = 2; k <= nsort; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < nsort; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l > i) {
                        const unsigned long long x = order[i], y = order[l];
                        if (((i & k) == 0) ? (x < y) : (x > y)) {
                            order[i] = y;
                            order[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        for (int q = warp; q < ntask; q += nwarps) {
            const int task = (int)(0xffffffffu - (uint32_t)order[q]);
            const unsigned long long bc =
                __shfl_sync(0xffffffffu, *reinterpret_cast<volatile unsigned long long *>(bestcn), 0);
            if (prunable(task, (uint32_t)(bc >> 32), (uint32_t)bc)) continue;  // warp-uniform
            eval_task(task);
            if (lane == 0) {
                atomicAdd(ntasks_done, 1u);
                if (best.valid && best.c > 0 && best.n > 0) {  // raise the shared best to this warp's
                    unsigned long long old = *reinterpret_cast<volatile unsigned long long *>(bestcn), seen;
                    do {
                        seen = old;
                        const uint32_t c0 = (uint32_t)(seen >> 32), n0 = (uint32_t)seen;
                        if (c0 && (uint64_t)best.c * best.c * n0 <= (uint64_t)c0 * c0 * best.n) break;
                        old = atomicCAS(bestcn, seen, ((unsigned long long)best.c << 32) | best.n);
                    } while (old != seen);
                }
            }
        }
        if (lane == 0) wb[warp] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            if (stats) {
                atomicAdd(stats + 2, (unsigned long long)*ntasks_done);
                atomicAdd(stats + 3, (unsigned long long)ntask);
            }
            Best b = wb[0];
            for (int w = 1; w < nwarps; ++w)
                if (before(wb[w], b, pa)) b = wb[w];
            rec.dx_dbu = b.dx * g.p;
            rec.dy_dbu = b.dy * g.p;
            rec.score = b.c;
            rec.reserved = b.n;
            uint16_t fl = PCL_F_ALIGNED;
            float sim = 0.0f;
            if (pa == 0 && b.n == 0) {
                sim = 1.0f;
                rec.pass = 1;
                fl |= PCL_F_EMPTY;
            } else if (pa && b.n) {
                sim = (float)b.c / sqrtf((float)pa * (float)b.n);
                const float T = (float)prm.cos_num / (float)prm.cos_den;
                if (fabsf(sim - T) < prm.near_band) {
                    fl |= PCL_F_NEAR_BAND;
                    sim = (float)((double)b.c / sqrt((double)pa * (double)b.n));
                }
                rec.pass = cos_exceeds(b.c, pa, b.n, prm.cos_num, prm.cos_den) ? 1 : 0;
            }
            rec.sim = sim;
            rec.flags = fl;
            out[pid] = rec;
        }
    }
}

size_t raster_smem(const Geo &g) {
    const int NH = halo_side(g.N, g.S), NWH = halo_words(g.N, g.S), K = 2 * g.S + 1;
    return 8ull * NH * NWH + 2ull * NH * K;
}

size_t pair_smem(const Geo &g) {
    const int NH = halo_side(g.N, g.S), NWH = halo_words(g.N, g.S), K = 2 * g.S + 1;
    return 8ull * g.N * a_stride(g.nw) + 8ull * NH * h_stride(NWH) + 4ull * (((size_t)K * K + 3) & ~size_t(3)) +
           sizeof(Best) * (kThreads / 32) + 8ull * 1024 + 8 + 4ull * (2 * NH + 2 * K + 1) + 2ull * 2 * g.N + 16;
}

template <int NW>
cudaError_t launch_pair(const pcl_params &prm, const Geo &g, const pcl_clipset &a, const pcl_clipset &b,
                        const uint64_t *hb, const uint32_t *nb, const pcl_pair *pairs, uint64_t n,
                        const unsigned long long *d_n, pcl_record *out, int num_sms, unsigned long long *stats,
                        cudaStream_t st) {
    const size_t sm = pair_smem(g);
    cudaError_t e = cudaFuncSetAttribute(halo_pair_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, halo_pair_kernel<NW>, kThreads, sm);
    if (e != cudaSuccess) return e;
    const uint64_t cap = (uint64_t)num_sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    halo_pair_kernel<NW><<<(unsigned)(n < cap ? n : cap), kThreads, sm, st>>>(prm, a, b, hb, nb, pairs, n, d_n, out,
                                                                             stats);
    return cudaGetLastError();
}

pcl_status fail(pcl_ctx *ctx, pcl_status s, const char *m) {
    ctx->err = m;
    return s;
}

pcl_status cuda_fail(pcl_ctx *ctx, cudaError_t e, const char *where) {
    ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
    return PCL_ERR_CUDA;
}

bool halo_geometry_ok(const Geo &g) { return g.S <= 32 && g.S <= g.N / 2; }

}  // namespace

extern "C" {

pcl_status pcl_halo_sizes_get(const pcl_params *P, uint32_t n_clips, uint64_t *hbits_bytes, uint64_t *norms_bytes) {
    if (pcl_params_validate(P) != PCL_OK || !hbits_bytes || !norms_bytes) return PCL_ERR_INVALID;
    const Geo g = make_geo(*P);
    if (!halo_geometry_ok(g)) return PCL_ERR_UNSUPPORTED;
    *hbits_bytes = 8ull * n_clips * halo_side(g.N, g.S) * halo_words(g.N, g.S);
    *norms_bytes = 4ull * n_clips * (uint64_t)norms_stride(g.N, g.S);
    return PCL_OK;
}

pcl_status pcl_rasterize_halo(pcl_ctx *ctx, const pcl_params *P, const pcl_clipset *cs, uint64_t *d_hbits,
                              uint32_t *d_norms, pcl_stream stream) {
    if (!ctx) return PCL_ERR_INVALID;
    ctx->err.clear();
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (pcl_params_validate(P) != PCL_OK) return fail(ctx, PCL_ERR_INVALID, "pcl_rasterize_halo: invalid parameters");
    const Geo g = make_geo(*P);
    if (!halo_geometry_ok(g)) return fail(ctx, PCL_ERR_UNSUPPORTED, "pcl_rasterize_halo: needs S <= 32 and S <= N/2");
    if (!cs || (cs->n_clips && (!cs->rect_off || !cs->rects || !d_hbits || !d_norms)))
        return fail(ctx, PCL_ERR_INVALID, "pcl_rasterize_halo: NULL buffer");
    if (cs->n_clips == 0) return PCL_OK;
    const size_t sm = raster_smem(g);
    e = cudaFuncSetAttribute(halo_raster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
        halo_raster_kernel<<<cs->n_clips, kThreads, sm, (cudaStream_t)stream>>>(*P, *cs, d_hbits, d_norms);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "halo raster kernel");
}

pcl_status pcl_match_halo(pcl_ctx *ctx, const pcl_params *P, const pcl_clipset *a, const pcl_clipset *b,
                          const uint64_t *d_hbits_b, const uint32_t *d_norms_b, const pcl_pair *d_pairs, uint64_t n,
                          const uint64_t *d_n, pcl_record *d_out, pcl_stream stream) {
    if (!ctx) return PCL_ERR_INVALID;
    ctx->err.clear();
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (pcl_params_validate(P) != PCL_OK) return fail(ctx, PCL_ERR_INVALID, "pcl_match_halo: invalid parameters");
    const Geo g = make_geo(*P);
    if (!halo_geometry_ok(g)) return fail(ctx, PCL_ERR_UNSUPPORTED, "pcl_match_halo: needs S <= 32 and S <= N/2");
    if (!a || !b || (n && (!d_pairs || !d_out || !d_hbits_b || !d_norms_b)) ||
        (a->n_clips && (!a->bits || !a->pop || !a->prof)))
        return fail(ctx, PCL_ERR_INVALID, "pcl_match_halo: NULL buffer");
    if (n == 0) return PCL_OK;
    const auto *dn = reinterpret_cast<const unsigned long long *>(d_n);
    cudaStream_t st = (cudaStream_t)stream;
    switch (g.nw) {
        case 1: e = launch_pair<1>(*P, g, *a, *b, d_hbits_b, d_norms_b, d_pairs, n, dn, d_out, ctx->num_sms,
                                       ctx->d_stats, st); break;
        case 2: e = launch_pair<2>(*P, g, *a, *b, d_hbits_b, d_norms_b, d_pairs, n, dn, d_out, ctx->num_sms,
                                       ctx->d_stats, st); break;
        case 4: e = launch_pair<4>(*P, g, *a, *b, d_hbits_b, d_norms_b, d_pairs, n, dn, d_out, ctx->num_sms,
                                       ctx->d_stats, st); break;
        case 8: e = launch_pair<8>(*P, g, *a, *b, d_hbits_b, d_norms_b, d_pairs, n, dn, d_out, ctx->num_sms,
                                       ctx->d_stats, st); break;
        default: return fail(ctx, PCL_ERR_UNSUPPORTED, "pcl_match_halo: raster side");
    }
    return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "halo pair kernel");
}

}  // extern "C"

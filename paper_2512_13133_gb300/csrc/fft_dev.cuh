// Device code of the FFT phase-correlation engine (Sec. 3.2.1, Eqs. 3-5) and
// the cosine decision at the optimal shift (Eq. 2), shared by the pair kernel
// and the mixed-batch kernel.  See fft.cu for the decomposition.
#pragma once

#include "gates.cuh"

namespace pcl {
namespace fft_dev {

constexpr float kPcmEps = 1e-6f;

// slot of (item, row r, column k) in a [item][9][P + 1] padded work buffer
template <int P>
__device__ __forceinline__ int vslot(int item, int r, int k) {
    return (item * 9 + r) * (P + 1) + k;
}

__device__ __forceinline__ void build_twiddles(float2 *tw, int L, int sign) {
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)L, &s, &c);
        tw[k] = make_float2((float)c, (float)(sign * s));
    }
}

__device__ __forceinline__ float bitf(const uint64_t *rows, int nw, int y, int x) {
    return (float)((rows[y * nw + (x >> 6)] >> (x & 63)) & 1ull);
}

// ---------------------------------------------------------------- per pair
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

__device__ __forceinline__ uint32_t float_order(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <int P>
struct PairSmem {
    static constexpr int L = 9 * P, LH = L / 2 + 1, NO = P + 1;  // NO outputs per axis
    static constexpr size_t tw = 0;                                          // L float2
    static constexpr size_t out1 = tw + sizeof(float2) * L;                  // [2][NO][LH] float2
    static constexpr size_t v2 = out1 + sizeof(float2) * 2 * NO * LH;        // [NO][9][P+1] float2
    static constexpr size_t misc = v2 + sizeof(float2) * NO * 9 * (P + 1);   // keys [2][32] u64, flags [8]
    static constexpr size_t two = misc + 2 * 32 * 8 + 8 * 4;                 // [9][NO] float2: pass-1 twiddles
    static constexpr size_t bytes = two + sizeof(float2) * 9 * NO;
    // pass 1's second half accumulates in v2 ([2][NO][LH] float2 fits its
    // NO * 9 * (P + 1) entries: 2 LH = 9P + 2); surfaces reuse out1 once
    // pass 2 has read it: [2][NO][NO] float
};

// One pair on the whole CTA.  gates_done: the caller has already checked the
// pair's indices, emptiness and gates (the mixed-batch kernel gates a warp's
// worth of pairs at a time).  RADIX selects the register DFT (2 or 4).
template <int P, int RADIX = 2>
__device__ __forceinline__ void pair_body(const pcl_params &prm, const pcl_clipset &A, const pcl_clipset &B,
                                          const pcl_pair pr, pcl_record *dst, bool gates_done = false) {
    using SM = PairSmem<P>;
    constexpr int L = SM::L, LH = SM::LH, NO = SM::NO, N = 8 * P, NW = N / 64;
    constexpr int LS = (LH + 3) & ~3;
    constexpr int HW = P / 2;  // half-width of the computed window
    constexpr int CHUNKS = (LH + 31) / 32;
    const Geo g = make_geo(prm);
    const int S = g.S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *tw = reinterpret_cast<float2 *>(smem + SM::tw);
    float2 *out1 = reinterpret_cast<float2 *>(smem + SM::out1);
    float2 *v2 = reinterpret_cast<float2 *>(smem + SM::v2);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem + SM::misc);  // [2][32]
    int *flags = reinterpret_cast<int *>(smem + SM::misc + 2 * 32 * 8);                 // [8]
    float *surf = reinterpret_cast<float *>(smem + SM::out1);                           // [2][NO][NO]

    if (threadIdx.x < 8) flags[threadIdx.x] = 0;
    pcl_record rec{};
    rec.a = pr.a;
    rec.b = pr.b;
    rec.mode = PCL_MODE_COSINE;
    if (pr.a >= A.n_clips || pr.b >= B.n_clips) {
        if (threadIdx.x == 0) {
            rec.flags = PCL_GATE_BAD_INDEX;
            *dst = rec;
        }
        return;
    }
    const uint64_t pa = A.pop[pr.a], pb = B.pop[pr.b];
    if (pa == 0 && pb == 0) {
        if (threadIdx.x == 0) {
            rec.sim = 1.0f;
            rec.pass = 1;
            rec.flags = PCL_F_EMPTY;
            *dst = rec;
        }
        return;
    }
    if (!gates_done && !(prm.flags & PCL_P_NO_GATES)) {
        if (warp == 0) {
            const int gate = warp_cosine_gate(A, pr.a, B, pr.b, g, prm.cos_num, prm.cos_den, lane);
            if (lane == 0) flags[0] = gate;
        }
        __syncthreads();
        const int gate = flags[0];
        if (gate) {
            if (threadIdx.x == 0) {
                rec.flags = (uint16_t)gate;
                *dst = rec;
            }
            return;
        }
    }
    build_twiddles(tw, L, +1);
    __syncthreads();
    // pass-1 twiddles of output row o = dy + HW at step k2: w^(k2 n), n = dy mod L
    float2 *two = reinterpret_cast<float2 *>(smem + SM::two);  // [9][NO]
    for (int t = threadIdx.x; t < 9 * NO; t += blockDim.x) {
        const int k2 = t / NO, dy = t % NO - HW;
        two[t] = tw[(k2 * (dy >= 0 ? dy : L + dy)) % L];
    }
    __syncthreads();

    const float2 *fa = reinterpret_cast<const float2 *>(A.spec) + (size_t)pr.a * L * LS;
    const float2 *fb = reinterpret_cast<const float2 *>(B.spec) + (size_t)pr.b * L * LS;
    const float thr = kPcmEps * (float)pa * (float)pb;
    const float thr2 = thr * thr;
    const bool want_pcm = !(prm.flags & PCL_P_NO_PCM);

    // ---- pass 1: along ky, pruned to |dy| <= HW.  Warp task = (column
    // chunk, half of the k2 steps): the task loads both spectra of its 32
    // columns once per step, forms C = F_A conj(F_B) and from it the phase-
    // correlation R = C/|C|, and runs the P-point DFT of both; the NO outputs
    // of each signal accumulate in shared memory (out1 for the first half of
    // the k2 steps, v2 for the second, added after the pass), not in
    // registers, so that the 2P loads of a step can all be in flight.
    {
        float2 *part = v2;  // [2][NO][LH] partial sums of the second half
        constexpr int K2H = 5;  // first half: k2 = 0..4, second half: 5..8
        for (int task = warp; task < 2 * CHUNKS; task += nwarps) {
            const int half = task / CHUNKS;
            const int kx = (task % CHUNKS) * 32 + lane;
            const bool valid = kx < LH;
            float2 *dst = (half ? part : out1) + kx;  // signal s, output o at dst[(s NO + o) LH]
            const int kb = half ? K2H : 0, ke = half ? 9 : K2H;
            if (!want_pcm && valid)
                for (int o = 0; o < NO; ++o) dst[(size_t)o * LH] = make_float2(0.f, 0.f);
            for (int k2 = kb; k2 < ke; ++k2) {
                float2 c[P];
                {
                    float2 ra[P], rb[P];
#pragma unroll
                    for (int k1 = 0; k1 < P; ++k1) {
                        const int ky = 9 * k1 + k2;
                        ra[k1] = valid ? __ldg(fa + (size_t)ky * LS + kx) : make_float2(0.f, 0.f);
                        rb[k1] = valid ? __ldg(fb + (size_t)ky * LS + kx) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int k1 = 0; k1 < P; ++k1) c[k1] = cmulc(ra[k1], rb[k1]);
                }
                const float2 *w2 = two + k2 * NO;
#pragma unroll
                for (int sig = 0; sig < 2; ++sig) {  // 0: phase correlation R, 1: correlation C
                    if (sig == 0 && !want_pcm) continue;
                    float2 v[P];
#pragma unroll
                    for (int k1 = 0; k1 < P; ++k1) {
                        float2 x = c[k1];
                        if (sig == 0) {
                            const float m2 = fmaf(x.x, x.x, x.y * x.y);
                            x = (m2 > thr2) ? cscale(x, rsqrtf(m2)) : make_float2(0.f, 0.f);
                        }
                        v[k1] = x;
                    }
                    dft_p<P, +1, RADIX>(v);
                    if (valid) {
                        float2 *d = dst + (size_t)sig * NO * LH;
#pragma unroll
                        for (int o = 0; o < NO; ++o) {
                            const int dy = o - HW;
                            const int n1 = dy >= 0 ? dy : P + dy;
                            const float2 t = cmul(v[n1], w2[o]);
                            d[(size_t)o * LH] = k2 == kb ? t : cadd(d[(size_t)o * LH], t);
                        }
                    }
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * NO * LH; t += blockDim.x) out1[t] = cadd(out1[t], part[t]);
    }
    __syncthreads();
    // ---- pass 2 step 1: along kx (packed R + iC), DFT_P per (row, k2)
    for (int task = threadIdx.x; task < NO * 9; task += blockDim.x) {
        const int oy = task / 9, k2 = task % 9;
        const float2 *h1 = out1 + (size_t)oy * LH;
        const float2 *h2 = out1 + ((size_t)NO + oy) * LH;
        float2 v[P];
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            const int kx = 9 * k1 + k2;
            if (kx <= L / 2) {
                const float2 a = h1[kx], b = h2[kx];
                v[k1] = make_float2(a.x - b.y, a.y + b.x);
            } else {
                const float2 a = h1[L - kx], b = h2[L - kx];
                v[k1] = make_float2(a.x + b.y, b.x - a.y);
            }
        }
        dft_p<P, +1, RADIX>(v);
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) v2[vslot<P>(oy, k2, n1)] = v[n1];
    }
    __syncthreads();
    // ---- pass 2 step 2: outputs (dy, dx) in the computed window
    const float inv = 1.0f / ((float)L * (float)L);
    for (int task = threadIdx.x; task < NO * NO; task += blockDim.x) {
        const int oy = task / NO, ox = task % NO;
        const int dx = ox - HW;
        const int n = dx >= 0 ? dx : L + dx;
        const int n1 = dx >= 0 ? dx : P + dx;
        float2 z = make_float2(0.f, 0.f);
#pragma unroll
        for (int k2 = 0; k2 < 9; ++k2) z = cadd(z, cmul(v2[vslot<P>(oy, k2, n1)], tw[(k2 * n) % L]));
        surf[oy * NO + ox] = z.x * inv;             // r_pcm
        surf[NO * NO + oy * NO + ox] = z.y * inv;   // c~
    }
    __syncthreads();
    // ---- exact argmax (rounded correlation) and phase-correlation peak
    unsigned long long kc = 0, kp = 0;
    int guard = 0;
    for (int task = threadIdx.x; task < NO * NO; task += blockDim.x) {
        const int oy = task / NO, ox = task % NO;
        const int dx = ox - HW, dy = oy - HW;
        if (dx < -S || dx > S || dy < -S || dy > S) continue;
        const float cf = surf[NO * NO + task];
        const float ci = rintf(cf);
        if (fabsf(cf - ci) > 0.25f || ci < 0.f) guard = 1;
        const uint32_t cu = ci < 0.f ? 0u : (uint32_t)ci;
        const unsigned long long k1 = shift_key(cu, dx, dy, S);
        kc = k1 > kc ? k1 : kc;
        const unsigned long long lo = k1 & 0xffffffffull;
        const unsigned long long k2 = ((unsigned long long)float_order(surf[task]) << 32) | lo;
        kp = k2 > kp ? k2 : kp;
    }
    kc = warp_max_u64(kc);
    kp = warp_max_u64(kp);
    guard = __reduce_or_sync(0xffffffffu, guard);
    if (lane == 0) {
        keys[warp] = kc;
        keys[32 + warp] = kp;
        if (guard) atomicOr(flags + 1, 1);
    }
    __syncthreads();
    // decode best keys
    unsigned long long bc = 0, bp = 0;
    for (int w = 0; w < nwarps; ++w) {
        bc = keys[w] > bc ? keys[w] : bc;
        bp = keys[32 + w] > bp ? keys[32 + w] : bp;
    }
    auto dec = [&](unsigned long long k, int &dx, int &dy) {
        dx = S - (int)(k & 0xffu);
        dy = S - (int)((k >> 8) & 0xffu);
    };
    int sdx, sdy, pdx, pdy;
    dec(bc, sdx, sdy);
    dec(bp, pdx, pdy);
    uint32_t cbest = (uint32_t)(bc >> 32);
    int gflag = flags[1];
    const uint64_t *ba = A.bits + (size_t)pr.a * N * NW;
    const uint64_t *bbits = B.bits + (size_t)pr.b * N * NW;
    // popcount check of the chosen shift (rows spread over the whole CTA),
    // fall back on mismatch
    if (!gflag) {
        if (threadIdx.x == 0) flags[4] = 0;
        __syncthreads();
        const uint32_t part = __reduce_add_sync(
            0xffffffffu, corr_rows_partial(ba, bbits, N, NW, sdx, sdy, (int)threadIdx.x, (int)blockDim.x));
        if (lane == 0) atomicAdd(flags + 4, (int)part);
        __syncthreads();
        if (threadIdx.x == 0 && (uint32_t)flags[4] != cbest) flags[2] = 1;
        __syncthreads();
        gflag = flags[2];
    }
    __syncthreads();
    if (gflag) {
        // exact popcount scan of the whole window, one shift per warp
        const int K = 2 * S + 1;
        unsigned long long kk = 0;
        for (int t = warp; t < K * K; t += nwarps) {
            const int dy = t / K - S, dx = t % K - S;
            const uint32_t ce = warp_corr_exact(ba, bbits, N, NW, dx, dy, lane);
            const unsigned long long k1 = shift_key(ce, dx, dy, S);
            kk = k1 > kk ? k1 : kk;
        }
        if (lane == 0) keys[warp] = kk;
        __syncthreads();
        bc = 0;
        for (int w = 0; w < nwarps; ++w) bc = keys[w] > bc ? keys[w] : bc;
        dec(bc, sdx, sdy);
        cbest = (uint32_t)(bc >> 32);
    }
    // phase-correlation rule: exact overlap at the PCM peak
    int rdx = sdx, rdy = sdy;
    uint32_t cdec = cbest;
    if (prm.shift_rule == PCL_SHIFT_PCM_PEAK && want_pcm) {
        rdx = pdx;
        rdy = pdy;
        if (warp == 0) {
            const uint32_t ce = warp_corr_exact(ba, bbits, N, NW, pdx, pdy, lane);
            if (lane == 0) flags[3] = (int)ce;
        }
        __syncthreads();
        cdec = (uint32_t)flags[3];
    }
    if (threadIdx.x == 0) {
        const int p = g.p;
        rec.dx_dbu = rdx * p;
        rec.dy_dbu = rdy * p;
        rec.pcm_dx_dbu = want_pcm ? pdx * p : 0;
        rec.pcm_dy_dbu = want_pcm ? pdy * p : 0;
        rec.score = cdec;
        float sim = (pa && pb) ? (float)cdec / sqrtf((float)pa * (float)pb) : 0.0f;
        uint16_t fl = PCL_F_ALIGNED;
        if (gflag) fl |= PCL_F_FFT_GUARD;
        if (want_pcm && pdx == sdx && pdy == sdy) fl |= PCL_F_PCM_AGREES;
        const float T = (float)prm.cos_num / (float)prm.cos_den;
        if (pa && pb && fabsf(sim - T) < prm.near_band) {
            fl |= PCL_F_NEAR_BAND;
            sim = (float)((double)cdec / sqrt((double)pa * (double)pb));
        }
        rec.sim = sim;
        rec.flags = fl;
        rec.pass = cos_exceeds(cdec, pa, pb, prm.cos_num, prm.cos_den) ? 1 : 0;
        *dst = rec;
    }
}


// Exact window scan for rasters the FFT body does not cover (N = 64 NW, here
// 512²): c(s) = sum_x A(x) B(x - s) counted with AND + popcount for every shift
// |dx|, |dy| <= S (S <= SMAX <= 32) -- the definition itself, so the record is
// the oracle's.  Both rasters are staged in shared memory (2 N²/8 bytes).  Warps
// take (dy, 8 consecutive dx starting at a multiple of 8); lanes take row pairs
// (A row y, B row y - dy) as 32-bit words and count the 8 shifts of a row pair
// from registers, one funnel shift per word and shift: B's row moved by
// dx = 32 q + r is word w - q funnel-shifted by r with word w - q - 1, and q is
// the same for the 8 shifts of a task because the chunk starts at a multiple
// of 8.  No phase-correlation surface is formed (pcm fields 0).  The caller has
// checked the indices, emptiness and gates.
template <int NW32, int Q>
__device__ __forceinline__ void exact_row_counts(const uint32_t (&a)[NW32], const uint32_t (&bp)[NW32 + 3], int rb,
                                                 uint32_t (&cnt)[8]) {
    // bp[i] = B's word i - 2 (zero outside the row); B moved by 32 Q + r has
    // word w = funnel(b[w - Q - 1], b[w - Q], r) = funnel(bp[w + 1 - Q], bp[w + 2 - Q], r)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int r = rb + u;  // 0..31
        uint32_t x[NW32];
#pragma unroll
        for (int w = 0; w < NW32; ++w) x[w] = a[w] & __funnelshift_l(bp[w + 1 - Q], bp[w + 2 - Q], r);
        cnt[u] += popc_sum<NW32>(x);
    }
}

template <int NW, int SMAX>
__device__ __forceinline__ void exact_body(const pcl_params &prm, const pcl_clipset &A, const pcl_clipset &B,
                                           const pcl_pair pr, pcl_record *dst,
                                           unsigned long long *stats = nullptr) {
    static_assert(SMAX <= 32 && NW >= 2, "shift words: q in {-1, 0, 1}; rows of whole 16-byte vectors");
    constexpr int N = 64 * NW, NW32 = 2 * NW, NV = NW32 / 4;  // 32-bit words and 16-byte vectors per row
    // row stride in shared memory: an odd number of vectors, so that the 8
    // lanes of a quarter-warp reading 8 consecutive rows hit 8 bank groups
    constexpr int SV = NV | 1;
    const Geo g = make_geo(prm);
    const int S = g.S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    extern __shared__ __align__(16) unsigned char smem[];
    uint4 *sa = reinterpret_cast<uint4 *>(smem);
    uint4 *sb = sa + N * SV;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(sb + N * SV);  // [32]
    uint32_t *rbound = reinterpret_cast<uint32_t *>(keys + 32);                      // [2 SMAX + 1]: R(dy)
    uint32_t *cbound = rbound + 2 * SMAX + 1;                                         // [2 SMAX + 1]: C(dx)
    uint32_t *lbest = cbound + 2 * SMAX + 1;  // [0]: L, [1]: tasks evaluated
    uint32_t *order = lbest + 4;                                                      // [1024] sort keys
    uint16_t *prof = reinterpret_cast<uint16_t *>(order + 1024);                      // [2][2N]: A's, B's
    const uint4 *ga = reinterpret_cast<const uint4 *>(A.bits + (size_t)pr.a * N * NW);
    const uint4 *gb = reinterpret_cast<const uint4 *>(B.bits + (size_t)pr.b * N * NW);
    __syncthreads();  // the shared memory may still be read by the previous item
    for (int t = threadIdx.x; t < N * NV; t += blockDim.x) {
        const int st = (t / NV) * SV + t % NV;
        sa[st] = __ldg(ga + t);
        sb[st] = __ldg(gb + t);
    }
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
        prof[t] = __ldg(A.prof + (size_t)pr.a * 2 * N + t);
        prof[2 * N + t] = __ldg(B.prof + (size_t)pr.b * 2 * N + t);
    }
    if (threadIdx.x == 0) lbest[0] = lbest[1] = 0u;
    __syncthreads();
    const int K = 2 * S + 1;
    // Upper bounds from the projection profiles (the bound of gate G2): rows y
    // of A and y - dy of B overlap in at most min(r_A(y), r_B(y - dy)) pixels,
    // so c(dx, dy) <= R(dy) = sum_y min(r_A(y), r_B(y - dy)), and likewise
    // c(dx, dy) <= C(dx) over the columns.
    for (int v = warp; v < 2 * K; v += nwarps) {
        const bool col = v >= K;
        const int d = (col ? v - K : v) - S;
        const uint16_t *pa_ = prof + (col ? N : 0), *pb_ = prof + 2 * N + (col ? N : 0);
        uint32_t sum = 0;
        for (int y = lane; y < N; y += 32) {
            const int yb = y - d;
            if (yb >= 0 && yb < N) sum += min((uint32_t)pa_[y], (uint32_t)pb_[yb]);
        }
        sum = __reduce_add_sync(0xffffffffu, sum);
        if (lane == 0) (col ? cbound : rbound)[d + S] = sum;
    }
    __syncthreads();
    // dx chunks [8 c, 8 c + 7] for c = floor(-S / 8) .. floor(S / 8); a task
    // (dy, chunk) is bounded by min(R(dy), max of C over its shifts)
    const int c0 = -((S + 7) / 8), nch = S / 8 - c0 + 1;
    auto task_bound = [&](int task) -> uint32_t {
        const int dy = task / nch - S, dx0 = (c0 + task % nch) * 8;
        uint32_t cm = 0;
        for (int u = 0; u < 8; ++u) {
            const int dx = dx0 + u;
            if (dx >= -S && dx <= S) cm = max(cm, cbound[dx + S]);
        }
        return min(rbound[dy + S], cm);
    };
    unsigned long long best = 0ull;
    // c(s) for the 8 shifts of one task; returns their largest overlap
    auto eval_task = [&](int task) -> uint32_t {
        const int dy = task / nch - S, dx0 = (c0 + task % nch) * 8;  // -32 <= dx0 <= 32
        const int q = (dx0 + 32) / 32 - 1, rb = dx0 - 32 * q;        // dx0 = 32 q + rb, rb in {0, 8, 16, 24}
        uint32_t cnt[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) cnt[u] = 0;
        const int j0 = dy > 0 ? dy : 0, j1 = dy < 0 ? N + dy : N;
        for (int j = j0 + lane; j < j1; j += 32) {
            uint32_t a[NW32], bp[NW32 + 3];
            bp[0] = bp[1] = bp[NW32 + 2] = 0u;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const uint4 x = sa[j * SV + v], y = sb[(j - dy) * SV + v];
                a[4 * v] = x.x, a[4 * v + 1] = x.y, a[4 * v + 2] = x.z, a[4 * v + 3] = x.w;
                bp[4 * v + 2] = y.x, bp[4 * v + 3] = y.y, bp[4 * v + 4] = y.z, bp[4 * v + 5] = y.w;
            }
            if (q < 0) exact_row_counts<NW32, -1>(a, bp, rb, cnt);
            else if (q == 0) exact_row_counts<NW32, 0>(a, bp, rb, cnt);
            else exact_row_counts<NW32, 1>(a, bp, rb, cnt);
        }
        uint32_t cmax = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int dx = dx0 + u;
            const uint32_t c = __reduce_add_sync(0xffffffffu, cnt[u]);
            if (dx >= -S && dx <= S) {
                const unsigned long long k = shift_key(c, dx, dy, S);
                best = k > best ? k : best;
                cmax = max(cmax, c);
            }
        }
        return cmax;
    };
    // Best first: the tasks sorted by bound, descending (bitonic sort of
    // keys bound << 12 | 4095 - task in shared memory; ties by task index);
    // warp w takes sorted positions w, w + nwarps, ...  The first round (the
    // nwarps largest bounds) sets L, the largest overlap counted so far, and
    // every counted task raises it (shared atomic max).  A warp stops at its
    // first position whose bound is below L: the positions after it have
    // bounds no larger, and a task below L holds no shift whose overlap
    // reaches the best, so the argmax and its ties are the full scan's.
    const int ntask = K * nch;  // <= 65 x 9 = 585
    int nsort = 32;
    while (nsort < ntask) nsort <<= 1;
    for (int t = threadIdx.x; t < nsort; t += blockDim.x)
        order[t] = t < ntask ? (task_bound(t) << 12) | (uint32_t)(4095 - t) : 0u;
    __syncthreads();
    for (int k = 2; k <= nsort; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < nsort; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const uint32_t x = order[i], y = order[l];
                    if (((i & k) == 0) ? (x < y) : (x > y)) {  // descending runs first
                        order[i] = y;
                        order[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (int p = warp; p < ntask; p += nwarps) {
        const uint32_t key = order[p];
        const uint32_t lnow = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile uint32_t *>(lbest), 0);
        if ((key >> 12) < lnow) break;  // warp-uniform
        const uint32_t cm = eval_task(4095 - (int)(key & 4095u));
        if (lane == 0) {
            atomicMax(lbest, cm);
            atomicAdd(lbest + 1, 1u);
        }
    }
    if (lane == 0) keys[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (stats) {
            atomicAdd(stats, (unsigned long long)lbest[1]);
            atomicAdd(stats + 1, (unsigned long long)(K * nch));
        }
        unsigned long long bk = 0ull;
        for (int w = 0; w < nwarps; ++w) bk = keys[w] > bk ? keys[w] : bk;
        const int dx = S - (int)(bk & 0xffu), dy = S - (int)((bk >> 8) & 0xffu);
        const uint32_t cb = (uint32_t)(bk >> 32);
        const uint64_t pa = A.pop[pr.a], pb = B.pop[pr.b];
        pcl_record rec{};
        rec.a = pr.a;
        rec.b = pr.b;
        rec.mode = PCL_MODE_COSINE;
        rec.dx_dbu = dx * g.p;
        rec.dy_dbu = dy * g.p;
        rec.score = cb;
        float sim = (pa && pb) ? (float)cb / sqrtf((float)pa * (float)pb) : 0.0f;
        uint16_t fl = PCL_F_ALIGNED;
        const float T = (float)prm.cos_num / (float)prm.cos_den;
        if (pa && pb && fabsf(sim - T) < prm.near_band) {
            fl |= PCL_F_NEAR_BAND;
            sim = (float)((double)cb / sqrt((double)pa * (double)pb));
        }
        rec.sim = sim;
        rec.flags = fl;
        rec.pass = cos_exceeds(cb, pa, pb, prm.cos_num, prm.cos_den) ? 1 : 0;
        *dst = rec;
    }
    __syncthreads();
}

// shared memory of exact_body
template <int NW>
constexpr size_t exact_smem() {
    // rasters (odd row stride), keys[32], R and C bounds (2 x 65), L and the task count (+ 2 pad),
    // 1024 sort keys, profiles [2][2N] u16
    return 2 * 16 * 64 * NW * ((NW / 2) | 1) + 32 * 8 + 4 * (2 * 65 + 4) + 4 * 1024 + 2 * 2 * 2 * 64 * NW;
}

}  // namespace fft_dev
}  // namespace pcl

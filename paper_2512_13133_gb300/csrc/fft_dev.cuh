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

}  // namespace fft_dev
}  // namespace pcl

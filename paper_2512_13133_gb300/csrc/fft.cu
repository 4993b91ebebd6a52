// a3-a6: FFT phase correlation (Sec. 3.2.1, Eqs. 3-5) and the cosine test at
// the optimal shift (Sec. 2.2.1, Eq. 2).
//
// FFT side L = 9P with P = N/8 a power of two: every shift |s| <= N/8 of the
// zero-padded linear correlation is alias-free (L >= N + S).  All transforms
// use one decomposition, index = 9*i1 + i2 on the input side and
// k = k1 + P*k2 on the output side:
//   X[k1 + P k2] = sum_i2 w9^(k2 i2) wL^(k1 i2) sum_i1 x[9 i1 + i2] wP^(k1 i1)
// i.e. nine P-point DFTs in registers (radix-2, compile-time twiddles), a
// twiddle, and P nine-point DFTs (3 x 3).
//
// Forward (per clip, cached): R2C of the raster zero-padded to L x L.  Rows
// are transformed two at a time as one complex sequence and split; then the
// L/2+1 columns.  The spectrum is stored [ky][kx] with kx contiguous.
//
// Per pair (one CTA): C = F_A conj(F_B) on the half spectrum; the phase-
// correlation spectrum R = C/|C| (Eq. 4; bins with |C| <= 1e-6 |A||B| set to
// 0, |A||B| = C(0) being the largest |C|).  Inverse pass 1 runs along ky for
// every kx column, pruned to the 2*(P/2)+1 output rows |dy| <= P/2: with
// outputs n = n1 + P n2 only n2 = 0 (dy >= 0) and n2 = 8 (dy < 0) are kept,
// so the nine-point stage collapses to one twiddled sum per output.  Pass 2
// packs the two Hermitian rows as R + iC into one complex sequence over kx
// and gives r_pcm(s) (real part) and c(s) (imaginary part), again pruned.
// The correlation is rounded to integers; the residual guard (any window
// entry more than 0.25 from an integer) and a popcount check of c at the
// chosen shift fall back to an exact popcount scan of the whole window.
#include <climits>

#include "gates.cuh"

namespace pcl {

namespace {

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

// ---------------------------------------------------------------- forward
template <int P>
__global__ void __launch_bounds__(256) spectra_kernel(pcl_params prm, pcl_clipset cs,
                                                      const uint32_t *list, uint32_t n_list,
                                                      uint8_t want_state) {
    constexpr int L = 9 * P, N = 8 * P, NW = N / 64, LH = L / 2 + 1;
    constexpr int LS = (LH + 3) & ~3;
    constexpr int CH = 32;  // rows pairs or columns per chunk
    uint32_t c;
    if (list) {
        if (blockIdx.x >= n_list) return;
        c = list[blockIdx.x];
    } else {
        c = blockIdx.x;
        if (c >= cs.n_clips) return;
        if (cs.spec_state[c] != want_state && !(want_state == 0 && cs.spec_state[c] == 2)) return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *tw = reinterpret_cast<float2 *>(smem);                 // L
    uint64_t *bits = reinterpret_cast<uint64_t *>(tw + L);          // N * NW
    float2 *vb = reinterpret_cast<float2 *>(bits + N * NW);         // CH * 9 * (P + 1)
    build_twiddles(tw, L, -1);
    const uint64_t *src = cs.bits + (size_t)c * N * NW;
    for (int t = threadIdx.x; t < N * NW; t += blockDim.x) bits[t] = src[t];
    float2 *spec = reinterpret_cast<float2 *>(cs.spec) + (size_t)c * L * LS;
    __syncthreads();

    // ---- rows: pairs (2t, 2t+1) as one complex sequence
    for (int t0 = 0; t0 < N / 2; t0 += CH) {
        for (int task = threadIdx.x; task < CH * 9; task += blockDim.x) {
            const int tl = task % CH, i2 = task / CH, t = t0 + tl;
            float2 v[P];
#pragma unroll
            for (int i1 = 0; i1 < P; ++i1) {
                const int x = 9 * i1 + i2;
                v[i1] = (x < N) ? make_float2(bitf(bits, NW, 2 * t, x), bitf(bits, NW, 2 * t + 1, x))
                                : make_float2(0.f, 0.f);
            }
            dft_pow2<P, -1>(v);
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) vb[vslot<P>(tl, i2, k1)] = v[k1];
        }
        __syncthreads();
        for (int task = threadIdx.x; task < CH * P; task += blockDim.x) {
            const int k1 = task % P, tl = task / P;
            float2 u[9];
#pragma unroll
            for (int i2 = 0; i2 < 9; ++i2) u[i2] = cmul(vb[vslot<P>(tl, i2, k1)], tw[(k1 * i2) % L]);
            dft9<-1>(u);
#pragma unroll
            for (int k2 = 0; k2 < 9; ++k2) vb[vslot<P>(tl, k2, k1)] = u[k2];
        }
        __syncthreads();
        for (int task = threadIdx.x; task < CH * LH; task += blockDim.x) {
            const int kx = task % LH, tl = task / LH, t = t0 + tl;
            const int km = (L - kx) % L;
            const float2 xk = vb[vslot<P>(tl, kx / P, kx % P)];
            const float2 xm = cconj(vb[vslot<P>(tl, km / P, km % P)]);
            const float2 fe = cscale(cadd(xk, xm), 0.5f);
            const float2 d = csub(xk, xm);
            const float2 fo = make_float2(0.5f * d.y, -0.5f * d.x);  // d / (2i)
            spec[(size_t)(2 * t) * LS + kx] = fe;
            spec[(size_t)(2 * t + 1) * LS + kx] = fo;
        }
        __syncthreads();
    }
    // ---- columns kx in chunks of CH; rows y < N hold the row transforms
    for (int c0 = 0; c0 < LH; c0 += CH) {
        for (int task = threadIdx.x; task < CH * 9; task += blockDim.x) {
            const int cl = task % CH, i2 = task / CH, kx = c0 + cl;
            float2 v[P];
#pragma unroll
            for (int i1 = 0; i1 < P; ++i1) {
                const int y = 9 * i1 + i2;
                v[i1] = (y < N && kx < LH) ? spec[(size_t)y * LS + kx] : make_float2(0.f, 0.f);
            }
            dft_pow2<P, -1>(v);
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) vb[vslot<P>(cl, i2, k1)] = v[k1];
        }
        __syncthreads();
        for (int task = threadIdx.x; task < CH * P; task += blockDim.x) {
            const int cl = task % CH, k1 = task / CH, kx = c0 + cl;
            float2 u[9];
#pragma unroll
            for (int i2 = 0; i2 < 9; ++i2) u[i2] = cmul(vb[vslot<P>(cl, i2, k1)], tw[(k1 * i2) % L]);
            dft9<-1>(u);
            if (kx < LH) {
#pragma unroll
                for (int k2 = 0; k2 < 9; ++k2) spec[(size_t)(k1 + P * k2) * LS + kx] = u[k2];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) cs.spec_state[c] = 1;
}

// mark clips referenced by a pair list whose spectrum is missing (state 2)
__global__ void mark_kernel(const pcl_pair *pairs, uint64_t n, const unsigned long long *d_n, uint8_t *state_a,
                            uint8_t *state_b, uint32_t na, uint32_t nb) {
    if (d_n && *d_n < n) n = *d_n;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const pcl_pair p = pairs[t];
        if (p.a < na && state_a[p.a] == 0) state_a[p.a] = 2;
        if (p.b < nb && state_b[p.b] == 0) state_b[p.b] = 2;
    }
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
    static constexpr size_t misc = v2 + sizeof(float2) * NO * 9 * (P + 1);   // keys [2][32] u64, flags [4]
    static constexpr size_t bytes = misc + 2 * 32 * 8 + 4 * 4;
    // surfaces reuse out1 once pass 2 has read it: [2][NO][NO] float
};

template <int P>
__device__ __forceinline__ void pair_body(const pcl_params &prm, const pcl_clipset &A, const pcl_clipset &B,
                                          const pcl_pair *pairs, uint64_t pid, pcl_record *out) {
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
    int *flags = reinterpret_cast<int *>(smem + SM::misc + 2 * 32 * 8);                 // [4]
    float *surf = reinterpret_cast<float *>(smem + SM::out1);                           // [2][NO][NO]

    if (threadIdx.x < 4) flags[threadIdx.x] = 0;
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
        return;
    }
    const uint64_t pa = A.pop[pr.a], pb = B.pop[pr.b];
    if (pa == 0 && pb == 0) {
        if (threadIdx.x == 0) {
            rec.sim = 1.0f;
            rec.pass = 1;
            rec.flags = PCL_F_EMPTY;
            out[pid] = rec;
        }
        return;
    }
    if (!(prm.flags & PCL_P_NO_GATES)) {
        if (warp == 0) {
            const int gate = warp_cosine_gate(A, pr.a, B, pr.b, g, prm.cos_num, prm.cos_den, lane);
            if (lane == 0) flags[0] = gate;
        }
        __syncthreads();
        const int gate = flags[0];
        if (gate) {
            if (threadIdx.x == 0) {
                rec.flags = (uint16_t)gate;
                out[pid] = rec;
            }
            return;
        }
    }
    build_twiddles(tw, L, +1);
    __syncthreads();

    const float2 *fa = reinterpret_cast<const float2 *>(A.spec) + (size_t)pr.a * L * LS;
    const float2 *fb = reinterpret_cast<const float2 *>(B.spec) + (size_t)pr.b * L * LS;
    const float thr = kPcmEps * (float)pa * (float)pb;
    const float thr2 = thr * thr;
    const bool want_pcm = !(prm.flags & PCL_P_NO_PCM);

    // ---- pass 1: along ky, pruned to |dy| <= HW; warp task = (signal, chunk)
    for (int task = warp; task < 2 * CHUNKS; task += nwarps) {
        const int sig = task / CHUNKS;  // 0: phase correlation R, 1: correlation C
        const int kx = (task % CHUNKS) * 32 + lane;
        const bool valid = kx < LH;
        if (sig == 0 && !want_pcm) {
            if (valid)
                for (int o = 0; o < NO; ++o) out1[(size_t)o * LH + kx] = make_float2(0.f, 0.f);
            continue;
        }
        float2 acc[NO];
#pragma unroll
        for (int o = 0; o < NO; ++o) acc[o] = make_float2(0.f, 0.f);
        for (int k2 = 0; k2 < 9; ++k2) {
            float2 v[P];
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) {
                const int ky = 9 * k1 + k2;
                float2 c = make_float2(0.f, 0.f);
                if (valid) c = cmulc(__ldg(fa + (size_t)ky * LS + kx), __ldg(fb + (size_t)ky * LS + kx));
                if (sig == 0) {
                    const float m2 = fmaf(c.x, c.x, c.y * c.y);
                    c = (m2 > thr2) ? cscale(c, rsqrtf(m2)) : make_float2(0.f, 0.f);
                }
                v[k1] = c;
            }
            dft_pow2<P, +1>(v);
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                const int dy = o - HW;
                const int n = dy >= 0 ? dy : L + dy;
                const int n1 = dy >= 0 ? dy : P + dy;
                const float2 w = tw[(k2 * n) % L];
                acc[o] = cadd(acc[o], cmul(v[n1], w));
            }
        }
        if (valid) {
#pragma unroll
            for (int o = 0; o < NO; ++o) out1[((size_t)sig * NO + o) * LH + kx] = acc[o];
        }
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
        dft_pow2<P, +1>(v);
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
    // popcount check of the chosen shift (warp 0), fall back on mismatch
    if (!gflag) {
        if (warp == 0) {
            const uint32_t ce = warp_corr_exact(ba, bbits, N, NW, sdx, sdy, lane);
            if (lane == 0 && ce != cbest) flags[2] = 1;
        }
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
        out[pid] = rec;
    }
}

// persistent: each CTA walks the pair list with a grid stride
template <int P>
__global__ void __launch_bounds__(32 * 2 * ((9 * P / 2 + 1 + 31) / 32), 1)
    pair_fft_kernel(pcl_params prm, pcl_clipset A, pcl_clipset B, const pcl_pair *pairs, uint64_t npairs,
                    const unsigned long long *d_n, pcl_record *out) {
    if (d_n && *d_n < npairs) npairs = *d_n;
    for (uint64_t pid = blockIdx.x; pid < npairs; pid += gridDim.x) {
        __syncthreads();
        pair_body<P>(prm, A, B, pairs, pid, out);
    }
}

template <int P>
size_t spectra_smem() {
    constexpr int L = 9 * P, N = 8 * P;
    return sizeof(float2) * L + 8 * (size_t)N * (N / 64) + sizeof(float2) * 32 * 9 * (P + 1);
}

template <int P>
cudaError_t spectra_t(const pcl_params &prm, const pcl_clipset &cs, const uint32_t *list, uint32_t n_list,
                      uint8_t want, cudaStream_t st) {
    const size_t sm = spectra_smem<P>();
    cudaError_t e = cudaFuncSetAttribute(spectra_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const uint32_t grid = list ? n_list : cs.n_clips;
    if (grid == 0) return cudaSuccess;
    spectra_kernel<P><<<grid, 256, sm, st>>>(prm, cs, list, n_list, want);
    return cudaGetLastError();
}

template <int P>
cudaError_t pair_t(const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b, const pcl_pair *pairs,
                   uint64_t n, const unsigned long long *d_n, pcl_record *out, int num_sms, cudaStream_t st) {
    const size_t sm = PairSmem<P>::bytes;
    cudaError_t e = cudaFuncSetAttribute(pair_fft_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    constexpr int LH = 9 * P / 2 + 1;
    const int threads = 32 * 2 * ((LH + 31) / 32);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_fft_kernel<P>, threads, sm);
    if (e != cudaSuccess) return e;
    const uint64_t cap = (uint64_t)num_sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)(n < cap ? n : cap);
    pair_fft_kernel<P><<<grid, threads, sm, st>>>(prm, a, b, pairs, n, d_n, out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_spectra(const pcl_params &prm, const pcl_clipset &cs, const uint32_t *list,
                           uint32_t n_list, bool requested_only, cudaStream_t st) {
    const Geo g = make_geo(prm);
    const uint8_t want = requested_only ? 2 : 0;
    switch (g.P) {
        case 8: return spectra_t<8>(prm, cs, list, n_list, want, st);
        case 16: return spectra_t<16>(prm, cs, list, n_list, want, st);
        case 32: return spectra_t<32>(prm, cs, list, n_list, want, st);
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_mark(const pcl_pair *pairs, uint64_t n, const unsigned long long *d_n, pcl_clipset &a,
                        pcl_clipset &b, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    mark_kernel<<<1024, 256, 0, st>>>(pairs, n, d_n, a.spec_state, b.spec_state, a.n_clips, b.n_clips);
    return cudaGetLastError();
}

cudaError_t launch_pair_fft(const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b,
                            const pcl_pair *pairs, uint64_t n, const unsigned long long *d_n, pcl_record *out,
                            int num_sms, cudaStream_t st) {
    const Geo g = make_geo(prm);
    switch (g.P) {
        case 8: return pair_t<8>(prm, a, b, pairs, n, d_n, out, num_sms, st);
        case 16: return pair_t<16>(prm, a, b, pairs, n, d_n, out, num_sms, st);
        case 32: return pair_t<32>(prm, a, b, pairs, n, d_n, out, num_sms, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace pcl

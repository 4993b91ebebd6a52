// Shared device helpers of the pcl CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "pcl.h"

namespace pcl {

// Derived geometry of a parameter block.
//   N  raster side (px)        S  shift half-range (px)     nw words per row
//   nb 16x16 blocks per side   rb block radius ceil(S/16)
//   L  FFT side 9N/8 = 9P      P  power-of-two factor N/8   Lh = L/2 + 1
//   Ls spectrum row stride (Lh rounded up to a multiple of 4 complex)
struct Geo {
    int p, W, M, N, S, nw, nb, rb, L, P, Lh, Ls;
};

__host__ __device__ inline Geo make_geo(const pcl_params &q) {
    Geo g;
    g.p = q.pitch_dbu;
    g.W = q.window_dbu;
    g.M = q.marker_dbu;
    g.N = (g.p > 0) ? g.W / g.p : 0;
    g.S = (g.p > 0) ? g.M / g.p : 0;
    g.nw = g.N / 64;
    g.nb = g.N / 16;
    g.rb = (g.S + 15) / 16;
    g.P = g.N / 8;
    g.L = 9 * g.P;
    g.Lh = g.L / 2 + 1;
    g.Ls = (g.Lh + 3) & ~3;
    return g;
}

// ------------------------------------------------------------ edge signature
enum { ES_N = 0, ES_HASX, ES_LOX, ES_HIX, ES_HASY, ES_LOY, ES_HIY, ES_BORDER };

// classes of the topological pre-screen: the polygon count, saturated
constexpr int kTopoClasses = 64;
__host__ __device__ inline int topo_class(int n_polygons) {
    return n_polygons < kTopoClasses - 1 ? n_polygons : kTopoClasses - 1;
}

// ------------------------------------------------------------ complex math
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// cos(2 pi k / 64) for k = 0..16 (first quadrant; float-rounded values of the
// mathematical constants)
__host__ __device__ constexpr float q64(int k) {
    return k == 0 ? 1.0f : k == 1 ? 0.9951847195625305f : k == 2 ? 0.9807852506637573f
         : k == 3 ? 0.9569403529167175f : k == 4 ? 0.9238795042037964f : k == 5 ? 0.8819212913513184f
         : k == 6 ? 0.8314695954322815f : k == 7 ? 0.7730104327201843f : k == 8 ? 0.7071067690849304f
         : k == 9 ? 0.6343932747840881f : k == 10 ? 0.5555702447891235f : k == 11 ? 0.4713967442512512f
         : k == 12 ? 0.3826834261417389f : k == 13 ? 0.290284663438797f : k == 14 ? 0.19509032368659973f
         : k == 15 ? 0.0980171412229538f : 0.0f;
}
__host__ __device__ constexpr float cos64(int k) {
    return (k & 63) <= 16 ? q64(k & 63)
         : (k & 63) <= 32 ? -q64(32 - (k & 63))
         : (k & 63) <= 48 ? -q64((k & 63) - 32)
                          : q64(64 - (k & 63));
}
__host__ __device__ constexpr float sin64(int k) { return cos64(k - 16); }

// x * exp(SIGN * 2 pi i K / 64), with the trivial rotations done exactly
template <int K, int SIGN>
__device__ __forceinline__ float2 rot64(float2 x) {
    constexpr int k = K & 63;
    if constexpr (k == 0) {
        return x;
    } else if constexpr (k == 16) {
        return SIGN > 0 ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    } else if constexpr (k == 32) {
        return make_float2(-x.x, -x.y);
    } else if constexpr (k == 48) {
        return SIGN > 0 ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
    } else {
        constexpr float c = cos64(k);
        constexpr float s = SIGN * sin64(k);
        return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
    }
}

__host__ __device__ constexpr int bitrev(int v, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
    return r;
}
__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

template <int P, int SIGN, int LEN>
__device__ __forceinline__ void dft_stage(float2 (&v)[P]) {
    constexpr int H = LEN / 2;
#pragma unroll
    for (int i = 0; i < P; i += LEN) {
        [&]<int... J>(std::integer_sequence<int, J...>) {
            ((void)([&] {
                 float2 u = v[i + J];
                 float2 t = rot64<J * (64 / LEN), SIGN>(v[i + J + H]);
                 v[i + J] = cadd(u, t);
                 v[i + J + H] = csub(u, t);
             }()),
             ...);
        }(std::make_integer_sequence<int, H>{});
    }
}

template <int P, int SIGN, int LEN>
__device__ __forceinline__ void dft_stages(float2 (&v)[P]) {
    if constexpr (LEN <= P) {
        dft_stage<P, SIGN, LEN>(v);
        dft_stages<P, SIGN, LEN * 2>(v);
    }
}

// In-register DFT of length P (power of two, <= 64):
//   v[k] <- sum_n v[n] exp(SIGN * 2 pi i n k / P)
// iterative radix-2 decimation in time; all indices are compile-time.
template <int P, int SIGN>
__device__ __forceinline__ void dft_pow2(float2 (&v)[P]) {
    static_assert(P >= 2 && P <= 64 && (P & (P - 1)) == 0, "P must be a power of two <= 64");
    constexpr int B = ilog2c(P);
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const int r = bitrev(i, B);
        if (i < r) {
            float2 t = v[i];
            v[i] = v[r];
            v[r] = t;
        }
    }
    dft_stages<P, SIGN, 2>(v);
}

// ---- radix-4 decimation in frequency (natural input, digit-reversed output
// reordered at compile time).  Radices: 4 while the block size is divisible
// by 4, then one radix-2 step (P = 8, 32).
__host__ __device__ constexpr int dif_freq(int p, int n) {
    // frequency held at position p of a DIF transform of size n
    return n == 1 ? 0
         : (n % 4 == 0) ? 4 * dif_freq(p % (n / 4), n / 4) + p / (n / 4)
                        : 2 * dif_freq(p % (n / 2), n / 2) + p / (n / 2);
}

template <int P, int SIGN, int BASE, int N>
__device__ __forceinline__ void dif_block(float2 (&v)[P]) {
    if constexpr (N == 2) {
        const float2 a = v[BASE], b = v[BASE + 1];
        v[BASE] = cadd(a, b);
        v[BASE + 1] = csub(a, b);
    } else if constexpr (N >= 4) {
        constexpr int Q = N / 4;
        [&]<int... J>(std::integer_sequence<int, J...>) {
            ((void)([&] {
                 const float2 a = v[BASE + J], b = v[BASE + J + Q], c = v[BASE + J + 2 * Q],
                              d = v[BASE + J + 3 * Q];
                 const float2 s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = csub(b, d);
                 // SIGN * i * d1
                 const float2 r = SIGN > 0 ? make_float2(-d1.y, d1.x) : make_float2(d1.y, -d1.x);
                 v[BASE + J] = cadd(s0, s1);
                 v[BASE + J + Q] = rot64<J * 1 * (64 / N), SIGN>(cadd(d0, r));
                 v[BASE + J + 2 * Q] = rot64<J * 2 * (64 / N), SIGN>(csub(s0, s1));
                 v[BASE + J + 3 * Q] = rot64<J * 3 * (64 / N), SIGN>(csub(d0, r));
             }()),
             ...);
        }(std::make_integer_sequence<int, Q>{});
        dif_block<P, SIGN, BASE, Q>(v);
        dif_block<P, SIGN, BASE + Q, Q>(v);
        dif_block<P, SIGN, BASE + 2 * Q, Q>(v);
        dif_block<P, SIGN, BASE + 3 * Q, Q>(v);
    }
}

// In-register DFT of length P by radix-4 DIF (same result as dft_pow2)
template <int P, int SIGN>
__device__ __forceinline__ void dft_pow2_r4(float2 (&v)[P]) {
    static_assert(P >= 4 && P <= 64 && (P & (P - 1)) == 0, "P must be a power of two in [4, 64]");
    dif_block<P, SIGN, 0, P>(v);
    float2 t[P];
#pragma unroll
    for (int p = 0; p < P; ++p) t[dif_freq(p, P)] = v[p];
#pragma unroll
    for (int p = 0; p < P; ++p) v[p] = t[p];
}

// DFT of length P with the radix chosen at compile time (2 or 4)
template <int P, int SIGN, int RADIX>
__device__ __forceinline__ void dft_p(float2 (&v)[P]) {
    if constexpr (RADIX == 4) dft_pow2_r4<P, SIGN>(v);
    else dft_pow2<P, SIGN>(v);
}

// 3-point DFT, sign SIGN
template <int SIGN>
__device__ __forceinline__ void dft3(float2 &a, float2 &b, float2 &c) {
    const float h = 0.8660253882408142f;  // sqrt(3)/2
    float2 s = cadd(b, c);
    float2 d = csub(b, c);
    float2 m = make_float2(fmaf(-0.5f, s.x, a.x), fmaf(-0.5f, s.y, a.y));
    // SIGN * i * h * d
    float2 r = SIGN > 0 ? make_float2(-h * d.y, h * d.x) : make_float2(h * d.y, -h * d.x);
    a = cadd(a, s);
    b = cadd(m, r);
    c = csub(m, r);
}

// 9-point DFT (3 x 3 Cooley-Tukey), v[k] <- sum_n v[n] exp(SIGN 2 pi i n k / 9)
template <int SIGN>
__device__ __forceinline__ void dft9(float2 (&v)[9]) {
    // inner 3-point transforms over a (x = 3a + b), one per b
#pragma unroll
    for (int b = 0; b < 3; ++b) dft3<SIGN>(v[b], v[3 + b], v[6 + b]);
    // after this, v[3c + b] = Y_b[c]; twiddle by exp(SIGN 2 pi i c b / 9)
    const float c1 = 0.7660444378852844f, s1 = 0.6427876353263855f;   // 2 pi / 9
    const float c2 = 0.1736481785774231f, s2 = 0.9848077297210693f;   // 4 pi / 9
    const float c4 = -0.9396926164627075f, s4 = 0.3420201539993286f;  // 8 pi / 9
    auto tw = [](float2 x, float c, float s) {
        return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
    };
    v[4] = tw(v[4], c1, SIGN * s1);  // c = 1, b = 1
    v[5] = tw(v[5], c2, SIGN * s2);  // c = 1, b = 2
    v[7] = tw(v[7], c2, SIGN * s2);  // c = 2, b = 1
    v[8] = tw(v[8], c4, SIGN * s4);  // c = 2, b = 2
    // outer 3-point transforms over b for each c -> X[c + 3d]
    float2 o[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 a0 = v[3 * c], a1 = v[3 * c + 1], a2 = v[3 * c + 2];
        dft3<SIGN>(a0, a1, a2);
        o[c] = a0;
        o[c + 3] = a1;
        o[c + 6] = a2;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = o[k];
}

// ------------------------------------------------------------ shift order
// (c1, dx1, dy1) before (c2, dx2, dy2): larger c, then smaller |dx|+|dy|, then
// smaller dy, then smaller dx.  Packs into one comparable 64-bit key (larger
// key = earlier) for warp reductions.
__device__ __forceinline__ unsigned long long shift_key(uint32_t c, int dx, int dy, int S) {
    const unsigned l = (unsigned)(abs(dx) + abs(dy));        // <= 2S
    const unsigned ry = (unsigned)(2 * S - (dy + S));        // smaller dy -> larger
    const unsigned rx = (unsigned)(2 * S - (dx + S));
    const unsigned rl = (unsigned)(4 * S - l);
    return ((unsigned long long)c << 32) | ((unsigned long long)rl << 16) |
           ((unsigned long long)ry << 8) | (unsigned long long)rx;
}

// exact overlap c(dx, dy) = sum_x A(x) B(x - s) of two bit-packed rasters,
// computed by one warp (lanes stride the rows); every lane gets the sum.
// this thread's share of c(dx, dy) over the rows j0 + first, j0 + first +
// step, ... (first in [0, step)): summed over all threads of a CTA (first =
// thread index, step = thread count) it gives the exact overlap
__device__ __forceinline__ uint32_t corr_rows_partial(const uint64_t *__restrict__ A,
                                                      const uint64_t *__restrict__ B, int N, int nw,
                                                      int dx, int dy, int first, int step) {
    uint32_t acc = 0;
    const int j0 = dy > 0 ? dy : 0, j1 = dy < 0 ? N + dy : N;
    const int base0 = -dx;
    const int wsh = base0 >= 0 ? base0 / 64 : -((-base0 + 63) / 64);
    const int off = base0 - 64 * wsh;
    for (int j = j0 + first; j < j1; j += step) {
        const uint64_t *ra = A + (size_t)j * nw;
        const uint64_t *rb = B + (size_t)(j - dy) * nw;
        for (int w = 0; w < nw; ++w) {
            const int wi = w + wsh;
            const uint64_t lo = (wi >= 0 && wi < nw) ? rb[wi] : 0ull;
            const uint64_t hi = (wi + 1 >= 0 && wi + 1 < nw) ? rb[wi + 1] : 0ull;
            const uint64_t sh = off ? ((lo >> off) | (hi << (64 - off))) : lo;
            acc += (uint32_t)__popcll(ra[w] & sh);
        }
    }
    return acc;
}

__device__ __forceinline__ uint32_t warp_corr_exact(const uint64_t *__restrict__ A,
                                                    const uint64_t *__restrict__ B, int N, int nw,
                                                    int dx, int dy, int lane) {
    uint32_t acc = 0;
    const int j0 = dy > 0 ? dy : 0, j1 = dy < 0 ? N + dy : N;
    // word w of B's row moved by dx: bits come from pixel 64 w - dx
    const int base0 = -dx;
    const int wsh = base0 >= 0 ? base0 / 64 : -((-base0 + 63) / 64);
    const int off = base0 - 64 * wsh;
    for (int j = j0 + lane; j < j1; j += 32) {
        const uint64_t *ra = A + (size_t)j * nw;
        const uint64_t *rb = B + (size_t)(j - dy) * nw;
        for (int w = 0; w < nw; ++w) {
            const int wi = w + wsh;
            const uint64_t lo = (wi >= 0 && wi < nw) ? rb[wi] : 0ull;
            const uint64_t hi = (wi + 1 >= 0 && wi + 1 < nw) ? rb[wi + 1] : 0ull;
            const uint64_t sh = off ? ((lo >> off) | (hi << (64 - off))) : lo;
            acc += (uint32_t)__popcll(ra[w] & sh);
        }
    }
    return __reduce_add_sync(0xffffffffu, acc);
}

// a * b as a 128-bit (hi, lo) pair
__device__ __forceinline__ void mul128(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo) {
    lo = a * b;
    hi = __umul64hi(a, b);
}

// integer cosine threshold test of Eq. 2 (strict >): den^2 c^2 > num^2 pa pb,
// exact for c, pa, pb < 2^32 and den < 2^16 (128-bit products)
__device__ __forceinline__ bool cos_exceeds(uint64_t c, uint64_t pa, uint64_t pb, uint32_t num,
                                            uint32_t den) {
    if (c == 0) return false;
    uint64_t lh, ll, rh, rl;
    mul128((uint64_t)den * den, c * c, lh, ll);
    mul128((uint64_t)num * num, pa * pb, rh, rl);
    return lh > rh || (lh == rh && ll > rl);
}

// sum of the popcounts of n words with fewer popcounts: per bit position a
// full adder gives x + y + z = (x ^ y ^ z) + 2 maj(x, y, z), so three words
// cost two popcounts and two logic operations.  Population counts issue at a
// quarter of the integer rate, so this balances the two pipes.
template <int n>
__device__ __forceinline__ uint32_t popc_sum(const uint32_t (&x)[n]) {
    uint32_t s1 = 0, s2 = 0;
#pragma unroll
    for (int w = 0; w + 2 < n; w += 3) {
        s1 += (uint32_t)__popc(x[w] ^ x[w + 1] ^ x[w + 2]);
        s2 += (uint32_t)__popc((x[w] & x[w + 1]) | (x[w + 2] & (x[w] ^ x[w + 1])));
    }
#pragma unroll
    for (int w = n / 3 * 3; w < n; ++w) s1 += (uint32_t)__popc(x[w]);
    return s1 + 2u * s2;
}

}  // namespace pcl

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

#include "exact_dev.cuh"
#include "fft_dev.cuh"

namespace pcl {

namespace {

using namespace fft_dev;
using namespace exact_dev;

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

// persistent: each CTA walks the pair list with a grid stride
template <int P>
__global__ void __launch_bounds__(32 * 2 * ((9 * P / 2 + 1 + 31) / 32), 1)
    pair_fft_kernel(pcl_params prm, pcl_clipset A, pcl_clipset B, const pcl_pair *pairs, uint64_t npairs,
                    const unsigned long long *d_n, pcl_record *out) {
    if (d_n && *d_n < npairs) npairs = *d_n;
    for (uint64_t pid = blockIdx.x; pid < npairs; pid += gridDim.x) {
        __syncthreads();
        pair_body<P>(prm, A, B, pairs[pid], out + pid);
    }
}

// The exact window scan: at 512² the FFT body's buffers exceed shared memory,
// and at 128² / 256² it is the exact-scan engine.  A pair passes the indices,
// emptiness and lossless gates as in pair_body and the survivors take the
// bound-pruned scan (exact_body<NW, SMAX>, N = 64 NW, S <= SMAX = N/16).  One
// pair per CTA iteration, persistent grid.
constexpr int kExactThreads = 320;

template <int NW, int SMAX>
__global__ void __launch_bounds__(kExactThreads, 2)
    exact_pair_kernel(pcl_params prm, pcl_clipset A, pcl_clipset B, const pcl_pair *pairs, uint64_t npairs,
                      const unsigned long long *d_n, pcl_record *out, unsigned long long *stats) {
    if (d_n && *d_n < npairs) npairs = *d_n;
    __shared__ int gate_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Geo g = make_geo(prm);
    for (uint64_t pid = blockIdx.x; pid < npairs; pid += gridDim.x) {
        const pcl_pair pr = pairs[pid];
        pcl_record rec{};
        rec.a = pr.a;
        rec.b = pr.b;
        rec.mode = PCL_MODE_COSINE;
        bool done = true;  // the same in every thread
        if (pr.a >= A.n_clips || pr.b >= B.n_clips) {
            rec.flags = PCL_GATE_BAD_INDEX;
        } else if (A.pop[pr.a] == 0 && B.pop[pr.b] == 0) {
            rec.flags = PCL_F_EMPTY;
            rec.sim = 1.0f;
            rec.pass = 1;
        } else if (!(prm.flags & PCL_P_NO_GATES)) {
            __syncthreads();
            if (warp == 0) {
                const int gt = warp_cosine_gate(A, pr.a, B, pr.b, g, prm.cos_num, prm.cos_den, lane);
                if (lane == 0) gate_s = gt;
            }
            __syncthreads();
            rec.flags = (uint16_t)gate_s;
            done = gate_s != 0;
        } else {
            done = false;
        }
        if (done) {
            if (threadIdx.x == 0) out[pid] = rec;
            continue;
        }
        exact_body<NW, SMAX>(prm, A, B, pr, out + pid, stats);
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

template <int NW, int SMAX>
cudaError_t exact_t(const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b, const pcl_pair *pairs,
                    uint64_t n, const unsigned long long *d_n, pcl_record *out, int num_sms,
                    unsigned long long *stats, cudaStream_t st) {
    const size_t sm = exact_smem<NW>();
    auto *kern = exact_pair_kernel<NW, SMAX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess || n == 0) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kExactThreads, sm);
    if (e != cudaSuccess) return e;
    const uint64_t cap = (uint64_t)num_sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)(n < cap ? n : cap);
    kern<<<grid, kExactThreads, sm, st>>>(prm, a, b, pairs, n, d_n, out, stats);
    return cudaGetLastError();
}

cudaError_t launch_exact_pairs(const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b,
                               const pcl_pair *pairs, uint64_t n, const unsigned long long *d_n, pcl_record *out,
                               int num_sms, unsigned long long *stats, cudaStream_t st) {
    const Geo g = make_geo(prm);
    if (g.S > g.N / 16) return cudaErrorNotSupported;
    switch (g.N) {
        case 128: return exact_t<2, 8>(prm, a, b, pairs, n, d_n, out, num_sms, stats, st);
        case 256: return exact_t<4, 16>(prm, a, b, pairs, n, d_n, out, num_sms, stats, st);
        case 512: return exact_t<8, 32>(prm, a, b, pairs, n, d_n, out, num_sms, stats, st);
        default: return cudaErrorNotSupported;
    }
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

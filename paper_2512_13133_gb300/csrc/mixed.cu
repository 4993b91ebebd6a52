// a9: one persistent launch over a mixed batch -- pairs of several raster
// size classes, cosine (FFT phase correlation) and edge (Min-Max) modes
// together, with uneven candidate lists.
//
// The work list holds the cosine items first, then the edge items.  Each CTA
// (320 threads, shared memory sized for the largest FFT) works in rounds:
// every warp claims a run of consecutive cosine items and checks their
// indices, emptiness and lossless gates one after the other; the round's
// survivors are then aligned one after the other by the whole CTA with the
// FFT body of their size class (512² rasters, beyond the FFT body's shared
// memory, take the exact window scan of exact_body instead).  When the cosine
// items are exhausted, every warp takes edge items 32 at a time: the lanes
// run their items' gates, and the whole warp evaluates the survivors.  The register DFT radix (2 or 4) and the number
// of CTAs per SM are tuning parameters (chosen by the autotuner).
#include "edge_dev.cuh"
#include "exact_dev.cuh"
#include "fft_dev.cuh"

namespace pcl {

namespace {

using namespace fft_dev;
using namespace exact_dev;
using namespace edge_dev;

constexpr int kMaxClasses = 4;
constexpr int kThreads = 320;  // ten warps: the pass-1 tasks of P = 32
constexpr int kWarps = kThreads / 32;
constexpr int kClaimMax = 64;  // cosine items a warp claims per round, at most (a tuning parameter)

struct MixedArgs {
    pcl_params prm[kMaxClasses];
    pcl_clipset cs[kMaxClasses];
    uint32_t n_classes;
};

__global__ void mark_mixed_kernel(MixedArgs args, const pcl_work *work, uint64_t n_cos) {
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_cos;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const pcl_work w = work[t];
        if (w.cls >= args.n_classes) continue;
        const pcl_clipset &c = args.cs[w.cls];
        if (!c.spec_state || make_geo(args.prm[w.cls]).P > 32) continue;
        if (w.a < c.n_clips && c.spec_state[w.a] == 0) c.spec_state[w.a] = 2;
        if (w.b < c.n_clips && c.spec_state[w.b] == 0) c.spec_state[w.b] = 2;
    }
}

template <int RADIX>
__global__ void __launch_bounds__(kThreads, 1)
    mixed_kernel(MixedArgs args, const pcl_work *work, uint64_t n_cos, uint64_t n, pcl_record *out,
                 unsigned long long *cursor, int claim) {
    __shared__ uint64_t surv[kWarps * kClaimMax];
    __shared__ int n_surv, exhausted;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // while gating, the alignment bodies' shared memory is free: each warp
    // takes a slice of it for the G2 profiles
    extern __shared__ __align__(16) unsigned char mixed_sm[];
    uint16_t *g2_scratch = reinterpret_cast<uint16_t *>(mixed_sm);
    // ---- cosine items, in rounds: every warp claims `claim` consecutive items
    // and gates them one after the other (the gate cost varies a lot between
    // items, so a round evens it out over `claim` items); the survivors of the
    // round are then aligned one after the other by the whole CTA
    for (;;) {
        if (threadIdx.x == 0) {
            n_surv = 0;
            exhausted = 0;
        }
        __syncthreads();
        uint64_t t0 = 0;
        if (lane == 0) t0 = atomicAdd(cursor, (unsigned long long)claim);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= n_cos && lane == 0) exhausted = 1;
        for (uint64_t t = t0; t < t0 + (uint64_t)claim && t < n_cos; ++t) {
            const pcl_work w = work[t];
            pcl_record rec{};
            rec.a = w.a;
            rec.b = w.b;
            rec.mode = PCL_MODE_COSINE;
            bool done = true;
            if (w.cls >= args.n_classes || w.a >= args.cs[w.cls].n_clips || w.b >= args.cs[w.cls].n_clips) {
                rec.flags = PCL_GATE_BAD_INDEX;
            } else {
                const pcl_params &prm = args.prm[w.cls];
                const pcl_clipset &cs = args.cs[w.cls];
                const Geo g = make_geo(prm);
                const uint64_t pa = cs.pop[w.a], pb = cs.pop[w.b];
                if ((g.P > 32 && (g.P != 64 || prm.shift_rule != PCL_SHIFT_EXACT_ARGMAX)) || g.S > g.N / 16) {
                    rec.flags = PCL_GATE_UNSUPPORTED;
                } else if (pa == 0 && pb == 0) {
                    rec.flags = PCL_F_EMPTY;
                    rec.sim = 1.0f;
                    rec.pass = 1;
                } else {
                    int gate = 0;
                    if (!(prm.flags & PCL_P_NO_GATES))
                        gate = warp_cosine_gate(cs, w.a, cs, w.b, g, prm.cos_num, prm.cos_den, lane,
                                                g2_scratch + warp * kG2Scratch);
                    if (gate) rec.flags = (uint16_t)gate;
                    else done = false;
                }
            }
            if (lane == 0) {
                if (done) out[t] = rec;
                else surv[atomicAdd(&n_surv, 1)] = t;
            }
        }
        __syncthreads();
        const int ns = n_surv;
        for (int k = 0; k < ns; ++k) {
            const uint64_t ti = surv[k];
            const pcl_work w = work[ti];
            const pcl_params &prm = args.prm[w.cls];
            const pcl_clipset &cs = args.cs[w.cls];
            switch (make_geo(prm).P) {
                case 8: pair_body<8, RADIX>(prm, cs, cs, pcl_pair{w.a, w.b}, out + ti, true); break;
                case 16: pair_body<16, RADIX>(prm, cs, cs, pcl_pair{w.a, w.b}, out + ti, true); break;
                case 64: exact_body<8, 32>(prm, cs, cs, pcl_pair{w.a, w.b}, out + ti); break;  // 512²
                default: pair_body<32, RADIX>(prm, cs, cs, pcl_pair{w.a, w.b}, out + ti, true); break;
            }
            __syncthreads();
        }
        if (exhausted) break;  // some warp found no items left: this round was the last
        __syncthreads();       // exhausted and n_surv are reset only after every warp read them
    }
    // ---- edge items: each lane takes one item and runs its gates (most items
    // end there); the whole warp then evaluates the survivors one at a time
    // (warp_edge_record).  Warps stride the list 32 items at a time.
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = n_cos + 32 * gw; base < n; base += 32 * nw) {
        const uint64_t t = base + lane;
        bool surv_e = false;
        pcl_work w{};
        if (t < n) {
            w = work[t];
            pcl_record r{};
            if (w.cls >= args.n_classes) {
                r.a = w.a;
                r.b = w.b;
                r.mode = PCL_MODE_EDGE;
                r.flags = PCL_GATE_BAD_INDEX;
            } else {
                surv_e = edge_gate_record(args.prm[w.cls], args.cs[w.cls], args.cs[w.cls], pcl_pair{w.a, w.b}, &r);
            }
            if (!surv_e) out[t] = r;
        }
        unsigned m = __ballot_sync(0xffffffffu, surv_e);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t cls = __shfl_sync(0xffffffffu, (uint32_t)w.cls, src);
            const uint32_t a = __shfl_sync(0xffffffffu, w.a, src), b = __shfl_sync(0xffffffffu, w.b, src);
            const pcl_record r = warp_edge_record(args.prm[cls], args.cs[cls], args.cs[cls], pcl_pair{a, b}, lane);
            if (lane == 0) out[base + src] = r;
        }
    }
}

size_t mixed_smem() {
    size_t b = PairSmem<32>::bytes > exact_smem<8>() ? PairSmem<32>::bytes : exact_smem<8>();
    const size_t g2 = sizeof(uint16_t) * kWarps * kG2Scratch;  // gating scratch, same memory
    return b > g2 ? b : g2;
}

}  // namespace

cudaError_t launch_spectra(const pcl_params &, const pcl_clipset &, const uint32_t *, uint32_t, bool, cudaStream_t);

cudaError_t launch_mixed(const pcl_params *prm, const pcl_clipset *sets, uint32_t n_classes, const pcl_work *work,
                         uint64_t n_cos, uint64_t n, pcl_record *out, unsigned long long *cursor, uint32_t radix,
                         uint32_t ctas_per_sm, uint32_t items_per_warp, int num_sms, cudaStream_t st) {
    if (n_classes == 0 || n_classes > kMaxClasses) return cudaErrorInvalidValue;
    const int claim = items_per_warp == 0 ? 16 : (int)items_per_warp;
    if (claim > kClaimMax) return cudaErrorInvalidValue;
    MixedArgs args{};
    args.n_classes = n_classes;
    for (uint32_t c = 0; c < n_classes; ++c) {
        args.prm[c] = prm[c];
        args.cs[c] = sets[c];
    }
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (n_cos) {
        mark_mixed_kernel<<<1024, 256, 0, st>>>(args, work, n_cos);
        for (uint32_t c = 0; c < n_classes; ++c) {
            if (!sets[c].spec_state || make_geo(prm[c]).P > 32) continue;
            if ((e = launch_spectra(prm[c], sets[c], nullptr, 0, true, st)) != cudaSuccess) return e;
        }
    }
    const size_t sm = mixed_smem();
    int per_sm = 0;
    if (radix == 4) {
        e = cudaFuncSetAttribute(mixed_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mixed_kernel<4>, kThreads, sm);
    } else {
        e = cudaFuncSetAttribute(mixed_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mixed_kernel<2>, kThreads, sm);
    }
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int ctas = (ctas_per_sm == 0 || (int)ctas_per_sm > per_sm) ? per_sm : (int)ctas_per_sm;
    const unsigned grid = (unsigned)(num_sms * ctas);
    if (n == 0) return cudaSuccess;
    if (radix == 4) mixed_kernel<4><<<grid, kThreads, sm, st>>>(args, work, n_cos, n, out, cursor, claim);
    else mixed_kernel<2><<<grid, kThreads, sm, st>>>(args, work, n_cos, n, out, cursor, claim);
    return cudaGetLastError();
}

}  // namespace pcl

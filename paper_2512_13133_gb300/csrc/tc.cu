// a8: direct windowed correlation on the 5th-generation tensor cores.
//
// For one representative A and a batch of NB members B_n sharing it,
//   D[t, n] = sum_u A(u + s_t) B_n(u)  =  c_n(s_t)      (c(s) = sum_x A(x) B(x - s))
// over every shift s_t of the marker window, as a GEMM with M = shifts (tiles
// of 128), N = members, K = pixels.  0/1 operands are exact in FP16 and the
// FP32 sums stay below 2^24, so the tensor cores return the exact integer
// overlaps (no rounding guard is needed).
//
// Per K stage (64 pixels of one image row) the CTA writes, in shared memory
// and in the canonical K-major no-swizzle layout (8-row x 16-byte core
// matrices, K-adjacent core matrices 128 B apart, 8-row groups 1024 B apart):
//   - the shifted-representative tile: row t holds A's row y + dy from column
//     x0 + dx (a 64-bit window of A's bit row), expanded bit -> FP16 by a
//     256-entry table;
//   - the member tile: row n holds member n's 64 pixels.
// One thread issues tcgen05.mma (kind::f16, M = 128, N = NB, K = 16) four
// times per (shift tile, stage) unit, accumulating in tensor memory; every
// shift tile of the representative has its own accumulator columns (tiles x NB
// <= 512), so all of them stay resident until the epilogue.  Two unit buffers alternate;
// tcgen05.commit arrives on the buffer's mbarrier, and a buffer is rewritten
// only after that barrier completes (waits are bounded; on time-out the CTA
// records an error and stops).  The epilogue reads the accumulators with
// tcgen05.ld (warp w sees rows 32w..32w+31) and reduces the exact argmax with
// the tie order (-c, |dx|+|dy|, dy, dx).
#include <climits>

#include "gates.cuh"

namespace pcl {

namespace {

constexpr int kThreads = 128;
constexpr int kStageK = 64;             // pixels per stage
constexpr int kTileBytesA = 128 * 128;  // 128 rows x 64 fp16
constexpr int kMaxNB = 256;
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitLimit = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// canonical K-major, no-swizzle shared-memory descriptor (tcgen05 format):
// start >> 4 [0,14), leading (K) core-matrix stride >> 4 [16,30), stride
// between 8-row groups >> 4 [32,46), version 1 at bit 46, layout 0 (none)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D = F32, A = B = F16, both K-major
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false on time-out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 64-bit window of a bit row starting at pixel `base` (zeros outside)
__device__ __forceinline__ uint64_t bit_window(const uint64_t *row, int nw, int base) {
    const int wi = base >= 0 ? base >> 6 : -((-base + 63) >> 6);
    const int off = base - 64 * wi;
    const uint64_t lo = (wi >= 0 && wi < nw) ? row[wi] : 0ull;
    const uint64_t hi = (wi + 1 >= 0 && wi + 1 < nw) ? row[wi + 1] : 0ull;
    return off ? ((lo >> off) | (hi << (64 - off))) : lo;
}

// shared-memory plan (dynamic): LUT 4 KB | A raster (N*N/8) | 2 x (A tile 16 KB +
// member tile NB*128 B) | keys | misc; padded to force one CTA per SM
struct TcSmem {
    uint32_t lut, araster, tiles, keys, misc, bytes;
};

__host__ __device__ inline TcSmem tc_smem(int N, int NB, int tiles) {
    TcSmem s;
    s.lut = 0;
    s.araster = 4096;
    const uint32_t ar = (uint32_t)N * N / 8;
    s.tiles = (s.araster + ar + 1023) & ~1023u;
    const uint32_t stage = kTileBytesA + (((uint32_t)NB * 128 + 1023) & ~1023u);
    s.keys = s.tiles + 2 * stage;
    s.misc = s.keys + (uint32_t)NB * 8;
    s.bytes = s.misc + 64;
    if (s.bytes < 120u * 1024) s.bytes = 120u * 1024;  // one CTA per SM: TMEM is taken whole
    (void)tiles;
    return s;
}

// work item: representative a, members pairs[first .. first+count) (all with pair.a == a)
struct TcItem {
    uint32_t first, count;
};

__global__ void __launch_bounds__(kThreads, 1)
    tc_corr_kernel(pcl_params prm, pcl_clipset A, pcl_clipset B, const pcl_pair *pairs, const uint32_t *surv,
                   const TcItem *items, const unsigned int *n_items, pcl_record *out, int NB, int *err) {
    const Geo g = make_geo(prm);
    const int N = g.N, nw = g.nw, S = g.S, K2 = 2 * S + 1, nshift = K2 * K2;
    const int tiles = (nshift + 127) / 128;
    const int nstage = N * N / kStageK;
    const TcSmem plan = tc_smem(N, NB, tiles);
    extern __shared__ __align__(1024) unsigned char sm[];
    uint4 *lut = reinterpret_cast<uint4 *>(sm + plan.lut);
    uint64_t *araster = reinterpret_cast<uint64_t *>(sm + plan.araster);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(sm + plan.keys);
    uint32_t *misc = reinterpret_cast<uint32_t *>(sm + plan.misc);  // [0] tmem base, [2..5] mbarriers
    const uint32_t stage_bytes = kTileBytesA + ((NB * 128 + 1023) & ~1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t mbar0 = smem_u32(misc + 2), mbar1 = smem_u32(misc + 4);

    // bit -> FP16 table: entry v holds 8 halves, element k = bit k of v
    for (int v = tid; v < 256; v += kThreads) {
        uint32_t w[4];
        for (int q = 0; q < 4; ++q) {
            const uint32_t lo = ((v >> (2 * q)) & 1) ? 0x3C00u : 0u;
            const uint32_t hi = ((v >> (2 * q + 1)) & 1) ? 0x3C00u : 0u;
            w[q] = lo | (hi << 16);
        }
        lut[v] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(misc)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = misc[0];
    const uint32_t idesc = idesc_f16(128, NB);
    bool failed = false;

    const unsigned int nit = *n_items;
    uint32_t u = 0;  // units (shift tile, stage) issued by this CTA, for the mbarrier phases
    for (unsigned int it = blockIdx.x; it < nit && !failed; it += gridDim.x) {
        const TcItem item = items[it];
        const uint32_t a = pairs[surv[item.first]].a;
        const uint64_t *abits = A.bits + (size_t)a * N * nw;
        for (int t = tid; t < N * nw; t += kThreads) araster[t] = abits[t];
        __syncthreads();
        // ---- main loop: shift tiles m (each with its own accumulator columns)
        //      x stages s (64 pixels of one image row)
        for (int m = 0; m < tiles && !failed; ++m) {
            for (int s = 0; s < nstage; ++s) {
                const int buf = u & 1;
                const uint32_t mb = buf ? mbar1 : mbar0;
                // this buffer was last read by the MMAs of unit u - 2
                if (u >= 2 && !mbar_wait(mb, ((u - 2) >> 1) & 1)) failed = true;
                failed = __syncthreads_or(failed);
                if (failed) break;
                unsigned char *tileA = sm + plan.tiles + buf * stage_bytes;
                unsigned char *tileB = tileA + kTileBytesA;
                const int y = s / nw, w0 = s % nw, x0 = 64 * w0;
                // member tile: row n = member n's 64 pixels of this stage
                for (int q = tid; q < NB * 8; q += kThreads) {
                    const int n = q >> 3, j = q & 7;
                    uint64_t bits = 0;
                    if (n < (int)item.count) {
                        const uint32_t b = pairs[surv[item.first + n]].b;
                        bits = B.bits[((size_t)b * N + y) * nw + w0];
                    }
                    const uint32_t byte = (uint32_t)(bits >> (8 * j)) & 0xFFu;
                    *reinterpret_cast<uint4 *>(tileB + (n >> 3) * 1024 + j * 128 + (n & 7) * 16) = lut[byte];
                }
                // shifted-representative tile: thread = row of the tile
                {
                    const int t = m * 128 + tid;
                    uint64_t bits = 0;
                    if (t < nshift) {
                        const int dy = t / K2 - S, dx = t % K2 - S;
                        const int yy = y + dy;
                        if (yy >= 0 && yy < N) bits = bit_window(araster + (size_t)yy * nw, nw, x0 + dx);
                    }
                    unsigned char *row = tileA + (tid >> 3) * 1024 + (tid & 7) * 16;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        *reinterpret_cast<uint4 *>(row + j * 128) = lut[(uint32_t)(bits >> (8 * j)) & 0xFFu];
                }
                fence_proxy_async();
                fence_before();
                __syncthreads();
                fence_after();
                if (tid == 0) {
                    const uint32_t aaddr = smem_u32(tileA), baddr = smem_u32(tileB);
                    const uint32_t dcol = tmem + (uint32_t)(m * NB);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = smem_desc(aaddr + kk * 256, 128, 1024);
                        const uint64_t bd = smem_desc(baddr + kk * 256, 128, 1024);
                        mma_f16(dcol, ad, bd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(mb);
                }
                ++u;
            }
        }
        // ---- drain: the commits of the last two units
        if (!failed) {
            for (uint32_t k = (u >= 2 ? u - 2 : 0); k < u; ++k)
                if (!mbar_wait((k & 1) ? mbar1 : mbar0, (k >> 1) & 1)) failed = true;
        }
        failed = __syncthreads_or(failed);
        if (failed) break;
        fence_after();
        // ---- epilogue: exact argmax per member over all shift tiles
        for (int n = tid; n < NB; n += kThreads) keys[n] = 0ull;
        __syncthreads();
        for (int m = 0; m < tiles; ++m) {
            for (int c0 = 0; c0 < NB; c0 += 16) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(m * NB + c0), r);
                tmem_wait_ld();
                const int t = m * 128 + warp * 32 + lane;
                const bool valid = t < nshift;
                const int dy = t / K2 - S, dx = t % K2 - S;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float f = __uint_as_float(r[q]);
                    const uint32_t c = valid ? (uint32_t)f : 0u;
                    unsigned long long k = valid ? shift_key(c, dx, dy, S) : 0ull;
#pragma unroll
                    for (int o = 16; o; o >>= 1) {
                        const unsigned long long w = __shfl_xor_sync(0xffffffffu, k, o);
                        k = w > k ? w : k;
                    }
                    if (lane == 0 && c0 + q < NB) atomicMax(keys + c0 + q, k);
                }
            }
        }
        fence_before();
        __syncthreads();
        fence_after();
        for (int n = tid; n < (int)item.count; n += kThreads) {
            const uint32_t pi = surv[item.first + n];
            const pcl_pair pr = pairs[pi];
            const unsigned long long k = keys[n];
            const int dx = S - (int)(k & 0xffu), dy = S - (int)((k >> 8) & 0xffu);
            const uint32_t cb = (uint32_t)(k >> 32);
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
            out[pi] = rec;
        }
        __syncthreads();
    }
    if (failed) {
        // let every MMA still in flight finish before the memory is released
        for (uint32_t k = (u >= 2 ? u - 2 : 0); k < u; ++k) (void)mbar_wait((k & 1) ? mbar1 : mbar0, (k >> 1) & 1);
        if (tid == 0) atomicExch(err, 1);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ---- preparation: gates, survivors (stable), representative segments, items

// warp per pair: indices, emptiness, gates; records for pairs that end here
__global__ void tc_gate_kernel(pcl_params prm, pcl_clipset A, pcl_clipset B, const pcl_pair *pairs, uint64_t n,
                               const unsigned long long *d_n, pcl_record *out, uint32_t *keep) {
    if (d_n && *d_n < n) n = *d_n;
    const Geo g = make_geo(prm);
    const int lane = threadIdx.x & 31;
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t t = wid; t < n; t += nwarps) {
        const pcl_pair pr = pairs[t];
        pcl_record rec{};
        rec.a = pr.a;
        rec.b = pr.b;
        rec.mode = PCL_MODE_COSINE;
        bool done = true;
        if (pr.a >= A.n_clips || pr.b >= B.n_clips) {
            rec.flags = PCL_GATE_BAD_INDEX;
        } else if (A.pop[pr.a] == 0 && B.pop[pr.b] == 0) {
            rec.flags = PCL_F_EMPTY;
            rec.sim = 1.0f;
            rec.pass = 1;
        } else {
            int gate = 0;
            if (!(prm.flags & PCL_P_NO_GATES)) gate = warp_cosine_gate(A, pr.a, B, pr.b, g, prm.cos_num, prm.cos_den, lane);
            if (gate) rec.flags = (uint16_t)gate;
            else done = false;
        }
        if (lane == 0) {
            if (done) out[t] = rec;
            keep[t] = done ? 0u : 1u;
        }
    }
}

// exclusive scan of v[0..m) into out[0..m] (out[m] = total), single CTA
__global__ void __launch_bounds__(1024) tc_scan_kernel(const uint32_t *v, uint32_t m, uint32_t *out) {
    __shared__ uint32_t wsum[32];
    const uint32_t per = (m + 1023) / 1024;
    const uint32_t lo = threadIdx.x * per, hi = min(m, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; ++i) s += v[i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t run = x - s + (wid ? wsum[wid - 1] : 0u);
    for (uint32_t i = lo; i < hi; ++i) {
        out[i] = run;
        run += v[i];
    }
    if (threadIdx.x == 1023) out[m] = run;
}

// survivors in list order; item starts where the representative changes or a
// batch of NB members is full
__global__ void tc_compact_kernel(const uint32_t *keep, const uint32_t *pos, uint64_t n,
                                  const unsigned long long *d_n, uint32_t *surv) {
    if (d_n && *d_n < n) n = *d_n;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x)
        if (keep[t]) surv[pos[t]] = (uint32_t)t;
}

__global__ void tc_seg_kernel(const pcl_pair *pairs, const uint32_t *surv, const uint32_t *n_surv, uint32_t *head) {
    const uint32_t ns = *n_surv;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x)
        head[i] = (i == 0 || pairs[surv[i]].a != pairs[surv[i - 1]].a) ? 1u : 0u;
}

// one item per (segment, batch of NB): written after a scan of segment heads;
// seg_end[k] found as the next head
__global__ void tc_items_kernel(const uint32_t *head, const uint32_t *hpos, const uint32_t *n_surv, int NB,
                                TcItem *items, unsigned int *n_items, uint32_t cap) {
    const uint32_t ns = *n_surv;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
        if (!head[i]) continue;
        uint32_t e = i + 1;
        while (e < ns && !head[e]) ++e;
        for (uint32_t f = i; f < e; f += (uint32_t)NB) {
            const unsigned int k = atomicAdd(n_items, 1u);
            if (k < cap) items[k] = TcItem{f, min((uint32_t)NB, e - f)};
        }
    }
    (void)hpos;
}

}  // namespace

int tc_batch(const Geo &g) {
    const int tiles = ((2 * g.S + 1) * (2 * g.S + 1) + 127) / 128;
    int nb = (int)(kTmemCols / (uint32_t)tiles) / 16 * 16;
    if (nb > kMaxNB) nb = kMaxNB;
    return nb;
}

size_t tc_workspace(uint64_t n) { return 4 * (3 * (size_t)n + 8) + sizeof(TcItem) * (size_t)(n + 1) + 256; }

cudaError_t launch_tc(const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b, const pcl_pair *pairs,
                      uint64_t n, const unsigned long long *d_n, pcl_record *out, void *ws, size_t ws_bytes,
                      int num_sms, int *d_err, cudaStream_t st) {
    const Geo g = make_geo(prm);
    const int NB = tc_batch(g);
    if (NB < 16 || n == 0) return n == 0 ? cudaSuccess : cudaErrorNotSupported;
    if (ws_bytes < tc_workspace(n) || n > 0xffffffffull) return cudaErrorInvalidValue;
    char *w = static_cast<char *>(ws);
    uint32_t *keep = reinterpret_cast<uint32_t *>(w);
    uint32_t *pos = keep + n;           // n + 1
    uint32_t *surv = pos + n + 1;       // n
    uint32_t *misc = surv + n;          // [0] n_items
    TcItem *items = reinterpret_cast<TcItem *>(((uintptr_t)(misc + 8) + 15) & ~uintptr_t(15));
    unsigned int *n_items = misc;
    cudaError_t e = cudaMemsetAsync(keep, 0, 4 * (size_t)n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(misc, 0, 32, st);
    if (e != cudaSuccess) return e;
    tc_gate_kernel<<<num_sms * 8, 256, 0, st>>>(prm, a, b, pairs, n, d_n, out, keep);
    tc_scan_kernel<<<1, 1024, 0, st>>>(keep, (uint32_t)n, pos);
    tc_compact_kernel<<<num_sms * 4, 256, 0, st>>>(keep, pos, n, d_n, surv);
    // segment heads over the survivors (keep reused as head flags)
    tc_seg_kernel<<<num_sms * 4, 256, 0, st>>>(pairs, surv, pos + n, keep);
    tc_items_kernel<<<num_sms * 4, 256, 0, st>>>(keep, nullptr, pos + n, NB, items, n_items, (uint32_t)n + 1);
    const int tiles = ((2 * g.S + 1) * (2 * g.S + 1) + 127) / 128;
    const TcSmem plan = tc_smem(g.N, NB, tiles);
    e = cudaFuncSetAttribute(tc_corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.bytes);
    if (e != cudaSuccess) return e;
    tc_corr_kernel<<<num_sms, kThreads, plan.bytes, st>>>(prm, a, b, pairs, surv, items, n_items, out, NB, d_err);
    return cudaGetLastError();
}

}  // namespace pcl

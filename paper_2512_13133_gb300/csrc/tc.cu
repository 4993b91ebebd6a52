// a8: direct windowed correlation on the 5th-generation tensor cores.
//
// For one representative A and the members B_n listed with it,
//   c_n(dy, dx) = sum_{y,x} A(y + dy, x + dx) B_n(y, x)     (c(s) = sum_x A(x) B(x - s))
// over the marker window |dx|, |dy| <= S is computed as a GEMM
//   D[m, col] = sum_k Aop[m, k] Bop[k, col]
// with K = pixels, M = 128 shifts and N = (member copy, member) columns.  0/1
// operands are exact in FP16 (1.0 = 0x3C00), BF16 (1.0 = 0x3F80) or E4M3
// (1.0 = 0x38), and the FP32
// sums stay below 2^24, so the tensor cores return the exact integer overlaps
// (no rounding guard is needed).
//
// M side, no per-stage writes: for each column phase (CH pixels = one 16-byte
// core-matrix row) the CTA keeps 16 copies of A's column strip, copy g shifted
// by dx_a = g - S, interleaved by image row ([row][copy][16 B], zero padded).
// An M tile is 8 consecutive image rows x 16 copies: M row m = (dy offset
// m >> 4, copy m & 15).  A core matrix is 8 copies of one row (128-byte
// aligned); the next K core matrix is the next row (256 bytes on) and the next
// image row of a stage moves the descriptor start by 256 bytes, so no operand
// is rewritten per stage.
// N side, a ring of member tiles: member n appears NBX x JB times, copy (i, jb)
// shifted by (16 i, 8 jb) pixels, so that with D's (copy g, dy offset r)
//   dx = -S + g + 16 i,   dy = -S + r + 8 jb,
// covering [-S, -S + 16 NBX) x [-S, -S + 8 JB).  A ring entry holds the jb = 0
// rows of one stage (8 image rows); the rows 8 jb above are the previous
// entries, and entry e sits at position RR - 1 - e % RR so that entries e,
// e - 1, .., e - JB + 1 are adjacent and one descriptor spans them (positions
// RR .. RR + JB - 2 mirror 0 .. JB - 2; each phase starts with JB - 1 zero
// entries).  The K loop runs over every row and column the member copies
// reach, so each product of the window is summed.  The rest of the window --
// the row dy = -S + 8 JB (= S) and, when -S + 16 NBX <= S, the column
// dx = -S + 16 NBX: an L of at most 4S + 1 shifts -- is counted exactly with
// AND + popcount on the CUDA cores, where its projection-profile bound can
// reach the best overlap of the core.
//
// Warp roles (one CTA per SM, 12 warps):
//   warps 0-1   one thread each issues tcgen05.mma (kind::f16, K = 16, or
//               kind::f8f6f4, K = 32) for alternate ring entries into its own
//               accumulator copy, and tcgen05.commit;
//   warps 2-3   write the 16 shifted copies of the next column phase (two
//               buffers);
//   warps 4-7   load member rows into registers a pair of entries ahead
//               (ping-pong buffers) and write the ring entries in pairs;
//   warps 8-11  the accumulators (tcgen05.ld; warp w reads TMEM lanes
//               32 (w % 4) ..; the two copies are added), the exact argmax with
//               the tie order (-c, |dx|+|dy|, dy, dx), the rest of the window,
//               and the records.
// Buffers change hands through mbarriers (producers arrive; tcgen05.commit
// releases), and the accumulators are double buffered in TMEM (2 x 256
// columns), so the epilogue of one item overlaps the MMAs of the next.  Every
// wait is bounded (one second unless the context sets another limit): on
// time-out the CTA records an error, each role leaves its loop, and the MMAs
// still in flight are waited for (always with the one-second limit) before the
// tensor memory is released.
#include <climits>

#include "gates.cuh"

namespace pcl {

namespace {

constexpr int kWarps = 12;
constexpr int kThreads = 32 * kWarps;
constexpr int kIssuers = 2;              // warps 0-1: one MMA-issuing thread each
constexpr int kAProd = 64;               // warps 2-3
constexpr int kBProd = 128;              // warps 4-7
constexpr int kEpi = 128;                // warps 8-11
constexpr int kKS = 4;                   // K steps (MMA K) per stage
constexpr int kCores = 2 * kKS;          // image rows (K core matrices) per stage
constexpr int kCopies = 16;              // shifted copies of the representative
constexpr int kMaxCols = 256;            // N of one MMA / one accumulator buffer
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kSmemMax = 227 * 1024;
constexpr unsigned long long kWaitNs = 1000000000ull;
enum { kBarB = 1, kBarEpi = 2 };
// mbarrier indices: a_full[2], a_empty[2], acc_full[2], acc_empty[2], fin, b_full[R], b_empty[R]
enum { kAFull = 0, kAEmpty = 2, kAccFull = 4, kAccEmpty = 6, kFin = 8, kBFull = 9 };

// operand types (both MMA operands always have the same one)
enum { kOpF16 = 0, kOpBF16 = 1, kOpE4M3 = 2 };

template <int S, int NW, int OP>
struct Tc {
    static constexpr int N = 64 * NW;
    static constexpr int NBX = (2 * S) / 16 > 0 ? (2 * S) / 16 : 1;  // x copies of a member (16 px apart)
    static constexpr int NBY = (2 * S) / 8 > 0 ? (2 * S) / 8 : 1;    // 8-row dy blocks of the core
    static constexpr int JB = NBY;                                    // dy blocks, all on the member side
    static constexpr int JA = 1;                                      // MMAs per K step
    static constexpr int NCOPY = NBX * JB;                            // member copies per MMA
    // members per item: each issuer accumulates into its own copy of the
    // N columns, and both copies fit one 256-column accumulator buffer
    static constexpr int NB = kMaxCols / kIssuers / (JA * NCOPY);
    static constexpr int NMAX = NCOPY * NB;                           // N of one MMA at most
    // member rounding: N % 16 == 0, and each ring entry (NBX * nbp columns) ends on an 8-column group
    static constexpr int RND = 16 / NCOPY > 8 / NBX ? 16 / NCOPY : 8 / NBX;
    static constexpr int DYL = -S + 8 * NBY;                          // rest row
    static constexpr int DXL = -S + 16 * NBX;                         // rest column, if <= S
    static constexpr bool COL = DXL <= S;
    static constexpr int CH = OP == kOpE4M3 ? 16 : 8;                 // pixels per 16-byte row
    static constexpr int YHI = (N + 8 * (JB - 1) + kCores - 1) / kCores * kCores;  // K image rows
    static constexpr int NST = YHI / kCores;                          // stages per phase
    static constexpr int ZE = JB - 1;                                 // zero entries per phase
    static constexpr int NPH = (N + 16 * (NBX - 1)) / CH;             // column phases
    static constexpr int ROWS = YHI + 8 + 8 * JB * (JA - 1);          // rows of one copy
    static constexpr uint32_t ABYTES = (uint32_t)kCopies * ROWS * 16;
    static constexpr int STRIP = 16 * (NBX - 1);                      // strip start left of the phase
    static constexpr int WPT = STRIP > 0 ? 2 : 1;                     // 64-bit words per staged strip
    static constexpr int TASKS = NB * kCores;                         // (member, row) tasks per stage
    static constexpr int TPT = TASKS / kBProd;                        // tasks per producer thread
    static constexpr uint32_t HBMAX = (uint32_t)(NMAX / JB) * 16;     // one entry, one K core, at most
    // ring residues: as many as shared memory holds (even, at most 18), so
    // that up to RR - JB entries are in flight between producers and MMAs
    static constexpr uint32_t OTHER = 2 * ABYTES + (uint32_t)NB * 8 + (uint32_t)(kBFull + 2 * 18) * 8 + 16;
    static constexpr int RFIT = (int)((kSmemMax - OTHER) / (kCores * HBMAX)) - (JB - 1);
    static constexpr int RR = (RFIT > 18 ? 18 : RFIT) & ~1;
    static constexpr int POS = RR + JB - 1;                           // ring positions (JB - 1 mirrors)
    static constexpr uint32_t RING = (uint32_t)POS * kCores * HBMAX;
    static constexpr int PD = TPT * WPT >= 16 ? 1 : 16 / (TPT * WPT);  // register prefetch depth (stages)
    static constexpr uint32_t OFF_RING = 2 * ABYTES;
    static constexpr uint32_t OFF_KEYS = OFF_RING + RING;
    static constexpr uint32_t OFF_BARS = OFF_KEYS + (uint32_t)NB * 8;
    static constexpr uint32_t BYTES = OFF_BARS + (uint32_t)(kBFull + 2 * RR) * 8 + 16;
    static_assert(CH + STRIP <= 32, "member strip exceeds 32 bits");
    static_assert(NPH * CH == N + 16 * (NBX - 1), "column phases do not cover the member copies");
    static_assert(kThreads == 32 * kIssuers + kAProd + kBProd + kEpi && kEpi == 128, "warp roles");
    static_assert(JA == 1 && (NST + ZE) % 2 == 0 && RR % kIssuers == 0, "issuers alternate entries, producers pair them");
    static_assert(TASKS % kBProd == 0 && NB % RND == 0 && JA * JB == NBY, "task split");
    static_assert((NBX * RND) % 8 == 0 || JB == 1, "an entry must end on an 8-column group");
    static_assert(RR - JB + 1 >= 3, "producers run at least three entries ahead");
    static_assert(kCores == 8, "the member-side dy copy (8 rows up) is the previous stage");
    static_assert(PD >= 2 && BYTES <= kSmemMax, "shared memory plan");
};

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

// instruction descriptor: D = F32 (bit 4), A and B formats in bits 7-9 and
// 10-12 (kind::f16: 0 = F16, 1 = BF16; kind::f8f6f4: 0 = E4M3), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_of(int M, int N, int op) {
    const uint32_t ab = op == kOpBF16 ? 1u : 0u;  // the same format for A and B
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <bool FP8>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (FP8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}

// the low CH pixels (bits) of b as one 16-byte core-matrix row of 0 / 1.0
template <int OP>
__device__ __forceinline__ uint4 expand(uint32_t b) {
    if constexpr (OP == kOpE4M3) {
        // a nibble times 0x00204081 puts bit k at bit 8k (no carries), masked to 0/1 bytes
        auto q = [](uint32_t nib) { return ((nib * 0x00204081u) & 0x01010101u) * 0x38u; };
        return make_uint4(q(b & 15u), q((b >> 4) & 15u), q((b >> 8) & 15u), q((b >> 12) & 15u));
    } else {
        constexpr uint32_t one = OP == kOpBF16 ? 0x3F80u : 0x3C00u;  // 1.0 in the 16-bit format
        auto h = [](uint32_t v) { return ((v & 1u) | ((v & 2u) << 15)) * one; };
        return make_uint4(h(b & 3u), h((b >> 2) & 3u), h((b >> 4) & 3u), h((b >> 6) & 3u));
    }
}

__device__ __forceinline__ void st16(unsigned char *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }
// 16-byte store to a shared-memory address (shared state space, not generic)
__device__ __forceinline__ void sts16(uint32_t a, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
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

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for the phase of the given parity; false after limit_ns or
// when another role has aborted (abort_flag may be null: wait regardless)
__device__ __forceinline__ bool wait_phase_slow(uint32_t mbar, uint32_t parity, const volatile uint32_t *abort_flag,
                                                unsigned long long limit_ns) {
    const uint64_t t0 = gtimer();
    for (;;) {
        for (int i = 0; i < 16; ++i)
            if (mbar_try_wait(mbar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if (gtimer() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity, const volatile uint32_t *abort_flag,
                                           unsigned long long limit_ns) {
    return mbar_try_wait(mbar, parity) || wait_phase_slow(mbar, parity, abort_flag, limit_ns);
}

// barrier over `count` threads of one role that also ORs a flag
__device__ __forceinline__ bool bar_any(int id, int count, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void bar_sync(int id, int count) {
    asm volatile("barrier.cta.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
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

// 64 bits of a bit row starting at pixel `base` (zeros outside the row)
template <int NW>
__device__ __forceinline__ uint64_t bit_window(const uint64_t *row, int base) {
    const int wi = base >= 0 ? base >> 6 : -((-base + 63) >> 6);
    const int off = base - 64 * wi;
    const uint64_t lo = (wi >= 0 && wi < NW) ? __ldg(row + wi) : 0ull;
    const uint64_t hi = (wi + 1 >= 0 && wi + 1 < NW) ? __ldg(row + wi + 1) : 0ull;
    return off ? ((lo >> off) | (hi << (64 - off))) : lo;
}

__device__ __forceinline__ unsigned long long warp_max64(unsigned long long k) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, k, o);
        k = w > k ? w : k;
    }
    return k;
}

// Row ya of A shifted left by SH pixels (pixels x + SH), zero outside the raster.
template <int NW, int SH>
__device__ __forceinline__ void shifted_row(const uint64_t *__restrict__ A, int ya, uint64_t (&o)[NW]) {
    uint64_t a[NW + 1];
    const bool in = ya >= 0 && ya < 64 * NW;
#pragma unroll
    for (int w = 0; w < NW; ++w) a[w] = in ? __ldg(A + (size_t)ya * NW + w) : 0ull;
    a[NW] = 0ull;
#pragma unroll
    for (int w = 0; w < NW; ++w) o[w] = (a[w] >> SH) | (a[w + 1] << (64 - SH));
}

// The rest of the window for one pair is counted exactly by one warp, lanes
// taking 32 consecutive rows y of B at a time.  Row part: dy = DYL for every
// dx in [-S, S], shifting A's row y + DYL in registers.  Returns the largest
// shift key among these shifts (the same in every lane).
template <int S, int NW, int DYL>
__device__ __forceinline__ unsigned long long rest_row_key(const uint64_t *__restrict__ A,
                                                           const uint64_t *__restrict__ B, int lane) {
    constexpr int N = 64 * NW;
    uint32_t cr[2 * S + 1];
#pragma unroll
    for (int d = 0; d <= 2 * S; ++d) cr[d] = 0;
    for (int y = lane; y + DYL < N; y += 32) {
        uint64_t b[NW];
        // a[w + 1] = word w of A's row y + DYL, zero words on both sides
        uint64_t a[NW + 2];
        a[0] = 0ull;
        a[NW + 1] = 0ull;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            b[w] = __ldg(B + (size_t)y * NW + w);
            a[w + 1] = __ldg(A + (size_t)(y + DYL) * NW + w);
        }
#pragma unroll
        for (int d = 0; d <= 2 * S; ++d) {
            const int dx = d - S;
            uint32_t sum = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                uint64_t sh;  // A's pixels x + dx for the x of word w
                if (dx > 0) sh = (a[w + 1] >> dx) | (a[w + 2] << (64 - dx));
                else if (dx < 0) sh = (a[w + 1] << (-dx)) | (a[w] >> (64 + dx));
                else sh = a[w + 1];
                sum += (uint32_t)__popcll(sh & b[w]);
            }
            cr[d] += sum;
        }
    }
    unsigned long long best = 0ull;
#pragma unroll
    for (int d = 0; d <= 2 * S; ++d) {
        const unsigned long long k = shift_key(__reduce_add_sync(0xffffffffu, cr[d]), d - S, DYL, S);
        best = k > best ? k : best;
    }
    return best;
}

// Column part: dx = DXL for dy in [-S, S).  Lane l needs A's row y0 + l + dy
// shifted by DXL; the warp holds two blocks of 32 shifted rows (y0 - S + l
// and y0 - S + 32 + l), and the row for dy is block row m = l + dy + S, i.e.
// lane (m & 31) of block m >> 5: a source lane j serves block 0 when
// j >= e (= dy + S), else block 1, so one shuffle per word suffices.
template <int S, int NW, int DXL>
__device__ __forceinline__ unsigned long long rest_col_key(const uint64_t *__restrict__ A,
                                                           const uint64_t *__restrict__ B, int lane) {
    constexpr int N = 64 * NW;
    static_assert(2 * S <= 32, "column rest spans more than two row blocks");
    uint32_t cc[2 * S];
#pragma unroll
    for (int e = 0; e < 2 * S; ++e) cc[e] = 0;
    for (int y0 = 0; y0 < N; y0 += 32) {
        const int y = y0 + lane;
        uint64_t b[NW], s0[NW], s1[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) b[w] = __ldg(B + (size_t)y * NW + w);
        shifted_row<NW, DXL>(A, y0 - S + lane, s0);
        shifted_row<NW, DXL>(A, y0 - S + 32 + lane, s1);
#pragma unroll
        for (int e = 0; e < 2 * S; ++e) {
            uint32_t sum = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint64_t v = __shfl_sync(0xffffffffu, lane >= e ? s0[w] : s1[w], (lane + e) & 31);
                sum += (uint32_t)__popcll(v & b[w]);
            }
            cc[e] += sum;
        }
    }
    unsigned long long best = 0ull;
#pragma unroll
    for (int e = 0; e < 2 * S; ++e) {
        const unsigned long long k = shift_key(__reduce_add_sync(0xffffffffu, cc[e]), DXL, e - S, S);
        best = k > best ? k : best;
    }
    return best;
}

// work item: representative a, members pairs[surv[first .. first+count)] (all with pair.a == a)
struct TcItem {
    uint32_t first, count;
};

template <int RND>
__device__ __forceinline__ int round_members(uint32_t count) {
    return (int)((count + RND - 1) / RND * RND);
}

// The strip words of one stage (phase ph, stage st) for one member-tile
// producer thread: rows st * kCores + q of its tasks' members, words w0 and
// w0 + 1 around the strip (zero outside the raster).  Plain read-only loads
// into registers, issued stages ahead of their use.
template <typename C>
__device__ __forceinline__ void stage_load(uint64_t (&o)[C::TPT][C::WPT], const uint64_t *const (&mb)[C::TPT], int bt,
                                           int ph, int st) {
    const int sb = ph * C::CH - C::STRIP;
    const int w0 = sb >= 0 ? sb >> 6 : -((-sb + 63) >> 6);
#pragma unroll
    for (int u = 0; u < C::TPT; ++u) {
        const int row = st * kCores + (bt + kBProd * u) / C::NB;
#pragma unroll
        for (int e = 0; e < C::WPT; ++e) {
            const int w = w0 + e;
            o[u][e] = (mb[u] && row < C::N && w >= 0 && w < C::N / 64) ? __ldg(mb[u] + (size_t)row * (C::N / 64) + w)
                                                                       : 0ull;
        }
    }
}

template <int S, int NW, int OP>
__global__ void __launch_bounds__(kThreads, 1)
    tc_corr_kernel(pcl_params prm, pcl_clipset A, pcl_clipset B, const pcl_pair *pairs, const uint32_t *surv,
                   const TcItem *items, const unsigned int *n_items, pcl_record *out, int *err,
                   unsigned long long wait_ns) {
    using C = Tc<S, NW, OP>;
    constexpr int N = C::N, RR = C::RR;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(sm + C::OFF_KEYS);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + C::OFF_BARS);
    volatile uint32_t *misc = reinterpret_cast<volatile uint32_t *>(bars + kBFull + 2 * RR);  // [0] tmem, [1] abort
    const volatile uint32_t *abortf = misc + 1;
    const uint32_t sbase = smem_u32(sm);
    const uint32_t bar0 = smem_u32(bars);
    auto bar = [&](int k) { return bar0 + 8u * (uint32_t)k; };
    auto raise_abort = [&]() {
        misc[1] = 1u;
        atomicExch(err, 1);
    };
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int n = tid; n < C::NB; n += kThreads) keys[n] = 0ull;
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(bar(kAFull + k), kAProd);
            mbar_init(bar(kAEmpty + k), kIssuers);
            mbar_init(bar(kAccFull + k), kIssuers);
            mbar_init(bar(kAccEmpty + k), kEpi);
        }
        mbar_init(bar(kFin), kIssuers);
        for (int k = 0; k < RR; ++k) {
            mbar_init(bar(kBFull + k), kBProd);
            mbar_init(bar(kBFull + RR + k), 1);
        }
        misc[1] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(
                         (const void *)misc)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = misc[0];
    const unsigned int nit = *n_items;

    if (warp < kIssuers) {
        // ---------------------------------------------------------------- MMA issue
        // Member tiles arrive as ring entries e (per phase: JB - 1 zero
        // entries, then one entry per stage).  Entry e sits at position
        // RR - 1 - e % RR, so entries e - 1, e - 2, .. follow it in memory
        // (positions RR .. RR + JB - 2 mirror 0 .. JB - 2): one descriptor
        // reads "this stage's rows | the rows 8 above | 16 above | .." as the
        // JB blocks of N.  An issuing thread can start one tcgen05 instruction
        // (MMA or commit) about every 150 cycles whatever N is, so two warps
        // issue: warp w takes the entries e = w (mod 2) into its own
        // accumulator copy (columns w * ncols of the buffer) and commits them;
        // the epilogue adds the copies.
        if (lane == 0) {
            const int iw = warp;
            bool ok = true;
            uint32_t pc = 0, e = 0, li = 0;
            for (unsigned int it = blockIdx.x; it < nit && ok; it += gridDim.x, ++li) {
                const TcItem item = items[it];
                const int ncols = C::NCOPY * round_members<C::RND>(item.count);  // N of each MMA
                const uint32_t hb = (uint32_t)(ncols / C::JB) * 16, lbo = (uint32_t)C::POS * hb;
                const uint32_t idesc = idesc_of(128, ncols, OP);
                uint32_t accum = 0;  // the first MMA of the item into this copy overwrites
                const uint32_t ab = li & 1;
                if (li >= 2 && !(ok = wait_phase(bar(kAccEmpty + ab), ((li >> 1) - 1) & 1, abortf, wait_ns))) break;
                fence_after();
                const uint32_t dcol = tmem + ab * (uint32_t)kMaxCols + (uint32_t)(iw * ncols);
                // descriptors: only the start field (16-byte units) moves below
                const uint64_t bd_item = smem_desc(sbase + C::OFF_RING, lbo, 128);
                for (int ph = 0; ph < C::NPH && ok; ++ph, ++pc) {
                    const uint32_t abf = pc & 1;
                    if (!(ok = wait_phase(bar(kAFull + abf), (pc >> 1) & 1, abortf, wait_ns))) break;
                    // A copies interleaved per image row ([row][copy][16 B]): a core
                    // matrix is 8 copies of one row (128-byte aligned), the next K
                    // core matrix the next row (256 bytes), the next group of 8 M
                    // rows the other 8 copies, then the next row (128 bytes)
                    const uint64_t ad_ph = smem_desc(sbase + abf * C::ABYTES, 256, 128);
                    // entries of this phase: e0 + (st + ZE); a phase (and an item) has an
                    // even number of entries, so issuer iw takes st = -ZE + iw, -ZE + iw + 2, ..
                    const uint32_t e0 = e;
                    for (int st = -C::ZE + iw; st < C::NST; st += kIssuers) {
                        const uint32_t e = e0 + (uint32_t)(st + C::ZE);
                        if (!(ok = wait_phase(bar(kBFull + e % RR), (e / RR) & 1, abortf, wait_ns))) break;
                        if (st >= 0) {
                            // the operands were published by the producers' proxy fence
                            // and arrival; no tcgen05 fence is needed on this path
                            const uint32_t pos = RR - 1 - e % RR;
                            const uint64_t bd_e = bd_item + (uint64_t)((pos * hb) >> 4);
                            const uint64_t ad_st = ad_ph + (uint64_t)(st * kCores * 16);
#pragma unroll
                            for (int t = 0; t < kKS; ++t) {
                                // K step t: image rows Y, Y + 1 with Y = st * kCores + 2 t;
                                // M row m = (dy offset m >> 4, copy m & 15) reads A's row
                                // Y + (m >> 4) - S
                                const uint64_t bd = bd_e + (uint64_t)((2 * t * lbo) >> 4);
                                const uint64_t ad = ad_st + (uint64_t)(2 * t * 16);
                                mma<OP == kOpE4M3>(dcol, ad, bd, idesc, accum);
                                accum = 1u;
                            }
                        }
                        mma_commit(bar(kBFull + RR + e % RR));
                    }
                    e = e0 + (uint32_t)(C::NST + C::ZE);
                    if (ok) mma_commit(bar(kAEmpty + abf));
                }
                if (ok) mma_commit(bar(kAccFull + ab));
            }
            if (!ok) raise_abort();
            // every MMA issued so far has completed before the tensor memory is released
            mma_commit(bar(kFin));
            if (!wait_phase(bar(kFin), 0, nullptr, kWaitNs)) raise_abort();  // always the full limit
        }
        __syncwarp();
    } else if (warp < kIssuers + kAProd / 32) {
        // ---------------------------------------------------------------- shifted copies of A
        const int pt = tid - 32 * kIssuers;
        bool ok = true;
        uint32_t pc = 0;
        for (unsigned int it = blockIdx.x; it < nit && ok; it += gridDim.x) {
            const TcItem item = items[it];
            const uint64_t *abits = A.bits + (size_t)pairs[surv[item.first]].a * N * NW;
            for (int ph = 0; ph < C::NPH; ++ph, ++pc) {
                const uint32_t abf = pc & 1;
                if (pc >= 2 && !(ok = wait_phase(bar(kAEmpty + abf), ((pc >> 1) - 1) & 1, abortf, wait_ns))) break;
                unsigned char *buf = sm + abf * C::ABYTES;
                const int base = ph * C::CH - S;  // copy g, pixel k = A column base + g + k
                // (row ridx, copy g) at 16 (16 ridx + g); a thread writes the 16
                // copies of its row, starting at copy (lane & 15) so that a warp's
                // stores spread over the banks
                for (int ridx = pt; ridx < C::ROWS; ridx += kAProd) {
                    const int yy = ridx - S;
                    uint64_t win = 0ull;
                    if (yy >= 0 && yy < N) win = bit_window<NW>(abits + (size_t)yy * NW, base);
#pragma unroll
                    for (int j = 0; j < kCopies; ++j) {
                        const int g = (j + lane) & 15;
                        st16(buf + (uint32_t)(ridx * kCopies + g) * 16, expand<OP>((uint32_t)(win >> g)));
                    }
                }
                fence_proxy_async();
                mbar_arrive(bar(kAFull + abf));
            }
        }
        if (!ok) raise_abort();
    } else if (warp < kIssuers + (kAProd + kBProd) / 32) {
        // ---------------------------------------------------------------- member tiles
        // Task k = (member n = k % NB, row q = k / NB of each stage); each
        // thread loads its own strip words (zero outside the raster) and writes
        // the NBX x copies of its row into the ring entry of the stage.  No
        // barrier among producers.
        const int bt = tid - (32 * kIssuers + kAProd);
        bool ok = true;
        uint32_t e = 0;
        const uint32_t ring_s = sbase + C::OFF_RING;
        for (unsigned int it = blockIdx.x; it < nit && ok; it += gridDim.x) {
            const TcItem item = items[it];
            const int nbp = round_members<C::RND>(item.count);
            const uint32_t hb = (uint32_t)(C::NBX * nbp) * 16, lbo = (uint32_t)C::POS * hb;
            const uint64_t *mb[C::TPT];
#pragma unroll
            for (int u = 0; u < C::TPT; ++u) {
                const int n = (bt + kBProd * u) % C::NB;
                mb[u] = n < (int)item.count ? B.bits + (size_t)pairs[surv[item.first + n]].b * N * NW : nullptr;
            }
            // Register ping-pong: the words of pair g + 1 are loaded into one
            // buffer while pair g is written from the other, so a load has a
            // whole pair of entries to arrive and no register in flight is moved.
            constexpr int PPP = (C::NST + C::ZE) / 2;  // pairs per phase
            uint64_t bufA[2][C::TPT][C::WPT], bufB[2][C::TPT][C::WPT];
            int nph = 0, nj = 0;  // next pair to load
            auto pair_load = [&](uint64_t(&b)[2][C::TPT][C::WPT]) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int st = -C::ZE + 2 * nj + h;
                    if (nph < C::NPH && st >= 0) {
                        stage_load<C>(b[h], mb, bt, nph, st);
                    } else {
#pragma unroll
                        for (int u = 0; u < C::TPT; ++u)
#pragma unroll
                            for (int w = 0; w < C::WPT; ++w) b[h][u][w] = 0ull;
                    }
                }
                if (++nj == PPP) {
                    nj = 0;
                    ++nph;
                }
            };
            bool first = true;  // the layout changes with the item: wait for the previous item's MMAs
            // done(x): the MMAs of entry x (by issuer x % 2) have completed
            auto done = [&](uint32_t x) { return wait_phase(bar(kBFull + RR + x % RR), (x / RR) & 1, abortf, wait_ns); };
            // entries e, e + 1 (stages st0, st0 + 1 of phase ph) from the words in b
            auto pair_step = [&](const uint64_t(&b)[2][C::TPT][C::WPT], int ph, int st0) -> bool {
                const int sb = ph * C::CH - C::STRIP;
                const int w0 = sb >= 0 ? sb >> 6 : -((-sb + 63) >> 6);
                const int off = sb - 64 * w0;
                uint32_t cur[2][C::TPT];
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int u = 0; u < C::TPT; ++u) {
                        const uint64_t lo = b[h][u][0];
                        const uint64_t hi = C::WPT == 2 ? b[h][u][C::WPT - 1] : 0ull;
                        cur[h][u] = (uint32_t)(off ? (lo >> off) | (hi << (64 - off)) : lo);
                    }
                // the position of entry x last held entry x - RR, read by the MMAs of
                // entries x - RR .. x - RR + JB - 1 = x - lag; with JB >= 2 those
                // come from both issuers, so the other issuer's last one, x - lag - 1,
                // is waited for too.  Every entry waited for is at least e - RR:
                // an older one shares its barrier with an entry already written,
                // and its phase parity would no longer tell the two apart.
                constexpr uint32_t lag = (uint32_t)(RR - C::JB + 1);
                bool okw = true;
                if (first) {
                    if (e >= 1) okw = done(e - 1);
                    if (okw && e >= 2) okw = done(e - 2);
                } else {
                    if (C::JB >= 2 && e >= lag + 1) okw = done(e - lag - 1);
                    if (okw && e >= lag) okw = done(e - lag);
                    if (okw && e + 1 >= lag) okw = done(e + 1 - lag);
                }
                first = false;
                if (!okw) return false;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t pos = RR - 1 - (e + h) % RR;
                    const uint32_t d0 = ring_s + pos * hb;
                    // positions RR .. RR + JB - 2 mirror 0 .. JB - 2
                    const bool mir = C::JB > 1 && pos + 1 < (uint32_t)C::JB;
                    const uint32_t d1 = ring_s + (pos + RR) * hb;
                    const int st = st0 + h, Ys = st * kCores;
#pragma unroll
                    for (int u = 0; u < C::TPT; ++u) {
                        const int k = bt + kBProd * u, n = k % C::NB, q = k / C::NB;
                        if (n >= nbp) continue;
                        const bool v = st >= 0 && n < (int)item.count && Ys + q < N;
                        const uint32_t strip = v ? cur[h][u] : 0u;
#pragma unroll
                        for (int i = 0; i < C::NBX; ++i) {
                            const int c0 = i * nbp + n;
                            const uint32_t o = (uint32_t)q * lbo + (uint32_t)(c0 >> 3) * 128 + (uint32_t)(c0 & 7) * 16;
                            const uint4 x = expand<OP>(strip >> (16 * (C::NBX - 1 - i)));
                            sts16(d0 + o, x);
                            if (mir) sts16(d1 + o, x);
                        }
                    }
                }
                fence_proxy_async();
                mbar_arrive(bar(kBFull + e % RR));
                mbar_arrive(bar(kBFull + (e + 1) % RR));
                return true;
            };
            pair_load(bufA);
            uint32_t gp = 0;  // pairs of this item so far
            for (int ph = 0; ph < C::NPH && ok; ++ph) {
                for (int j = 0; j < PPP; ++j, ++gp, e += 2) {
                    const int st0 = -C::ZE + 2 * j;
                    if (gp & 1) {
                        pair_load(bufA);
                        ok = pair_step(bufB, ph, st0);
                    } else {
                        pair_load(bufB);
                        ok = pair_step(bufA, ph, st0);
                    }
                    if (!ok) break;
                }
            }
        }
        if (!ok) raise_abort();
    } else {
        // ---------------------------------------------------------------- epilogue + rest of the window
        const int et = tid - (32 * kIssuers + kAProd + kBProd), ew = et >> 5, quarter = warp & 3;
        const Geo g = make_geo(prm);
        bool ok = true;
        uint32_t li = 0;
        for (unsigned int it = blockIdx.x; it < nit; it += gridDim.x, ++li) {
            const TcItem item = items[it];
            const uint32_t a = pairs[surv[item.first]].a;
            const uint32_t ab = li & 1;
            const bool w = wait_phase(bar(kAccFull + ab), (li >> 1) & 1, abortf, wait_ns);
            if (bar_any(kBarEpi, kEpi, !w)) {
                ok = false;
                break;
            }
            fence_after();
            const int nbp = round_members<C::RND>(item.count);
            const int ncols = C::NCOPY * nbp;
            const int m = 32 * quarter + lane, gg = m & 15, rr = m >> 4;  // copy, dy offset
            // column (jb * NBX + i) * nbp + n of each accumulator copy holds
            // member n at dx = -S + g + 16 i, dy = -S + r + 8 jb
            constexpr int nacc = kIssuers;
            const uint32_t tbase = tmem + ((uint32_t)(32 * quarter) << 16) + ab * (uint32_t)kMaxCols;
            for (int c0 = 0; c0 < ncols; c0 += 16) {
                uint32_t v[16], w[16];
                tmem_ld16(tbase + (uint32_t)c0, v);
                tmem_wait_ld();
                for (int cp = 1; cp < nacc; ++cp) {
                    tmem_ld16(tbase + (uint32_t)(cp * ncols + c0), w);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = __float_as_uint(__uint_as_float(v[q]) + __uint_as_float(w[q]));
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int col = c0 + q;
                    const int b = col / nbp, n = col - b * nbp;
                    const int dx = -S + gg + 16 * (b % C::NBX);
                    const int dy = -S + rr + 8 * (b / C::NBX);
                    // the kernel's window is S = N/16; a smaller marker (g.S < S)
                    // keeps the shifts within it
                    const bool valid = dx <= S && abs(dx) <= g.S && abs(dy) <= g.S;
                    const unsigned long long k =
                        warp_max64(valid ? shift_key((uint32_t)__uint_as_float(v[q]), dx, dy, S) : 0ull);
                    if (lane == 0 && n < (int)item.count) atomicMax(keys + n, k);
                }
            }
            // the accumulators are free for item li + 2 as soon as they are read
            fence_before();
            mbar_arrive(bar(kAccEmpty + ab));
            bar_sync(kBarEpi, kEpi);
            // The rest of the window (row dy = DYL, column dx = DXL) only
            // matters where it can reach the best core overlap c*: it is
            // skipped when the projection-profile bound, which holds for every
            // shift of that row (column), is below c* -- an exact, lossless test.
            const uint64_t *abits = A.bits + (size_t)a * N * NW;
            const uint16_t *pa = A.prof + (size_t)a * 2 * N;
            for (int n = ew; n < (int)item.count; n += 4) {
                const uint32_t bi = pairs[surv[item.first + n]].b;
                const uint16_t *pb = B.prof + (size_t)bi * 2 * N;
                const unsigned long long kc = keys[n];
                const uint32_t cstar = (uint32_t)(kc >> 32);
                uint32_t brow = 0, bcol = 0;
                for (int y = lane; y < N - C::DYL; y += 32) brow += min((uint32_t)pa[y + C::DYL], (uint32_t)pb[y]);
                if constexpr (C::COL)
                    for (int x = lane; x < N - C::DXL; x += 32)
                        bcol += min((uint32_t)pa[N + x + C::DXL], (uint32_t)pb[N + x]);
                brow = __reduce_add_sync(0xffffffffu, brow);
                bcol = __reduce_add_sync(0xffffffffu, bcol);
                const uint64_t *bbits = B.bits + (size_t)bi * N * NW;
                unsigned long long k = kc;
                // the rest lies at |dy| = S or |dx| = S: outside a smaller window
                if (g.S == S && brow >= cstar) {
                    const unsigned long long r = rest_row_key<S, NW, C::DYL>(abits, bbits, lane);
                    k = r > k ? r : k;
                }
                if constexpr (C::COL) {
                    if (g.S == S && bcol >= cstar) {
                        const unsigned long long r = rest_col_key<S, NW, C::DXL>(abits, bbits, lane);
                        k = r > k ? r : k;
                    }
                }
                if (lane == 0) keys[n] = k;
            }
            bar_sync(kBarEpi, kEpi);
            for (int n = et; n < (int)item.count; n += kEpi) {
                const uint32_t pi = surv[item.first + n];
                const pcl_pair pr = pairs[pi];
                const unsigned long long k = keys[n];
                keys[n] = 0ull;
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
            bar_sync(kBarEpi, kEpi);
        }
        if (!ok) raise_abort();
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

// rasters of 64^2, 128^2 or 256^2 px with S <= N/16: the kernel of that size
// (window S = N/16) keeps the shifts of the smaller window
bool tc_supported(const Geo &g) { return (g.N == 64 || g.N == 128 || g.N == 256) && g.S >= 0 && g.S <= g.N / 16; }

size_t tc_workspace(uint64_t n) { return 4 * (3 * (size_t)n + 8) + sizeof(TcItem) * (size_t)(n + 1) + 256; }

namespace {

template <int S, int NW, int OP>
cudaError_t launch_corr(const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b, const pcl_pair *pairs,
                        const uint32_t *surv, const TcItem *items, const unsigned int *n_items, pcl_record *out,
                        int num_sms, int *d_err, unsigned long long wait_ns, cudaStream_t st) {
    using C = Tc<S, NW, OP>;
    cudaError_t e = cudaFuncSetAttribute(tc_corr_kernel<S, NW, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::BYTES);
    if (e != cudaSuccess) return e;
    tc_corr_kernel<S, NW, OP><<<num_sms, kThreads, C::BYTES, st>>>(prm, a, b, pairs, surv, items, n_items, out, d_err,
                                                                                wait_ns);
    return cudaGetLastError();
}

template <int S, int NW>
cudaError_t launch_corr_op(int op, const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b,
                           const pcl_pair *pairs, const uint32_t *surv, const TcItem *items,
                           const unsigned int *n_items, pcl_record *out, int num_sms, int *d_err,
                           unsigned long long wait_ns, cudaStream_t st) {
    switch (op) {
        case kOpE4M3: return launch_corr<S, NW, kOpE4M3>(prm, a, b, pairs, surv, items, n_items, out, num_sms, d_err, wait_ns, st);
        case kOpBF16: return launch_corr<S, NW, kOpBF16>(prm, a, b, pairs, surv, items, n_items, out, num_sms, d_err, wait_ns, st);
        default: return launch_corr<S, NW, kOpF16>(prm, a, b, pairs, surv, items, n_items, out, num_sms, d_err, wait_ns, st);
    }
}

template <int S, int NW>
int members_of() {
    return Tc<S, NW, kOpF16>::NB;  // the same for every operand type
}

}  // namespace

cudaError_t launch_tc(const pcl_params &prm, const pcl_clipset &a, const pcl_clipset &b, const pcl_pair *pairs,
                      uint64_t n, const unsigned long long *d_n, pcl_record *out, void *ws, size_t ws_bytes,
                      int num_sms, int *d_err, unsigned long long wait_ns, cudaStream_t st) {
    const Geo g = make_geo(prm);
    if (!tc_supported(g)) return cudaErrorNotSupported;
    if (wait_ns == 0) wait_ns = kWaitNs;
    if (n == 0) return cudaSuccess;
    if (ws_bytes < tc_workspace(n) || n > 0xffffffffull) return cudaErrorInvalidValue;
    const int op = prm.cos_engine == PCL_ENGINE_TC_DIRECT_FP8   ? kOpE4M3
                   : prm.cos_engine == PCL_ENGINE_TC_DIRECT_BF16 ? kOpBF16
                                                                 : kOpF16;
    const int NB = g.N == 64 ? members_of<4, 1>() : g.N == 128 ? members_of<8, 2>() : members_of<16, 4>();
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
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    switch (g.N) {
        case 64: return launch_corr_op<4, 1>(op, prm, a, b, pairs, surv, items, n_items, out, num_sms, d_err, wait_ns, st);
        case 128: return launch_corr_op<8, 2>(op, prm, a, b, pairs, surv, items, n_items, out, num_sms, d_err, wait_ns, st);
        default: return launch_corr_op<16, 4>(op, prm, a, b, pairs, surv, items, n_items, out, num_sms, d_err, wait_ns, st);
    }
}

}  // namespace pcl

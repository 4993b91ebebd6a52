// a10: serving loop -- resident representative libraries, one per raster
// size class, and continuously batched query requests (cosine mode with the
// FFT phase-correlation engine, the tensor-core direct correlation or, for
// 512^2 px clips, the exact window scan; or edge mode with the Min-Max
// procedure).  Every request names its size class; all classes share the
// request slots and the memory budget, so requests of different sizes are
// admitted together as slots and memory free up.
//
// The library's rasters and signatures stay in device memory (with the FFT
// engine also its spectra), with its clips sorted by area once.  The
// tensor-core engine reads the bit-packed rasters only, so its library costs
// N^2/8 bytes of rasters plus ~2.6 KB of signatures per clip (2,000,000 clips
// of 256^2 px: ~21 GB) instead of ~350 KB with spectra.  Each admitted request gets a slot: its own
// stream and a region of a fixed device arena holding the query clip set,
// candidates and records.  Admission needs a free slot and room in the arena
// (the memory budget), so requests that arrive while others run are admitted
// as slots and memory free up, and their kernels overlap on the device.  A
// request's work: host->device copy of its rectangles, rasterisation,
// query x library candidate join, spectra of the referenced query clips,
// phase-correlation matching, pass compaction, device->host copy of the pass
// list; a host callback on the stream stamps the completion time.  With the
// tensor-core engine the spectra and phase-correlation steps are replaced by
// the grouped direct correlation of the candidates (exact argmax).
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace pcl {
cudaError_t launch_raster(const pcl_params &, const pcl_clipset &, cudaStream_t);
cudaError_t launch_spectra(const pcl_params &, const pcl_clipset &, const uint32_t *, uint32_t, bool, cudaStream_t);
cudaError_t launch_mark(const pcl_pair *, uint64_t, const unsigned long long *, pcl_clipset &, pcl_clipset &,
                        cudaStream_t);
cudaError_t launch_pair_fft(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const pcl_pair *, uint64_t,
                            const unsigned long long *, pcl_record *, int, cudaStream_t);
cudaError_t launch_compact(const pcl_record *, uint64_t, const unsigned long long *, pcl_pair *, uint64_t,
                           unsigned long long *, cudaStream_t);
cudaError_t launch_area_sort(const uint32_t *, uint32_t, uint32_t, uint32_t *, uint32_t *, uint32_t *, uint32_t *,
                             int, cudaStream_t);
size_t cross_join_workspace(const Geo &, uint32_t, uint32_t);
bool tc_supported(const Geo &);
size_t tc_workspace(uint64_t);
cudaError_t launch_tc(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const pcl_pair *, uint64_t,
                      const unsigned long long *, pcl_record *, void *, size_t, int, int *, unsigned long long,
                      cudaStream_t);
cudaError_t launch_edge_screen_cross(const pcl_params &, const pcl_clipset &, const pcl_clipset &, pcl_pair *,
                                     uint64_t, unsigned long long *, unsigned long long *, cudaStream_t, void *,
                                     size_t, int);
cudaError_t launch_edge_match(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const pcl_pair *, uint64_t,
                              const unsigned long long *, pcl_record *, int, cudaStream_t);
cudaError_t launch_cross_join(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const uint32_t *,
                              const uint32_t *, const uint32_t *, void *, size_t, pcl_pair *, uint64_t,
                              unsigned long long *, unsigned long long *, int, cudaStream_t);
cudaError_t launch_exact_pairs(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const pcl_pair *,
                               uint64_t, const unsigned long long *, pcl_record *, int, unsigned long long *,
                               cudaStream_t);
}  // namespace pcl

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// first-fit allocator over one device region, 256-byte granules
struct Arena {
    char *base = nullptr;
    size_t bytes = 0;
    std::map<size_t, size_t> free_;  // offset -> size
    void init(char *b, size_t n) {
        base = b;
        bytes = n;
        free_.clear();
        free_[0] = n;
    }
    bool alloc(size_t n, size_t *off) {
        n = align256(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = align256(n);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Slot {
    bool busy = false, done = false;
    uint64_t id = 0;
    uint32_t cls = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    size_t off = 0, bytes = 0;
    uint32_t nq = 0;
    uint64_t cap = 0;
    pcl_clipset q{};
    pcl_pair *cand = nullptr, *pass = nullptr;
    pcl_record *rec = nullptr;
    unsigned long long *counts = nullptr;  // [0] candidates, [1] pass, [2] device error word of the request
    void *ws = nullptr;
    size_t ws_bytes = 0;
    // pinned host staging
    uint32_t *h_off = nullptr;
    int32_t *h_rects = nullptr;
    pcl_pair *h_pass = nullptr;
    pcl_record *h_rec = nullptr;
    unsigned long long *h_counts = nullptr;
    std::vector<pcl_pair> overflow;
    std::vector<pcl_record> rec_overflow;
    int64_t t_submit = 0;
    int64_t t_done = 0;  // written by the stream's host callback
    pcl_completion comp{};
};

void CUDART_CB stamp_done(void *p) { static_cast<Slot *>(p)->t_done = now_ns(); }

}  // namespace

// one resident library of one raster size class
struct ServerClass {
    pcl_params P{};
    pcl::Geo g{};
    pcl_clipset lib{};
    int engine = 0;  // kEdge, kFft, kTc or kExact
    uint32_t *lib_cum = nullptr, *lib_fill = nullptr, *lib_order = nullptr, *lib_spop = nullptr;
};

struct pcl_server {
    pcl_ctx *ctx = nullptr;
    pcl_server_cfg cfg{};
    std::vector<ServerClass> cls;
    char *arena_mem = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    std::mutex mu;
};

namespace {

// request pipelines (kExact: the exact window scan of 512^2 px cosine pairs)
constexpr int kEdge = 0, kFft = 1, kTc = 2, kExact = 3;

// workspace of a cosine request: the band join's, then (same stream, after
// it) the tensor-core engine's grouping buffers in the same bytes
size_t request_ws(const pcl::Geo &g, int engine, uint32_t nq, uint32_t n_lib, uint64_t cap) {
    if (engine == kEdge) return 0;
    const size_t cj = pcl::cross_join_workspace(g, nq, n_lib);
    if (engine == kFft || engine == kExact) return cj;
    const size_t tc = pcl::tc_workspace(cap);
    return cj > tc ? cj : tc;
}

// device bytes of one request of nq clips and R rectangles with candidate capacity cap
size_t footprint(const pcl::Geo &g, uint32_t nq, uint64_t R, uint64_t cap, int engine, uint32_t n_lib) {
    size_t b = 0;
    b += align256(4ull * (nq + 1));                 // rect_off
    b += align256(16ull * (R ? R : 1));             // rects
    b += align256(8ull * nq * g.N * g.nw);          // bits
    b += align256(4ull * nq);                       // pop
    b += align256(4ull * nq * g.N);                 // prof
    b += align256(4ull * nq * g.nb * g.nb);         // blk
    b += align256(32ull * nq);                      // esig
    b += align256(512ull * nq);                     // occ
    b += align256(2ull * (R ? R : 1));              // rorder
    b += engine == kFft ? align256(8ull * nq * g.L * g.Ls) : 0;  // spec (FFT engine only)
    b += align256(nq);                              // spec_state
    b += align256(8ull * cap) * 2;                  // cand, pass
    b += align256(40ull * cap);                     // records
    b += align256(64);                              // counts
    b += align256(request_ws(g, engine, nq, n_lib, cap));     // band join / tensor-core workspace (cosine only)
    return b;
}

void carve(Slot &s, const pcl::Geo &g, char *base, uint32_t nq, uint64_t R, uint64_t cap, int engine,
           uint32_t n_lib) {
    char *p = base;
    auto take = [&](size_t n) {
        char *r = p;
        p += align256(n);
        return r;
    };
    s.q.n_clips = nq;
    s.q.rect_off = reinterpret_cast<uint32_t *>(take(4ull * (nq + 1)));
    s.q.rects = reinterpret_cast<int32_t *>(take(16ull * (R ? R : 1)));
    s.q.bits = reinterpret_cast<uint64_t *>(take(8ull * nq * g.N * g.nw));
    s.q.pop = reinterpret_cast<uint32_t *>(take(4ull * nq));
    s.q.prof = reinterpret_cast<uint16_t *>(take(4ull * nq * g.N));
    s.q.blk = reinterpret_cast<uint16_t *>(take(4ull * nq * g.nb * g.nb));
    s.q.esig = reinterpret_cast<int32_t *>(take(32ull * nq));
    s.q.occ = reinterpret_cast<uint64_t *>(take(512ull * nq));
    s.q.rorder = reinterpret_cast<uint16_t *>(take(2ull * (R ? R : 1)));
    s.q.spec = engine == kFft ? take(8ull * nq * g.L * g.Ls) : nullptr;
    s.q.spec_state = reinterpret_cast<uint8_t *>(take(nq));
    s.cand = reinterpret_cast<pcl_pair *>(take(8ull * cap));
    s.pass = reinterpret_cast<pcl_pair *>(take(8ull * cap));
    s.rec = reinterpret_cast<pcl_record *>(take(40ull * cap));
    s.counts = reinterpret_cast<unsigned long long *>(take(64));
    s.ws_bytes = request_ws(g, engine, nq, n_lib, cap);
    s.ws = s.ws_bytes ? take(s.ws_bytes) : nullptr;
}

pcl_status fail(pcl_ctx *ctx, pcl_status s, const std::string &m) {
    if (ctx) ctx->err = m;
    return s;
}

}  // namespace

extern "C" {

pcl_status pcl_server_create_classes(pcl_ctx *ctx, const pcl_params *params, const pcl_clipset *libraries,
                                     uint32_t n_classes, const pcl_server_cfg *cfg, pcl_server **out) {
    if (!ctx || !out) return PCL_ERR_INVALID;
    *out = nullptr;
    ctx->err.clear();
    if (!params || !libraries || n_classes == 0 || n_classes > 16)
        return fail(ctx, PCL_ERR_INVALID, "pcl_server_create: 1 to 16 size classes");
    if (!cfg || cfg->max_inflight == 0 || cfg->max_inflight > 64 || cfg->max_query_clips == 0 ||
        cfg->cand_per_query == 0)
        return fail(ctx, PCL_ERR_INVALID, "pcl_server_create: invalid configuration");
    const bool edge = cfg->mode == PCL_MODE_EDGE;
    if (cfg->mode != 0 && cfg->mode != PCL_MODE_COSINE && !edge)
        return fail(ctx, PCL_ERR_INVALID, "pcl_server_create: mode must be PCL_MODE_COSINE or PCL_MODE_EDGE");
    std::vector<ServerClass> classes(n_classes);
    for (uint32_t c = 0; c < n_classes; ++c) {
        const pcl_params *P = params + c;
        const pcl_clipset *library = libraries + c;
        const std::string who = "pcl_server_create (class " + std::to_string(c) + "): ";
        if (pcl_params_validate(P) != PCL_OK) return fail(ctx, PCL_ERR_INVALID, who + "invalid parameters");
        const pcl::Geo g = pcl::make_geo(*P);
        const bool tc = P->cos_engine == PCL_ENGINE_TC_DIRECT || P->cos_engine == PCL_ENGINE_TC_DIRECT_FP8 ||
                        P->cos_engine == PCL_ENGINE_TC_DIRECT_BF16;
        int engine = kEdge;
        if (edge) {
            if (!library->rect_off || !library->rects || !library->bits || !library->esig || !library->occ ||
                !library->rorder)
                return fail(ctx, PCL_ERR_INVALID, who + "edge library needs rectangles and edge signatures");
        } else {
            if (!library->pop || !library->blk || !library->prof || !library->bits)
                return fail(ctx, PCL_ERR_INVALID, who + "library needs rasters and signatures");
            if (g.S > g.N / 16)
                return fail(ctx, PCL_ERR_UNSUPPORTED, who + "cosine serving covers S <= N/16");
            if (g.N == 512 || (P->cos_engine == PCL_ENGINE_EXACT_SCAN && g.N >= 128)) {
                // 512^2 px, or the exact-scan engine: the bound-pruned exact
                // window scan (no spectra, no tensor-core geometry)
                if (P->shift_rule != PCL_SHIFT_EXACT_ARGMAX)
                    return fail(ctx, PCL_ERR_UNSUPPORTED, who + "the exact window scan takes the exact argmax rule");
                engine = kExact;
            } else if (tc) {
                if (!pcl::tc_supported(g) || P->shift_rule != PCL_SHIFT_EXACT_ARGMAX)
                    return fail(ctx, PCL_ERR_UNSUPPORTED,
                                who + "tensor-core engine covers N = 64, 128, 256 with S <= N/16, exact argmax");
                engine = kTc;
            } else {
                if (P->cos_engine != PCL_ENGINE_FFT_PCM)
                    return fail(ctx, PCL_ERR_UNSUPPORTED,
                                who + "cosine serving takes the FFT, tensor-core or exact-scan engine (the "
                                      "exact scan from 128^2 px)");
                if (!library->spec || !library->spec_state)
                    return fail(ctx, PCL_ERR_INVALID, who + "FFT engine needs the library's spectra");
                engine = kFft;
            }
        }
        classes[c].P = *P;
        classes[c].g = g;
        classes[c].lib = *library;
        classes[c].engine = engine;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail(ctx, PCL_ERR_CUDA, "cudaSetDevice");
    pcl_server *s = new (std::nothrow) pcl_server;
    if (!s) return PCL_ERR_OOM;
    s->ctx = ctx;
    s->cfg = *cfg;
    s->cls = classes;
    auto cleanup = [&](pcl_status st, const std::string &m) {
        pcl_server_destroy(s);
        return fail(ctx, st, m);
    };
    if (cudaMalloc(&s->arena_mem, cfg->mem_budget ? cfg->mem_budget : 1)) {
        cudaGetLastError();
        return cleanup(PCL_ERR_OOM, "pcl_server_create: device allocation failed");
    }
    s->arena.init(s->arena_mem, cfg->mem_budget);
    // resident libraries (cosine): each class's area order, and with the FFT
    // engine the spectra of every clip, once
    for (auto &k : s->cls) {
        if (edge) continue;
        const uint32_t V = (uint32_t)k.g.N * k.g.N + 2;
        const uint32_t nl = k.lib.n_clips;
        if (cudaMalloc(&k.lib_cum, 4ull * V) || cudaMalloc(&k.lib_fill, 4ull * V) ||
            cudaMalloc(&k.lib_order, 4ull * (nl ? nl : 1)) || cudaMalloc(&k.lib_spop, 4ull * (nl ? nl : 1))) {
            cudaGetLastError();
            return cleanup(PCL_ERR_OOM, "pcl_server_create: device allocation failed");
        }
        if (k.engine == kFft) e = pcl::launch_spectra(k.P, k.lib, nullptr, 0, false, 0);
        if (e == cudaSuccess)
            e = pcl::launch_area_sort(k.lib.pop, nl, V, k.lib_cum, k.lib_fill, k.lib_order, k.lib_spop,
                                      ctx->num_sms, 0);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cleanup(PCL_ERR_CUDA, std::string("library preparation: ") + cudaGetErrorString(e));
    s->slots.resize(cfg->max_inflight);
    const uint32_t pass_copy = cfg->pass_copy ? cfg->pass_copy : 1;
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) ||
            cudaMallocHost(&sl.h_off, 4ull * (cfg->max_query_clips + 1)) ||
            cudaMallocHost(&sl.h_rects, 16ull * (cfg->max_query_rects ? cfg->max_query_rects : 1)) ||
            cudaMallocHost(&sl.h_pass, 8ull * pass_copy) || cudaMallocHost(&sl.h_rec, 40ull * pass_copy) ||
            cudaMallocHost(&sl.h_counts, 64)) {
            cudaGetLastError();
            return cleanup(PCL_ERR_OOM, "pcl_server_create: stream / pinned allocation failed");
        }
    }
    *out = s;
    return PCL_OK;
}

pcl_status pcl_server_create(pcl_ctx *ctx, const pcl_params *P, const pcl_clipset *library,
                             const pcl_server_cfg *cfg, pcl_server **out) {
    return pcl_server_create_classes(ctx, P, library, 1, cfg, out);
}

pcl_status pcl_server_submit_class(pcl_server *s, uint32_t cls, const uint32_t *h_rect_off, const int32_t *h_rects,
                                   uint32_t n_clips, uint64_t request_id) {
    if (!s) return PCL_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    pcl_ctx *ctx = s->ctx;
    ctx->err.clear();
    if (cls >= s->cls.size()) return fail(ctx, PCL_ERR_INVALID, "pcl_server_submit: no such size class");
    ServerClass &k = s->cls[cls];
    if (n_clips == 0 || n_clips > s->cfg.max_query_clips || !h_rect_off)
        return fail(ctx, PCL_ERR_INVALID, "pcl_server_submit: clip count out of range");
    const uint64_t R = h_rect_off[n_clips] - h_rect_off[0];
    if (h_rect_off[n_clips] < h_rect_off[0] || R > s->cfg.max_query_rects || (R && !h_rects))
        return fail(ctx, PCL_ERR_INVALID, "pcl_server_submit: rectangle count out of range");
    Slot *sl = nullptr;
    for (auto &x : s->slots)
        if (!x.busy) {
            sl = &x;
            break;
        }
    if (!sl) return fail(ctx, PCL_ERR_BUSY, "pcl_server_submit: no free slot");
    const uint64_t cap = (uint64_t)s->cfg.cand_per_query * n_clips + 64;
    const size_t bytes = footprint(k.g, n_clips, R, cap, k.engine, k.lib.n_clips);
    size_t off = 0;
    if (!s->arena.alloc(bytes, &off)) return fail(ctx, PCL_ERR_BUSY, "pcl_server_submit: memory budget full");
    cudaError_t e = cudaSetDevice(ctx->device);
    sl->busy = true;
    sl->done = false;
    sl->id = request_id;
    sl->cls = cls;
    sl->off = off;
    sl->bytes = bytes;
    sl->nq = n_clips;
    sl->cap = cap;
    sl->overflow.clear();
    sl->rec_overflow.clear();
    sl->t_done = 0;
    sl->t_submit = now_ns();
    carve(*sl, k.g, s->arena.base + off, n_clips, R, cap, k.engine, k.lib.n_clips);
    std::memcpy(sl->h_off, h_rect_off, 4ull * (n_clips + 1));
    const uint32_t base = h_rect_off[0];
    if (R) std::memcpy(sl->h_rects, h_rects + 4ull * base, 16ull * R);
    cudaStream_t st = sl->st;
    // rect offsets of the request relative to its own rectangle array
    if (base)
        for (uint32_t i = 0; i <= n_clips; ++i) sl->h_off[i] -= base;
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)sl->q.rect_off, sl->h_off, 4ull * (n_clips + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && R)
        e = cudaMemcpyAsync((void *)sl->q.rects, sl->h_rects, 16ull * R, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl->counts, 0, 64, st);
    if (e == cudaSuccess) e = pcl::launch_raster(k.P, sl->q, st);
    if (k.engine == kEdge) {
        // every (query, library) pair through the edge gates (the tiled screen
        // of the self-join, rows = queries, columns = library clips), then
        // the Min-Max record of each survivor, one pair per warp
        if (e == cudaSuccess)
            e = pcl::launch_edge_screen_cross(k.P, sl->q, k.lib, sl->cand, cap, sl->counts + 0, nullptr, st,
                                              nullptr, 0, ctx->num_sms);
        if (e == cudaSuccess)
            e = pcl::launch_edge_match(k.P, sl->q, k.lib, sl->cand, cap, sl->counts + 0, sl->rec, ctx->num_sms, st);
    } else {
        if (e == cudaSuccess)
            e = pcl::launch_cross_join(k.P, sl->q, k.lib, k.lib_order, k.lib_spop, k.lib_cum, sl->ws, sl->ws_bytes,
                                       sl->cand, cap, sl->counts + 0, nullptr, ctx->num_sms, st);
        if (k.engine == kTc) {
            // candidates grouped by query clip through the direct correlation;
            // a bounded wait that runs out sets the request's own error word
            if (e == cudaSuccess)
                e = pcl::launch_tc(k.P, sl->q, k.lib, sl->cand, cap, sl->counts + 0, sl->rec, sl->ws, sl->ws_bytes,
                                   ctx->num_sms, reinterpret_cast<int *>(sl->counts + 2), ctx->wait_ns, st);
        } else if (k.engine == kExact) {
            if (e == cudaSuccess)
                e = pcl::launch_exact_pairs(k.P, sl->q, k.lib, sl->cand, cap, sl->counts + 0, sl->rec, ctx->num_sms,
                                            ctx->d_stats, st);
        } else {
            if (e == cudaSuccess) e = pcl::launch_mark(sl->cand, cap, sl->counts + 0, sl->q, k.lib, st);
            if (e == cudaSuccess) e = pcl::launch_spectra(k.P, sl->q, nullptr, 0, true, st);
            if (e == cudaSuccess)
                e = pcl::launch_pair_fft(k.P, sl->q, k.lib, sl->cand, cap, sl->counts + 0, sl->rec, ctx->num_sms,
                                         st);
        }
    }
    if (e == cudaSuccess) e = pcl::launch_compact(sl->rec, cap, sl->counts + 0, sl->pass, cap, sl->counts + 1, st);
    const uint32_t pass_copy = s->cfg.pass_copy ? s->cfg.pass_copy : 1;
    const uint64_t first = pass_copy < cap ? pass_copy : cap;
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl->h_counts, sl->counts, 24, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl->h_pass, sl->pass, 8ull * first, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl->h_rec, sl->rec, 40ull * first, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, stamp_done, sl);
    if (e == cudaSuccess) e = cudaEventRecord(sl->ev, st);
    if (e != cudaSuccess) {
        // the slot keeps its memory until its stream is idle
        cudaStreamSynchronize(st);
        s->arena.release(sl->off, sl->bytes);
        sl->busy = false;
        return fail(ctx, PCL_ERR_CUDA, std::string("pcl_server_submit: ") + cudaGetErrorString(e));
    }
    return PCL_OK;
}

pcl_status pcl_server_submit(pcl_server *s, const uint32_t *h_rect_off, const int32_t *h_rects, uint32_t n_clips,
                             uint64_t request_id) {
    return pcl_server_submit_class(s, 0, h_rect_off, h_rects, n_clips, request_id);
}

pcl_status pcl_server_poll(pcl_server *s, pcl_completion *out, uint32_t cap, uint32_t *n_out) {
    if (!s || !n_out || (cap && !out)) return PCL_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    *n_out = 0;
    cudaSetDevice(s->ctx->device);
    const uint32_t pass_copy = s->cfg.pass_copy ? s->cfg.pass_copy : 1;
    for (auto &sl : s->slots) {
        if (!sl.busy || sl.done || *n_out >= cap) continue;
        const cudaError_t q = cudaEventQuery(sl.ev);
        if (q == cudaErrorNotReady) continue;
        pcl_completion &c = sl.comp;
        c = pcl_completion{};
        c.request_id = sl.id;
        c.size_class = sl.cls;
        c.n_queries = sl.nq;
        c.t_submit_ns = sl.t_submit;
        c.t_done_ns = sl.t_done;
        if (q != cudaSuccess) {
            c.status = PCL_ERR_CUDA;
        } else {
            c.n_candidates = sl.h_counts[0];
            const uint64_t np = sl.h_counts[1];
            c.status = sl.h_counts[2] ? PCL_ERR_TIMEOUT : (c.n_candidates > sl.cap) ? PCL_ERR_BUSY : PCL_OK;
            const uint64_t got = np < sl.cap ? np : sl.cap;
            c.n_pass = got;
            if (got <= pass_copy) {
                c.pass = sl.h_pass;
            } else {
                sl.overflow.resize(got);
                cudaMemcpy(sl.overflow.data(), sl.pass, 8ull * got, cudaMemcpyDeviceToHost);
                c.pass = sl.overflow.data();
            }
            // one record per candidate (those within the capacity)
            const uint64_t nr = c.n_candidates < sl.cap ? c.n_candidates : sl.cap;
            c.n_records = nr;
            if (nr <= pass_copy) {
                c.records = sl.h_rec;
            } else {
                sl.rec_overflow.resize(nr);
                cudaMemcpy(sl.rec_overflow.data(), sl.rec, 40ull * nr, cudaMemcpyDeviceToHost);
                c.records = sl.rec_overflow.data();
            }
        }
        sl.done = true;
        out[(*n_out)++] = c;
    }
    return PCL_OK;
}

pcl_status pcl_server_release(pcl_server *s, uint64_t request_id) {
    if (!s) return PCL_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto &sl : s->slots) {
        if (sl.busy && sl.done && sl.id == request_id) {
            s->arena.release(sl.off, sl.bytes);
            sl.busy = false;
            sl.done = false;
            return PCL_OK;
        }
    }
    return fail(s->ctx, PCL_ERR_INVALID, "pcl_server_release: no completed request with that id");
}

pcl_status pcl_server_stats(pcl_server *s, uint32_t *inflight, uint64_t *free_bytes) {
    if (!s) return PCL_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    uint32_t k = 0;
    for (auto &sl : s->slots) k += sl.busy ? 1u : 0u;
    uint64_t f = 0;
    for (auto &kv : s->arena.free_) f += kv.second;
    if (inflight) *inflight = k;
    if (free_bytes) *free_bytes = f;
    return PCL_OK;
}

void pcl_server_destroy(pcl_server *s) {
    if (!s) return;
    cudaSetDevice(s->ctx->device);
    for (auto &sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.h_off) cudaFreeHost(sl.h_off);
        if (sl.h_rects) cudaFreeHost(sl.h_rects);
        if (sl.h_pass) cudaFreeHost(sl.h_pass);
        if (sl.h_rec) cudaFreeHost(sl.h_rec);
        if (sl.h_counts) cudaFreeHost(sl.h_counts);
    }
    for (auto &k : s->cls) {
        cudaFree(k.lib_cum);
        cudaFree(k.lib_fill);
        cudaFree(k.lib_order);
        cudaFree(k.lib_spop);
    }
    cudaFree(s->arena_mem);
    delete s;
}

}  // extern "C"

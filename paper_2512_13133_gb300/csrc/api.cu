// C ABI of the pcl library: context, parameter checks, clip-set sizes and the
// entry points of include/pcl.h.  Kernels live in raster.cu, gates.cu,
// edge.cu and fft.cu; the host set cover and loop in host_scp.cpp.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "common.cuh"

namespace pcl {
cudaError_t launch_raster(const pcl_params &, const pcl_clipset &, cudaStream_t);
size_t band_join_workspace(const Geo &, uint32_t, bool);
cudaError_t launch_band_join(const pcl_params &, const pcl_clipset &, void *, size_t, pcl_pair *, uint64_t,
                             unsigned long long *, unsigned long long *, int, cudaStream_t, uint32_t, uint32_t);
size_t edge_checks_workspace(uint64_t);
cudaError_t launch_edge_screen(const pcl_params &, const pcl_clipset &, pcl_pair *, uint64_t,
                               unsigned long long *, unsigned long long *, cudaStream_t, uint32_t, uint32_t, void *,
                               size_t, int);
cudaError_t launch_edge_screen_cross(const pcl_params &, const pcl_clipset &, const pcl_clipset &, pcl_pair *,
                                     uint64_t, unsigned long long *, unsigned long long *, cudaStream_t, void *,
                                     size_t, int);
cudaError_t launch_area_sort(const uint32_t *, uint32_t, uint32_t, uint32_t *, uint32_t *, uint32_t *, uint32_t *,
                             int, cudaStream_t);
size_t cross_join_workspace(const Geo &, uint32_t, uint32_t);
cudaError_t launch_cross_join(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const uint32_t *,
                              const uint32_t *, const uint32_t *, void *, size_t, pcl_pair *, uint64_t,
                              unsigned long long *, unsigned long long *, int, cudaStream_t);
cudaError_t launch_edge_match(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const pcl_pair *, uint64_t,
                              const unsigned long long *, pcl_record *, int, cudaStream_t);
cudaError_t launch_spectra(const pcl_params &, const pcl_clipset &, const uint32_t *, uint32_t, bool,
                           cudaStream_t);
cudaError_t launch_mark(const pcl_pair *, uint64_t, const unsigned long long *, pcl_clipset &, pcl_clipset &,
                        cudaStream_t);
cudaError_t launch_pair_fft(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const pcl_pair *,
                            uint64_t, const unsigned long long *, pcl_record *, int, cudaStream_t);
cudaError_t launch_compact(const pcl_record *, uint64_t, const unsigned long long *, pcl_pair *, uint64_t,
                           unsigned long long *, cudaStream_t);
bool tc_supported(const Geo &);
cudaError_t launch_exact_pairs(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const pcl_pair *,
                               uint64_t, const unsigned long long *, pcl_record *, int, unsigned long long *,
                               cudaStream_t);
size_t tc_workspace(uint64_t);
cudaError_t launch_tc(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const pcl_pair *, uint64_t,
                      const unsigned long long *, pcl_record *, void *, size_t, int, int *, unsigned long long,
                      cudaStream_t);
cudaError_t launch_xysep(const pcl_params &, const pcl_clipset &, const pcl_clipset &, const pcl_pair *, uint64_t,
                         const unsigned long long *, pcl_record *, int, cudaStream_t);
cudaError_t launch_mixed(const pcl_params *, const pcl_clipset *, uint32_t, const pcl_work *, uint64_t, uint64_t,
                         pcl_record *, unsigned long long *, uint32_t, uint32_t, uint32_t, int, cudaStream_t);
}  // namespace pcl

#include "ctx.h"

using namespace pcl;

namespace {

pcl_status fail(pcl_ctx *ctx, pcl_status s, const char *fmt, const char *a = "", long long b = 0) {
    if (ctx) {
        char buf[512];
        snprintf(buf, sizeof buf, fmt, a, b);
        ctx->err = buf;
    }
    return s;
}

pcl_status cuda_fail(pcl_ctx *ctx, cudaError_t e, const char *where) {
    if (ctx) ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
    return PCL_ERR_CUDA;
}

pcl_status enter(pcl_ctx *ctx) {
    if (!ctx) return PCL_ERR_INVALID;
    ctx->err.clear();
    const cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return PCL_OK;
}

pcl_status ensure_ws(pcl_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return PCL_OK;
    if (ctx->ws) {
        cudaFree(ctx->ws);  // synchronises the device: no kernel still uses it
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    const size_t want = bytes + bytes / 4 + 4096;
    const cudaError_t e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return fail(ctx, PCL_ERR_OOM, "workspace allocation of %s%lld bytes failed", "", (long long)want);
    }
    ctx->ws_bytes = want;
    return PCL_OK;
}

bool pow2_raster(int N) { return N == 64 || N == 128 || N == 256 || N == 512; }

pcl_status check_clipset(pcl_ctx *ctx, const pcl_clipset *cs, bool need_edge_or_raster) {
    if (!cs) return fail(ctx, PCL_ERR_INVALID, "clip set is NULL%s%lld");
    if (cs->n_clips && (!cs->rect_off || !cs->rects || !cs->bits || !cs->pop || !cs->prof || !cs->blk ||
                        (need_edge_or_raster && (!cs->esig || !cs->occ || !cs->rorder))))
        return fail(ctx, PCL_ERR_INVALID, "clip set has a NULL buffer%s%lld");
    // kernels read rects and esig (and the 8-byte arrays) with 16-byte vector loads
    const uintptr_t mis = (uintptr_t)cs->rects | (uintptr_t)cs->bits | (uintptr_t)cs->esig | (uintptr_t)cs->occ;
    if (cs->n_clips && (mis & 15u))
        return fail(ctx, PCL_ERR_INVALID, "clip set buffer not 16-byte aligned%s%lld");
    return PCL_OK;
}

}  // namespace

extern "C" {

const char *pcl_status_string(pcl_status s) {
    switch (s) {
        case PCL_OK: return "ok";
        case PCL_ERR_INVALID: return "invalid argument";
        case PCL_ERR_OOM: return "out of device memory";
        case PCL_ERR_CUDA: return "CUDA error";
        case PCL_ERR_TIMEOUT: return "device wait timed out";
        case PCL_ERR_BUSY: return "busy / capacity too small";
        case PCL_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

pcl_status pcl_create(pcl_ctx **out, int device) {
    if (!out) return PCL_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return PCL_ERR_INVALID;
    }
    pcl_ctx *c = new (std::nothrow) pcl_ctx;
    if (!c) return PCL_ERR_OOM;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&c->d_err, 256) != cudaSuccess || cudaMemset(c->d_err, 0, 256) != cudaSuccess ||
        cudaMalloc(&c->d_stats, 64) != cudaSuccess || cudaMemset(c->d_stats, 0, 64) != cudaSuccess) {
        cudaGetLastError();
        if (c->d_err) cudaFree(c->d_err);
        if (c->d_stats) cudaFree(c->d_stats);
        delete c;
        return PCL_ERR_CUDA;
    }
    *out = c;
    return PCL_OK;
}

void pcl_destroy(pcl_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_stats) cudaFree(ctx->d_stats);
    delete ctx;
}

const char *pcl_last_error(const pcl_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

pcl_status pcl_stats_get(pcl_ctx *ctx, uint64_t *out, int reset) {
    if (!ctx || !out) return PCL_ERR_INVALID;
    cudaSetDevice(ctx->device);
    unsigned long long h[4] = {0ull, 0ull, 0ull, 0ull};
    cudaError_t e = cudaMemcpy(h, ctx->d_stats, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset) e = cudaMemset(ctx->d_stats, 0, sizeof(h));
    if (e != cudaSuccess) {
        ctx->err = std::string("pcl_stats_get: ") + cudaGetErrorString(e);
        return PCL_ERR_CUDA;
    }
    for (int k = 0; k < 4; ++k) out[k] = h[k];
    return PCL_OK;
}

pcl_status pcl_set_wait_limit(pcl_ctx *ctx, uint64_t ns) {
    if (!ctx) return PCL_ERR_INVALID;
    ctx->wait_ns = ns;
    return PCL_OK;
}

pcl_status pcl_params_validate(const pcl_params *P) {
    if (!P) return PCL_ERR_INVALID;
    if (P->pitch_dbu <= 0 || P->window_dbu <= 0 || P->window_dbu % P->pitch_dbu) return PCL_ERR_INVALID;
    if (!pow2_raster(P->window_dbu / P->pitch_dbu)) return PCL_ERR_INVALID;
    if (P->marker_dbu < 0 || P->marker_dbu % P->pitch_dbu) return PCL_ERR_INVALID;
    if (P->marker_dbu / P->pitch_dbu > 64) return PCL_ERR_INVALID;
    if (P->cos_den == 0 || P->cos_den > 65535 || P->cos_num == 0 || P->cos_num >= P->cos_den)
        return PCL_ERR_INVALID;
    if (P->edge_tol_dbu < 0) return PCL_ERR_INVALID;
    if (P->cos_engine > PCL_ENGINE_EXACT_SCAN || P->shift_rule > PCL_SHIFT_PCM_PEAK) return PCL_ERR_INVALID;
    if (!(P->near_band >= 0.0f)) return PCL_ERR_INVALID;
    return PCL_OK;
}

pcl_status pcl_clipset_sizes_get(const pcl_params *P, uint32_t n, uint64_t n_rects, pcl_clipset_sizes *o) {
    if (!o || pcl_params_validate(P) != PCL_OK) return PCL_ERR_INVALID;
    const Geo g = make_geo(*P);
    o->bits = 8ull * n * g.N * g.nw;
    o->pop = 4ull * n;
    o->prof = 2ull * n * 2 * g.N;
    o->blk = 2ull * n * 2 * g.nb * g.nb;
    o->esig = 32ull * n;
    o->occ = 8ull * 64 * n;
    o->rorder = 2ull * n_rects;
    o->spec = 8ull * n * g.L * g.Ls;
    o->spec_state = n;
    o->N = g.N;
    o->S = g.S;
    o->L = g.L;
    o->Ls = g.Ls;
    return PCL_OK;
}

pcl_status pcl_rasterize(pcl_ctx *ctx, const pcl_params *P, pcl_clipset *cs, pcl_stream stream) {
    pcl_status s = enter(ctx);
    if (s) return s;
    if (pcl_params_validate(P)) return fail(ctx, PCL_ERR_INVALID, "invalid parameters%s%lld");
    if ((s = check_clipset(ctx, cs, true))) return s;
    const cudaError_t e = launch_raster(*P, *cs, (cudaStream_t)stream);
    return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "raster kernel");
}

pcl_status pcl_spectra(pcl_ctx *ctx, const pcl_params *P, pcl_clipset *cs, const uint32_t *d_list,
                       uint32_t n_list, pcl_stream stream) {
    pcl_status s = enter(ctx);
    if (s) return s;
    if (pcl_params_validate(P)) return fail(ctx, PCL_ERR_INVALID, "invalid parameters%s%lld");
    if ((s = check_clipset(ctx, cs, false))) return s;
    if (!cs->spec || !cs->spec_state) return fail(ctx, PCL_ERR_INVALID, "spec / spec_state buffers missing%s%lld");
    const Geo g = make_geo(*P);
    if (g.N > 256) return fail(ctx, PCL_ERR_UNSUPPORTED, "FFT engine covers N <= 256 (got N = %s%lld)", "", g.N);
    const cudaError_t e = launch_spectra(*P, *cs, d_list, n_list, false, (cudaStream_t)stream);
    return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "spectra kernel");
}

pcl_status pcl_candidates(pcl_ctx *ctx, const pcl_params *P, uint32_t mode, const pcl_clipset *a,
                          const pcl_clipset *b, pcl_pair *d_out, uint64_t cap, uint64_t *d_count,
                          uint64_t *d_gate_counts, pcl_stream stream) {
    if (!b) return pcl_candidates_shard(ctx, P, mode, a, 0, 1, d_out, cap, d_count, d_gate_counts, stream);
    pcl_status s = enter(ctx);
    if (s) return s;
    if (pcl_params_validate(P)) return fail(ctx, PCL_ERR_INVALID, "invalid parameters%s%lld");
    const bool edge = mode == PCL_MODE_EDGE;
    if (!edge && mode != PCL_MODE_COSINE) return fail(ctx, PCL_ERR_INVALID, "unknown mode%s %lld", "", mode);
    if (P->flags & PCL_P_TOPO_HASH)
        return fail(ctx, PCL_ERR_UNSUPPORTED, "the topological pre-screen is a self-join screen%s%lld");
    if ((s = check_clipset(ctx, a, edge)) || (s = check_clipset(ctx, b, edge))) return s;
    if (!d_count || (cap && !d_out)) return fail(ctx, PCL_ERR_INVALID, "NULL output%s%lld");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
    auto *cnt = reinterpret_cast<unsigned long long *>(d_count);
    auto *gates = reinterpret_cast<unsigned long long *>(d_gate_counts);
    if (edge) {
        // the workspace holds the list of pairs for the correspondence check
        if ((s = ensure_ws(ctx, edge_checks_workspace((uint64_t)a->n_clips * b->n_clips)))) return s;
        e = launch_edge_screen_cross(*P, *a, *b, d_out, cap, cnt, gates, st, ctx->ws, ctx->ws_bytes, ctx->num_sms);
        return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "edge screen (two sets)");
    }
    const Geo g = make_geo(*P);
    if (g.S > g.N / 16) return fail(ctx, PCL_ERR_UNSUPPORTED, "cosine gates need S <= N/16%s%lld");
    // workspace: B's area histogram, fill counters, area order and sorted
    // areas, then the cross join's own part (16-byte aligned)
    const uint32_t V = (uint32_t)g.N * g.N + 2, nb = b->n_clips;
    const size_t sort_bytes = ((4 * (2 * (size_t)V + 2 * (size_t)nb)) + 15) & ~(size_t)15;
    const size_t join_bytes = cross_join_workspace(g, a->n_clips, nb);
    if ((s = ensure_ws(ctx, sort_bytes + join_bytes))) return s;
    uint32_t *cum = static_cast<uint32_t *>(ctx->ws), *fill = cum + V, *order = fill + V, *spop = order + nb;
    e = launch_area_sort(b->pop, nb, V, cum, fill, order, spop, ctx->num_sms, st);
    if (e == cudaSuccess)
        e = launch_cross_join(*P, *a, *b, order, spop, cum, static_cast<char *>(ctx->ws) + sort_bytes,
                              ctx->ws_bytes - sort_bytes, d_out, cap, cnt, gates, ctx->num_sms, st);
    return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "band join (two sets)");
}

pcl_status pcl_candidates_shard(pcl_ctx *ctx, const pcl_params *P, uint32_t mode, const pcl_clipset *cs,
                                uint32_t shard, uint32_t n_shards, pcl_pair *d_out, uint64_t cap, uint64_t *d_count,
                                uint64_t *d_gate_counts, pcl_stream stream) {
    pcl_status s = enter(ctx);
    if (s) return s;
    if (pcl_params_validate(P)) return fail(ctx, PCL_ERR_INVALID, "invalid parameters%s%lld");
    if (n_shards == 0 || shard >= n_shards) return fail(ctx, PCL_ERR_INVALID, "shard out of range%s%lld");
    const bool topo = (P->flags & PCL_P_TOPO_HASH) != 0;
    if ((s = check_clipset(ctx, cs, mode == PCL_MODE_EDGE || topo))) return s;
    if (topo && n_shards != 1)
        return fail(ctx, PCL_ERR_UNSUPPORTED, "the topological pre-screen takes the whole self-join%s%lld");
    if (!d_count || (cap && !d_out)) return fail(ctx, PCL_ERR_INVALID, "NULL output%s%lld");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
    auto *cnt = reinterpret_cast<unsigned long long *>(d_count);
    auto *gates = reinterpret_cast<unsigned long long *>(d_gate_counts);
    if (mode == PCL_MODE_COSINE) {
        const Geo g = make_geo(*P);
        if (g.S > g.N / 16) return fail(ctx, PCL_ERR_UNSUPPORTED, "cosine gates need S <= N/16%s%lld");
        const size_t need = band_join_workspace(g, cs->n_clips, topo);
        if ((s = ensure_ws(ctx, need))) return s;
        e = launch_band_join(*P, *cs, ctx->ws, ctx->ws_bytes, d_out, cap, cnt, gates, ctx->num_sms, st, shard,
                             n_shards);
        return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "band join");
    }
    if (mode == PCL_MODE_EDGE) {
        const uint64_t n = cs->n_clips;
        if ((s = ensure_ws(ctx, edge_checks_workspace(n * (n - (n > 0)) / 2 / n_shards)))) return s;
        e = launch_edge_screen(*P, *cs, d_out, cap, cnt, gates, st, shard, n_shards, ctx->ws, ctx->ws_bytes,
                               ctx->num_sms);
        return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "edge screen");
    }
    return fail(ctx, PCL_ERR_INVALID, "unknown mode%s %lld", "", mode);
}

pcl_status pcl_match_pairs(pcl_ctx *ctx, const pcl_params *P, uint32_t mode, pcl_clipset *a, pcl_clipset *b,
                           const pcl_pair *d_pairs, uint64_t n, const uint64_t *d_n, pcl_record *d_out,
                           pcl_stream stream) {
    const auto *dn = reinterpret_cast<const unsigned long long *>(d_n);
    pcl_status s = enter(ctx);
    if (s) return s;
    if (pcl_params_validate(P)) return fail(ctx, PCL_ERR_INVALID, "invalid parameters%s%lld");
    const bool geo = mode == PCL_MODE_EDGE || P->cos_engine == PCL_ENGINE_XYSEP;  // needs the polygons
    if ((s = check_clipset(ctx, a, geo)) || (s = check_clipset(ctx, b, geo))) return s;
    if (n && (!d_pairs || !d_out)) return fail(ctx, PCL_ERR_INVALID, "NULL pair list or output%s%lld");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (mode == PCL_MODE_EDGE) {
        e = launch_edge_match(*P, *a, *b, d_pairs, n, dn, d_out, ctx->num_sms, st);
        return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "edge match");
    }
    if (mode != PCL_MODE_COSINE) return fail(ctx, PCL_ERR_INVALID, "unknown mode%s %lld", "", mode);
    const Geo g = make_geo(*P);
    if (P->cos_engine == PCL_ENGINE_TC_DIRECT || P->cos_engine == PCL_ENGINE_TC_DIRECT_FP8 ||
        P->cos_engine == PCL_ENGINE_TC_DIRECT_BF16) {
        if (!tc_supported(g) || P->shift_rule != PCL_SHIFT_EXACT_ARGMAX)
            return fail(ctx, PCL_ERR_UNSUPPORTED,
                        "tensor-core engine covers N = 64, 128, 256 with S <= N/16, exact argmax%s%lld");
        if (n == 0) return PCL_OK;
        if ((s = ensure_ws(ctx, tc_workspace(n)))) return s;
        e = launch_tc(*P, *a, *b, d_pairs, n, dn, d_out, ctx->ws, ctx->ws_bytes, ctx->num_sms, ctx->d_err,
                      ctx->wait_ns, st);
        return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "tensor-core correlation");
    }
    if (P->cos_engine == PCL_ENGINE_XYSEP) {
        e = launch_xysep(*P, *a, *b, d_pairs, n, dn, d_out, ctx->num_sms, st);
        return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "interval-competition shift");
    }
    if (P->cos_engine != PCL_ENGINE_FFT_PCM && P->cos_engine != PCL_ENGINE_EXACT_SCAN)
        return fail(ctx, PCL_ERR_UNSUPPORTED, "cosine engine %s%lld not built", "", P->cos_engine);
    if ((g.N == 512 || (P->cos_engine == PCL_ENGINE_EXACT_SCAN && g.N >= 128)) && g.S <= g.N / 16) {
        // 512² (or the exact-scan engine): gates, then the bound-pruned exact
        // window scan (no phase-correlation surface, no spectra)
        if (P->shift_rule != PCL_SHIFT_EXACT_ARGMAX)
            return fail(ctx, PCL_ERR_UNSUPPORTED, "the exact window scan takes the exact argmax only%s%lld");
        e = launch_exact_pairs(*P, *a, *b, d_pairs, n, dn, d_out, ctx->num_sms, ctx->d_stats, st);
        return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "exact window scan");
    }
    if (P->cos_engine == PCL_ENGINE_EXACT_SCAN)
        return fail(ctx, PCL_ERR_UNSUPPORTED, "exact-scan engine covers N = 128, 256, 512 and S <= N/16%s%lld");
    if (g.N > 256 || g.S > g.N / 16)
        return fail(ctx, PCL_ERR_UNSUPPORTED, "FFT engine covers N <= 256 (512 by exact scan) and S <= N/16%s%lld");
    if (!a->spec || !a->spec_state || !b->spec || !b->spec_state)
        return fail(ctx, PCL_ERR_INVALID, "spec / spec_state buffers missing%s%lld");
    if ((e = launch_mark(d_pairs, n, dn, *a, *b, st)) != cudaSuccess) return cuda_fail(ctx, e, "mark");
    if ((e = launch_spectra(*P, *a, nullptr, 0, true, st)) != cudaSuccess) return cuda_fail(ctx, e, "spectra");
    if (b->spec_state != a->spec_state &&
        (e = launch_spectra(*P, *b, nullptr, 0, true, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "spectra");
    e = launch_pair_fft(*P, *a, *b, d_pairs, n, dn, d_out, ctx->num_sms, st);
    return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "pair fft");
}

pcl_status pcl_match_mixed(pcl_ctx *ctx, const pcl_params *params, pcl_clipset *sets, uint32_t n_classes,
                           const pcl_work *d_work, uint64_t n_cosine, uint64_t n, pcl_record *d_out,
                           const pcl_tuning *tune, pcl_stream stream) {
    pcl_status s = enter(ctx);
    if (s) return s;
    if (!params || !sets || n_classes == 0 || n_classes > 4 || n_cosine > n || (n && (!d_work || !d_out)))
        return fail(ctx, PCL_ERR_INVALID, "pcl_match_mixed: invalid arguments%s%lld");
    for (uint32_t c = 0; c < n_classes; ++c) {
        if (pcl_params_validate(&params[c])) return fail(ctx, PCL_ERR_INVALID, "pcl_match_mixed: class %s%lld params", "", c);
        if ((s = check_clipset(ctx, &sets[c], true))) return s;
        const Geo gc = make_geo(params[c]);
        if (n_cosine && gc.N <= 256 && (!sets[c].spec || !sets[c].spec_state))
            return fail(ctx, PCL_ERR_INVALID, "pcl_match_mixed: class %s%lld lacks spectra buffers", "", c);
    }
    const uint32_t radix = tune && tune->fft_radix == 4 ? 4 : 2;
    const uint32_t ctas = tune ? tune->ctas_per_sm : 0;
    const uint32_t ipw = tune ? tune->items_per_warp : 0;
    if (ipw > 64) return fail(ctx, PCL_ERR_INVALID, "pcl_match_mixed: items_per_warp above 64%s%lld");
    if ((s = ensure_ws(ctx, 256))) return s;
    const cudaError_t e = launch_mixed(params, sets, n_classes, d_work, n_cosine, n, d_out,
                                       static_cast<unsigned long long *>(ctx->ws), radix, ctas, ipw, ctx->num_sms,
                                       (cudaStream_t)stream);
    return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "mixed batch");
}

pcl_status pcl_device_error(pcl_ctx *ctx, int *flag) {
    pcl_status s = enter(ctx);
    if (s) return s;
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pcl_device_error");
    if (flag) *flag = h;
    return h ? fail(ctx, PCL_ERR_TIMEOUT, "a device-side wait ran out%s%lld") : PCL_OK;
}

pcl_status pcl_compact_pass(pcl_ctx *ctx, const pcl_record *d_rec, uint64_t n, const uint64_t *d_n,
                            pcl_pair *d_out, uint64_t cap, uint64_t *d_count, pcl_stream stream) {
    pcl_status s = enter(ctx);
    if (s) return s;
    if (!d_count || (n && !d_rec) || (cap && !d_out)) return fail(ctx, PCL_ERR_INVALID, "NULL argument%s%lld");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st);
    if (e == cudaSuccess)
        e = launch_compact(d_rec, n, reinterpret_cast<const unsigned long long *>(d_n), d_out, cap,
                           reinterpret_cast<unsigned long long *>(d_count), st);
    return e == cudaSuccess ? PCL_OK : cuda_fail(ctx, e, "compact");
}

}  // extern "C"

namespace pcl {
namespace {
__global__ void compact_kernel(const pcl_record *rec, uint64_t n, const unsigned long long *d_n, pcl_pair *out,
                               uint64_t cap, unsigned long long *count) {
    if (d_n && *d_n < n) n = *d_n;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = base + threadIdx.x;
        const bool keep = t < n && rec[t].pass;
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        if (!mask) continue;
        const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
        unsigned long long b0 = 0;
        if (lane == leader) b0 = atomicAdd(count, (unsigned long long)__popc(mask));
        b0 = __shfl_sync(0xffffffffu, b0, leader);
        if (keep) {
            const unsigned long long idx = b0 + __popc(mask & ((1u << lane) - 1u));
            if (idx < cap) out[idx] = pcl_pair{rec[t].a, rec[t].b};
        }
    }
}
}  // namespace

cudaError_t launch_compact(const pcl_record *rec, uint64_t n, const unsigned long long *d_n, pcl_pair *out,
                           uint64_t cap, unsigned long long *count, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    compact_kernel<<<1024, 256, 0, st>>>(rec, n, d_n, out, cap, count);
    return cudaGetLastError();
}
}  // namespace pcl

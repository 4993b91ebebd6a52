// Cosine candidate generation for callers that cannot allocate device memory.
//
// pcl_candidates (mode COSINE) needs scratch memory for the area histogram and
// the area-sorted clip order, which it takes from a workspace the context
// grows with cudaMalloc.  Some callers cannot let a library allocate: their
// device memory is owned by another allocator (a framework's caching
// allocator running with a fixed budget, where a raw cudaMalloc either fails
// or escapes its accounting), or they run a latency-critical service loop in
// which a cudaMalloc/cudaFree pair would synchronise the device in the middle
// of a request.  This entry point serves them: its scratch is a file-scope
// __device__ array of fixed size, so the call allocates nothing.  Inputs and
// outputs still come from the caller.
#include <mutex>

#include "common.cuh"
#include "ctx.h"

namespace pcl {
size_t band_join_workspace(const Geo &, uint32_t, bool);
cudaError_t launch_band_join(const pcl_params &, const pcl_clipset &, void *, size_t, pcl_pair *, uint64_t,
                             unsigned long long *, unsigned long long *, int, cudaStream_t, uint32_t, uint32_t);
}  // namespace pcl

namespace {

// 8 MiB: the histogram of areas (8 (N^2 + 2) bytes) plus 8 bytes per clip,
// e.g. up to ~980,000 clips of 256^2 px or ~780,000 clips of 512^2 px.
constexpr size_t kScratchBytes = size_t(8) << 20;

// Every GPU that loads the library holds this array until the process exits.
// Host code must not pass the symbol itself to a kernel (on the host it names
// a host-side stand-in); its device address is looked up per device below.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// device address of g_scratch on the current device (resolved once per device)
pcl_status scratch_address(pcl_ctx *ctx, void **out) {
    if (ctx->device < 0 || ctx->device >= kMaxDevices) {
        ctx->err = "pcl_candidates_cosine_noalloc: device ordinal out of range";
        return PCL_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[ctx->device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            ctx->err = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
            return PCL_ERR_CUDA;
        }
        g_addr[ctx->device] = p;
    }
    *out = g_addr[ctx->device];
    return PCL_OK;
}

}  // namespace

extern "C" pcl_status pcl_candidates_cosine_noalloc(pcl_ctx *ctx, const pcl_params *P, const pcl_clipset *cs,
                                                    pcl_pair *d_out, uint64_t cap, uint64_t *d_count,
                                                    uint64_t *d_gate_counts, pcl_stream stream) {
    if (!ctx) return PCL_ERR_INVALID;
    ctx->err.clear();
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        ctx->err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return PCL_ERR_CUDA;
    }
    if (pcl_params_validate(P) != PCL_OK) {
        ctx->err = "pcl_candidates_cosine_noalloc: invalid parameters";
        return PCL_ERR_INVALID;
    }
    if (!cs || (cs->n_clips && (!cs->pop || !cs->prof || !cs->blk)) || !d_count || (cap && !d_out)) {
        ctx->err = "pcl_candidates_cosine_noalloc: NULL buffer";
        return PCL_ERR_INVALID;
    }
    const pcl::Geo g = pcl::make_geo(*P);
    if (g.S > g.N / 16) {
        ctx->err = "pcl_candidates_cosine_noalloc: cosine gates need S <= N/16";
        return PCL_ERR_UNSUPPORTED;
    }
    const bool topo = (P->flags & PCL_P_TOPO_HASH) != 0;
    if (topo && cs->n_clips && !cs->esig) {
        ctx->err = "pcl_candidates_cosine_noalloc: the topological pre-screen needs esig";
        return PCL_ERR_INVALID;
    }
    const size_t need = pcl::band_join_workspace(g, cs->n_clips, topo);
    if (need > kScratchBytes) {
        ctx->err = "pcl_candidates_cosine_noalloc: " + std::to_string(cs->n_clips) + " clips of " +
                   std::to_string(g.N) + "^2 px need " + std::to_string(need) +
                   " bytes of scratch, above the fixed 8 MiB; use pcl_candidates";
        return PCL_ERR_INVALID;
    }
    void *ws = nullptr;
    pcl_status s = scratch_address(ctx, &ws);
    if (s != PCL_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st);
    // launch_band_join zeroes the counters, histogram and fill slots it uses
    // before its kernels run; the sorted order is fully rewritten each call
    if (e == cudaSuccess)
        e = pcl::launch_band_join(*P, *cs, ws, kScratchBytes, d_out, cap,
                                  reinterpret_cast<unsigned long long *>(d_count),
                                  reinterpret_cast<unsigned long long *>(d_gate_counts), ctx->num_sms, st, 0, 1);
    if (e != cudaSuccess) {
        ctx->err = std::string("band join: ") + cudaGetErrorString(e);
        return PCL_ERR_CUDA;
    }
    return PCL_OK;
}

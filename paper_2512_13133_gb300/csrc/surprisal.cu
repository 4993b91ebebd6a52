// Degrees, surprisal weights and first-step scores of the pass graph on the
// GPU (Sec. 3.3.1, Eqs. 7-9), the step that feeds the host set cover: the
// graph of passing pairs can hold millions of edges, and its per-node sums
// are a scatter over the edge list.
//
// deg(i)   edges at node i (each listed edge once per endpoint)
// S_i      floor(2^32 / (1 + deg(i)))   (Eq. 8 in 32-bit fixed point)
// Score_j  S_j + sum of S_k over the neighbours k of j   (Eq. 9, all nodes
//          uncovered: the scores the lazy greedy starts from)
// Integer atomics only, so the results are exact and independent of the
// order in which the edges are visited.
#include "common.cuh"
#include "ctx.h"

namespace {

__device__ __forceinline__ uint64_t edge_count(uint64_t n, const unsigned long long *d_n) {
    return (d_n && *d_n < n) ? *d_n : n;
}

__global__ void degree_kernel(const pcl_pair *e, uint64_t n, const unsigned long long *d_n, uint32_t n_nodes,
                              unsigned int *deg) {
    const uint64_t m = edge_count(n, d_n);
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < m; k += (uint64_t)gridDim.x * blockDim.x) {
        const pcl_pair p = e[k];
        if (p.a >= n_nodes || p.b >= n_nodes || p.a == p.b) continue;
        atomicAdd(deg + p.a, 1u);
        atomicAdd(deg + p.b, 1u);
    }
}

__global__ void weight_kernel(const unsigned int *deg, uint32_t n_nodes, unsigned long long *w,
                              unsigned long long *score) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += gridDim.x * blockDim.x) {
        const unsigned long long s = (1ull << 32) / (1ull + deg[i]);
        w[i] = s;
        score[i] = s;
    }
}

__global__ void score_kernel(const pcl_pair *e, uint64_t n, const unsigned long long *d_n, uint32_t n_nodes,
                             const unsigned long long *w, unsigned long long *score) {
    const uint64_t m = edge_count(n, d_n);
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < m; k += (uint64_t)gridDim.x * blockDim.x) {
        const pcl_pair p = e[k];
        if (p.a >= n_nodes || p.b >= n_nodes || p.a == p.b) continue;
        atomicAdd(score + p.a, w[p.b]);
        atomicAdd(score + p.b, w[p.a]);
    }
}

}  // namespace

extern "C" pcl_status pcl_surprisal(pcl_ctx *ctx, const pcl_pair *d_edges, uint64_t n_edges, const uint64_t *d_n,
                                    uint32_t n_nodes, uint32_t *d_degree, uint64_t *d_weight, uint64_t *d_score,
                                    pcl_stream stream) {
    if (!ctx) return PCL_ERR_INVALID;
    ctx->err.clear();
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        ctx->err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return PCL_ERR_CUDA;
    }
    if ((n_edges && !d_edges) || (n_nodes && (!d_degree || !d_weight || !d_score))) {
        ctx->err = "pcl_surprisal: NULL buffer";
        return PCL_ERR_INVALID;
    }
    if (n_nodes == 0) return PCL_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const auto *dn = reinterpret_cast<const unsigned long long *>(d_n);
    auto *w = reinterpret_cast<unsigned long long *>(d_weight);
    auto *sc = reinterpret_cast<unsigned long long *>(d_score);
    const unsigned grid_e = (unsigned)(ctx->num_sms * 8), grid_n = (unsigned)((n_nodes + 255) / 256);
    e = cudaMemsetAsync(d_degree, 0, 4ull * n_nodes, st);
    if (e == cudaSuccess && n_edges) degree_kernel<<<grid_e, 256, 0, st>>>(d_edges, n_edges, dn, n_nodes, d_degree);
    if (e == cudaSuccess) weight_kernel<<<grid_n < 65535u ? grid_n : 65535u, 256, 0, st>>>(d_degree, n_nodes, w, sc);
    if (e == cudaSuccess && n_edges) score_kernel<<<grid_e, 256, 0, st>>>(d_edges, n_edges, dn, n_nodes, w, sc);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->err = std::string("pcl_surprisal: ") + cudaGetErrorString(e);
        return PCL_ERR_CUDA;
    }
    return PCL_OK;
}

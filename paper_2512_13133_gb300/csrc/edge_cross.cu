// Query x library edge screen of the serving loop (Sec. 2.2.2 gates E2/E1 and
// the Min-Max procedure of Sec. 3.2.2, Eq. 6, for every pair of a query set
// and a resident library).
#include "edge_dev.cuh"

namespace pcl {

namespace {
using namespace edge_dev;

// Query x library screen of edge mode for the serving loop: every pair
// (q, l) of the query set Q and the library L.  Lanes take pairs and run the
// gates of one record (edge_gate_record); the whole warp then evaluates each
// survivor (warp_edge_record).  Pairs that no gate rejects are appended with
// their records (the candidates and their alignment in one pass).
__device__ __forceinline__ void append_pair(bool keep, uint32_t q, uint32_t l, const pcl_record &r, pcl_pair *out,
                                            pcl_record *rec, uint64_t cap, unsigned long long *count) {
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    const unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
    if (keep && idx < cap) {
        out[idx] = pcl_pair{q, l};
        rec[idx] = r;
    }
}

__global__ void __launch_bounds__(256) edge_cross_kernel(pcl_params prm, pcl_clipset Q, pcl_clipset L,
                                                         pcl_pair *out, pcl_record *rec, uint64_t cap,
                                                         unsigned long long *count) {
    const uint64_t nl = L.n_clips, total = (uint64_t)Q.n_clips * nl;
    const int lane = threadIdx.x & 31;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = 32 * w0; base < total; base += 32 * nw) {  // warp-uniform
        const uint64_t p = base + lane;
        bool surv = false, keep = false;
        pcl_record r{};
        uint32_t q = 0, l = 0;
        if (p < total) {
            q = (uint32_t)(p / nl);
            l = (uint32_t)(p % nl);
            surv = edge_gate_record(prm, Q, L, pcl_pair{q, l}, &r);
            keep = !surv && (r.flags & PCL_F_EMPTY);  // both clips empty: similar by definition
        }
        append_pair(keep, q, l, r, out, rec, cap, count);
        unsigned m = __ballot_sync(0xffffffffu, surv);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t qs = __shfl_sync(0xffffffffu, q, src), ls = __shfl_sync(0xffffffffu, l, src);
            const pcl_record rs = warp_edge_record(prm, Q, L, pcl_pair{qs, ls}, lane);
            append_pair(lane == 0 && (rs.flags & 15) == 0, qs, ls, rs, out, rec, cap, count);
        }
    }
}

}  // namespace

// query x library edge screen + records of its candidates (serving)
cudaError_t launch_edge_cross(const pcl_params &prm, const pcl_clipset &q, const pcl_clipset &lib, pcl_pair *out,
                              pcl_record *rec, uint64_t cap, unsigned long long *count, int num_sms,
                              cudaStream_t st) {
    if ((uint64_t)q.n_clips * lib.n_clips == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_cross_kernel, 256, 0);
    if (e != cudaSuccess) return e;
    const uint64_t need = ((uint64_t)q.n_clips * lib.n_clips + 255) / 256;
    const uint64_t grid = (uint64_t)num_sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    edge_cross_kernel<<<(unsigned)(need < grid ? need : grid), 256, 0, st>>>(prm, q, lib, out, rec, cap, count);
    return cudaGetLastError();
}

}  // namespace pcl

// Hash index of the adjacency lists: one bucketed open-addressing table per
// list of at least HASH_MIN_LEN ids, so that a membership test against a long
// list (a probe of a candidate-set intersection) is one 32-byte sector read
// instead of a binary search.
#include "xm_kernels.cuh"

namespace xm {

namespace {

// One warp per list; lanes insert the list's ids with atomicCAS into the
// first free slot of their bucket (or of the following buckets).
__global__ void k_hash_build(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                             const int64_t* __restrict__ hoff, int32_t* __restrict__ htab, int32_t n) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nwarps) {
        const int64_t t0 = hoff[v];
        const uint32_t T = (uint32_t)(hoff[v + 1] - t0);
        if (T == 0) continue;
        const uint32_t nb = T / HASH_BUCKET;
        int32_t* tab = htab + t0;
        for (int i = off[v] + lane; i < off[v + 1]; i += 32) {
            const int32_t x = adj[i];
            uint32_t b = hash_bucket(x, nb);
            // a table is at most half full, so a free slot is always found
            bool placed = false;
            for (uint32_t step = 0; step < nb && !placed; step++) {
                for (int s = 0; s < HASH_BUCKET; s++) {
                    const int32_t old = atomicCAS(tab + (size_t)b * HASH_BUCKET + s, -1, x);
                    if (old == -1 || old == x) { placed = true; break; }
                }
                b = (b + 1) & (nb - 1);
            }
        }
    }
}

}  // namespace

cudaError_t build_hash_index(const int32_t* off, const int32_t* adj, const int64_t* hoff, int32_t* htab, int32_t n,
                             cudaStream_t stream) {
    int dev = 0, nsm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    k_hash_build<<<nsm * 8, 256, 0, stream>>>(off, adj, hoff, htab, n);
    return cudaGetLastError();
}

}  // namespace xm

// Hash index of the adjacency lists: one bucketed open-addressing table per
// list of at least HASH_MIN_LEN ids, so that a membership test against a long
// list (a probe of a candidate-set intersection) is one 32-byte sector read
// instead of a binary search.
#include <algorithm>

#include "xm_kernels.cuh"

namespace xm {

namespace {

// Slots 4q..4q+3 of a bucket, read from L2 (where the atomics land), not L1.
__device__ __forceinline__ int4 ld_l2(const int32_t* p) {
    int4 r;
    asm volatile("ld.global.cg.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

// One thread per list entry, over all lists at once, so that hub lists are
// spread over the whole grid instead of one warp each. The thread finds its
// list by a binary search of the offsets, reads the id's bucket (two 16-byte
// loads from L2) and claims the first empty slot with atomicCAS; a failed
// claim reads the bucket again, and a full bucket continues in the next one.
// Slots are only ever claimed in order within a bucket, so the filled slots
// of every bucket stay a prefix, which is what a search relies on.
__global__ void k_hash_build(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                             const int64_t* __restrict__ hoff, int32_t* __restrict__ htab, int32_t n, int64_t m) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        // list v holding entry i: the last v with off[v] <= i
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(off + mid) <= i) lo = mid; else hi = mid;
        }
        const int v = lo;
        const int64_t t0 = __ldg(hoff + v);
        const uint32_t T = (uint32_t)(__ldg(hoff + v + 1) - t0);
        if (T == 0) continue;
        const uint32_t nb = T / HASH_BUCKET;
        int32_t* tab = htab + t0;
        const int32_t x = __ldg(adj + i);
        uint32_t b = hash_bucket(x, nb);
        // a table is at most half full, so a free slot is always found
        for (uint32_t step = 0; step < nb; step++) {
            int32_t* bk = tab + (size_t)b * HASH_BUCKET;
            bool placed = false;
            for (;;) {
                const int4 a0 = ld_l2(bk), a1 = ld_l2(bk + 4);
                const int32_t y[HASH_BUCKET] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                int s = HASH_BUCKET;
#pragma unroll
                for (int j = HASH_BUCKET - 1; j >= 0; j--)
                    if (y[j] == -1) s = j;  // the first empty slot
#pragma unroll
                for (int j = 0; j < HASH_BUCKET; j++)
                    if (y[j] == x) placed = true;
                if (placed || s == HASH_BUCKET) break;
                const int32_t old = atomicCAS(bk + s, -1, x);
                if (old == -1 || old == x) { placed = true; break; }
            }
            if (placed) break;
            b = (b + 1) & (nb - 1);
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
    int32_t m32 = 0;  // the list entries: off[n]
    if ((e = cudaMemcpyAsync(&m32, off + n, sizeof m32, cudaMemcpyDeviceToHost, stream)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return e;
    const int64_t m = m32;
    if (m <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((m + 255) / 256, (int64_t)nsm * 64);
    k_hash_build<<<(int)blocks, 256, 0, stream>>>(off, adj, hoff, htab, n, m);
    return cudaGetLastError();
}

}  // namespace xm

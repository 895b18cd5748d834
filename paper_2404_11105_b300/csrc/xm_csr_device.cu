// Device construction of the dual sorted CSR (the out_arcs / in_arcs lists
// that plan execution reads, Alg. 2): repeats and self-loops dropped, every
// list ascending, int32 offsets.
//
// Each arc (u, v) becomes one 64-bit key u * 2^b + v (2^b >= n). A stable
// least-significant-digit radix sort over the key's 2b bits, 8 bits a pass,
// orders the keys by (u, v); equal neighbours are repeats. Self-loops get
// the key (2^b - 1, 2^b - 1), which sorts after every arc and is dropped
// with the repeats. The surviving keys give out_adj (their low halves) and
// out_off (the first position of every row). The in-CSR takes the surviving
// keys with the halves swapped and sorts them stably by their high half.
//
// One radix pass: every warp owns a tile of RADIX_TILE consecutive keys.
// k_radix_hist counts the tile's digits into hist[digit * tiles + tile]; an
// exclusive scan of hist (digit-major) gives each (digit, tile) its first
// output position; k_radix_scatter walks the tile again 32 keys at a time in
// order, ranks each key among the tile's keys of the same digit so far
// (__match_any_sync within the 32, a running count per digit in shared
// memory before them) and writes it to its position. Keys of one digit keep
// their order, so the sort is stable.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <string>

#include "xm_internal.h"
#include "xm_kernels.cuh"

namespace xm {

namespace {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int RADIX_TILE = 32 * 64;    // keys per warp tile
constexpr int RADIX_WARPS = 8;         // warps per block

// keys of the arcs; an endpoint outside [0, n) raises STATUS_BAD_ID in
// *status (its key is then meaningless and the build is rejected)
__global__ void k_pack_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m, int b,
                            int32_t n, unsigned long long* __restrict__ keys, unsigned long long* status) {
    const unsigned long long loop = ((1ull << b) - 1) << b | ((1ull << b) - 1);
    const unsigned long long mask = (1ull << b) - 1;
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = __ldg(src + i), v = __ldg(dst + i);
        bad |= (uint32_t)u >= (uint32_t)n || (uint32_t)v >= (uint32_t)n;
        keys[i] = u == v ? loop : (((unsigned long long)(uint32_t)u & mask) << b | ((uint32_t)v & mask));
    }
    if (bad) atomicOr(status, (unsigned long long)STATUS_BAD_ID);
}

__global__ void __launch_bounds__(32 * RADIX_WARPS) k_radix_hist(const unsigned long long* __restrict__ keys,
                                                                 int64_t m, int shift, int ntiles,
                                                                 int32_t* __restrict__ hist) {
    __shared__ int32_t cnt[RADIX_WARPS][RADIX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x * RADIX_WARPS + w;
    for (int d = lane; d < RADIX; d += 32) cnt[w][d] = 0;
    __syncwarp();
    if (tile < ntiles) {
        const int64_t base = (int64_t)tile * RADIX_TILE;
        for (int j = lane; j < RADIX_TILE; j += 32) {
            const int64_t i = base + j;
            if (i < m) atomicAdd(&cnt[w][(int)((__ldg(keys + i) >> shift) & (RADIX - 1))], 1);
        }
        __syncwarp();
        for (int d = lane; d < RADIX; d += 32) hist[(int64_t)d * ntiles + tile] = cnt[w][d];
    }
}

__global__ void __launch_bounds__(32 * RADIX_WARPS) k_radix_scatter(const unsigned long long* __restrict__ in,
                                                                    int64_t m, int shift, int ntiles,
                                                                    const int32_t* __restrict__ pos,
                                                                    unsigned long long* __restrict__ out) {
    __shared__ int32_t base_of[RADIX_WARPS][RADIX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x * RADIX_WARPS + w;
    if (tile >= ntiles) return;
    for (int d = lane; d < RADIX; d += 32) base_of[w][d] = __ldg(pos + (int64_t)d * ntiles + tile);
    __syncwarp();
    const int64_t base = (int64_t)tile * RADIX_TILE;
    const unsigned lt = (1u << lane) - 1;
    for (int j = 0; j < RADIX_TILE; j += 32) {
        const int64_t i = base + j + lane;
        const bool valid = i < m;
        const unsigned long long k = valid ? __ldg(in + i) : 0ull;
        // invalid lanes take a digit of their own (RADIX) so they join no group
        const int d = valid ? (int)((k >> shift) & (RADIX - 1)) : RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid) {
            const int at = base_of[w][d] + __popc(peers & lt);
            out[at] = k;
        }
        __syncwarp();
        if (valid && (peers & lt) == 0) base_of[w][d] += __popc(peers);  // the group's first lane
        __syncwarp();
    }
}

// flags[i] = 1 for the first copy of each arc (not a self-loop), else 0
__global__ void k_first_copies(const unsigned long long* __restrict__ keys, int64_t m, unsigned long long loop,
                               int32_t* __restrict__ flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = __ldg(keys + i);
        flags[i] = (k != loop && (i == 0 || __ldg(keys + i - 1) != k)) ? 1 : 0;
    }
}

// Compacts the first copies into out: `at` holds the exclusive scan of the
// first-copy flags, so key i is a first copy when at[i + 1] > at[i] (the
// last key: when last_flag).
__global__ void k_compact(const unsigned long long* __restrict__ keys, int64_t m, const int32_t* __restrict__ at,
                          int32_t last_flag, unsigned long long* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const bool first = i + 1 < m ? __ldg(at + i + 1) > __ldg(at + i) : last_flag != 0;
        if (first) out[__ldg(at + i)] = __ldg(keys + i);
    }
}

// From m ascending distinct keys: adj[p] = low half, and off[r] = the first
// position whose row is >= r, for r in [0, n] (rows between two keys' rows
// are filled by the later key's thread; the last key's thread fills the
// rows after it).
__global__ void k_csr_from_keys(const unsigned long long* __restrict__ keys, int64_t m, int b, int32_t n,
                                int32_t* __restrict__ off, int32_t* __restrict__ adj) {
    const unsigned long long mask = (1ull << b) - 1;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = __ldg(keys + p);
        adj[p] = (int32_t)(k & mask);
        const int32_t r = (int32_t)(k >> b);
        const int32_t rprev = p > 0 ? (int32_t)(__ldg(keys + p - 1) >> b) : -1;
        for (int32_t rr = rprev + 1; rr <= r; rr++) off[rr] = (int32_t)p;
    }
}

// off[r] = m for the rows after the last key's row (the last key's row is
// read on the device)
__global__ void k_fill_tail(const unsigned long long* __restrict__ keys, int64_t m, int b, int32_t n,
                            int32_t* __restrict__ off) {
    const int32_t r_last = (int32_t)(__ldg(keys + m - 1) >> b);
    for (int64_t r = r_last + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= n;
         r += (int64_t)gridDim.x * blockDim.x)
        off[r] = (int32_t)m;
}

// buckets[v] = hash-table buckets of node v's list (v < n), buckets[n] = 0
__global__ void k_table_buckets(const int32_t* __restrict__ off, int32_t n, int32_t* __restrict__ buckets) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x)
        buckets[v] = v < n ? (int32_t)(hash_table_size(__ldg(off + v + 1) - __ldg(off + v)) / HASH_BUCKET) : 0;
}

__global__ void k_hoff(const int32_t* __restrict__ buckets, int32_t n, int64_t* __restrict__ hoff) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x)
        hoff[v] = (int64_t)HASH_BUCKET * __ldg(buckets + v);
}

__global__ void k_fill(int32_t* __restrict__ off, int32_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        off[i] = v;
}

// swapped keys (v, u) of the out-CSR's keys
__global__ void k_swap_keys(const unsigned long long* __restrict__ keys, int64_t m, int b,
                            unsigned long long* __restrict__ out) {
    const unsigned long long mask = (1ull << b) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = __ldg(keys + i);
        out[i] = (k & mask) << b | (k >> b);
    }
}

int grid_for(int64_t items, int nsm) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, (int64_t)nsm * 32));
}

}  // namespace

// Sorts keys[0..m) by their bits [lo_bit, hi_bit) (stable LSD radix sort:
// keys equal in those bits keep their order), using tmp[m] and hist of
// ceil(m / RADIX_TILE) * RADIX ints; the result ends in *sorted (keys or tmp).
static cudaError_t radix_sort(unsigned long long* keys, unsigned long long* tmp, int64_t m, int lo_bit, int hi_bit,
                              int32_t* hist, const RunArgs& sa, unsigned long long** sorted, cudaStream_t stream) {
    const int ntiles = (int)((m + RADIX_TILE - 1) / RADIX_TILE);
    const int blocks = (ntiles + RADIX_WARPS - 1) / RADIX_WARPS;
    unsigned long long* a = keys;
    unsigned long long* o = tmp;
    for (int shift = lo_bit; shift < hi_bit; shift += RADIX_BITS) {
        k_radix_hist<<<blocks, 32 * RADIX_WARPS, 0, stream>>>(a, m, shift, ntiles, hist);
        cudaError_t e = scan_int32_in_place(hist, (int64_t)ntiles * RADIX, sa, stream);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<blocks, 32 * RADIX_WARPS, 0, stream>>>(a, m, shift, ntiles, hist, o);
        std::swap(a, o);
    }
    *sorted = a;
    return cudaGetLastError();
}

int csr_key_bits(int32_t n) {
    int b = 1;
    while ((1ll << b) < (int64_t)n) b++;
    return b;
}

int64_t csr_int_scratch(int64_t m, int32_t n) {
    const int64_t ntiles = (m + RADIX_TILE - 1) / RADIX_TILE;
    return std::max<int64_t>(std::max<int64_t>(ntiles * RADIX, m + 1), (int64_t)n + 2);
}

cudaError_t csr_sort_unique(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, unsigned long long* k0,
                            unsigned long long* k1, int32_t* ints, const RunArgs& sa, unsigned long long** keys_out,
                            int64_t* m_out, cudaStream_t stream) {
    cudaError_t e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *keys_out = k0;
    *m_out = 0;
    if (m == 0) return cudaSuccess;
    const int b = csr_key_bits(n);
    const unsigned long long loop = ((1ull << b) - 1) << b | ((1ull << b) - 1);
    k_pack_keys<<<grid_for(m, nsm), 256, 0, stream>>>(src, dst, m, b, n, k0, sa.ctl + CTL_STATUS);
    unsigned long long* sorted = nullptr;
    if ((e = radix_sort(k0, k1, m, 0, 2 * b, ints, sa, &sorted, stream)) != cudaSuccess) return e;
    unsigned long long* other = sorted == k0 ? k1 : k0;
    k_first_copies<<<grid_for(m, nsm), 256, 0, stream>>>(sorted, m, loop, ints);
    int32_t last[2] = {0, 0};  // the last key's flag, then its scanned position
    if ((e = cudaMemcpyAsync(&last[0], ints + m - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return e;
    if ((e = scan_int32_in_place(ints, m, sa, stream)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&last[1], ints + m - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return e;
    k_compact<<<grid_for(m, nsm), 256, 0, stream>>>(sorted, m, ints, last[0], other);
    *keys_out = other;
    *m_out = (int64_t)last[1] + last[0];
    return cudaGetLastError();
}

cudaError_t csr_emit(int32_t n, unsigned long long* keys, unsigned long long* spare, int64_t mm, int32_t* ints,
                     const RunArgs& sa, int32_t* out_off, int32_t* out_adj, int32_t* in_off, int32_t* in_adj,
                     cudaStream_t stream) {
    cudaError_t e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (mm == 0) {
        k_fill<<<grid_for((int64_t)n + 1, nsm), 256, 0, stream>>>(out_off, n, 0);
        k_fill<<<grid_for((int64_t)n + 1, nsm), 256, 0, stream>>>(in_off, n, 0);
        return cudaGetLastError();
    }
    const int b = csr_key_bits(n);
    k_csr_from_keys<<<grid_for(mm, nsm), 256, 0, stream>>>(keys, mm, b, n, out_off, out_adj);
    k_fill_tail<<<grid_for((int64_t)n + 1, nsm), 256, 0, stream>>>(keys, mm, b, n, out_off);
    k_swap_keys<<<grid_for(mm, nsm), 256, 0, stream>>>(keys, mm, b, spare);
    // the swapped keys (v, u) come in ascending u within each v (the keys were
    // sorted by (u, v)), so a stable sort by their high half v completes the
    // order: half the passes of a full sort
    unsigned long long* sorted = nullptr;
    if ((e = radix_sort(spare, keys, mm, b, 2 * b, ints, sa, &sorted, stream)) != cudaSuccess) return e;
    k_csr_from_keys<<<grid_for(mm, nsm), 256, 0, stream>>>(sorted, mm, b, n, in_off, in_adj);
    k_fill_tail<<<grid_for((int64_t)n + 1, nsm), 256, 0, stream>>>(sorted, mm, b, n, in_off);
    return cudaGetLastError();
}

cudaError_t hash_offsets(const int32_t* off, int32_t n, int32_t* ints, const RunArgs& sa, int64_t* hoff,
                         cudaStream_t stream) {
    cudaError_t e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    k_table_buckets<<<grid_for((int64_t)n + 1, nsm), 256, 0, stream>>>(off, n, ints);
    if ((e = scan_int32_in_place(ints, (int64_t)n + 1, sa, stream)) != cudaSuccess) return e;
    k_hoff<<<grid_for((int64_t)n + 1, nsm), 256, 0, stream>>>(ints, n, hoff);
    return cudaGetLastError();
}

}  // namespace xm

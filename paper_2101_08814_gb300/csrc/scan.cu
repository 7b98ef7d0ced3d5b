// Device-wide exclusive prefix sum (three passes, no inter-block waiting): per-block scans, a single-block scan
// of the block totals, then a uniform add. out[0..n] with out[n] = total; in and out may alias.
#include "common.cuh"

namespace rascal {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline int64_t block_exclusive_scan(int64_t v, int64_t* warp_tot, int64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t t = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = t;
        if (lane == kScanThreads / 32 - 1) *total = t;
    }
    __syncthreads();
    const int64_t before = warp ? warp_tot[warp - 1] : 0;
    return before + x - v;
}

template <typename Tin>
__global__ void k_scan_tiles(const Tin* in, int64_t* out, int64_t n, int64_t* tile_sums) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    __shared__ int64_t total;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? (int64_t)in[base + k] : 0;
        s += v[k];
    }
    int64_t ex = block_exclusive_scan(s, warp_tot, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// one block: exclusive scan of the tile sums in place, total to *grand
__global__ void k_scan_tile_sums(int64_t* sums, int64_t n_tiles, int64_t* grand) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    __shared__ int64_t total;
    int64_t carry = 0;
    for (int64_t start = 0; start < n_tiles; start += kScanThreads) {
        const int64_t i = start + threadIdx.x;
        const int64_t v = (i < n_tiles) ? sums[i] : 0;
        const int64_t ex = block_exclusive_scan(v, warp_tot, &total);
        if (i < n_tiles) sums[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int64_t add = tile_sums[blockIdx.x];
    for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
        const int64_t i = base + k;
        if (i < n) out[i] += add;
    }
}

template <typename Tin>
static int scan_impl(const Tin* in, int64_t* out, int64_t n, cudaStream_t stream, Arena& scratch) {
    const int64_t tiles = div_up(n > 0 ? n : 1, kScanTile);
    void* buf;
    int st = arena_get(scratch, sizeof(int64_t) * (tiles + 1), &buf);
    if (st) return st;
    int64_t* sums = static_cast<int64_t*>(buf);
    k_scan_tiles<Tin><<<(unsigned)tiles, kScanThreads, 0, stream>>>(in, out, n, sums);
    RASCAL_LAUNCH_CHECK("k_scan_tiles");
    k_scan_tile_sums<<<1, kScanThreads, 0, stream>>>(sums, tiles, out + n);
    RASCAL_LAUNCH_CHECK("k_scan_tile_sums");
    if (tiles > 1) {
        k_scan_add<<<(unsigned)tiles, kScanThreads, 0, stream>>>(out, n, sums);
        RASCAL_LAUNCH_CHECK("k_scan_add");
    }
    return RASCAL_OK;
}

// Same scan with a caller-provided buffer for the tile sums (scan_tile_sums_len(n) int64 words); allocates nothing.
template <typename Tin>
static int scan_into_impl(const Tin* in, int64_t* out, int64_t n, cudaStream_t stream, int64_t* sums) {
    const int64_t tiles = div_up(n > 0 ? n : 1, kScanTile);
    k_scan_tiles<Tin><<<(unsigned)tiles, kScanThreads, 0, stream>>>(in, out, n, sums);
    RASCAL_LAUNCH_CHECK("k_scan_tiles");
    k_scan_tile_sums<<<1, kScanThreads, 0, stream>>>(sums, tiles, out + n);
    RASCAL_LAUNCH_CHECK("k_scan_tile_sums");
    if (tiles > 1) {
        k_scan_add<<<(unsigned)tiles, kScanThreads, 0, stream>>>(out, n, sums);
        RASCAL_LAUNCH_CHECK("k_scan_add");
    }
    return RASCAL_OK;
}

int64_t scan_tile_sums_len(int64_t n) { return div_up(n > 0 ? n : 1, kScanTile) + 1; }
int scan_exclusive_into(const int* in, int64_t* out, int64_t n, cudaStream_t stream, int64_t* sums) {
    return scan_into_impl<int>(in, out, n, stream, sums);
}
int scan_exclusive_into(const int64_t* in, int64_t* out, int64_t n, cudaStream_t stream, int64_t* sums) {
    return scan_into_impl<int64_t>(in, out, n, stream, sums);
}

int scan_exclusive(const int* in, int64_t* out, int64_t n, cudaStream_t stream, Arena& scratch) {
    return scan_impl<int>(in, out, n, stream, scratch);
}
int scan_exclusive(const int64_t* in, int64_t* out, int64_t n, cudaStream_t stream, Arena& scratch) {
    return scan_impl<int64_t>(in, out, n, stream, scratch);
}

}  // namespace rascal

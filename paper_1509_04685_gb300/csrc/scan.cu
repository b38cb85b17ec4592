// Exclusive prefix sum of int32 counts on the device (used by the FoF cell
// list and by the particle binning of the PM step): a[0..n) is replaced by
// its exclusive scan and a[n] receives the total, in three launches (tile
// sums, a one-block scan of the tile sums, the tiles' own scans).
#include "cola_common.cuh"

namespace cola {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// ---------------------------------------------------------------------------
// exclusive scan of a[0..n) in place, a[n] = total (int32, n + 1 entries)
// ---------------------------------------------------------------------------
// block-wide exclusive scan of one value per thread; returns the block total
__device__ __forceinline__ int block_exclusive_scan(int v, int* excl) {
    __shared__ int warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const int before = w ? warp_tot[w - 1] : 0;
    *excl = before + x - v;
    const int total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();  // warp_tot is reused by the next call
    return total;
}

__device__ __forceinline__ void tile_load(const int* a, long long n, long long base, int v[kScanItems]) {
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const long long i = base + (long long)threadIdx.x * kScanItems + r;
        v[r] = i < n ? a[i] : 0;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int* a, long long n, int* sums) {
    int v[kScanItems];
    tile_load(a, n, (long long)blockIdx.x * kScanTile, v);
    int s = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) s += v[r];
    int ex;
    const int tot = block_exclusive_scan(s, &ex);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// one block: exclusive scan of the nb tile sums in place; a[n] = total
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int* sums, int nb, int* a, long long n) {
    int carry = 0;
    for (long long base = 0; base < nb; base += kScanTile) {
        int v[kScanItems];
        tile_load(sums, nb, base, v);
        int s = 0;
#pragma unroll
        for (int r = 0; r < kScanItems; ++r) s += v[r];
        int ex;
        const int tot = block_exclusive_scan(s, &ex);
        int run = carry + ex;
#pragma unroll
        for (int r = 0; r < kScanItems; ++r) {
            const long long i = base + (long long)threadIdx.x * kScanItems + r;
            if (i < nb) sums[i] = run;
            run += v[r];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) a[n] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int* a, long long n, const int* sums) {
    const long long base = (long long)blockIdx.x * kScanTile;
    int v[kScanItems];
    tile_load(a, n, base, v);
    int s = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) s += v[r];
    int ex;
    block_exclusive_scan(s, &ex);
    int run = sums[blockIdx.x] + ex;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const long long i = base + (long long)threadIdx.x * kScanItems + r;
        if (i < n) a[i] = run;
        run += v[r];
    }
}

}  // namespace

size_t scan_sums_bytes(long long n) { return (size_t)((n + kScanTile - 1) / kScanTile) * sizeof(int); }

int exclusive_scan(int* a, long long n, int* sums, cudaStream_t s) {
    const int nb = (int)((n + kScanTile - 1) / kScanTile);
    if (nb > 0) {
        k_scan_tiles<<<nb, kScanThreads, 0, s>>>(a, n, sums);
        if (int rc = check_launch()) return rc;
    }
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, nb, a, n);
    if (int rc = check_launch()) return rc;
    if (nb > 0) {
        k_scan_apply<<<nb, kScanThreads, 0, s>>>(a, n, sums);
        return check_launch();
    }
    return COLA_OK;
}

}  // namespace cola

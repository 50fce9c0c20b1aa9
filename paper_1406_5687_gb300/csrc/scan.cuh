// scan.cuh -- device-wide exclusive prefix sum over a generated sequence.
//
// out[i] = sum_{j<i} f(j) for i in [0, n], uint64, where f is a device functor
// `uint64_t operator()(int64_t i) const`.  Three phases (tile reduce, scan of the
// tile sums, tile downsweep); f is evaluated twice per element.  No inter-block
// waiting, so nothing can spin.
#pragma once

#include "common.cuh"

namespace tcg {

constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = (int64_t)kScanBlock * kScanItems;

template <class F>
__global__ void __launch_bounds__(kScanBlock) k_scan_tile_sums(F f, int64_t n, uint64_t* tile_sums) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)warp * 32 * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * 32 + lane;
        if (i < n) s += f(i);
    }
    s = warp_sum(s);
    __shared__ uint64_t ws[kScanBlock / 32];
    if (lane == 0) ws[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < kScanBlock / 32; ++w) t += ws[w];
        tile_sums[blockIdx.x] = t;
    }
}

// In-place exclusive scan of v[0..n) by one block; v[n] receives the total.
__global__ void k_scan_single_block(uint64_t* v, int64_t n);

template <class F>
__global__ void __launch_bounds__(kScanBlock) k_scan_downsweep(F f, int64_t n, const uint64_t* tile_prefix,
                                                                uint64_t* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)warp * 32 * kScanItems;
    uint64_t ex[kScanItems];
    uint64_t carry = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * 32 + lane;
        uint64_t v = i < n ? f(i) : 0;
        uint64_t incl = warp_inclusive_scan(v, lane);
        ex[k] = carry + incl - v;
        carry += __shfl_sync(kFull, incl, 31);
    }
    __shared__ uint64_t ws[kScanBlock / 32];
    if (lane == 0) ws[warp] = carry;
    __syncthreads();
    uint64_t woff = tile_prefix[blockIdx.x];
    for (int w = 0; w < warp; ++w) woff += ws[w];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * 32 + lane;
        if (i < n) out[i] = woff + ex[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = tile_prefix[gridDim.x];
}

// Scratch needed by scan_exclusive for n elements (uint64 words).
inline int64_t scan_scratch_words(int64_t n) {
    int64_t tiles = ceil_div(n > 0 ? n : 1, kScanTile);
    int64_t words = tiles + 1;
    // large inputs scan their tile sums recursively into a second array of tiles+1 words
    if (tiles > 4096) words += (tiles + 1) + scan_scratch_words(tiles);
    return words;
}

struct IdentityU64 {
    const uint64_t* v;
    __device__ uint64_t operator()(int64_t i) const { return v[i]; }
};

// out: n+1 uint64 (out[n] = total).  scratch: scan_scratch_words(n) uint64.
template <class F>
cudaError_t scan_exclusive(F f, int64_t n, uint64_t* out, uint64_t* scratch, cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(uint64_t), s);
    const int64_t tiles = ceil_div(n, kScanTile);
    uint64_t* tile = scratch;  // tiles + 1
    k_scan_tile_sums<<<(unsigned)tiles, kScanBlock, 0, s>>>(f, n, tile);
    note_launch();
    if (tiles <= 4096) {
        k_scan_single_block<<<1, 1024, 0, s>>>(tile, tiles);
        note_launch();
    } else {
        // scan the tile sums with the same machinery; the result lands in place
        uint64_t* tmp = scratch + tiles + 1;
        cudaError_t e = scan_exclusive(IdentityU64{tile}, tiles, tmp, tmp + tiles + 1, s);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(tile, tmp, (tiles + 1) * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    k_scan_downsweep<<<(unsigned)tiles, kScanBlock, 0, s>>>(f, n, tile, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tcg

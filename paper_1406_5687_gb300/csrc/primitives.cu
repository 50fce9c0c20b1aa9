// primitives.cu -- LSD radix sort (step a2's sort) and the single-block scan.
//
// Each 8-bit pass is reduce-then-scan: a per-tile digit histogram, one device-wide
// exclusive scan of the digit-major counts, and a scatter that ranks the tile's keys
// stably in shared memory (warp match + per-warp digit counters) and writes every digit
// run contiguously.  No block waits on another block.
#include <atomic>
#include <mutex>

#include "primitives.cuh"
#include "scan.cuh"

namespace tcg {

static std::atomic<long long> g_launches{0};
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void retain_pool_memory() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    (void)cudaGetLastError();
    done[dev] = true;
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

__global__ void k_scan_single_block(uint64_t* v, int64_t n) {
    // n <= 4096: each of the 1024 threads scans four consecutive values
    __shared__ uint64_t part[1024];
    const int t = threadIdx.x;
    uint64_t x[4];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int64_t i = (int64_t)t * 4 + k;
        x[k] = i < n ? v[i] : 0;
        s += x[k];
    }
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        uint64_t add = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += add;
        __syncthreads();
    }
    uint64_t run = part[t] - s;  // exclusive prefix of this thread's group
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int64_t i = (int64_t)t * 4 + k;
        if (i < n) v[i] = run;
        run += x[k];
    }
    if (t == 1023) v[n] = part[1023];
}

// --------------------------------------------------------------------------- radix sort

constexpr int kRsBlock = 512;
constexpr int kRsWarps = kRsBlock / 32;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsBlock * kRsItems;  // 8192 keys
constexpr int kRsRadix = 256;

struct IdentityU32 {
    const uint32_t* v;
    __device__ uint64_t operator()(int64_t i) const { return v[i]; }
};

__global__ void __launch_bounds__(kRsBlock) k_rs_hist(const uint64_t* __restrict__ in, int64_t n, int shift,
                                                      int64_t ntiles, uint32_t* __restrict__ counts) {
    __shared__ uint32_t h[kRsWarps][kRsRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * kRsRadix; i += kRsBlock) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int j = 0; j < kRsItems; ++j) {
        int64_t i = base + (int64_t)j * kRsBlock + threadIdx.x;
        unsigned d = i < n ? (unsigned)((in[i] >> shift) & 0xFF) : 256u;
        unsigned peers = __match_any_sync(kFull, d);
        if (d < 256u && lane == __ffs(peers) - 1) h[warp][d] += __popc(peers);
    }
    __syncthreads();
    if (threadIdx.x < kRsRadix) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) s += h[w][threadIdx.x];
        counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = s;
    }
}

constexpr size_t kRsScatterSmem = (size_t)kRsTile * 8 + (size_t)kRsWarps * kRsRadix * 4 + 264 * 4 + kRsRadix * 8;

__global__ void __launch_bounds__(kRsBlock) k_rs_scatter(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                         int64_t n, int shift, int64_t ntiles,
                                                         const uint64_t* __restrict__ offs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* skeys = (uint64_t*)smem_raw;                    // kRsTile
    uint32_t* wcnt = (uint32_t*)(skeys + kRsTile);            // kRsWarps * 256
    uint32_t* dstart = wcnt + kRsWarps * kRsRadix;            // 256 (+ 8 for the warp totals)
    uint64_t* goff = (uint64_t*)(dstart + 264);               // 256
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tbase = (int64_t)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsWarps * kRsRadix; i += kRsBlock) wcnt[i] = 0;
    if (threadIdx.x < kRsRadix) goff[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();

    // warp-striped load: lane l holds the warp's keys j*32 + l, j = 0..15 (memory order j-major)
    const int64_t wbase = tbase + (int64_t)warp * 32 * kRsItems;
    uint64_t key[kRsItems];
    uint32_t rank[kRsItems];
    uint32_t* mycnt = wcnt + warp * kRsRadix;
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
        int64_t i = wbase + j * 32 + lane;
        bool valid = i < n;
        key[j] = valid ? in[i] : 0;
        unsigned d = valid ? (unsigned)((key[j] >> shift) & 0xFF) : 256u;
        unsigned peers = __match_any_sync(kFull, d);
        int leader = __ffs(peers) - 1;
        uint32_t b = 0;
        if (lane == leader && d < 256u) {
            b = mycnt[d];
            mycnt[d] = b + __popc(peers);
        }
        b = __shfl_sync(kFull, b, leader);
        rank[j] = b + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    // per digit: exclusive scan over warps, then over digits
    if (threadIdx.x < kRsRadix) {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            uint32_t t = wcnt[w * kRsRadix + d];
            wcnt[w * kRsRadix + d] = run;
            run += t;
        }
        uint32_t incl = warp_inclusive_scan(run, lane);
        if (lane == 31) dstart[256 + warp] = incl;  // warp totals (8 warps cover 256 digits)
        dstart[d] = incl - run;
    }
    __syncthreads();
    if (threadIdx.x < kRsRadix) {
        uint32_t add = 0;
        for (int w = 0; w < warp; ++w) add += dstart[256 + w];
        dstart[threadIdx.x] += add;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
        int64_t i = wbase + j * 32 + lane;
        if (i < n) {
            unsigned d = (unsigned)((key[j] >> shift) & 0xFF);
            skeys[dstart[d] + mycnt[d] + rank[j]] = key[j];
        }
    }
    __syncthreads();
    const int64_t valid = n - tbase < kRsTile ? n - tbase : kRsTile;
    for (int i = threadIdx.x; i < valid; i += kRsBlock) {
        uint64_t k = skeys[i];
        unsigned d = (unsigned)((k >> shift) & 0xFF);
        out[goff[d] + (uint64_t)(i - (int)dstart[d])] = k;
    }
}

int64_t radix_sort_scratch_bytes(int64_t n) {
    int64_t ntiles = ceil_div(n > 0 ? n : 1, kRsTile);
    int64_t cnt = ntiles * kRsRadix;
    return (int64_t)align_up(cnt * 4, 256) + (int64_t)align_up((cnt + 1) * 8, 256) +
           (int64_t)align_up(scan_scratch_words(cnt) * 8, 256);
}

tc_status radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int nbits, Allocator* al, cudaStream_t s,
                         uint64_t** result) {
    *result = keys;
    if (n <= 1 || nbits <= 0) return TC_OK;
    TC_CUDA_TRY(cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRsScatterSmem));
    const int64_t ntiles = ceil_div(n, kRsTile);
    const int64_t cnt = ntiles * kRsRadix;
    DevBuf<uint32_t> counts;
    DevBuf<uint64_t> offs, scr;
    TC_TRY(counts.alloc(al, cnt, s));
    TC_TRY(offs.alloc(al, cnt + 1, s));
    TC_TRY(scr.alloc(al, scan_scratch_words(cnt), s));
    uint64_t* a = keys;
    uint64_t* b = tmp;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_rs_hist<<<(unsigned)ntiles, kRsBlock, 0, s>>>(a, n, shift, ntiles, counts.ptr);
        note_launch();
        TC_CUDA_TRY(scan_exclusive(IdentityU32{counts.ptr}, cnt, offs.ptr, scr.ptr, s));
        k_rs_scatter<<<(unsigned)ntiles, kRsBlock, kRsScatterSmem, s>>>(a, b, n, shift, ntiles, offs.ptr);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
        uint64_t* t = a;
        a = b;
        b = t;
    }
    *result = a;
    return TC_OK;
}

}  // namespace tcg

extern "C" int64_t tc_kernel_launches(void) { return (int64_t)tcg::g_launches.load(); }

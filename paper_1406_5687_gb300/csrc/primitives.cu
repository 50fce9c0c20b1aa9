// primitives.cu -- LSD radix sort (the sorts of steps a2 and a5 and of the task array), the
// single-block scan, the library's bounded device wait and its launch counter.
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
    // initialised once, thread-safely (slot threads of a server may ask at the same time)
    static const int sms = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
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
//
// LSD radix sort with 8-bit digits and one kernel per digit (the "onesweep" arrangement of
// Adinets and Merrill, 2022).  One upfront pass counts every digit of every key.  Each
// digit pass then takes tiles of 4096 keys in the order blocks start (an atomic tile
// counter), counts the tile's digits and publishes them at once, ranks the tile's keys
// stably in shared memory while the first look-back load is in flight, and obtains the
// count of each digit in all earlier tiles by a decoupled look-back over their published
// words (flag in the top two bits: aggregate of the tile alone, or inclusive prefix), then
// writes every digit run of the tile contiguously.
// A tile waits only on tiles taken earlier, whose blocks are already running; every wait
// is bounded and sets the error word when it gives up.

// Tile shape: threads per block, keys per thread, and the blocks per SM the register
// budget is sized for (the block must have at least 256 threads: one per digit).
#ifndef TC_OS_BLOCK
#define TC_OS_BLOCK 256
#endif
#ifndef TC_OS_ITEMS
#define TC_OS_ITEMS 16
#endif
#ifndef TC_OS_MINB
#define TC_OS_MINB 4
#endif
constexpr int kOsBlock = TC_OS_BLOCK;
constexpr int kOsWarps = kOsBlock / 32;
constexpr int kOsItems = TC_OS_ITEMS;
constexpr int kOsTile = kOsBlock * kOsItems;
static_assert(kOsBlock >= 256 && kOsBlock % 32 == 0, "one thread per digit");
constexpr int kRadix = 256;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kCountMask = (1ull << 62) - 1;

// Counts of every digit of every pass (npass * 256, uint64).  Each warp counts into its
// own shared-memory copy, so atomics only collide between lanes of one warp.
__global__ void __launch_bounds__(kOsBlock) k_os_hist(const uint64_t* __restrict__ keys, int64_t n, int lo_bit,
                                                      int npass, unsigned long long* __restrict__ ghist) {
    extern __shared__ unsigned hs[];  // kOsWarps * npass * 256
    const int warp = threadIdx.x >> 5;
    const int per_warp = npass * kRadix;
    for (int i = threadIdx.x; i < kOsWarps * per_warp; i += kOsBlock) hs[i] = 0;
    __syncthreads();
    unsigned* h = hs + warp * per_warp;
    for (int64_t i = (int64_t)blockIdx.x * kOsBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kOsBlock) {
        const uint64_t k = keys[i] >> lo_bit;
        for (int p = 0; p < npass; ++p) atomicAdd(&h[p * kRadix + (unsigned)((k >> (8 * p)) & 0xFF)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < per_warp; i += kOsBlock) {
        unsigned t = 0;
        for (int w = 0; w < kOsWarps; ++w) t += hs[w * per_warp + i];
        if (t) atomicAdd(&ghist[i], (unsigned long long)t);
    }
}

// Exclusive scan of each pass's 256 digit counts, in place (one block per pass).
__global__ void k_os_bases(unsigned long long* ghist) {
    __shared__ unsigned long long v[kRadix];
    unsigned long long* g = ghist + (int64_t)blockIdx.x * kRadix;
    const int d = threadIdx.x;
    const unsigned long long own = g[d];
    v[d] = own;
    __syncthreads();
    for (int o = 1; o < kRadix; o <<= 1) {
        const unsigned long long t = d >= o ? v[d - o] : 0ull;
        __syncthreads();
        v[d] += t;
        __syncthreads();
    }
    g[d] = v[d] - own;
}

constexpr size_t kOsSmem = (size_t)kOsTile * 8 + (size_t)kOsWarps * kRadix * 4 + 264 * 4 + kRadix * 8;

// Poll *p until it is nonzero; give up (return 0) once `spins`, shared by the caller's
// successive waits, exceeds `limit`.  Every device wait of the library goes through here.
__device__ __forceinline__ unsigned long long wait_nonzero(const unsigned long long* p, long long limit,
                                                           long long& spins) {
    for (;;) {
        const unsigned long long v = *(const volatile unsigned long long*)p;
        if (v != 0) return v;
        if (++spins > limit) return 0;
    }
}

// One thread waits on a flag that nothing sets: the wait must give up after `limit` polls
// and record TC_ERR_TIMEOUT.
__global__ void k_wait_selftest(const unsigned long long* flag, long long limit, DevStatus* err) {
    long long spins = 0;
    if (wait_nonzero(flag, limit, spins) == 0) set_error(err, TC_ERR_TIMEOUT, spins);
}

__global__ void __launch_bounds__(kOsBlock, TC_OS_MINB) k_os_pass(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                      int64_t n, int shift, const unsigned long long* __restrict__ base,
                                                      unsigned long long* status, unsigned* tile_counter,
                                                      DevStatus* err, long long spin_limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* skeys = (uint64_t*)smem_raw;                           // kOsTile
    uint32_t* wcnt = (uint32_t*)(skeys + kOsTile);                   // kOsWarps * 256
    uint32_t* dstart = wcnt + kOsWarps * kRadix;                     // 256 + 8 warp totals
    unsigned long long* goff = (unsigned long long*)(dstart + 264);  // 256
    __shared__ unsigned s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    for (int i = threadIdx.x; i < kOsWarps * kRadix; i += kOsBlock) wcnt[i] = 0;
    __syncthreads();
    const long long tile = (long long)s_tile;
    const int64_t tbase = tile * kOsTile;

    // warp-striped load: lane l holds the warp's keys j*32 + l (memory order j-major)
    const int64_t wbase = tbase + (int64_t)warp * 32 * kOsItems;
    uint64_t key[kOsItems];
    uint32_t rank[kOsItems];
    uint32_t* mycnt = wcnt + warp * kRadix;
    __shared__ uint32_t s_hist[kRadix];
    if (threadIdx.x < kRadix) s_hist[threadIdx.x] = 0;
#pragma unroll
    for (int j = 0; j < kOsItems; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        key[j] = i < n ? in[i] : 0;
    }
    __syncthreads();
    // early counts: the tile's digit histogram, published before the ranking so that later
    // tiles find it sooner; the first look-back load is issued before ranking too
#pragma unroll
    for (int j = 0; j < kOsItems; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        if (i < n) atomicAdd(&s_hist[(unsigned)((key[j] >> shift) & 0xFF)], 1u);
    }
    __syncthreads();
    unsigned long long* st = status + tile * kRadix;
    uint32_t run = 0;
    unsigned long long lb_first = 0;
    if (threadIdx.x < kRadix) {
        run = s_hist[threadIdx.x];
        if (tile == 0) {
            *(volatile unsigned long long*)&st[threadIdx.x] = kFlagPrefix | run;
        } else {
            *(volatile unsigned long long*)&st[threadIdx.x] = kFlagAgg | run;
            lb_first = *(const volatile unsigned long long*)&status[(tile - 1) * kRadix + threadIdx.x];
        }
    }
#pragma unroll
    for (int j = 0; j < kOsItems; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        const bool valid = i < n;
        const unsigned d = valid ? (unsigned)((key[j] >> shift) & 0xFF) : 256u;
        // lanes holding the same digit: one ballot per digit bit (cheaper than a warp match);
        // lanes past the end form a group of their own
        const unsigned vmask = __ballot_sync(kFull, valid);
        unsigned peers = valid ? vmask : ~vmask;
#pragma unroll
        for (int bt = 0; bt < 8; ++bt) {
            const unsigned bit = (d >> bt) & 1u;
            peers &= __ballot_sync(kFull, bit) ^ (bit - 1u);
        }
        const int leader = __ffs(peers) - 1;
        uint32_t b = 0;
        if (lane == leader && d < 256u) {
            b = mycnt[d];
            mycnt[d] = b + __popc(peers);
        }
        b = __shfl_sync(kFull, b, leader);
        rank[j] = b + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    if (threadIdx.x < kRadix) {
        const int d = threadIdx.x;
        // per digit: exclusive scan over the warps
        uint32_t r2 = 0;
#pragma unroll
        for (int w = 0; w < kOsWarps; ++w) {
            const uint32_t t = wcnt[w * kRadix + d];
            wcnt[w * kRadix + d] = r2;
            r2 += t;
        }
        unsigned long long excl = 0;
        if (tile != 0) {
            long long j = tile - 1;
            long long spins = 0;
            unsigned long long v = lb_first;
            for (;;) {
                if (v == 0) v = wait_nonzero(&status[j * kRadix + d], spin_limit, spins);
                if (v == 0) {
                    set_error(err, TC_ERR_TIMEOUT, tile);
                    break;
                }
                const unsigned long long f = v & ~kCountMask;
                excl += v & kCountMask;
                if (f == kFlagPrefix || j == 0) break;
                --j;
                v = *(const volatile unsigned long long*)&status[j * kRadix + d];
            }
            *(volatile unsigned long long*)&st[d] = kFlagPrefix | (excl + run);
        }
        goff[d] = base[d] + excl;
        // tile-local start of each digit: scan over the digits
        const uint32_t incl = warp_inclusive_scan(run, lane);
        if (lane == 31) dstart[256 + warp] = incl;
        dstart[d] = incl - run;
    }
    __syncthreads();
    if (threadIdx.x < kRadix) {
        uint32_t add = 0;
        for (int w = 0; w < warp; ++w) add += dstart[256 + w];
        dstart[threadIdx.x] += add;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kOsItems; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        if (i < n) {
            const unsigned d = (unsigned)((key[j] >> shift) & 0xFF);
            skeys[dstart[d] + mycnt[d] + rank[j]] = key[j];
        }
    }
    __syncthreads();
    const int64_t valid = n - tbase < kOsTile ? n - tbase : kOsTile;
    for (int i = threadIdx.x; i < valid; i += kOsBlock) {
        const uint64_t k = skeys[i];
        const unsigned d = (unsigned)((k >> shift) & 0xFF);
        out[goff[d] + (uint64_t)(i - (int)dstart[d])] = k;
    }
}

int64_t radix_sort_scratch_bytes(int64_t n) {
    const int64_t ntiles = ceil_div(n > 0 ? n : 1, kOsTile);
    return (int64_t)align_up((size_t)ntiles * kRadix * 8, 256) + 4096 + 256;
}

tc_status radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int lo_bit, int nbits, Allocator* al,
                         cudaStream_t s, uint64_t** result, DevStatus* err, long long spin_limit,
                         unsigned long long* counts) {
    *result = keys;
    if (n <= 1 || nbits <= 0) return TC_OK;
    if (lo_bit < 0 || lo_bit + nbits > 64) return TC_ERR_INVALID_ARG;
    const int npass = (nbits + 7) / 8;
    const int64_t ntiles = ceil_div(n, kOsTile);
    if (ntiles > 0xFFFFFFFFll) return TC_ERR_UNSUPPORTED;
    TC_CUDA_TRY(cudaFuncSetAttribute(k_os_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOsSmem));
    DevBuf<unsigned long long> own_hist, status;
    DevBuf<unsigned> counters;
    unsigned long long* ghist = counts;
    if (!counts) {
        TC_TRY(own_hist.alloc(al, (size_t)npass * kRadix, s));
        ghist = own_hist.ptr;
    }
    TC_TRY(status.alloc(al, (size_t)ntiles * kRadix, s));
    TC_TRY(counters.alloc(al, (size_t)npass, s));
    TC_CUDA_TRY(cudaMemsetAsync(counters.ptr, 0, sizeof(unsigned) * npass, s));
    if (!counts) {
        TC_CUDA_TRY(cudaMemsetAsync(ghist, 0, sizeof(unsigned long long) * npass * kRadix, s));
        const int64_t hblocks = ntiles < (int64_t)num_sms() * 8 ? ntiles : (int64_t)num_sms() * 8;
        const size_t hsmem = (size_t)kOsWarps * npass * kRadix * sizeof(unsigned);
        TC_CUDA_TRY(cudaFuncSetAttribute(k_os_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem));
        k_os_hist<<<(unsigned)hblocks, kOsBlock, hsmem, s>>>(keys, n, lo_bit, npass, ghist);
        note_launch();
    }
    k_os_bases<<<npass, kRadix, 0, s>>>(ghist);
    note_launch();
    TC_CUDA_TRY(cudaGetLastError());
    uint64_t* a = keys;
    uint64_t* b = tmp;
    for (int p = 0; p < npass; ++p) {
        TC_CUDA_TRY(cudaMemsetAsync(status.ptr, 0, sizeof(unsigned long long) * ntiles * kRadix, s));
        k_os_pass<<<(unsigned)ntiles, kOsBlock, kOsSmem, s>>>(a, b, n, lo_bit + 8 * p, ghist + (int64_t)p * kRadix,
                                                               status.ptr, counters.ptr + p, err, spin_limit);
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

extern "C" tc_status tc_wait_selftest(int64_t spin_limit, tc_stream_t stream) {
    using namespace tcg;
    if (spin_limit < 1) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Allocator al;
    DevBuf<unsigned long long> buf;  // [0]: the flag (never set), [1..]: the status word
    TC_TRY(buf.alloc(&al, 1 + (sizeof(DevStatus) + 7) / 8, s));
    TC_CUDA_TRY(cudaMemsetAsync(buf.ptr, 0, buf.count * 8, s));
    k_wait_selftest<<<1, 1, 0, s>>>(buf.ptr, (long long)spin_limit, (DevStatus*)(buf.ptr + 1));
    note_launch();
    TC_CUDA_TRY(cudaGetLastError());
    DevStatus h;
    TC_CUDA_TRY(cudaMemcpyAsync(&h, buf.ptr + 1, sizeof(h), cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    return (tc_status)h.code;
}

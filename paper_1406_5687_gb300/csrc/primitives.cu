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
// Adinets and Merrill, 2022).  The digit counts of every pass are known before the first
// pass (gathered by the kernel that wrote the keys, or by one counting pass).  Each digit
// pass takes tiles of 8192 keys in the order blocks start (an atomic tile counter), ranks
// the tile's keys stably within each warp (lanes with equal digits found through a shared
// word of peer bits per digit),
// publishes the tile's count of each digit, and obtains the count of each digit in all
// earlier tiles by a decoupled look-back over their published words (flag in the top two
// bits: aggregate of the tile alone, or inclusive prefix; then a 6-bit pass tag, so one
// zeroed status array serves every pass of a sort), then writes every digit run of the tile
// contiguously.  A tile waits only on tiles taken earlier, whose blocks are already running;
// every wait is bounded and sets the error word when it gives up.
//
// The pass is bound by its work inside the SM (ranking, the shared-memory scatter of the
// tile, instruction issue) more than by its 16 bytes of traffic per key, so the work per key
// is kept small: one digit extraction per phase, ranks packed two to a register, full tiles
// without bounds checks, per (warp, digit) one shared word that turns a rank into the key's
// position in the tile, and tiles of 8192 keys, which halve the per-tile work of the digit
// phase and the look-back against 4096.

// Tile shape: 256 threads (one per digit in the per-digit phase), keys per thread, and the
// blocks per SM the register budget is sized for.
#ifndef TC_OS_ITEMS
#define TC_OS_ITEMS 32
#endif
#ifndef TC_OS_MINB
#define TC_OS_MINB 2
#endif
#ifndef TC_OS_RANK
#define TC_OS_RANK 1  // 0: eight ballots per key; 1: shared peer words
#endif
#ifndef TC_OS_SAMECHECK
#define TC_OS_SAMECHECK 0
#endif
constexpr int kOsBlock = 256;
constexpr int kOsWarps = kOsBlock / 32;
constexpr int kOsItems = TC_OS_ITEMS;
static_assert(kOsItems % 2 == 0, "ranks are packed two to a register");
constexpr int kOsTile = kOsBlock * kOsItems;
constexpr int kRadix = 256;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr int kTagShift = 56;
constexpr unsigned long long kCountMask = (1ull << kTagShift) - 1;

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

constexpr int kOsWarpWords = 2 * kRadix + 2;  // per warp: (peer bits, count) of each digit, and a spare pair
constexpr size_t kOsSmem = (size_t)kOsTile * 8 + (size_t)kOsWarps * kOsWarpWords * 4 + (size_t)kRadix * 8 + 64;

// Poll *p until its 6-bit tag (bits 56..61) equals `tag`; give up (return 0) once `spins`,
// shared by the caller's successive waits, exceeds `limit`.  Every device wait of the
// library goes through here.
__device__ __forceinline__ unsigned long long wait_tag(const unsigned long long* p, unsigned tag, long long limit,
                                                       long long& spins) {
    for (;;) {
        const unsigned long long v = *(const volatile unsigned long long*)p;
        if (((unsigned)(v >> kTagShift) & 0x3Fu) == tag) return v;
        if (++spins > limit) return 0;
    }
}

// One thread waits on a flag that nothing sets: the wait must give up after `limit` polls
// and record TC_ERR_TIMEOUT.
__global__ void k_wait_selftest(const unsigned long long* flag, long long limit, DevStatus* err) {
    long long spins = 0;
    if (wait_tag(flag, 1u, limit, spins) == 0) set_error(err, TC_ERR_TIMEOUT, spins);
}

__device__ __forceinline__ uint32_t os_digit(uint64_t k, int shift) { return (uint32_t)(k >> shift) & 0xFFu; }

// One tile of a digit pass.  FULL: the tile holds kOsTile keys (no bounds checks).
template <bool FULL>
__device__ __forceinline__ void os_tile(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int64_t n,
                                        int shift, const unsigned long long* __restrict__ base,
                                        unsigned long long* status, unsigned tag, long long tile, DevStatus* err,
                                        long long spin_limit, const OsOut& po, unsigned char* smem) {
    uint64_t* skeys = (uint64_t*)smem;                           // kOsTile
    uint32_t* wcnt = (uint32_t*)(skeys + kOsTile);               // kOsWarps * kOsWarpWords: counts, then bases
    long long* gofs = (long long*)(wcnt + kOsWarps * kOsWarpWords);  // 256: output index minus tile index
    uint32_t* wsum = (uint32_t*)(gofs + kRadix);                 // kOsWarps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tbase = tile * kOsTile;
    const int tvalid = FULL ? kOsTile : (int)(n - tbase);
    uint32_t* mycnt = wcnt + warp * kOsWarpWords;
    // each warp clears its own words
    for (int i = lane; i < kOsWarpWords / 2; i += 32) reinterpret_cast<uint2*>(mycnt)[i] = make_uint2(0u, 0u);
    // warp-striped load: lane l holds the warp's keys j*32 + l (memory order j-major)
    const int wofs = warp * 32 * kOsItems + lane;
    const uint64_t* src = in + tbase + wofs;
    uint64_t key[kOsItems];
#pragma unroll
    for (int j = 0; j < kOsItems; ++j) key[j] = (FULL || wofs + j * 32 < tvalid) ? src[j * 32] : 0ull;
    __syncwarp();
    // rank within the warp, stably.  The lanes holding the same digit are found either by one
    // ballot per digit bit, or (the default) by each lane setting its bit in a shared word of
    // its digit; a row whose lanes all hold one digit skips both.  The group's highest lane
    // advances the warp's counter of that digit.
    const unsigned lt = lanemask_lt();
    uint32_t rank2[kOsItems / 2];
#pragma unroll
    for (int j = 0; j < kOsItems; ++j) {
        const bool valid = FULL || wofs + j * 32 < tvalid;
        const uint32_t d = os_digit(key[j], shift);
        unsigned peers;
        uint32_t old;
#if TC_OS_RANK == 0
        peers = kFull;
        if (!FULL) {
            const unsigned vmask = __ballot_sync(kFull, valid);
            peers = valid ? vmask : ~vmask;
        }
#pragma unroll
        for (int bt = 0; bt < 8; ++bt) {
            const bool bit = (d >> bt) & 1u;
            const unsigned b = __ballot_sync(kFull, bit);
            peers &= bit ? b : ~b;
        }
        old = mycnt[2 * d + 1];
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) mycnt[2 * d + 1] = old + (uint32_t)__popc(peers);
#else
        // (peer bits, count) of digit d in one 8-byte word; invalid lanes use a word of their own
        const uint32_t slot = valid ? d : (uint32_t)kRadix;
        const bool same = TC_OS_SAMECHECK && __all_sync(kFull, valid && d == __shfl_sync(kFull, d, 0));
        if (same) {
            peers = kFull;
            old = mycnt[2 * d + 1];
        } else {
            atomicOr(&mycnt[2 * slot], 1u << lane);
            __syncwarp();
            const uint2 w = reinterpret_cast<const uint2*>(mycnt)[slot];
            peers = w.x;
            old = w.y;
        }
        __syncwarp();
        if (valid && lane == 31 - __clz(peers))
            reinterpret_cast<uint2*>(mycnt)[slot] = make_uint2(0u, old + (uint32_t)__popc(peers));
#endif
        __syncwarp();
        const uint32_t r = old + (uint32_t)__popc(peers & lt);
        if (j & 1) rank2[j >> 1] |= r << 16;
        else rank2[j >> 1] = r;
    }
    __syncthreads();
    // per digit d (thread d): exclusive scan over the warps, publish the tile's count, scan
    // over the digits, look back for the count in all earlier tiles
    const int d = threadIdx.x;
    const unsigned long long tagbits = (unsigned long long)tag << kTagShift;
    unsigned long long lb = 0;
    if (tile > 0) lb = *(const volatile unsigned long long*)&status[(tile - 1) * kRadix + d];
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kOsWarps; ++w) {
        const uint32_t c = wcnt[w * kOsWarpWords + 2 * d + 1];
        wcnt[w * kOsWarpWords + 2 * d + 1] = tot;
        tot += c;
    }
    unsigned long long* st = status + tile * kRadix;
    *(volatile unsigned long long*)&st[d] = (tile == 0 ? kFlagPrefix : kFlagAgg) | tagbits | tot;
    const uint32_t incl = warp_inclusive_scan(tot, lane);
    if (lane == 31) wsum[warp] = incl;
    unsigned long long excl = 0;
    if (tile != 0) {
        long long j = tile - 1;
        long long spins = 0;
        unsigned long long v = lb;
        for (;;) {
            if (((unsigned)(v >> kTagShift) & 0x3Fu) != tag) v = wait_tag(&status[j * kRadix + d], tag, spin_limit, spins);
            if (v == 0) {
                set_error(err, TC_ERR_TIMEOUT, tile);
                break;
            }
            excl += v & kCountMask;
            if ((v & ~(kCountMask | (0x3Full << kTagShift))) == kFlagPrefix || j == 0) break;
            --j;
            v = *(const volatile unsigned long long*)&status[j * kRadix + d];
        }
        *(volatile unsigned long long*)&st[d] = kFlagPrefix | tagbits | (excl + tot);
    }
    __syncthreads();
    uint32_t dstart = incl - tot;
    for (int w = 0; w < warp; ++w) dstart += wsum[w];
    gofs[d] = (long long)(base[d] + excl) - (long long)dstart;
#pragma unroll
    for (int w = 0; w < kOsWarps; ++w) wcnt[w * kOsWarpWords + 2 * d + 1] += dstart;
    __syncthreads();
    // the tile in digit order in shared memory, then every digit run to its place
#pragma unroll
    for (int j = 0; j < kOsItems; ++j) {
        if (FULL || wofs + j * 32 < tvalid) {
            const uint32_t r = (rank2[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
            skeys[mycnt[2 * os_digit(key[j], shift) + 1] + r] = key[j];
        }
    }
    __syncthreads();
    // consecutive lanes hold consecutive positions of the tile's sorted order
    if (po.mode == OS_OUT_KEYS) {
#pragma unroll
        for (int k = 0; k < kOsItems; ++k) {
            const int i = k * kOsBlock + threadIdx.x;
            if (FULL || i < tvalid) {
                const uint64_t x = skeys[i];
                out[gofs[os_digit(x, shift)] + i] = x;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kOsItems; ++k) {
            const int i = k * kOsBlock + threadIdx.x;
            const bool v = FULL || i < tvalid;
            const uint64_t x = v ? skeys[i] : 0ull;
            if (v) {
                const long long g = gofs[os_digit(x, shift)] + i;
                out[g] = x;
                if (po.mode == OS_OUT_LISTS) po.cols[g] = (int32_t)(x & ((1ull << po.b) - 1ull));
            }
            // runs of one field value are consecutive lanes: the first lane of each adds its length
            const bool counted = v && x != po.skip;
            const uint32_t f = counted ? (uint32_t)((x >> po.fshift) & po.fmask) : 0xFFFFFFFFu;
            const uint32_t prev = __shfl_up_sync(kFull, f, 1);
            const bool edge = lane == 0 || f != prev;
            const unsigned after = __ballot_sync(kFull, edge) & ~lanemask_le();
            const int end = after ? __ffs(after) - 1 : 32;
            if (counted && edge && f < po.nvert) atomicAdd(&po.cnt[f], end - lane);
        }
    }
}

__global__ void __launch_bounds__(kOsBlock, TC_OS_MINB) k_os_pass(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                      int64_t n, int shift, const unsigned long long* __restrict__ base,
                                                      unsigned long long* status, unsigned tag, unsigned* tile_counter,
                                                      DevStatus* err, long long spin_limit, OsOut po) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned s_tile;
    __shared__ int s_skip;
    // once a wait of this sort has given up, later passes leave the keys alone
    if (threadIdx.x == 0) {
        s_skip = *(volatile int*)&err->code != 0;
        s_tile = s_skip ? 0u : atomicAdd(tile_counter, 1u);
    }
    __syncthreads();
    if (s_skip) return;
    const long long tile = (long long)s_tile;
    if ((tile + 1) * kOsTile <= n) os_tile<true>(in, out, n, shift, base, status, tag, tile, err, spin_limit, po, smem_raw);
    else os_tile<false>(in, out, n, shift, base, status, tag, tile, err, spin_limit, po, smem_raw);
}

int64_t radix_sort_scratch_bytes(int64_t n) {
    const int64_t ntiles = ceil_div(n > 0 ? n : 1, kOsTile);
    return (int64_t)align_up((size_t)ntiles * kRadix * 8, 256) + 4096 + 256;
}

tc_status radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int lo_bit, int nbits, Allocator* al,
                         cudaStream_t s, uint64_t** result, DevStatus* err, long long spin_limit,
                         unsigned long long* counts, const OsOut* wout, bool* applied) {
    *result = keys;
    if (applied) *applied = false;
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
    // one zeroed status array for every pass: pass p tags its words with p + 1
    TC_CUDA_TRY(cudaMemsetAsync(status.ptr, 0, sizeof(unsigned long long) * ntiles * kRadix, s));
    for (int p = 0; p < npass; ++p) {
        OsOut po;
        if (wout && p == (wout->pass < 0 ? npass - 1 : wout->pass)) {
            po = *wout;
            if (applied) *applied = true;
        }
        k_os_pass<<<(unsigned)ntiles, kOsBlock, kOsSmem, s>>>(a, b, n, lo_bit + 8 * p, ghist + (int64_t)p * kRadix,
                                                               status.ptr, (unsigned)(p + 1), counters.ptr + p, err,
                                                               spin_limit, po);
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

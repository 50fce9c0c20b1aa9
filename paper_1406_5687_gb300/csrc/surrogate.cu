// surrogate.cu -- the space-efficient count of Sec. IV over a non-overlapping partition
// (Def. 1), for N+ lists that need not fit in device memory.
//
// The vertices are split into P sets of consecutive ids V_j = [cuts[j], cuts[j+1]).  Part j's
// lists (N_u for u in V_j) are one contiguous slice of cols, because the sets are consecutive:
// that slice is the partition G_j.  The parts are taken one after another on this GPU.  Part
// j's slice is copied into a device buffer (the copy of part j+1 overlaps the count of part j);
// every list N_v with an entry in V_j is then a data message to part j, which adds
// SurrogateCount(N_v, j) = sum over u in N_v ∩ V_j of |N_u ∩ N_v| (Sec. IV-C, Fig. 2).  Messages
// are read where they are: device memory, or page-locked host memory over the host link.
//
// Each list goes to a part once (Sec. IV-C's LastProc).  Lists are ascending and the parts
// consecutive, so the entries of N_v in V_j form one run, and the parts are visited in
// increasing order: a per-vertex cursor at the first entry not yet sent replaces LastProc.  The
// routing kernel finds, for every list whose next entry lies in V_j, the end of that run, emits
// work items (v, s, e) of at most kItemU entries, and advances the cursor.
//
// Count kernel.  A warp takes 32 items at a time.  The message list X = N_v of an item is staged
// into an open-addressing hash table in the warp's shared memory (short lists side by side in
// regions of their own, a long list a piece at a time).  The lists N_u of the item's entries u
// (resident, in HBM), trimmed to X's [first, last] range, are streamed through it as 16-byte
// units.  Hits go to a per-block counter of the sender's part i; each block adds its counters to
// table[i][j] once, at its end.
//
// Planning (Sec. IV-B): cuts[k] is the first vertex whose exclusive prefix of a per-vertex cost f
// reaches k / P of the total, so every part gets about 1 / P of it.  With Sec. IV-F's f(u) = sum
// over the lists N_v holding u of (d^_u + d^_v), the work part j does for u, the parts take equal
// work; with f(v) = |N_v| they hold equal shares of the lists (about m / P entries each).
#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "graph.cuh"
#include "scan.cuh"

namespace tcg {
namespace {

constexpr uint32_t kSEmpty = 0xFFFFFFFFu;
constexpr uint32_t kSHashMul = 0x9E3779B1u;   // 2^32 / golden ratio (multiplicative hashing)
#ifndef TC_SURR_UNITS
#define TC_SURR_UNITS 2
#endif
#ifndef TC_SURR_MIN_BLOCKS
#define TC_SURR_MIN_BLOCKS 4
#endif
constexpr int kSWarps = 8;                          // warps per block of the count kernel
constexpr uint32_t kSCap = TC_SURROGATE_PIECE;      // longest message staged whole; longer ones in pieces
constexpr uint32_t kSSlots = 4 * kSCap;             // hash slots of one warp's table (load <= 1/4)
constexpr uint32_t kItemU = 256;              // entries u of one work item
constexpr int kSUnits = TC_SURR_UNITS;        // 16-byte units a lane loads per step
constexpr uint32_t kSTrimMin = 16;            // shorter resident lists are streamed whole
constexpr int kRouteBlock = 256;

// One work item: entries [s, e) of N_v lie in the receiving part; i is v's part.
struct __align__(16) SItem {
    uint32_t v;
    uint32_t i;
    uint32_t s;
    uint32_t e;
};

struct SArgs {
    const int64_t* off;                 // device, n + 1
    const int32_t* msrc;                // every list, device-readable (device or mapped host memory)
    const int32_t* res;                 // part j's lists: res[k] = cols[e0 + k]; 16-byte aligned
    long long e0;                       // first entry held by res (a multiple of 4)
    long long res_len;                  // entries readable from res
    const SItem* items;
    const unsigned long long* n_items;  // items of this part (written by the routing kernel)
    unsigned long long cap;             // capacity of items
    unsigned long long* claim;          // next unclaimed item
    int32_t c_lo, c_hi;                 // V_j
    int32_t nparts, j;
    unsigned long long* table;          // device, nparts * nparts
    unsigned long long* counters;       // device (staged, streamed) entries, or null
    DevStatus* st;
};

__device__ __forceinline__ int s_nth_set_bit(unsigned m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (k >= c) {
            k -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// A table region packed in 32 bits: slot offset in the low 16 bits, log2(slots) above.
__device__ __forceinline__ uint32_t s_region(uint32_t base, uint32_t cap) {
    return base | ((uint32_t)(__ffs(cap) - 1) << 16);
}

struct SView {
    uint32_t* tbl;
    uint32_t mask;
    int shift;
};

__device__ __forceinline__ SView s_view(uint32_t* tbl, uint32_t reg) {
    const uint32_t lg = reg >> 16;
    SView h;
    h.tbl = tbl + (reg & 0xFFFFu);
    h.mask = (1u << lg) - 1u;
    h.shift = 32 - (int)lg;
    return h;
}

// Linear probing from an even slot: the table is read as buckets of two slots, so one 8-byte
// shared load covers the first two probes of a lookup.  A region holds at most a quarter of its
// slots, so the loops end and most lookups end at their first bucket.
__device__ __forceinline__ uint32_t s_start(const SView& h, uint32_t x) {
    return ((x * kSHashMul) >> (h.shift + 1)) << 1;
}

__device__ __forceinline__ void s_insert(const SView& h, uint32_t x) {
    uint32_t p = s_start(h, x);
    while (atomicCAS(&h.tbl[p], kSEmpty, x) != kSEmpty) p = (p + 1u) & h.mask;
}

// The rest of a lookup whose first bucket held two other keys.
__device__ __forceinline__ bool s_find_rest(const SView& h, uint32_t x, uint32_t p) {
    for (;;) {
        const uint32_t y = h.tbl[p];
        if (y == x) return true;
        if (y == kSEmpty) return false;
        p = (p + 1u) & h.mask;
    }
}

// Lookups of the four entries of a unit (those flagged in `ok`), their first buckets loaded
// together; returns the hits.
__device__ __forceinline__ uint32_t s_find4(const SView& h, const uint32_t (&x)[4], const bool (&ok)[4]) {
    uint32_t p[4];
    uint2 b[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) p[t] = s_start(h, x[t]);
#pragma unroll
    for (int t = 0; t < 4; ++t) b[t] = *reinterpret_cast<const uint2*>(h.tbl + p[t]);
    uint32_t hits = 0u;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (!ok[t]) continue;
        if (b[t].x == x[t] || b[t].y == x[t]) ++hits;
        else if (b[t].x != kSEmpty && b[t].y != kSEmpty && s_find_rest(h, x[t], (p[t] + 2u) & h.mask)) ++hits;
    }
    return hits;
}

// Both lists are ascending, so only the entries of the resident list r[ps, ps + len) inside
// [xmin, xmax] (the message's first and last entry) can match: shrink it to that sub-list with
// two binary searches run side by side.
__device__ __forceinline__ void s_trim(const int32_t* __restrict__ r, uint32_t& ps, uint32_t& len, uint32_t xmin,
                                       uint32_t xmax) {
    const uint32_t first = (uint32_t)__ldg(&r[ps]), last = (uint32_t)__ldg(&r[ps + len - 1u]);
    if (first >= xmin && last <= xmax) return;
    if (last < xmin || first > xmax) {
        len = 0u;
        return;
    }
    uint32_t lb = ps, nl = first < xmin ? len : 0u;  // lb: first entry >= xmin
    uint32_t ub = ps + len, nu = last > xmax ? len : 0u;  // ub: first entry > xmax
    if (nu) ub = ps;
    while (nl | nu) {
        if (nl) {
            const uint32_t h = nl >> 1;
            if ((uint32_t)__ldg(&r[lb + h]) < xmin) {
                lb += h + 1u;
                nl -= h + 1u;
            } else {
                nl = h;
            }
        }
        if (nu) {
            const uint32_t h = nu >> 1;
            if ((uint32_t)__ldg(&r[ub + h]) <= xmax) {
                ub += h + 1u;
                nu -= h + 1u;
            } else {
                nu = h;
            }
        }
    }
    ps = lb;
    len = ub > lb ? ub - lb : 0u;
}

// The warp streams the resident lists N_u of up to 32 receiver entries (lane t holds u when
// `valid`), each through the table region `reg` of its message, whose first and last entries
// are xmin and xmax.  The trimmed lists are read as one stream of 16-byte units: list k covers
// the aligned units from res[ps_k & ~3] to its end, the lists' units numbered one after
// another; a unit's list is the last list starting at or before it, found from an OR-reduced
// mask of the list starts in each 32-unit window.  Returns this lane's hits.
__device__ uint32_t s_batch(const SArgs& a, bool valid, uint32_t u, uint32_t reg, uint32_t xmin, uint32_t xmax,
                            uint32_t* __restrict__ tbl, int lane) {
    uint32_t ps = 0u, len = 0u;
    if (valid) {
        const long long ob = a.off[u];
        ps = (uint32_t)(ob - a.e0);
        len = (uint32_t)(a.off[u + 1] - ob);
        if (len >= kSTrimMin) s_trim(a.res, ps, len, xmin, xmax);
    }
    const unsigned act = __ballot_sync(kFull, len != 0u);
    const int na = __popc(act);
    if (na == 0) return 0u;
    {  // the k-th nonempty list into lane k
        const int src = lane < na ? s_nth_set_bit(act, lane) : 0;
        const uint32_t gl = __shfl_sync(kFull, len, src);
        ps = __shfl_sync(kFull, ps, src);
        reg = __shfl_sync(kFull, reg, src);
        len = lane < na ? gl : 0u;
    }
    if (a.counters) {
        const uint32_t tot = warp_sum(len);
        if (lane == 0) atomicAdd(&a.counters[1], (unsigned long long)tot);
    }
    const uint32_t units = len != 0u ? (((ps & 3u) + len + 3u) >> 2) : 0u;
    const uint32_t uincl = warp_inclusive_scan(units, lane);
    const uint32_t ustart = uincl - units;
    const uint32_t U = __shfl_sync(kFull, uincl, 31);
    uint32_t before = 0u, hits = 0u;
    for (uint32_t w0 = 0; w0 < U; w0 += 32u * kSUnits) {
        int4 val[kSUnits];
        uint32_t lo[kSUnits], ln[kSUnits], rg[kSUnits], e0[kSUnits];
        bool in[kSUnits];
#pragma unroll
        for (int k = 0; k < kSUnits; ++k) {
            const uint32_t wb = w0 + 32u * (uint32_t)k;
            const uint32_t rel = ustart - wb;
            const uint32_t bit = (units != 0u && rel < 32u) ? (1u << rel) : 0u;
            const uint32_t starts = __reduce_or_sync(kFull, bit);
            const int q = ((int)(before + __popc(starts & lanemask_le())) - 1) & 31;
            before += __popc(starts);
            lo[k] = __shfl_sync(kFull, ps, q);
            ln[k] = __shfl_sync(kFull, len, q);
            rg[k] = __shfl_sync(kFull, reg, q);
            const uint32_t us = __shfl_sync(kFull, ustart, q);
            const uint32_t unit = wb + (uint32_t)lane;
            in[k] = unit < U;
            e0[k] = (lo[k] & ~3u) + 4u * (unit - us);
            val[k] = make_int4(-1, -1, -1, -1);
            if (in[k]) {
                if ((long long)e0[k] + 4 <= a.res_len) {
                    val[k] = __ldg(reinterpret_cast<const int4*>(a.res + e0[k]));
                } else {  // the last unit of the slice: only its entries inside the slice
                    if ((long long)e0[k] + 0 < a.res_len) val[k].x = __ldg(&a.res[e0[k] + 0]);
                    if ((long long)e0[k] + 1 < a.res_len) val[k].y = __ldg(&a.res[e0[k] + 1]);
                    if ((long long)e0[k] + 2 < a.res_len) val[k].z = __ldg(&a.res[e0[k] + 2]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kSUnits; ++k) {
            if (!in[k]) continue;
            const SView hv = s_view(tbl, rg[k]);
            const uint32_t xs[4] = {(uint32_t)val[k].x, (uint32_t)val[k].y, (uint32_t)val[k].z, (uint32_t)val[k].w};
            bool ok[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) ok[t] = e0[k] + (uint32_t)t - lo[k] < ln[k];
            hits += s_find4(hv, xs, ok);
        }
    }
    return hits;
}

// Stage entries [p0, p0 + cnt) of the flattened message lists into their regions; list q of
// the window (lane q holds it: start xb in msrc, exclusive prefix excl of the staged lengths,
// region reg) covers staged entries [excl_q, excl_q + len_q).  Checks that each list ascends
// strictly (the entry before a staged one is in the lane below, or reloaded by lane 0).
__device__ __forceinline__ void s_stage(const SArgs& a, uint32_t* __restrict__ tbl, long long xb, uint32_t pos0,
                                        uint32_t len, uint32_t excl, uint32_t reg, uint32_t tot, int lane) {
    if (a.counters && lane == 0) atomicAdd(&a.counters[0], (unsigned long long)tot);
    uint32_t before = 0u;
    for (uint32_t base = 0; base < tot; base += 32u) {
        const uint32_t rel = excl - base;
        const uint32_t bit = (len != 0u && rel < 32u) ? (1u << rel) : 0u;
        const uint32_t starts = __reduce_or_sync(kFull, bit);
        const int q = ((int)(before + __popc(starts & lanemask_le())) - 1) & 31;
        before += __popc(starts);
        const long long xq = __shfl_sync(kFull, xb, q);
        const uint32_t pq = __shfl_sync(kFull, pos0, q);
        const uint32_t eq = __shfl_sync(kFull, excl, q);
        const uint32_t rq = __shfl_sync(kFull, reg, q);
        const uint32_t g = base + (uint32_t)lane;
        const bool ok = g < tot;
        const uint32_t k = pq + (g - eq);  // position in the list
        int32_t x = -1;
        if (ok) x = a.msrc[xq + k];
        const int32_t xp = __shfl_up_sync(kFull, x, 1);
        if (ok && k > 0u) {
            const int32_t prev = (lane > 0 && g - eq > 0u) ? xp : a.msrc[xq + k - 1];
            if (x <= prev) set_error(a.st, TC_ERR_INVALID_ARG, xq + k);
        }
        if (ok) {
            if (x >= 0) s_insert(s_view(tbl, rq), (uint32_t)x);
            else set_error(a.st, TC_ERR_VERTEX_RANGE, xq + k);
        }
    }
}

// Receiver entries [r0, r0 + R) flattened over the window's items (lane q holds item q: start
// xb, first entry s, exclusive prefix rexcl of the entry counts, region, range): each batch of
// 32 entries u is checked to lie in V_j and streamed by s_batch.
__device__ __forceinline__ unsigned long long s_receivers(const SArgs& a, uint32_t* __restrict__ tbl, long long xb,
                                                          uint32_t s, uint32_t r, uint32_t rexcl, uint32_t reg,
                                                          uint32_t xmin, uint32_t xmax, uint32_t R, int lane) {
    uint32_t before = 0u;
    unsigned long long acc = 0ull;
    for (uint32_t tb = 0; tb < R; tb += 32u) {
        const uint32_t rel = rexcl - tb;
        const uint32_t bit = (r != 0u && rel < 32u) ? (1u << rel) : 0u;
        const uint32_t starts = __reduce_or_sync(kFull, bit);
        const int q = ((int)(before + __popc(starts & lanemask_le())) - 1) & 31;
        before += __popc(starts);
        const long long xq = __shfl_sync(kFull, xb, q);
        const uint32_t sq = __shfl_sync(kFull, s, q);
        const uint32_t eq = __shfl_sync(kFull, rexcl, q);
        const uint32_t rq = __shfl_sync(kFull, reg, q);
        const uint32_t mn = __shfl_sync(kFull, xmin, q);
        const uint32_t mx = __shfl_sync(kFull, xmax, q);
        const uint32_t g = tb + (uint32_t)lane;
        bool valid = false;
        uint32_t u = 0u;
        if (g < R) {
            const int32_t uu = a.msrc[xq + sq + (g - eq)];
            valid = uu >= a.c_lo && uu < a.c_hi;
            if (!valid) set_error(a.st, TC_ERR_INVALID_ARG, xq + sq + (g - eq));
            u = (uint32_t)uu;
        }
        acc += s_batch(a, valid, u, rq, mn, mx, tbl, lane);
    }
    return acc;
}

// Four blocks of 8 warps per SM (64 registers, 4 KB of table per warp): the kernel is bound by
// its probe stream, and the extra warps hide its latency better than the registers they cost.
__global__ void __launch_bounds__(kSWarps * 32, TC_SURR_MIN_BLOCKS) k_surrogate_count(SArgs a) {
    extern __shared__ uint32_t s_dyn[];
    uint32_t* const tbl = s_dyn + (threadIdx.x >> 5) * kSSlots;
    unsigned long long* const acc = reinterpret_cast<unsigned long long*>(s_dyn + kSWarps * kSSlots);
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < a.nparts; k += blockDim.x) acc[k] = 0ull;
    __syncthreads();
    const unsigned long long N = *a.n_items < a.cap ? *a.n_items : a.cap;
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(a.claim, 32ull);
        b = __shfl_sync(kFull, b, 0);
        if (b >= N) break;
        const int nc = (int)(N - b < 32ull ? N - b : 32ull);
        SItem it = {0u, 0u, 0u, 0u};
        long long xb = 0;
        uint32_t d = 0u;
        if (lane < nc) {
            it = a.items[b + lane];
            xb = a.off[it.v];
            d = (uint32_t)(a.off[it.v + 1] - xb);
        }
        // short messages: windows of items of one sender part whose regions fit the table
        unsigned pending = __ballot_sync(kFull, lane < nc && d <= kSCap);
        while (pending) {
            const uint32_t i0 = __shfl_sync(kFull, it.i, __ffs(pending) - 1);
            const bool cand = ((pending >> lane) & 1u) && it.i == i0;
            uint32_t cap = 0u;
            if (cand) {
                cap = 32u;
                while (cap < 4u * d) cap <<= 1;
            }
            const uint32_t cend = warp_inclusive_scan(cap, lane);
            const unsigned win = __ballot_sync(kFull, cand && cend <= kSSlots);  // never empty
            const uint32_t used = __shfl_sync(kFull, cend, 31 - __clz(win));
            for (uint32_t k = lane; k < used; k += 32u) tbl[k] = kSEmpty;
            __syncwarp();
            const int ng = __popc(win);
            const int src = lane < ng ? s_nth_set_bit(win, lane) : 0;
            const uint32_t my_reg = cand ? s_region(cend - cap, cap) : 0u;
            const long long g_xb = __shfl_sync(kFull, xb, src);
            const uint32_t g_d0 = __shfl_sync(kFull, d, src);
            const uint32_t g_reg = __shfl_sync(kFull, my_reg, src);
            const uint32_t g_s = __shfl_sync(kFull, it.s, src);
            const uint32_t g_e = __shfl_sync(kFull, it.e, src);
            const uint32_t g_d = lane < ng ? g_d0 : 0u;
            const uint32_t incl = warp_inclusive_scan(g_d, lane);
            s_stage(a, tbl, g_xb, 0u, g_d, incl - g_d, g_reg, __shfl_sync(kFull, incl, 31), lane);
            uint32_t xmin = 0u, xmax = 0u;
            if (lane < ng) {
                xmin = (uint32_t)a.msrc[g_xb];
                xmax = (uint32_t)a.msrc[g_xb + g_d - 1];
            }
            __syncwarp();
            const uint32_t r = lane < ng ? g_e - g_s : 0u;
            const uint32_t rincl = warp_inclusive_scan(r, lane);
            unsigned long long wh = s_receivers(a, tbl, g_xb, g_s, r, rincl - r, g_reg, xmin, xmax,
                                                __shfl_sync(kFull, rincl, 31), lane);
            wh = warp_sum(wh);
            if (lane == 0 && wh) atomicAdd(&acc[i0], wh);
            pending &= ~win;
            __syncwarp();
        }
        // long messages: one at a time, staged a piece of kSCap entries at a time
        unsigned bigm = __ballot_sync(kFull, lane < nc && d > kSCap);
        while (bigm) {
            const int f = __ffs(bigm) - 1;
            bigm &= bigm - 1u;
            const long long bxb = __shfl_sync(kFull, xb, f);
            const uint32_t bd = __shfl_sync(kFull, d, f);
            const uint32_t bs = __shfl_sync(kFull, it.s, f);
            const uint32_t be = __shfl_sync(kFull, it.e, f);
            const uint32_t bi = __shfl_sync(kFull, it.i, f);
            const uint32_t reg = s_region(0u, kSSlots);
            unsigned long long wh = 0ull;
            for (uint32_t p0 = 0; p0 < bd; p0 += kSCap) {
                const uint32_t pl = bd - p0 < kSCap ? bd - p0 : kSCap;
                for (uint32_t k = lane; k < kSSlots; k += 32u) tbl[k] = kSEmpty;
                __syncwarp();
                s_stage(a, tbl, bxb, p0, lane == 0 ? pl : 0u, 0u, reg, pl, lane);
                const uint32_t mn = (uint32_t)a.msrc[bxb + p0], mx = (uint32_t)a.msrc[bxb + p0 + pl - 1];
                __syncwarp();
                wh += s_receivers(a, tbl, bxb, bs, lane == 0 ? be - bs : 0u, 0u, reg, mn, mx, be - bs, lane);
                __syncwarp();
            }
            wh = warp_sum(wh);
            if (lane == 0 && wh) atomicAdd(&acc[bi], wh);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < a.nparts; k += blockDim.x)
        if (acc[k]) atomicAdd(&a.table[(size_t)k * a.nparts + a.j], acc[k]);
}

// Sender side for part j (Sec. IV-C): every list whose next unsent entry lies in V_j is sent
// once.  The end e of its run in V_j is found by galloping from the cursor, then a binary
// search; items of at most kItemU entries are appended (one atomic per warp) and the cursor
// moves to e.
__global__ void __launch_bounds__(kRouteBlock) k_surrogate_route(const int64_t* __restrict__ off,
                                                                 const int32_t* __restrict__ msrc, int32_t n,
                                                                 const int32_t* __restrict__ cuts, int32_t nparts,
                                                                 int32_t c_lo, int32_t c_hi, uint32_t* cur,
                                                                 int32_t* nx, SItem* items,
                                                                 unsigned long long* n_items,
                                                                 unsigned long long cap,
                                                                 unsigned long long* items_total, DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
        const long long v = base + threadIdx.x;
        bool act = false;
        uint32_t c = 0u, e = 0u, d = 0u, ip = 0u;
        long long b = 0;
        if (v < n) {
            const int32_t x = nx[v];
            if (x < c_hi) {
                if (x < c_lo) {
                    set_error(st, x < 0 ? TC_ERR_VERTEX_RANGE : TC_ERR_INVALID_ARG, v);  // not ascending
                } else {
                    act = true;
                    b = off[v];
                    d = (uint32_t)(off[v + 1] - b);
                    c = cur[v];
                    if (msrc[b + d - 1] < c_hi) {
                        e = d;
                    } else {
                        uint32_t lo = c, hi = d - 1u, step = 1u;  // msrc[b + lo] < c_hi <= msrc[b + hi]
                        for (;;) {
                            const uint32_t p = lo + step;
                            if (p >= hi) break;
                            if (msrc[b + p] >= c_hi) {
                                hi = p;
                                break;
                            }
                            lo = p;
                            step <<= 1;
                        }
                        uint32_t l = lo + 1u, h = hi;
                        while (l < h) {
                            const uint32_t mid = l + ((h - l) >> 1);
                            if (msrc[b + mid] >= c_hi) h = mid; else l = mid + 1u;
                        }
                        e = l;
                    }
                    int klo = 0, khi = nparts - 1;  // v's part: the last k with cuts[k] <= v
                    while (klo < khi) {
                        const int mid = (klo + khi + 1) >> 1;
                        if (cuts[mid] <= v) klo = mid; else khi = mid - 1;
                    }
                    ip = (uint32_t)klo;
                }
            }
        }
        const uint32_t nit = act ? (e - c + kItemU - 1u) / kItemU : 0u;
        const uint32_t incl = warp_inclusive_scan(nit, lane);
        const uint32_t tot = __shfl_sync(kFull, incl, 31);
        unsigned long long wb = 0;
        if (lane == 31 && tot) {
            wb = atomicAdd(n_items, (unsigned long long)tot);
            if (items_total) atomicAdd(items_total, (unsigned long long)tot);
        }
        wb = __shfl_sync(kFull, wb, 31);
        if (tot && wb + tot > cap) {
            if (lane == 0) set_error(st, TC_ERR_INVALID_ARG, -1);
            continue;
        }
        if (act) {
            unsigned long long o = wb + (incl - nit);
            for (uint32_t s = c; s < e; s += kItemU, ++o) {
                SItem itm;
                itm.v = (uint32_t)v;
                itm.i = ip;
                itm.s = s;
                itm.e = e - s > kItemU ? s + kItemU : e;
                items[o] = itm;
            }
            cur[v] = e;
            nx[v] = e < d ? msrc[b + e] : INT_MAX;
        }
    }
}

// Cursor of every list at its first entry >= c_first (the first part counted), and that entry.
__global__ void k_surrogate_init(const int64_t* __restrict__ off, const int32_t* __restrict__ msrc, int32_t n,
                                 int32_t c_first, uint32_t* cur, int32_t* nx) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const long long b = off[v];
        const uint32_t d = (uint32_t)(off[v + 1] - b);
        uint32_t l = 0u;
        if (c_first > 0) {
            uint32_t h = d;
            while (l < h) {
                const uint32_t mid = l + ((h - l) >> 1);
                if (msrc[b + mid] >= c_first) h = mid; else l = mid + 1u;
            }
        }
        cur[v] = l;
        nx[v] = l < d ? msrc[b + l] : INT_MAX;
    }
}

// off[0] = 0, off non-decreasing, off[n] = m: every list position then lies in [0, m).
__global__ void k_surrogate_check_off(const int64_t* __restrict__ off, int32_t n, long long m, DevStatus* st) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += (long long)gridDim.x * blockDim.x) {
        const long long o = off[v];
        if ((v == 0 && o != 0) || (v == n && o != m) || (v < n && off[v + 1] < o)) set_error(st, TC_ERR_INVALID_ARG, v);
    }
}

// After the last part every entry of every list has been sent; one left over is >= n.
__global__ void k_surrogate_done(const int32_t* __restrict__ nx, int32_t n, DevStatus* st) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        if (nx[v] != INT_MAX) set_error(st, TC_ERR_VERTEX_RANGE, v);
}

__global__ void k_surrogate_cut_offsets(const int64_t* __restrict__ off, const int32_t* __restrict__ cuts, int32_t P,
                                        int64_t* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= P) out[k] = off[cuts[k]];
}

// Per-vertex costs for the cuts: f(v) = 1 (TC_FN_ONE), |N_v| (TC_FN_LIST) or the list part of
// d_v (TC_FN_DEGREE, completed by k_surrogate_cost); 0 for the sums over entries.
__global__ void k_surrogate_cost_init(const int64_t* __restrict__ off, int32_t n, int fn, unsigned long long* f) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        f[v] = fn == TC_FN_ONE ? 1ull
                               : (fn == TC_FN_LIST || fn == TC_FN_DEGREE) ? (unsigned long long)(off[v + 1] - off[v])
                                                                          : 0ull;
}

// Sums over the entries u of every list N_w: d_u = |N_u| + #{w : u in N_w} (TC_FN_DEGREE, Sec.
// V-A); PATRIC's f(w) = sum over u in N_w of (d^_w + d^_u) (Sec. IV-B); the new f(u) = sum over
// the w with u in N_w of (d^_u + d^_w) (Sec. IV-F).  A warp takes 32 consecutive lists, whose
// entries are one contiguous range of cols; an entry's list is found by a binary search over the
// lanes' list starts.
__global__ void k_surrogate_cost(const int64_t* __restrict__ off, const int32_t* __restrict__ msrc, int32_t n, int fn,
                                 unsigned long long* f, DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)n + 31) / 32;
    const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nw; w += wstride) {
        const long long w0 = w * 32;
        const long long os = off[w0 + lane < n ? w0 + lane : n];
        const long long oe = off[w0 + 32 < n ? w0 + 32 : n];
        const long long o0 = __shfl_sync(kFull, os, 0);
        for (long long p0 = o0; p0 < oe; p0 += 32) {
            const long long p = p0 + lane;
            int lo = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const long long t = __shfl_sync(kFull, os, lo + step);
                if (t <= p) lo += step;
            }
            if (p < oe) {
                const long long w1 = w0 + lo;
                const long long dw = off[w1 + 1] - off[w1];
                const int32_t u = msrc[p];
                if (u < 0 || u >= n) {
                    set_error(st, TC_ERR_VERTEX_RANGE, p);
                } else if (fn == TC_FN_DEGREE) {
                    atomicAdd(&f[u], 1ull);
                } else {
                    const unsigned long long c = (unsigned long long)(off[u + 1] - off[u] + dw);
                    atomicAdd(&f[fn == TC_FN_PATRIC ? w1 : u], c);
                }
            }
        }
    }
}

struct CostAt {
    const unsigned long long* f;
    __device__ uint64_t operator()(int64_t i) const { return f[i]; }
};

// cuts[k] = the first q in [0, n] with F[q] >= ceil(k F[n] / P); cuts[0] = 0, cuts[P] = n.
__global__ void k_surrogate_cuts(const uint64_t* __restrict__ F, int32_t n, int32_t P, int32_t* cuts) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > P) return;
    if (k == 0 || k == P) {
        cuts[k] = k == 0 ? 0 : n;
        return;
    }
    const unsigned __int128 num = (unsigned __int128)F[n] * (unsigned)k;
    const uint64_t t = (uint64_t)((num + (unsigned)P - 1) / (unsigned)P);
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (F[mid] >= t) hi = mid; else lo = mid + 1;
    }
    cuts[k] = lo;
}

__global__ void k_surrogate_part_sizes(const int64_t* __restrict__ off, const int32_t* __restrict__ cuts, int32_t P,
                                       unsigned long long* max_entries) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) atomicMax(max_entries, (unsigned long long)(off[cuts[k + 1]] - off[cuts[k]]));
}

// Small device block of one call: error word and counters.
struct SDev {
    DevStatus status;
    unsigned long long n_items;
    unsigned long long claim;
    unsigned long long max_entries;
    unsigned long long counters[3];  // staged, streamed, items (with stats)
};

// Pageable host lists are page-locked for the duration of a call.  Calls may overlap (several
// threads, the same lists), so the library's registrations are counted: a call inside a range
// that another call registered takes a reference, the last call to finish unregisters, and no
// call releases memory another still reads.  A range that only partly overlaps a registered one
// is refused.
std::mutex g_reg_mu;
struct RegEntry {
    size_t bytes;
    int refs;
};
std::map<uintptr_t, RegEntry>& registrations() {
    static std::map<uintptr_t, RegEntry> m;
    return m;
}

// Page-lock [p, p + bytes) or take a reference on a registration covering it; *key receives the
// registration to release (0: none needed, the caller's memory was already page-locked).
tc_status acquire_host(const void* p, size_t bytes, uintptr_t* key) {
    *key = 0;
    const uintptr_t a = (uintptr_t)p, b = a + bytes;
    std::lock_guard<std::mutex> lk(g_reg_mu);
    auto& m = registrations();
    auto it = m.upper_bound(a);  // first registration starting after a
    if (it != m.begin()) {
        auto pr = std::prev(it);
        const uintptr_t e = pr->first + pr->second.bytes;
        if (e > a) {
            if (b > e) return TC_ERR_INVALID_ARG;  // runs past the registered range
            ++pr->second.refs;
            *key = pr->first;
            return TC_OK;
        }
    }
    if (it != m.end() && it->first < b) return TC_ERR_INVALID_ARG;  // a registered range starts inside
    if (pinned_device_view(p)) return TC_OK;  // page-locked by the caller
    cudaError_t err = cudaHostRegister(const_cast<void*>(p), bytes, cudaHostRegisterPortable | cudaHostRegisterMapped);
    if (err != cudaSuccess) {
        (void)cudaGetLastError();
        return err == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA;
    }
    m[a] = RegEntry{bytes, 1};
    *key = a;
    return TC_OK;
}

void release_host(uintptr_t key) {
    if (!key) return;
    std::lock_guard<std::mutex> lk(g_reg_mu);
    auto& m = registrations();
    auto it = m.find(key);
    if (it == m.end()) return;
    if (--it->second.refs == 0) {
        cudaHostUnregister((void*)key);
        m.erase(it);
    }
}

// Device-readable views of the caller's lists for one call.
struct Lists {
    const int64_t* off_host = nullptr;  // non-null when off is host memory
    const int32_t* msrc = nullptr;      // device-readable cols
    bool cols_device = false;
    uintptr_t registered = 0;  // registration this call holds (release_host)
    ~Lists() { release_host(registered); }
};

// Declared after a Lists, so that no kernel still reads the lists when they are released.
struct SyncOnExit {
    cudaStream_t s;
    ~SyncOnExit() { cudaStreamSynchronize(s); }
};

tc_status device_cols(const int32_t* cols, int64_t m, Lists* L) {
    if (m == 0) return TC_OK;
    if (is_device_pointer(cols)) {
        L->msrc = cols;
        L->cols_device = true;
        return TC_OK;
    }
    TC_TRY(acquire_host(cols, (size_t)m * 4, &L->registered));
    const void* pin = pinned_device_view(cols);
    if (!pin) return TC_ERR_CUDA;
    L->msrc = (const int32_t*)pin;
    return TC_OK;
}

// off as a device array (copied when it is host memory), checked by k_surrogate_check_off.
tc_status device_offsets(const int64_t* off, int32_t n, int64_t m, Allocator* al, cudaStream_t s,
                         DevBuf<int64_t>* buf, const int64_t** off_d, Lists* L, DevStatus* st) {
    if (is_device_pointer(off)) {
        *off_d = off;
    } else {
        L->off_host = off;
        TC_TRY(buf->alloc(al, (size_t)n + 1, s));
        TC_CUDA_TRY(cudaMemcpyAsync(buf->ptr, off, ((size_t)n + 1) * 8, cudaMemcpyDefault, s));
        *off_d = buf->ptr;
    }
    const int grid = (int)std::min<int64_t>(ceil_div((int64_t)n + 1, 256), (int64_t)num_sms() * 8);
    k_surrogate_check_off<<<grid, 256, 0, s>>>(*off_d, n, (long long)m, st);
    note_launch();
    return TC_OK;
}

tc_status read_sdev(SDev* dev, cudaStream_t s, SDev* host) {
    TC_CUDA_TRY(cudaMemcpyAsync(host, dev, sizeof(SDev), cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    return host->status.code ? (tc_status)host->status.code : TC_OK;
}

tc_status check_cuts(const int32_t* cuts, int32_t nparts, int32_t n) {
    if (!cuts || nparts < 1 || nparts > TC_SURROGATE_MAX_PARTS) return TC_ERR_INVALID_ARG;
    if (cuts[0] != 0 || cuts[nparts] != n) return TC_ERR_INVALID_ARG;
    for (int32_t k = 0; k < nparts; ++k)
        if (cuts[k] > cuts[k + 1]) return TC_ERR_INVALID_ARG;
    return TC_OK;
}

struct StreamEvents {
    cudaStream_t cs = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr};
    cudaEvent_t counted[2] = {nullptr, nullptr};
    tc_status create() {
        TC_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            TC_CUDA_TRY(cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming));
            TC_CUDA_TRY(cudaEventCreateWithFlags(&counted[b], cudaEventDisableTiming));
        }
        return TC_OK;
    }
    ~StreamEvents() {
        if (cs) cudaStreamSynchronize(cs);
        for (int b = 0; b < 2; ++b) {
            if (copied[b]) cudaEventDestroy(copied[b]);
            if (counted[b]) cudaEventDestroy(counted[b]);
        }
        if (cs) cudaStreamDestroy(cs);
    }
};

// CUDA events around every routing and count kernel of a call (stats only).
struct KernelTimes {
    std::vector<cudaEvent_t> ev;
    ~KernelTimes() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    tc_status mark(cudaStream_t s) {
        cudaEvent_t e;
        TC_CUDA_TRY(cudaEventCreate(&e));
        ev.push_back(e);
        TC_CUDA_TRY(cudaEventRecord(e, s));
        return TC_OK;
    }
    // events are recorded as (route start, count start, count end) per part
    void sum(float* route, float* count) const {
        *route = *count = 0.f;
        for (size_t k = 0; k + 2 < ev.size(); k += 3) {
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, ev[k], ev[k + 1]);
            cudaEventElapsedTime(&b, ev[k + 1], ev[k + 2]);
            *route += a;
            *count += b;
        }
    }
};

tc_status surrogate_count(const int64_t* off, const int32_t* cols, int32_t n, int64_t m, const int32_t* cuts,
                          int32_t P, int32_t lo, int32_t hi, const tc_options& o, cudaStream_t s,
                          std::vector<unsigned long long>* table, tc_surrogate_stats* stats) {
    Allocator al;
    al.alloc = o.alloc;
    al.release = o.release;
    al.ctx = o.alloc_ctx;
    al.budget = o.hbm_budget_bytes;
    retain_pool_memory();
    DevBuf<SDev> dev;
    TC_TRY(dev.alloc(&al, 1, s));
    TC_CUDA_TRY(cudaMemsetAsync(dev.ptr, 0, sizeof(SDev), s));
    DevStatus* st = &dev.ptr->status;
    Lists L;
    SyncOnExit sync_guard{s};
    DevBuf<int64_t> offbuf;
    const int64_t* off_d = nullptr;
    TC_TRY(device_offsets(off, n, m, &al, s, &offbuf, &off_d, &L, st));
    SDev h;
    TC_TRY(read_sdev(dev.ptr, s, &h));  // the offsets are valid before any list is read
    // each part's first entry and slice (host values)
    std::vector<int64_t> oc((size_t)P + 1);
    if (L.off_host) {
        for (int32_t k = 0; k <= P; ++k) oc[k] = L.off_host[cuts[k]];
    } else {
        DevBuf<int32_t> cd;
        DevBuf<int64_t> od;
        TC_TRY(cd.alloc(&al, (size_t)P + 1, s));
        TC_TRY(od.alloc(&al, (size_t)P + 1, s));
        TC_CUDA_TRY(cudaMemcpyAsync(cd.ptr, cuts, ((size_t)P + 1) * 4, cudaMemcpyHostToDevice, s));
        k_surrogate_cut_offsets<<<(P + 256) / 256, 256, 0, s>>>(off_d, cd.ptr, P, od.ptr);
        note_launch();
        TC_CUDA_TRY(cudaMemcpyAsync(oc.data(), od.ptr, ((size_t)P + 1) * 8, cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    table->assign((size_t)P * P, 0ull);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (m == 0 || lo == hi) return TC_OK;
    TC_TRY(device_cols(cols, m, &L));
    const bool direct = L.cols_device && ((uintptr_t)cols & 15u) == 0;
    int64_t max_len = 0;
    for (int32_t j = lo; j < hi; ++j) {
        const int64_t len = oc[j + 1] - (oc[j] & ~(int64_t)3);
        if (len > ((int64_t)1 << 32) - 8) return TC_ERR_UNSUPPORTED;
        max_len = std::max(max_len, len);
    }
    DevBuf<int32_t> cuts_d;
    TC_TRY(cuts_d.alloc(&al, (size_t)P + 1, s));
    TC_CUDA_TRY(cudaMemcpyAsync(cuts_d.ptr, cuts, ((size_t)P + 1) * 4, cudaMemcpyHostToDevice, s));
    DevBuf<uint32_t> cur;
    DevBuf<int32_t> nx;
    DevBuf<SItem> items;
    DevBuf<unsigned long long> tab;
    DevBuf<int32_t> res[2];
    const unsigned long long cap = (unsigned long long)n + (unsigned long long)m / kItemU + 1ull;
    TC_TRY(cur.alloc(&al, (size_t)std::max(n, 1), s));
    TC_TRY(nx.alloc(&al, (size_t)std::max(n, 1), s));
    TC_TRY(items.alloc(&al, (size_t)cap, s));
    TC_TRY(tab.alloc(&al, (size_t)P * P, s));
    TC_CUDA_TRY(cudaMemsetAsync(tab.ptr, 0, (size_t)P * P * 8, s));
    if (!direct) {
        for (int b = 0; b < (hi - lo > 1 ? 2 : 1); ++b) TC_TRY(res[b].alloc(&al, (size_t)max_len + 4, s));
    }
    const int sms = num_sms();
    const int ngrid = (int)std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), kRouteBlock), (int64_t)sms * 8);
    k_surrogate_init<<<ngrid, kRouteBlock, 0, s>>>(off_d, L.msrc, n, cuts[lo], cur.ptr, nx.ptr);
    note_launch();

    const size_t smem = (size_t)kSWarps * kSSlots * 4 + (size_t)P * 8;
    TC_CUDA_TRY(cudaFuncSetAttribute(k_surrogate_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_surrogate_count, kSWarps * 32, smem));
    const int cgrid = sms * std::max(per_sm, 1);

    StreamEvents ev;
    KernelTimes kt;
    int64_t copied = 0;
    auto copy_part = [&](int32_t j) -> tc_status {
        const int b = (j - lo) & 1;
        const int64_t e0 = oc[j] & ~(int64_t)3, len = oc[j + 1] - e0;
        if (j - lo >= 2) TC_CUDA_TRY(cudaStreamWaitEvent(ev.cs, ev.counted[b], 0));
        if (len > 0)
            TC_CUDA_TRY(cudaMemcpyAsync(res[b].ptr, cols + e0, (size_t)len * 4, cudaMemcpyDefault, ev.cs));
        copied += 4 * std::max<int64_t>(len, 0);
        TC_CUDA_TRY(cudaEventRecord(ev.copied[b], ev.cs));
        return TC_OK;
    };
    if (!direct) {
        TC_TRY(ev.create());
        TC_CUDA_TRY(cudaEventRecord(ev.counted[0], s));  // the copy stream starts after the set-up above
        TC_CUDA_TRY(cudaStreamWaitEvent(ev.cs, ev.counted[0], 0));
        TC_TRY(copy_part(lo));
    }
    for (int32_t j = lo; j < hi; ++j) {
        const int b = (j - lo) & 1;
        const int64_t e0 = oc[j] & ~(int64_t)3;
        SArgs a;
        a.off = off_d;
        a.msrc = L.msrc;
        a.e0 = e0;
        a.res_len = oc[j + 1] - e0;
        if (direct) {
            a.res = cols + e0;
        } else {
            TC_CUDA_TRY(cudaStreamWaitEvent(s, ev.copied[b], 0));
            a.res = res[b].ptr;
        }
        a.items = items.ptr;
        a.n_items = &dev.ptr->n_items;
        a.cap = cap;
        a.claim = &dev.ptr->claim;
        a.c_lo = cuts[j];
        a.c_hi = cuts[j + 1];
        a.nparts = P;
        a.j = j;
        a.table = tab.ptr;
        a.counters = stats ? dev.ptr->counters : nullptr;
        a.st = st;
        TC_CUDA_TRY(cudaMemsetAsync(&dev.ptr->n_items, 0, 2 * sizeof(unsigned long long), s));
        if (stats) TC_TRY(kt.mark(s));
        k_surrogate_route<<<ngrid, kRouteBlock, 0, s>>>(off_d, L.msrc, n, cuts_d.ptr, P, a.c_lo, a.c_hi, cur.ptr,
                                                       nx.ptr, items.ptr, &dev.ptr->n_items, cap,
                                                       stats ? &dev.ptr->counters[2] : nullptr, st);
        if (stats) TC_TRY(kt.mark(s));
        k_surrogate_count<<<cgrid, kSWarps * 32, smem, s>>>(a);
        if (stats) TC_TRY(kt.mark(s));
        note_launch(2);
        TC_CUDA_TRY(cudaGetLastError());
        if (!direct) {
            TC_CUDA_TRY(cudaEventRecord(ev.counted[b], s));
            if (j + 1 < hi) TC_TRY(copy_part(j + 1));
        }
    }
    if (hi == P) {
        k_surrogate_done<<<ngrid, kRouteBlock, 0, s>>>(nx.ptr, n, st);
        note_launch();
    }
    TC_CUDA_TRY(cudaMemcpyAsync(table->data(), tab.ptr, (size_t)P * P * 8, cudaMemcpyDeviceToHost, s));
    const tc_status r = read_sdev(dev.ptr, s, &h);
    if (stats) {
        stats->staged = (int64_t)h.counters[0];
        stats->streamed = (int64_t)h.counters[1];
        stats->items = (int64_t)h.counters[2];
        stats->copied_bytes = copied;
        kt.sum(&stats->route_ms, &stats->count_ms);
    }
    return r;
}

tc_status surrogate_plan(const int64_t* off, const int32_t* cols, int32_t n, int64_t m, int fn, int32_t nparts,
                         int64_t part_bytes, int32_t max_parts, cudaStream_t s, int32_t* cuts, int32_t* nparts_out) {
    Allocator al;
    retain_pool_memory();
    DevBuf<SDev> dev;
    TC_TRY(dev.alloc(&al, 1, s));
    TC_CUDA_TRY(cudaMemsetAsync(dev.ptr, 0, sizeof(SDev), s));
    DevStatus* st = &dev.ptr->status;
    Lists L;
    SyncOnExit sync_guard{s};
    DevBuf<int64_t> offbuf;
    const int64_t* off_d = nullptr;
    TC_TRY(device_offsets(off, n, m, &al, s, &offbuf, &off_d, &L, st));
    SDev h;
    TC_TRY(read_sdev(dev.ptr, s, &h));
    const bool entries = fn == TC_FN_DEGREE || fn == TC_FN_PATRIC || fn == TC_FN_NEW;
    if (entries) TC_TRY(device_cols(cols, m, &L));
    DevBuf<unsigned long long> f;
    DevBuf<uint64_t> F, scr;
    DevBuf<int32_t> cd;
    TC_TRY(f.alloc(&al, (size_t)std::max(n, 1), s));
    TC_TRY(F.alloc(&al, (size_t)n + 1, s));
    TC_TRY(scr.alloc(&al, (size_t)scan_scratch_words(n), s));
    if (n > 0) {
        const int grid = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8);
        k_surrogate_cost_init<<<grid, 256, 0, s>>>(off_d, n, fn, f.ptr);
        note_launch();
    }
    if (entries && m > 0) {
        const int grid = (int)std::min<int64_t>(ceil_div(ceil_div(n, 32), 8), (int64_t)num_sms() * 16);
        k_surrogate_cost<<<grid, 256, 0, s>>>(off_d, L.msrc, n, fn, f.ptr, st);
        note_launch();
    }
    TC_CUDA_TRY(scan_exclusive(CostAt{f.ptr}, n, F.ptr, scr.ptr, s));
    const int32_t pmax = nparts > 0 ? nparts : max_parts;
    TC_TRY(cd.alloc(&al, (size_t)pmax + 1, s));
    TC_TRY(read_sdev(dev.ptr, s, &h));
    // the smallest part count whose cost-balanced cuts keep every part's lists within part_bytes
    int32_t P = nparts > 0 ? nparts : (int32_t)std::max<int64_t>(1, std::min<int64_t>(ceil_div(4 * m, part_bytes), pmax));
    for (;; ++P) {
        TC_CUDA_TRY(cudaMemsetAsync(&dev.ptr->max_entries, 0, 8, s));
        k_surrogate_cuts<<<(P + 256) / 256, 256, 0, s>>>(F.ptr, n, P, cd.ptr);
        k_surrogate_part_sizes<<<(P + 255) / 256, 256, 0, s>>>(off_d, cd.ptr, P, &dev.ptr->max_entries);
        note_launch(2);
        TC_CUDA_TRY(cudaMemcpyAsync(cuts, cd.ptr, ((size_t)P + 1) * 4, cudaMemcpyDeviceToHost, s));
        TC_TRY(read_sdev(dev.ptr, s, &h));
        const bool fits = part_bytes <= 0 || (int64_t)h.max_entries * 4 <= part_bytes;
        if (fits) {
            *nparts_out = P;
            return TC_OK;
        }
        if (nparts > 0 || P >= pmax) {
            *nparts_out = P;
            return TC_ERR_BUDGET;
        }
    }
}

}  // namespace
}  // namespace tcg

using namespace tcg;

extern "C" {

tc_status tc_surrogate_plan(const int64_t* off, const int32_t* cols, int32_t n, int64_t m, int32_t fn,
                            int32_t nparts, int64_t part_bytes, int32_t max_parts, tc_stream_t stream, int32_t* cuts,
                            int32_t* nparts_out) {
    if (!off || !cuts || !nparts_out || n < 0 || m < 0 || (m > 0 && !cols)) return TC_ERR_INVALID_ARG;
    if (fn < TC_FN_ONE || fn > TC_FN_LIST) return TC_ERR_INVALID_ARG;
    if (n == INT32_MAX) return TC_ERR_UNSUPPORTED;
    if (nparts < 0 || nparts > TC_SURROGATE_MAX_PARTS || part_bytes < 0) return TC_ERR_INVALID_ARG;
    if (nparts == 0 && (part_bytes == 0 || max_parts < 1 || max_parts > TC_SURROGATE_MAX_PARTS))
        return TC_ERR_INVALID_ARG;
    *nparts_out = 0;
    tc_status r = surrogate_plan(off, cols, n, m, fn, nparts, part_bytes, max_parts, (cudaStream_t)stream, cuts,
                                 nparts_out);
    if (r != TC_OK) (void)cudaGetLastError();
    return r;
}

tc_status tc_surrogate_plan_both(const int64_t* off, const int32_t* cols, int32_t n, int64_t m, int32_t fn,
                                 int32_t work_parts, int64_t part_bytes, int32_t max_parts, tc_stream_t stream,
                                 int32_t* cuts, int32_t* nparts_out) {
    if (!off || !cuts || !nparts_out || n < 0 || m < 0 || (m > 0 && !cols)) return TC_ERR_INVALID_ARG;
    if (fn < TC_FN_ONE || fn > TC_FN_LIST) return TC_ERR_INVALID_ARG;
    if (n == INT32_MAX) return TC_ERR_UNSUPPORTED;
    if (work_parts < 1 || work_parts > TC_SURROGATE_MAX_PARTS || part_bytes <= 0 || max_parts < 1 ||
        max_parts > TC_SURROGATE_MAX_PARTS)
        return TC_ERR_INVALID_ARG;
    *nparts_out = 0;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> cw((size_t)work_parts + 1), cb((size_t)max_parts + 1);
    int32_t pw = 0, pb = 0;
    tc_status r = surrogate_plan(off, cols, n, m, fn, work_parts, 0, work_parts, s, cw.data(), &pw);
    if (r == TC_OK) r = surrogate_plan(off, cols, n, m, TC_FN_LIST, 0, part_bytes, max_parts, s, cb.data(), &pb);
    if (r != TC_OK) {
        (void)cudaGetLastError();
        return r;
    }
    // the union of both cut sets: every part lies inside one part of each
    std::vector<int32_t> u;
    u.reserve((size_t)pw + pb + 2);
    size_t i = 0, j = 0;
    while (i <= (size_t)pw || j <= (size_t)pb) {
        int32_t x;
        if (j > (size_t)pb || (i <= (size_t)pw && cw[i] <= cb[j])) x = cw[i++];
        else x = cb[j++];
        if (u.empty() || x != u.back()) u.push_back(x);
    }
    if (u.size() == 1) u.push_back(u[0]);  // n = 0: one empty part
    if ((int64_t)u.size() - 1 > TC_SURROGATE_MAX_PARTS) return TC_ERR_BUDGET;
    std::memcpy(cuts, u.data(), u.size() * sizeof(int32_t));
    *nparts_out = (int32_t)u.size() - 1;
    return TC_OK;
}

tc_status tc_count_surrogate(const int64_t* off, const int32_t* cols, int32_t n, int64_t m, const int32_t* cuts,
                             int32_t nparts, int32_t part_lo, int32_t part_hi, const tc_options* opt,
                             tc_stream_t stream, uint64_t* table, uint64_t* total, tc_surrogate_stats* stats) {
    if (!off || !total || n < 0 || m < 0 || (m > 0 && !cols)) return TC_ERR_INVALID_ARG;
    if (n == INT32_MAX) return TC_ERR_UNSUPPORTED;
    TC_TRY(check_cuts(cuts, nparts, n));
    if (part_lo < 0 || part_lo > part_hi || part_hi > nparts) return TC_ERR_INVALID_ARG;
    tc_options o;
    tc_options_default(&o);
    if (opt) o = *opt;
    TC_TRY(check_options(o));
    std::vector<unsigned long long> tab;
    tc_status r = surrogate_count(off, cols, n, m, cuts, nparts, part_lo, part_hi, o, (cudaStream_t)stream, &tab,
                                  stats);
    if (r != TC_OK) {
        (void)cudaGetLastError();
        return r;
    }
    uint64_t t = 0;
    for (unsigned long long x : tab) t += x;
    if (table) std::memcpy(table, tab.data(), tab.size() * 8);
    *total = t;
    return TC_OK;
}

}  // extern "C"

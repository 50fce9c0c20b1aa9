// count.cu -- steps a6-a8: task costs and their prefix, the Eq. 1 / Eq. 2 schedule, the
// persistent intersection kernels and the exact reduction.
//
// Work unit.  Fig. 1 sums |N_v ∩ N_u| over oriented edges (v,u).  Each oriented edge is one
// task owned by the endpoint whose list is longer; the owner's list is staged into an
// open-addressing hash table in shared memory (load at most 1/8, so a lookup almost
// always ends at its first or second slot) and the partner lists of the owner's tasks are
// streamed through it.  Each edge thus costs min(|N_v|, |N_u|) streamed entries instead of
// the |N_v| + |N_u| of a merge (Sec. III-A).
//
// Two task classes, two kernels.  Owners with at most small_max entries: each warp takes
// windows of up to 32 consecutive tasks and stages the lists of all the window's owners
// at once, each in its own region of the warp's table.  Longer owners: a block stages a
// window of consecutive owners into regions of one shared table and its warps pull
// batches of 32 of the window's tasks from a block counter.
// Inside a batch, the partner lists are read as one stream of 16-byte units spread over the
// lanes (warp_batch_count); a big owner's partner lists are first trimmed to the part inside
// the owner list's [first, last] range, the only part that can match.
//
// Schedule (Sec. V-B), per class.  The persistent grid has W workers, one per block (the
// warps of a block share its chunk).  Task costs are prefix-summed (uint64).  The first
// H = floor(C * static_percent / 100) cost units (Eq. 1, default one half) are split into W
// equal initial chunks, one per worker, taken without coordination; the rest is handed out
// by a compare-and-swap on a device head, each pop taking max(min_chunk,
// floor((C - head) / W)) (Eq. 2), so chunks shrink as the work drains.  A cost boundary maps
// to the first task whose exclusive prefix reaches it.
//
// Reduction.  Each warp sums its hits in registers, then one uint64 atomicAdd per warp:
// exact and independent of order.
#include <mutex>

#include "graph.cuh"
#include "scan.cuh"

namespace tcg {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kHashMul = 0x9E3779B1u;  // Knuth's multiplicative constant, 2^32 / golden ratio
#ifndef TC_UNITS
#define TC_UNITS 4
#endif
constexpr int kStageItems = 4;  // list entries a thread loads before inserting them (staging)
constexpr int kUnits = TC_UNITS;  // 16-byte units of partner lists a lane loads per step of warp_batch_count
#ifndef TC_UNITS_X
#define TC_UNITS_X 3
#endif
constexpr int kUnitsX = TC_UNITS_X;  // the same for per-vertex / per-edge counts, whose per-hit path needs more registers
#ifndef TC_UNITS_XS
#define TC_UNITS_XS 2
#endif
constexpr int kUnitsXS = TC_UNITS_XS;  // ... in the small-owner kernel (3 and 2: no register spills)
#ifndef TC_COUNT_MINB
#define TC_COUNT_MINB 2
#endif
constexpr int kCountMinBlocks = TC_COUNT_MINB;  // resident 512-thread blocks per SM the count kernels' registers allow

struct CountArgs {
    const int64_t* off;
    const int32_t* cols;
    const TaskRec* tasks;
    long long t_begin, t_end;  // this class's tasks
    const int32_t* deg;
    const uint64_t* P;   // exclusive prefix of all task costs (T + 1)
    Sched* sched;        // this class's schedule
    Sched* trace_sched;  // holds the shared trace record counter
    long long W;
    int cls;
    int piece;
    int table_slots;
    int warps_per_block;
    unsigned long long* total;
    unsigned long long* t_v;
    uint32_t* per_edge;
    uint64_t* trace_chunks;
    long long trace_cap;
    uint64_t* trace_busy;
    long long busy_offset;
    DevStatus* status;
    long long retry_limit;
    const uint32_t* own_first;  // big class: first task of each owner, then T
    long long n_owners;         // big class: owners
    const int64_t* gtask;       // packs: this class's first task of each graph, then its end
    unsigned long long* streamed;  // traced counts only: partner entries read, summed per class
    int cnt_off;                   // per-vertex counts: words from a table slot to its hit count (0: none)
    int hits_off;                  // per-vertex / per-edge counts: the warps' task-hit counters, in words
    long long n_sub;            // packs: graphs (0: one graph, one total)
    // multi-pack counts (a batch's packs in one launch): the packs, and per class each pack's
    // first task in the class's concatenated order (then the end) and the class cost before it
    // (then the total)
    const PackDev* packs;
    int n_packs;
    const long long* tbase;
    const unsigned long long* cbase;
};

// First index q in [lo, hi] with pred(q), for pred false..false true..true and pred(hi) true.
// Each round every lane tests one sample and the warp keeps the gap between the last false
// and the first true sample, so a range of R shrinks to R/32.
template <class Pred>
__device__ __forceinline__ long long warp_first_true(long long lo, long long hi, Pred pred, int lane) {
    while (hi - lo > 31) {
        const long long step = (hi - lo + 31) / 32;
        long long q = lo + (long long)lane * step;
        if (q > hi) q = hi;
        const unsigned b = __ballot_sync(kFull, pred(q));
        if (b == 0) {
            const long long q31 = lo + 31 * step;
            lo = (q31 > hi ? hi : q31) + 1;
        } else {
            const int f = __ffs(b) - 1;
            if (f == 0) return lo;
            const long long qf = lo + (long long)f * step;
            hi = qf > hi ? hi : qf;
            lo = lo + (long long)(f - 1) * step + 1;
        }
    }
    const long long q = lo + lane;
    const unsigned b = __ballot_sync(kFull, q <= hi ? pred(q) : true);
    return lo + (__ffs(b) - 1);
}

// Cost boundary x (class-local) -> task index: the first task of the class whose exclusive
// prefix reaches x; x >= C maps to the end of the class.
__device__ __forceinline__ long long class_bound(const CountArgs& a, unsigned long long x, unsigned long long C,
                                                 unsigned long long base, int lane) {
    if (x >= C && a.sched->at_end) return a.t_end;
    const uint64_t* __restrict__ P = a.P;
    const unsigned long long target = x + base;
    return warp_first_true(a.t_begin, a.t_end, [&](long long q) { return P[q] >= target; }, lane);
}

// Multi-pack counts: cost boundary x of the class (counted over the packs one after another)
// -> the first task, in the class's concatenated order, whose exclusive prefix reaches x.
__device__ __forceinline__ long long class_bound_multi(const CountArgs& a, unsigned long long x, unsigned long long C,
                                                       int lane) {
    const int np = a.n_packs;
    if (x >= C) return a.tbase[np];
    // the pack holding cost x: the first whose end lies beyond x
    const unsigned long long* __restrict__ cb = a.cbase;
    const long long p = warp_first_true(0, np - 1, [&](long long q) { return cb[q + 1] > x; }, lane);
    const PackDev& pk = a.packs[p];
    const long long lb = a.cls == 0 ? 0 : pk.Ts, ub = a.cls == 0 ? pk.Ts : pk.T;
    const uint64_t* __restrict__ P = pk.P;
    const unsigned long long target = P[lb] + (x - cb[p]);
    const long long j = warp_first_true(lb, ub, [&](long long q) { return P[q] >= target; }, lane);
    return a.tbase[p] + (j - lb);
}

// Multi-pack counts: call fn(b, l0, l1) for every pack piece of the class's tasks [g0, g1)
// (concatenated order), b the arguments of that pack and [l0, l1) its local tasks.  Every
// thread of the block calls this.  Warp 0 prepares each piece in shared memory (the pack's
// arguments in one copy the block shares, the piece's bounds, where the next piece starts),
// so that no loop state stays live in registers while the block counts a piece.
template <class Fn>
__device__ __forceinline__ void for_pack_pieces(const CountArgs& a, long long g0, long long g1, int lane, Fn fn) {
    __shared__ CountArgs s_b;
    __shared__ long long s_piece[3];  // local first and end task, then where the next piece starts
    if (threadIdx.x == 0) s_piece[2] = g0;
    __syncthreads();
    for (;;) {
        if (threadIdx.x < 32) {
            const long long g = s_piece[2];
            long long e = g;
            if (g < g1) {
                // the pack of g: the first whose end lies beyond g (packs without tasks skipped)
                const long long* __restrict__ tb = a.tbase;
                const int np = a.n_packs;
                const long long p = warp_first_true(0, np - 1, [&](long long q) { return tb[q + 1] > g; }, lane);
                e = tb[p + 1] < g1 ? tb[p + 1] : g1;
                if (lane == 0) {
                    const PackDev& pk = a.packs[p];
                    s_b = a;
                    s_b.off = pk.off;
                    s_b.cols = pk.cols;
                    s_b.tasks = pk.tasks;
                    s_b.deg = pk.deg;
                    s_b.P = pk.P;
                    s_b.own_first = pk.own_first;
                    s_b.n_owners = pk.n_owners;
                    s_b.n_sub = pk.n_sub;
                    s_b.gtask = pk.sub_task + (a.cls == 0 ? 0 : pk.n_sub + 1);
                    s_b.total = pk.total;
                    s_b.t_begin = a.cls == 0 ? 0 : pk.Ts;
                    s_b.t_end = a.cls == 0 ? pk.Ts : pk.T;
                    s_piece[0] = s_b.t_begin + (g - tb[p]);
                    s_piece[1] = s_b.t_begin + (e - tb[p]);
                }
            }
            if (lane == 0) s_piece[2] = e == g ? g1 : e;  // nothing left (g >= g1): stop
            if (lane == 0 && e == g) s_piece[0] = s_piece[1] = 0;
        }
        __syncthreads();
        // read before the barrier below: warp 0 rewrites the piece words after it
        const long long l0 = s_piece[0], l1 = s_piece[1];
        const bool last = s_piece[2] >= g1;
        if (l1 > l0) fn(s_b, l0, l1);
        __syncthreads();  // every thread is done with this piece's arguments
        if (last) break;
    }
}

// Position of u in the sorted list N+(v).
__device__ __forceinline__ long long edge_position(const CountArgs& a, uint32_t v, uint32_t u) {
    long long lo = a.off[v], hi = a.off[v + 1];
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if ((uint32_t)a.cols[mid] < u) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The block's dynamic shared memory: hash tables, then (per-vertex counts) the tables' slot
// counts, then (per-vertex / per-edge counts) the warps' task-hit counters.
extern __shared__ uint32_t smem_dyn[];

// Per-vertex and per-edge outputs.  A triangle found at task (owner, partner) with third vertex
// w adds 1 to T_owner, T_partner and T_w (Theorem 1's attribution) and 1 to its oriented edge.
// Every w is an entry of the owner's staged list, so its hits are counted at w's own table slot
// (a count array beside the table, one shared atomic per hit) and added to T_w once per staged
// list.  A task's hits are summed in the warp's shared counter of that task and added to its
// owner, its partner and its edge once per batch.
// Position of x in the sorted list cols[p, p + len), or -1.
__device__ __forceinline__ long long list_position(const int32_t* __restrict__ cols, uint32_t p, uint32_t len,
                                                   uint32_t x) {
    uint32_t lo = p, hi = p + len;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if ((uint32_t)__ldg(&cols[mid]) < x) lo = mid + 1; else hi = mid;
    }
    return (lo < p + len && (uint32_t)__ldg(&cols[lo]) == x) ? (long long)lo : -1ll;
}

__device__ __forceinline__ uint32_t* warp_task_hits(const CountArgs& a) {
    return smem_dyn + a.hits_off + 32 * (threadIdx.x >> 5);
}

struct HashView {
    uint32_t* tbl;
    uint32_t cmask;
    int shift;
};

// Table of `cap` slots (a power of two) for a list of at most cap / 8 entries.
__device__ __forceinline__ HashView make_view(uint32_t* tbl, uint32_t cap) {
    HashView hv;
    hv.tbl = tbl;
    hv.cmask = cap - 1;
    hv.shift = 33 - __ffs(cap);  // 32 - log2(cap)
    return hv;
}

// Linear probing that starts at an even slot: the table is read as buckets of two slots,
// so one 8-byte shared load covers the first two probes of a lookup.
__device__ __forceinline__ uint32_t hash_start(const HashView& hv, uint32_t x) {
    return ((x * kHashMul) >> (hv.shift + 1)) << 1;
}

__device__ __forceinline__ void hash_insert(const HashView& hv, uint32_t x) {
    uint32_t h = hash_start(hv, x);
    while (atomicCAS(&hv.tbl[h], kEmpty, x) != kEmpty) h = (h + 1) & hv.cmask;
}

// Continue a lookup of w from slot h (the first bucket was full of other keys).
__device__ __noinline__ bool hash_probe_rest(const HashView& hv, uint32_t w, uint32_t h) {
    for (;;) {
        const uint32_t s = hv.tbl[h];
        if (s == w) return true;
        if (s == kEmpty) return false;
        h = (h + 1) & hv.cmask;
    }
}

__device__ __forceinline__ bool hash_probe(const HashView& hv, uint32_t w) {
    const uint32_t h = hash_start(hv, w);
    const uint2 b = *reinterpret_cast<const uint2*>(hv.tbl + h);
    if (b.x == w || b.y == w) return true;
    if (b.x == kEmpty || b.y == kEmpty) return false;
    return hash_probe_rest(hv, w, (h + 2) & hv.cmask);
}

// Slot of w in the table, or -1.
__device__ __noinline__ int hash_find_rest(const HashView& hv, uint32_t w, uint32_t h) {
    for (;;) {
        const uint32_t s = hv.tbl[h];
        if (s == w) return (int)h;
        if (s == kEmpty) return -1;
        h = (h + 1) & hv.cmask;
    }
}

__device__ __forceinline__ int hash_find(const HashView& hv, uint32_t w) {
    const uint32_t h = hash_start(hv, w);
    const uint2 b = *reinterpret_cast<const uint2*>(hv.tbl + h);
    if (b.x == w) return (int)h;
    if (b.y == w) return (int)h + 1;
    if (b.x == kEmpty || b.y == kEmpty) return -1;
    return hash_find_rest(hv, w, (h + 2) & hv.cmask);
}

// Add the hit counts of a staged list's entries to T_v (one atomic per entry that was hit)
// and clear them; entries [e0, ol) step `step` of the list at cols[ob].
__device__ __forceinline__ void flush_slot_hits(const CountArgs& a, const HashView& hv, long long ob, uint32_t ol,
                                                uint32_t e0, uint32_t step) {
    for (uint32_t e = e0; e < ol; e += step) {
        const uint32_t x = (uint32_t)__ldg(&a.cols[ob + e]);
        const int sl = hash_find(hv, x);
        if (sl < 0) continue;
        uint32_t* c = hv.tbl + a.cnt_off + sl;
        if (*c) {
            atomicAdd(&a.t_v[x], (unsigned long long)*c);
            *c = 0u;
        }
    }
}

// First-bucket lookups of N entries issued together.  Returns the hits; entries whose
// bucket held two other keys are flagged in `more` (bit k) for hash_probe_rest.
template <int N>
__device__ __forceinline__ uint32_t probe_batch(const HashView& hv, const uint32_t (&w)[N], const bool (&valid)[N],
                                                uint32_t& more) {
    uint32_t h[N];
    uint2 b[N];
#pragma unroll
    for (int k = 0; k < N; ++k) h[k] = hash_start(hv, w[k]);
#pragma unroll
    for (int k = 0; k < N; ++k) b[k] = *reinterpret_cast<const uint2*>(hv.tbl + h[k]);
    uint32_t hits = 0;
    more = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const bool hit = b[k].x == w[k] || b[k].y == w[k];
        const bool end = b[k].x == kEmpty || b[k].y == kEmpty;
        hits += (valid[k] && hit) ? 1u : 0u;
        more |= (valid[k] && !hit && !end) ? (1u << k) : 0u;
    }
    return hits;
}

// First-bucket lookups of N entries issued together, returning each entry's slot (-1: absent);
// entries whose bucket held two other keys are flagged in `more` for hash_find_rest.
template <int N>
__device__ __forceinline__ void find_batch(const HashView& hv, const uint32_t (&w)[N], const bool (&valid)[N],
                                           int (&slot)[N], uint32_t& more) {
    uint32_t h[N];
    uint2 b[N];
#pragma unroll
    for (int k = 0; k < N; ++k) h[k] = hash_start(hv, w[k]);
#pragma unroll
    for (int k = 0; k < N; ++k) b[k] = *reinterpret_cast<const uint2*>(hv.tbl + h[k]);
    more = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        slot[k] = !valid[k] ? -1 : b[k].x == w[k] ? (int)h[k] : b[k].y == w[k] ? (int)h[k] + 1 : -1;
        const bool end = b[k].x == kEmpty || b[k].y == kEmpty;
        more |= (valid[k] && slot[k] < 0 && !end) ? (1u << k) : 0u;
    }
}

// Bit position of the set bit of m that has exactly k set bits below it (0 <= k < popc(m)):
// halve the window five times, skipping the low half when the target is above it.
__device__ __forceinline__ int nth_set_bit(unsigned m, int k) {
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
__device__ __forceinline__ uint32_t pack_region(uint32_t base, uint32_t cap) {
    return base | ((uint32_t)(__ffs(cap) - 1) << 16);
}

__device__ __forceinline__ HashView region_view(uint32_t* tbl, uint32_t reg) {
    const uint32_t lg = reg >> 16;
    HashView hv;
    hv.tbl = tbl + (reg & 0xFFFFu);
    hv.cmask = (1u << lg) - 1u;
    hv.shift = 32 - (int)lg;
    return hv;
}

// Both lists are ascending, so only the partner entries within [omin, omax] (the owner
// list's first and last entry) can be in the owner's list: shrink the partner list
// cols[ps, ps + len) to that sub-list.  The two bounds are found by binary searches run
// side by side; lists already inside the range (the usual case) cost two loads.  Lists
// shorter than kTrimMin are left whole.
#ifndef TC_TRIM_MIN
#define TC_TRIM_MIN TC_TRIM_MIN_ENTRIES
#endif
constexpr uint32_t kTrimMin = TC_TRIM_MIN;  // shorter partner lists are read whole: a search would cost about as much

__device__ __forceinline__ void trim_to_range(const int32_t* __restrict__ cols, uint32_t& ps, uint32_t& len,
                                              uint32_t omin, uint32_t omax) {
    if (len < kTrimMin) return;
    const uint32_t first = (uint32_t)__ldg(&cols[ps]), last = (uint32_t)__ldg(&cols[ps + len - 1u]);
    if (first >= omin && last <= omax) return;
    if (last < omin || first > omax) {
        len = 0u;
        return;
    }
    // lb: first entry >= omin; ub: first entry > omax
    uint32_t lb = ps, nl = first < omin ? len : 0u;
    uint32_t ub = ps + len, nu = last > omax ? len : 0u;
    if (nu) ub = ps;
    while (nl | nu) {
        if (nl) {
            const uint32_t h = nl >> 1;
            if ((uint32_t)__ldg(&cols[lb + h]) < omin) {
                lb += h + 1u;
                nl -= h + 1u;
            } else {
                nl = h;
            }
        }
        if (nu) {
            const uint32_t h = nu >> 1;
            if ((uint32_t)__ldg(&cols[ub + h]) <= omax) {
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

// One warp counts a batch of nb <= 32 tasks (lane i holds task i's record and, in
// `reg`, the table region of that task's owner) against the staged owner lists.  With
// TRIM (big owners), each partner list is first trimmed to its owner's range [omin, omax];
// lists left empty drop out and the others are gathered into the low lanes.  Lists of
// small owners are short and seldom trimmed, so they are read whole.
//
// The partner lists are read as one stream of 16-byte units: list j covers the aligned
// units from cols[pstart_j & ~3] to its end, and the lists' units are numbered one after
// another.  Each step a lane takes four units, 32 apart; the list of its unit is the last
// list that starts at or before it, found from a bit mask of the lists starting in the
// 32-unit window (one OR-reduction) and a population count.  Entries of a unit outside its
// list (before pstart, after the end) are masked.
template <bool EXTRA, bool TRIM>
__device__ __forceinline__ void warp_batch_count(const CountArgs& a, const TaskRec& rin, int nb, uint32_t* __restrict__ tbl,
                                                 uint32_t reg_in, uint32_t omin, uint32_t omax, int lane, uint32_t& cnt) {
    uint32_t ps = rin.pstart, len = lane < nb ? rin.plen : 0u;
    if (TRIM) trim_to_range(a.cols, ps, len, omin, omax);
    // the k-th nonempty list in lane k (untrimmed lists are never empty)
    const unsigned act = __ballot_sync(kFull, len != 0u);
    const int na = __popc(act);
    TaskRec r = rin;
    uint32_t reg = reg_in;
    uint32_t p0 = rin.pstart;  // per-edge counts: the untrimmed partner list is cols[p0, p0 + r.plen)
    if (TRIM && act != (na == 32 ? kFull : (1u << na) - 1u)) {
        const int src = lane < na ? nth_set_bit(act, lane) : 0;
        const uint32_t gl = __shfl_sync(kFull, len, src);
        ps = __shfl_sync(kFull, ps, src);
        reg = __shfl_sync(kFull, reg_in, src);
        if (EXTRA) {
            r.owner = __shfl_sync(kFull, rin.owner, src);
            r.partner = __shfl_sync(kFull, rin.partner, src);
            r.plen = __shfl_sync(kFull, rin.plen, src);
            p0 = __shfl_sync(kFull, rin.pstart, src);
        }
        len = lane < na ? gl : 0u;
    }
    r.pstart = ps;
    if (a.streamed) {
        const uint32_t tot = warp_sum(len);
        if (lane == 0 && tot) atomicAdd(a.streamed, (unsigned long long)tot);
    }
    uint32_t* thits = EXTRA ? warp_task_hits(a) : nullptr;
    // per-vertex / per-edge: this lane's hits of its current list, added to the list's task counter
    // when the lane moves on (a lane's units come in increasing order, so its lists do too)
    int cur_q = 0;
    uint32_t cur_h = 0;
    const uint32_t units = len != 0u ? (((ps & 3u) + len + 3u) >> 2) : 0u;
    const uint32_t uincl = warp_inclusive_scan(units, lane);
    const uint32_t ustart = uincl - units;
    const uint32_t U = __shfl_sync(kFull, uincl, 31);
    uint32_t before = 0;  // lists that start before the current window
    constexpr int NU = EXTRA ? (TRIM ? kUnitsX : kUnitsXS) : kUnits;
    for (uint32_t w0 = 0; w0 < U; w0 += 32u * NU) {
        int4 v[NU];
        uint32_t lo[NU], ln[NU], e0[NU], rg[NU];
        int qk[NU];
        bool in[NU];
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const uint32_t wb = w0 + 32u * (uint32_t)u;
            const uint32_t rel = ustart - wb;
            const uint32_t bit = (units != 0u && rel < 32u) ? (1u << rel) : 0u;
            const uint32_t starts = __reduce_or_sync(kFull, bit);
            const int q = ((int)(before + __popc(starts & lanemask_le())) - 1) & 31;
            before += __popc(starts);
            lo[u] = __shfl_sync(kFull, r.pstart, q);
            ln[u] = __shfl_sync(kFull, len, q);
            rg[u] = __shfl_sync(kFull, reg, q);
            const uint32_t us = __shfl_sync(kFull, ustart, q);
            const uint32_t unit = wb + (uint32_t)lane;
            in[u] = unit < U;
            if (EXTRA) qk[u] = q;
            e0[u] = (lo[u] & ~3u) + 4u * (unit - us);
            v[u] = in[u] ? __ldg(reinterpret_cast<const int4*>(a.cols + e0[u])) : make_int4(-1, -1, -1, -1);
        }
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            if (w0 + 32u * (uint32_t)u >= U) break;
            const HashView hv = region_view(tbl, rg[u]);
            const uint32_t xs[4] = {(uint32_t)v[u].x, (uint32_t)v[u].y, (uint32_t)v[u].z, (uint32_t)v[u].w};
            bool ok[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) ok[k] = in[u] && e0[u] + (uint32_t)k - lo[u] < ln[u];
            if (!EXTRA) {
                uint32_t more;
                cnt += probe_batch<4>(hv, xs, ok, more);
                // entries whose first bucket held two other keys (rare); every index is static so
                // that the four entries stay in registers
                if (more) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if ((more >> k) & 1u) cnt += hash_probe_rest(hv, xs[k], (hash_start(hv, xs[k]) + 2) & hv.cmask) ? 1u : 0u;
                }
            } else {
                // per-vertex / per-edge: each hit counted at its slot, the unit's hits at its task
                int sl[4];
                uint32_t more;
                find_batch<4>(hv, xs, ok, sl, more);
                if (more) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if ((more >> k) & 1u) sl[k] = hash_find_rest(hv, xs[k], (hash_start(hv, xs[k]) + 2) & hv.cmask);
                }
                uint32_t h = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (sl[k] >= 0) {
                        ++h;
                        if (a.cnt_off) atomicAdd(hv.tbl + a.cnt_off + sl[k], 1u);
                    }
                }
                cnt += h;
                if (qk[u] != cur_q) {
                    if (cur_h) atomicAdd(&thits[cur_q], cur_h);
                    cur_q = qk[u];
                    cur_h = 0;
                }
                cur_h += h;
            }
        }
    }
    if (EXTRA) {
        if (cur_h) atomicAdd(&thits[cur_q], cur_h);
        // each task's hits to its owner, its partner and its oriented edge, once per batch
        __syncwarp();
        const uint32_t th = lane < na ? thits[lane] : 0u;
        if (lane < na) thits[lane] = 0u;
        __syncwarp();
        if (th) {
            if (a.t_v) {
                atomicAdd(&a.t_v[r.owner], (unsigned long long)th);
                atomicAdd(&a.t_v[r.partner], (unsigned long long)th);
            }
            if (a.per_edge) {
                // the oriented edge is partner -> owner when the owner is in the partner's list
                // (found in the list this task streamed), else owner -> partner
                long long pos = list_position(a.cols, p0, r.plen, r.owner);
                if (pos < 0) pos = edge_position(a, r.owner, r.partner);
                atomicAdd(&a.per_edge[pos], th);
            }
        }
    }
}

template <bool EXTRA, bool TRIM>
__device__ void warp_batch(const CountArgs& a, const TaskRec& r, int nb, uint32_t* __restrict__ tbl, uint32_t reg,
                           uint32_t omin, uint32_t omax, int lane, unsigned long long& acc) {
    uint32_t cnt = 0;  // this lane's hits in the batch (fits 32 bits: at most 32 lists of < 2^17 entries)
    warp_batch_count<EXTRA, TRIM>(a, r, nb, tbl, reg, omin, omax, lane, cnt);
    acc += cnt;
}

// Eq. 2: take the next chunk of the class's remaining cost (one thread; bounded retries).
__device__ __forceinline__ int pop_chunk(const CountArgs& a, unsigned long long C, unsigned long long minc,
                                         unsigned long long& c, unsigned long long& e) {
    const unsigned long long W = (unsigned long long)a.W;
    c = *(volatile unsigned long long*)&a.sched->head;
    for (long long tries = 0;; ++tries) {
        if (c >= C) return 0;
        unsigned long long sz = (C - c) / W;
        if (sz < minc) sz = minc;
        e = (C - c > sz) ? c + sz : C;
        const unsigned long long old = atomicCAS(&a.sched->head, c, e);
        if (old == c) return 1;
        c = old;
        if (tries >= a.retry_limit) {
            set_error(a.status, TC_ERR_TIMEOUT, tries);
            return 0;
        }
    }
}

__device__ __forceinline__ void trace_chunk(const CountArgs& a, unsigned long long lo, unsigned long long hi,
                                            long long t0, long long t1) {
    if (!a.trace_chunks) return;
    const unsigned long long idx = atomicAdd(&a.trace_sched->n_chunks, 1ull);
    if ((long long)idx < a.trace_cap) {
        a.trace_chunks[4 * idx] = ((uint64_t)a.cls << 56) | lo;
        a.trace_chunks[4 * idx + 1] = hi;
        a.trace_chunks[4 * idx + 2] = (uint64_t)t0;
        a.trace_chunks[4 * idx + 3] = (uint64_t)t1;
    }
}

// ------------------------------------------------------------------ small owners: one warp each

// A warp takes windows of up to 32 consecutive tasks.  The distinct owners of a window get
// separate regions of the warp's table (each sized for a load of at most 1/8); their lists
// are staged together, then all the window's tasks are counted.  One chain of dependent
// loads per window instead of one per owner.
template <bool EXTRA>
__device__ void process_small(const CountArgs& a, long long t0, long long t1, uint32_t* __restrict__ tbl, int lane,
                              unsigned long long& acc) {
    const uint32_t slots = (uint32_t)a.table_slots;
    long long t = t0;
    while (t < t1) {
        const long long j = t + lane;
        const bool in = j < t1;
        TaskRec r = {0u, 0u, 0u, 0u};
        if (in) r = a.tasks[j];
        const uint32_t prev = __shfl_up_sync(kFull, r.owner, 1);
        const bool lead = in && (lane == 0 || r.owner != prev);  // first task of an owner in the window
        long long ob = 0;
        uint32_t ol = 0, cap = 0;
        if (lead) {
            ob = a.off[r.owner];
            ol = (uint32_t)(a.off[r.owner + 1] - ob);
            cap = 32;
            while (cap < 8 * ol) cap <<= 1;
        }
        const uint32_t cend = warp_inclusive_scan(cap, lane);  // end of each leader's region
        const unsigned lead_m = __ballot_sync(kFull, lead);
        const unsigned fit_m = __ballot_sync(kFull, lead && cend <= slots);
        // the window stops before the first owner whose region does not fit (lane 0's always does)
        const unsigned over = lead_m & ~fit_m;
        const int nt = over ? (__ffs(over) - 1) : __popc(__ballot_sync(kFull, in));
        const unsigned kept = fit_m & (nt >= 32 ? kFull : ((1u << nt) - 1u));
        // each task's region is its leader's
        const int leader = 31 - __clz(lead_m & lanemask_le());
        const uint32_t my_reg = lead ? pack_region(cend - cap, cap) : 0u;
        const uint32_t reg = __shfl_sync(kFull, my_reg, leader);
        const uint32_t used = __shfl_sync(kFull, cend, 31 - __clz(kept));
        for (uint32_t i = lane; i < used; i += 32) tbl[i] = kEmpty;
        __syncwarp();
        // stage: gather the kept leaders into lanes 0..ng-1, spread their lists over the lanes
        const int ng = __popc(kept);
        const int src = lane < ng ? nth_set_bit(kept, lane) : 0;
        const long long s_ob = __shfl_sync(kFull, ob, src);
        const uint32_t s_len0 = __shfl_sync(kFull, ol, src);
        const uint32_t s_reg = __shfl_sync(kFull, my_reg, src);
        const uint32_t s_len = lane < ng ? s_len0 : 0u;
        const uint32_t incl = warp_inclusive_scan(s_len, lane);
        const uint32_t excl = incl - s_len;
        const uint32_t tot = __shfl_sync(kFull, incl, 31);
        uint32_t before = 0;
        for (uint32_t base0 = 0; base0 < tot; base0 += 32u * kStageItems) {
            // each lane's entries of kStageItems rows loaded before any is inserted
            uint32_t xs[kStageItems], rqs[kStageItems];
#pragma unroll
            for (int k = 0; k < kStageItems; ++k) {
                const uint32_t base = base0 + 32u * (uint32_t)k;
                const uint32_t rel = excl - base;
                const uint32_t bit = (s_len != 0u && rel < 32u) ? (1u << rel) : 0u;
                const uint32_t starts = __reduce_or_sync(kFull, bit);
                const int q = ((int)(before + __popc(starts & lanemask_le())) - 1) & 31;
                const long long obq = __shfl_sync(kFull, s_ob, q);
                const uint32_t eq = __shfl_sync(kFull, excl, q);
                rqs[k] = __shfl_sync(kFull, s_reg, q);
                const uint32_t g = base + lane;
                xs[k] = g < tot ? (uint32_t)__ldg(&a.cols[obq + (g - eq)]) : 0u;
                before += __popc(starts);
            }
#pragma unroll
            for (int k = 0; k < kStageItems; ++k)
                if (base0 + 32u * (uint32_t)k + lane < tot) hash_insert(region_view(tbl, rqs[k]), xs[k]);
        }
        __syncwarp();
        warp_batch<EXTRA, false>(a, r, nt, tbl, reg, 0u, 0xFFFFFFFFu, lane, acc);
        __syncwarp();
        if (EXTRA && a.cnt_off) {
            // the staged entries' hit counts to T_v, spread over the lanes as when they were staged
            before = 0;
            for (uint32_t base = 0; base < tot; base += 32u) {
                const uint32_t rel = excl - base;
                const uint32_t bit = (s_len != 0u && rel < 32u) ? (1u << rel) : 0u;
                const uint32_t starts = __reduce_or_sync(kFull, bit);
                const int q = ((int)(before + __popc(starts & lanemask_le())) - 1) & 31;
                const long long obq = __shfl_sync(kFull, s_ob, q);
                const uint32_t eq = __shfl_sync(kFull, excl, q);
                const uint32_t rq = __shfl_sync(kFull, s_reg, q);
                const uint32_t g = base + lane;
                if (g < tot) flush_slot_hits(a, region_view(tbl, rq), obq + (g - eq), 1u, 0u, 1u);
                before += __popc(starts);
            }
            __syncwarp();
        }
        t += nt;
    }
}

// The warps of a block pull 32-task slices of the block's chunk [t0, t1) from a shared
// counter and count each slice with process_small.
template <bool EXTRA>
__device__ void process_small_block(const CountArgs& a, long long t0, long long t1, uint32_t* __restrict__ tbl,
                                    unsigned* s_claim, int lane, unsigned long long& acc) {
    if (threadIdx.x == 0) *s_claim = 0u;
    __syncthreads();
    for (;;) {
        unsigned o = 0;
        if (lane == 0) o = atomicAdd(s_claim, 32u);
        o = __shfl_sync(kFull, o, 0);
        const long long t = t0 + (long long)o;
        if (t >= t1) break;
        process_small<EXTRA>(a, t, t + 32 < t1 ? t + 32 : t1, tbl, lane, acc);
    }
    __syncthreads();
}

// ------------------------------------------------------------------ big owners: one block each

constexpr int kWinOwners = 32;

// A window of consecutive big owners staged together into regions of the block's table.
struct BigWindow {
    long long first[kWinOwners + 1];  // owner i's tasks of the window: [first[i], first[i + 1])
    long long ob[kWinOwners];         // owner i's list: cols[ob[i], ob[i] + ol[i])
    uint32_t ol[kWinOwners];
    uint32_t reg[kWinOwners];         // owner i's table region
    uint32_t lmin[kWinOwners];        // owner i's first and last list entry
    uint32_t lmax[kWinOwners];
    uint32_t epre[kWinOwners + 1];    // list entries of the owners before owner i (then the total)
    long long k;                      // owner index of the window's first owner
    uint32_t used;                    // table slots in use
    int nown;                         // owners in the window; 0: one owner needs several pieces
};

// A warp's next batch of 32 tasks of the block's task range [t, tend) (s_next: tasks claimed
// so far).  Returns the batch's size (0: the range is done).  (Smaller batches near the end of
// the range, to even out the warps' arrival at the barrier after it, measured slower: a batch
// has a fixed cost of record loads, trims and scans.)
__device__ __forceinline__ int claim_batch(unsigned* s_next, long long t, long long tend, int lane, long long& tb) {
    unsigned b = 0;
    if (lane == 0) b = atomicAdd(s_next, 32u);
    b = __shfl_sync(kFull, b, 0);
    tb = t + (long long)b;
    if (tb >= tend) return 0;
    return (int)(tend - tb < 32 ? tend - tb : 32);
}

// Count the tasks [t, tend) of one owner whose list (cols[ob, ob + ol)) is longer than a
// piece: the table holds one piece at a time and every partner list is streamed per piece.
template <bool EXTRA>
__device__ void big_owner_pieces(const CountArgs& a, long long t, long long tend, long long ob, uint32_t ol,
                                 uint32_t* __restrict__ tbl, unsigned* s_next, int lane, unsigned long long& acc) {
    for (uint32_t ps = 0; ps < ol; ps += (uint32_t)a.piece) {
        const uint32_t pl = min((uint32_t)a.piece, ol - ps);
        uint32_t cap = 1024;
        while (cap < 8 * pl) cap <<= 1;
        const HashView hv = make_view(tbl, cap);
        const uint32_t reg = pack_region(0u, cap);
        for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) tbl[i] = kEmpty;
        if (threadIdx.x == 0) *s_next = 0;
        __syncthreads();
        for (uint32_t i0 = threadIdx.x; i0 < pl; i0 += kStageItems * blockDim.x) {
            uint32_t xs[kStageItems];  // each thread's entries loaded before any is inserted
#pragma unroll
            for (int k = 0; k < kStageItems; ++k) {
                const uint32_t i = i0 + (uint32_t)k * blockDim.x;
                xs[k] = i < pl ? (uint32_t)__ldg(&a.cols[ob + ps + i]) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kStageItems; ++k)
                if (i0 + (uint32_t)k * blockDim.x < pl) hash_insert(hv, xs[k]);
        }
        const uint32_t pmin = (uint32_t)__ldg(&a.cols[ob + ps]), pmax = (uint32_t)__ldg(&a.cols[ob + ps + pl - 1]);
        __syncthreads();
        for (;;) {
            long long tb;
            const int nb = claim_batch(s_next, t, tend, lane, tb);
            if (nb == 0) break;
            TaskRec r = {0u, 0u, 0u, 0u};
            if (lane < nb) r = a.tasks[tb + lane];
            warp_batch<EXTRA, true>(a, r, nb, tbl, reg, pmin, pmax, lane, acc);
        }
        __syncthreads();
        if (EXTRA && a.cnt_off) {
            flush_slot_hits(a, hv, ob + ps, pl, threadIdx.x, blockDim.x);
            __syncthreads();
        }
    }
}

// Count the big-class tasks [t0, t1) (every thread of the block calls this).  Consecutive
// owners are taken in windows: as many as fit the block table at a load of at most 1/8
// each; their lists are staged together and the block's warps pull batches of 32 of the
// window's tasks from a block counter, each task probing its own owner's region.
template <bool EXTRA>
__device__ void process_big(const CountArgs& a, long long t0, long long t1, uint32_t* __restrict__ tbl,
                            BigWindow* w, unsigned* s_next, int lane, int warp, unsigned long long& acc) {
    if (t0 >= t1) return;
    const int nwarps = blockDim.x >> 5;
    if (warp == 0) {
        // owner of t0: the last owner whose first task is at or before t0
        const uint32_t* __restrict__ of = a.own_first;
        const long long K = a.n_owners;
        const long long k = warp_first_true(0, K, [&](long long q) { return q >= K || (long long)of[q] > t0; }, lane) - 1;
        if (lane == 0) w->k = k;
    }
    __syncthreads();
    long long k = w->k;
    long long t = t0;
    while (t < t1) {
        if (warp == 0) {
            const long long kq = k + lane;
            const bool exists = kq < a.n_owners && (long long)a.own_first[kq] < t1;
            long long ob = 0, first = 0;
            uint32_t ol = 0, cap = 0, lmin = 0u, lmax = 0u;
            if (exists) {
                first = (long long)a.own_first[kq];
                const uint32_t owner = a.tasks[first].owner;
                ob = a.off[owner];
                ol = (uint32_t)(a.off[owner + 1] - ob);
                cap = 1024;
                while (cap < 8 * ol) cap <<= 1;
                if (ol) {
                    lmin = (uint32_t)__ldg(&a.cols[ob]);
                    lmax = (uint32_t)__ldg(&a.cols[ob + ol - 1]);
                }
            }
            const uint32_t cend = warp_inclusive_scan(cap, lane);
            const unsigned fit = __ballot_sync(kFull, exists && cend <= (uint32_t)a.table_slots);
            const int nown = fit == kFull ? 32 : __ffs(~fit) - 1;  // leading run of owners that fit
            const uint32_t used = __shfl_sync(kFull, cend, (nown - 1) & 31);
            const uint32_t eincl = warp_inclusive_scan(lane < nown ? ol : 0u, lane);
            if (lane < nown) w->epre[lane] = eincl - ol;
            if (lane == 31) w->epre[nown] = eincl;  // nown <= 32: the window's entries
            if (lane < (nown > 0 ? nown : 1)) {
                w->first[lane] = lane == 0 ? t : first;
                w->ob[lane] = ob;
                w->ol[lane] = ol;
                w->reg[lane] = pack_region(cend - cap, cap);
                w->lmin[lane] = lmin;
                w->lmax[lane] = lmax;
            }
            if (lane == 0) {
                const long long nk = k + (nown > 0 ? nown : 1);
                const long long nf = (long long)a.own_first[nk];  // own_first[n_owners] = T
                w->first[nown > 0 ? nown : 1] = nf < t1 ? nf : t1;
                w->nown = nown;
                w->used = nown > 0 ? used : 0u;
            }
        }
        __syncthreads();
        const int nown = w->nown;
        const long long tend = w->first[nown > 0 ? nown : 1];
        if (nown == 0) {
            big_owner_pieces<EXTRA>(a, t, tend, w->ob[0], w->ol[0], tbl, s_next, lane, acc);
        } else {
            const uint32_t used = w->used;
            for (uint32_t i = threadIdx.x; i < used; i += blockDim.x) tbl[i] = kEmpty;
            if (threadIdx.x == 0) *s_next = 0;
            __syncthreads();
            // stage the window's lists: its entries numbered one after another and spread over
            // the block's threads, each thread's entries loaded before any is inserted
            const uint32_t etot = w->epre[nown];
            for (uint32_t e0 = threadIdx.x; e0 < etot; e0 += kStageItems * blockDim.x) {
                uint32_t xs[kStageItems];
                int oi[kStageItems];
#pragma unroll
                for (int k = 0; k < kStageItems; ++k) {
                    const uint32_t e = e0 + (uint32_t)k * blockDim.x;
                    int lo = 0, hi = nown - 1;  // the last owner whose entries start at or before e
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (w->epre[mid] <= e) lo = mid; else hi = mid - 1;
                    }
                    oi[k] = lo;
                    xs[k] = e < etot ? (uint32_t)__ldg(&a.cols[w->ob[lo] + (e - w->epre[lo])]) : 0u;
                }
#pragma unroll
                for (int k = 0; k < kStageItems; ++k)
                    if (e0 + (uint32_t)k * blockDim.x < etot) hash_insert(region_view(tbl, w->reg[oi[k]]), xs[k]);
            }
            __syncthreads();
            for (;;) {
                long long tb;
                const int nb = claim_batch(s_next, t, tend, lane, tb);
                if (nb == 0) break;
                TaskRec r = {0u, 0u, 0u, 0u};
                uint32_t reg = 0u, omin = 0u, omax = 0u;
                if (lane < nb) {
                    const long long j = tb + lane;
                    r = a.tasks[j];
                    int lo = 0, hi = nown - 1;  // the last window owner whose tasks start at or before j
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (w->first[mid] <= j) lo = mid; else hi = mid - 1;
                    }
                    reg = w->reg[lo];
                    omin = w->lmin[lo];
                    omax = w->lmax[lo];
                }
                warp_batch<EXTRA, true>(a, r, nb, tbl, reg, omin, omax, lane, acc);
            }
            __syncthreads();
            if (EXTRA && a.cnt_off) {
                for (int i = warp; i < nown; i += nwarps)
                    flush_slot_hits(a, region_view(tbl, w->reg[i]), w->ob[i], w->ol[i], lane, 32u);
                __syncthreads();  // before warp 0 rewrites the window record
            }
        }
        t = tend;
        k += nown > 0 ? nown : 1;
    }
}

// Scheduling loop of one block-wide worker (Sec. V-B): its Eq. 1 initial chunk, then Eq. 2
// chunks popped by thread 0 until the class's cost is exhausted.  `process(t0, t1)` is
// called by every thread of the block.
template <bool MULTI, class Process>
__device__ __forceinline__ void block_worker(const CountArgs& a, Process process, int lane, int warp,
                                             long long& busy, long long& nch) {
    __shared__ long long s_t[2];
    __shared__ unsigned long long s_c[2];
    __shared__ int s_got;
    const long long wid = blockIdx.x;
    const unsigned long long C = a.sched->C, H = a.sched->H, minc = a.sched->min_chunk, base = a.sched->base;
    const unsigned long long W = (unsigned long long)a.W;
    // Eq. 1: the initial share split into W parts of equal cost, one per block
    if (warp == 0) {
        const unsigned long long q = H / W, r = H % W, w0 = (unsigned long long)wid;
        const unsigned long long lo = w0 * q + (w0 < r ? w0 : r);
        const unsigned long long hi = (w0 + 1) * q + (w0 + 1 < r ? w0 + 1 : r);
        // worker 0 starts at the schedule's first task: the class's first, or for a later part the
        // first task whose prefix reaches the part's base -- even when the part's cost is zero, where
        // its start boundary would otherwise map to the class end and its zero-cost tasks be lost
        long long t0;
        if (wid == 0 && a.sched->at_start) {
            t0 = a.t_begin;
        } else if (MULTI) {
            t0 = class_bound_multi(a, lo, C, lane);
        } else if (wid == 0) {
            const uint64_t* __restrict__ P = a.P;
            t0 = warp_first_true(a.t_begin, a.t_end, [&](long long q) { return P[q] >= base; }, lane);
        } else {
            t0 = class_bound(a, lo, C, base, lane);
        }
        const long long t1 = MULTI ? class_bound_multi(a, hi, C, lane) : class_bound(a, hi, C, base, lane);
        if (lane == 0) {
            s_t[0] = t0;
            s_t[1] = t1;
            trace_chunk(a, lo, hi, t0, t1);
        }
    }
    __syncthreads();
    long long c0 = clock64();
    process(s_t[0], s_t[1]);
    busy += clock64() - c0;
    ++nch;
    // Eq. 2: guided chunks of the remaining cost
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long c = 0, e = 0;
            s_got = pop_chunk(a, C, minc, c, e);
            s_c[0] = c;
            s_c[1] = e;
        }
        __syncthreads();
        if (!s_got) break;
        if (warp == 0) {
            const long long t0 = MULTI ? class_bound_multi(a, s_c[0], C, lane) : class_bound(a, s_c[0], C, base, lane);
            const long long t1 = MULTI ? class_bound_multi(a, s_c[1], C, lane) : class_bound(a, s_c[1], C, base, lane);
            if (lane == 0) {
                s_t[0] = t0;
                s_t[1] = t1;
                trace_chunk(a, s_c[0], s_c[1], t0, t1);
            }
        }
        __syncthreads();
        c0 = clock64();
        process(s_t[0], s_t[1]);
        busy += clock64() - c0;
        ++nch;
    }
}

// Packs: count the chunk [t0, t1) one graph at a time, adding each graph's hits into its own
// total.  With one graph the chunk is processed as it is.  Packs count totals only, so the
// per-vertex / per-edge instantiations (EXTRA) leave the split out.
template <bool EXTRA, class Process>
__device__ __forceinline__ void by_graph(const CountArgs& a, long long t0, long long t1, Process process,
                                         unsigned long long& acc, int lane, int warp) {
    if (EXTRA || a.n_sub == 0) {
        process(t0, t1);
        return;
    }
    __shared__ long long s_g;
    if (warp == 0) {
        const int64_t* __restrict__ gt = a.gtask;
        const long long K = a.n_sub;
        // the graph holding task t0: the first graph whose tasks end after t0
        const long long gq = warp_first_true(0, K - 1, [&](long long q) { return q >= K - 1 || gt[q + 1] > t0; }, lane);
        if (lane == 0) s_g = gq;
    }
    __syncthreads();
    long long g = s_g;
    for (long long t = t0; t < t1; ++g) {
        const long long ge = a.gtask[g + 1];
        const long long te = ge < t1 ? ge : t1;
        if (te > t) {
            process(t, te);
            const unsigned long long v = warp_sum(acc);
            if (lane == 0 && v) atomicAdd(&a.total[g], v);
            acc = 0;
        }
        t = te;
    }
}

template <bool EXTRA>
__device__ __forceinline__ void worker_epilogue(const CountArgs& a, unsigned long long acc, int lane, long long busy,
                                                long long nch) {
    acc = warp_sum(acc);
    if (lane == 0 && acc) atomicAdd(a.total, acc);
    if (threadIdx.x == 0 && a.trace_busy) {
        a.trace_busy[2 * (a.busy_offset + blockIdx.x)] = (uint64_t)busy;
        a.trace_busy[2 * (a.busy_offset + blockIdx.x) + 1] = (uint64_t)nch;
    }
}

// Per-vertex / per-edge counts: zero the warps' task-hit counters and the slot counts (flushes
// leave them zero again).  `slots`: the words of the block's tables.
__device__ __forceinline__ void extra_init(const CountArgs& a, int slots) {
    if (a.cnt_off)
        for (int i = threadIdx.x; i < slots; i += blockDim.x) smem_dyn[a.cnt_off + i] = 0u;
    for (int i = threadIdx.x; i < 32 * (int)(blockDim.x >> 5); i += blockDim.x) smem_dyn[a.hits_off + i] = 0u;
    __syncthreads();
}

// Small owners: one worker per block, a table per warp.  MULTI: the packs of a batch.
template <bool EXTRA, bool MULTI>
__global__ void __launch_bounds__(512, kCountMinBlocks) k_count_small(CountArgs a) {
    __shared__ unsigned s_claim;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* tbl = smem_dyn + (size_t)warp * a.table_slots;
    unsigned long long acc = 0;
    long long busy = 0, nch = 0;
    if (EXTRA) extra_init(a, a.warps_per_block * a.table_slots);
    if (MULTI) {
        block_worker<true>(a, [&](long long g0, long long g1) {
            for_pack_pieces(a, g0, g1, lane, [&](const CountArgs& b, long long l0, long long l1) {
                by_graph<false>(b, l0, l1, [&](long long u0, long long u1) {
                    process_small_block<false>(b, u0, u1, tbl, &s_claim, lane, acc);
                }, acc, lane, warp);
            });
        }, lane, warp, busy, nch);
    } else {
        block_worker<false>(a, [&](long long t0, long long t1) {
            by_graph<EXTRA>(a, t0, t1, [&](long long u0, long long u1) { process_small_block<EXTRA>(a, u0, u1, tbl, &s_claim, lane, acc); },
                     acc, lane, warp);
        }, lane, warp, busy, nch);
    }
    worker_epilogue<EXTRA>(a, acc, lane, busy, nch);
}

// Big owners: one worker per block, one table per block.  MULTI: the packs of a batch.
template <bool EXTRA, bool MULTI>
__global__ void __launch_bounds__(512, kCountMinBlocks) k_count_big(CountArgs a) {
    uint32_t* smem_tbl = smem_dyn;
    __shared__ BigWindow s_win;
    __shared__ unsigned s_next;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long acc = 0;
    long long busy = 0, nch = 0;
    if (EXTRA) extra_init(a, a.table_slots);
    if (MULTI) {
        block_worker<true>(a, [&](long long g0, long long g1) {
            for_pack_pieces(a, g0, g1, lane, [&](const CountArgs& b, long long l0, long long l1) {
                by_graph<false>(b, l0, l1, [&](long long u0, long long u1) {
                    process_big<false>(b, u0, u1, smem_tbl, &s_win, &s_next, lane, warp, acc);
                }, acc, lane, warp);
            });
        }, lane, warp, busy, nch);
    } else {
        block_worker<false>(a, [&](long long t0, long long t1) {
            by_graph<EXTRA>(a, t0, t1, [&](long long u0, long long u1) {
                process_big<EXTRA>(a, u0, u1, smem_tbl, &s_win, &s_next, lane, warp, acc);
            }, acc, lane, warp);
        }, lane, warp, busy, nch);
    }
    worker_epilogue<EXTRA>(a, acc, lane, busy, nch);
}

// --------------------------------------------------------------------------- costs (a6)

struct TaskCost {
    const TaskRec* tasks;
    long long T;
    const int64_t* off;
    const uint64_t* f;
    int model;
    uint32_t piece, small_max, c_task, c_owner;
    __device__ uint64_t operator()(int64_t t) const {
        const TaskRec r = tasks[t];
        const bool last = (t + 1 == T) || tasks[t + 1].owner != r.owner;
        if (model == TC_COST_EDGE) {
            const uint64_t dho = (uint64_t)(off[r.owner + 1] - off[r.owner]);
            const uint64_t pieces = dho <= small_max ? 1ull : (dho + piece - 1) / piece;
            uint64_t c = pieces * ((uint64_t)r.plen + c_task);
            if (last) c += dho + c_owner;
            return c;
        }
        if (model == TC_COST_MERGE) return (uint64_t)(off[r.owner + 1] - off[r.owner]) + (uint64_t)r.plen;
        return last ? f[r.owner] : 0ull;  // per-vertex models: the owner's cost on its last task
    }
};

// Schedule state of both classes: class 0 is tasks [0, Ts), class 1 is [Ts, T).  With
// nparts > 1, only part `part` of each class's cost: [Cc part / nparts, Cc (part + 1) / nparts).
__global__ void k_sched_init(Sched* sc, const uint64_t* P, long long Ts, long long T, long long W0, long long W1,
                             int static_percent, long long min_chunk, int part, int nparts) {
    const unsigned long long sp = (unsigned long long)static_percent;
    for (int c = 0; c < 2; ++c) {
        const unsigned long long cbase = c == 0 ? 0ull : P[Ts];
        const unsigned long long Cc = (c == 0 ? P[Ts] : P[T]) - cbase;
        // part boundaries without overflow: Cc * p / nparts as (Cc / np) p + ((Cc % np) p) / np
        const unsigned long long np = (unsigned long long)nparts, p0 = (unsigned long long)part;
        const unsigned long long lo = (Cc / np) * p0 + ((Cc % np) * p0) / np;
        const unsigned long long hi = (Cc / np) * (p0 + 1) + ((Cc % np) * (p0 + 1)) / np;
        const unsigned long long base = cbase + lo;
        const unsigned long long C = hi - lo;
        const unsigned long long W = (unsigned long long)(c == 0 ? W0 : W1);
        const unsigned long long H = (C / 100ull) * sp + ((C % 100ull) * sp) / 100ull;
        unsigned long long minc = (unsigned long long)min_chunk;
        if (min_chunk <= 0) {
            minc = C / (W * 128ull);
            if (minc < 32ull) minc = 32ull;
        }
        sc[c].C = C;
        sc[c].H = H;
        sc[c].min_chunk = minc;
        sc[c].head = H;
        sc[c].n_chunks = 0;
        sc[c].base = base;
        sc[c].streamed = 0;
        sc[c].at_start = part == 0 ? 1ull : 0ull;
        sc[c].at_end = part == nparts - 1 ? 1ull : 0ull;
    }
}

// Per-vertex cost functions (Sec. IV-B, IV-F, V-A); f must be zeroed for TC_FN_NEW.
__global__ void k_vertex_cost(int fn, int32_t n, const int32_t* __restrict__ deg, const int64_t* __restrict__ off,
                              const int32_t* __restrict__ cols, uint64_t* __restrict__ f) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = off[v], e = off[v + 1];
        const uint64_t dv = (uint64_t)(e - b);
        if (fn == TC_FN_ONE) {
            f[v] = 1;
        } else if (fn == TC_FN_DEGREE) {
            f[v] = (uint64_t)deg[v];
        } else if (fn == TC_FN_PATRIC) {
            uint64_t s = 0;
            for (int64_t i = b; i < e; ++i) {
                const int32_t u = cols[i];
                s += dv + (uint64_t)(off[u + 1] - off[u]);
            }
            f[v] = s;
        } else {
            // v in N_u  <=>  u in Nfull_v - N_v: each oriented edge (v,u) charges u
            for (int64_t i = b; i < e; ++i) {
                const int32_t u = cols[i];
                atomicAdd((unsigned long long*)&f[u], (unsigned long long)(dv + (uint64_t)(off[u + 1] - off[u])));
            }
        }
    }
}

__global__ void k_clustering(int32_t n, const int32_t* __restrict__ deg, const uint64_t* __restrict__ t_v,
                             double* __restrict__ cc) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)deg[v];
        cc[v] = deg[v] < 2 ? 0.0 : 2.0 * (double)t_v[v] / (d * (d - 1.0));
    }
}

static unsigned blocks_for(int64_t n) {
    int64_t want = ceil_div(n > 0 ? n : 1, 256);
    int64_t cap = (int64_t)num_sms() * 16;
    return (unsigned)(want < cap ? want : cap);
}

tc_status vertex_cost_enqueue(tc_graph* g, int fn, cudaStream_t s, uint64_t* f) {
    if (fn < TC_FN_ONE || fn > TC_FN_NEW) return TC_ERR_INVALID_ARG;
    if (g->n == 0) return TC_OK;
    if (fn == TC_FN_NEW) TC_CUDA_TRY(cudaMemsetAsync(f, 0, sizeof(uint64_t) * g->n, s));
    k_vertex_cost<<<blocks_for(g->n), 256, 0, s>>>(fn, g->n, g->deg, g->off, g->cols, f);
    note_launch();
    TC_CUDA_TRY(cudaGetLastError());
    return TC_OK;
}

tc_status clustering_enqueue(tc_graph* g, const uint64_t* t_v, double* cc, cudaStream_t s) {
    if (g->n == 0) return TC_OK;
    k_clustering<<<blocks_for(g->n), 256, 0, s>>>(g->n, g->deg, t_v, cc);
    note_launch();
    TC_CUDA_TRY(cudaGetLastError());
    return TC_OK;
}

tc_status ensure_count_work(tc_graph* g, const tc_options& opt, cudaStream_t s) {
    CountWork& w = g->work;
    if (!w.prefix) {
        void* p = nullptr;
        TC_TRY(g->al.get(&p, (size_t)(g->tasks + 1) * 8, s));
        w.prefix = (uint64_t*)p;
        w.prefix_len = g->tasks + 1;
        g->bytes += (int64_t)align_up((size_t)(g->tasks + 1) * 8, 256);
        w.scan_words = scan_scratch_words(g->tasks);
        TC_TRY(g->al.get(&p, (size_t)w.scan_words * 8, s));
        w.scan_scr = (uint64_t*)p;
        g->bytes += (int64_t)align_up((size_t)w.scan_words * 8, 256);
    }
    const bool vertex_model = opt.cost_model >= TC_COST_ONE;
    if (vertex_model && !w.fcost) {
        void* p = nullptr;
        TC_TRY(g->al.get(&p, (size_t)(g->n > 0 ? g->n : 1) * 8, s));
        w.fcost = (uint64_t*)p;
        g->bytes += (int64_t)align_up((size_t)(g->n > 0 ? g->n : 1) * 8, 256);
    }
    return TC_OK;
}

template <class K>
static tc_status grid_for_kernel(K kernel, int threads, size_t smem, int cap_per_sm, int* blocks) {
    TC_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    if (per_sm < 1) return TC_ERR_INVALID_ARG;
    if (cap_per_sm > 0 && cap_per_sm < per_sm) per_sm = cap_per_sm;
    *blocks = num_sms() * per_sm;
    return TC_OK;
}

tc_status count_enqueue(tc_graph* g, const tc_options& opt, cudaStream_t s, unsigned long long* total_dev,
                        unsigned long long* t_v, uint32_t* per_edge, tc_count_trace* trace, int part, int nparts) {
    if (nparts < 1 || part < 0 || part >= nparts) return TC_ERR_INVALID_ARG;
    const bool extra = t_v != nullptr || per_edge != nullptr;
    if (g->n_sub > 0 && (extra || trace)) return TC_ERR_UNSUPPORTED;
    TC_TRY(ensure_count_work(g, opt, s));
    CountWork& w = g->work;
    const long long T = g->tasks, Ts = g->tasks_small;
    // Per-vertex counts keep a hit count beside every table slot, so their tables take twice the
    // shared memory: they run with at most 8 warps per small-class block and pieces of at most
    // 1024 entries (the block table of 8 * piece slots), which keeps two blocks per SM.
    const int wpb = (t_v && opt.warps_per_block > 8) ? 8 : opt.warps_per_block;
    const int piece = (t_v && opt.piece > 1024) ? 1024 : opt.piece;
    const int tab = t_v ? 2 : 1;
    // small class: blocks whose warps each have a table
    const int slots_s = small_table_slots(g->opt.small_max);
    const size_t smem_s = (size_t)wpb * slots_s * sizeof(uint32_t);
    // big class: blocks sharing one table of 8 * piece slots
    const int threads_b = opt.big_warps * 32;
    const int slots_b = 8 * piece;
    const size_t smem_b = (size_t)slots_b * sizeof(uint32_t);
    // per-vertex / per-edge counts: slot counts after the tables, then 32 task-hit counters per warp
    const size_t smem_s_x = smem_s * tab + (size_t)32 * wpb * sizeof(uint32_t);
    const size_t smem_b_x = smem_b * tab + (size_t)32 * opt.big_warps * sizeof(uint32_t);
    int blocks_s = 0, blocks_b = 0;
    if (extra) {
        TC_TRY(grid_for_kernel(k_count_small<true, false>, wpb * 32, smem_s_x, opt.blocks_per_sm, &blocks_s));
        TC_TRY(grid_for_kernel(k_count_big<true, false>, threads_b, smem_b_x, opt.blocks_per_sm, &blocks_b));
    } else {
        TC_TRY(grid_for_kernel(k_count_small<false, false>, wpb * 32, smem_s, opt.blocks_per_sm, &blocks_s));
        TC_TRY(grid_for_kernel(k_count_big<false, false>, threads_b, smem_b, opt.blocks_per_sm, &blocks_b));
    }
    const long long W_s = blocks_s, W_b = blocks_b;  // one worker per block in both classes

    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (trace) {
        for (auto& e : ev) TC_CUDA_TRY(cudaEventCreate(&e));
        TC_CUDA_TRY(cudaEventRecord(ev[0], s));
    }
    // a6: costs, prefix, schedule state of both classes
    if (opt.cost_model >= TC_COST_ONE) {
        const int fn = opt.cost_model - TC_COST_ONE;  // ONE, DEGREE, PATRIC, NEW in enum order
        TC_TRY(vertex_cost_enqueue(g, fn, s, w.fcost));
    }
    TaskCost tcf{g->trec, T, g->off, w.fcost, opt.cost_model, (uint32_t)opt.piece, (uint32_t)g->opt.small_max,
                 (uint32_t)opt.c_task, (uint32_t)opt.c_owner};
    TC_CUDA_TRY(scan_exclusive(tcf, T, w.prefix, w.scan_scr, s));
    k_sched_init<<<1, 1, 0, s>>>(w.sched, w.prefix, Ts, T, W_s, W_b, opt.static_percent, opt.min_chunk, part, nparts);
    note_launch();
    TC_CUDA_TRY(cudaGetLastError());
    TC_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(unsigned long long) * (g->n_sub > 0 ? g->n_sub : 1), s));
    if (t_v && g->n > 0) TC_CUDA_TRY(cudaMemsetAsync(t_v, 0, sizeof(unsigned long long) * g->n, s));
    if (per_edge && g->m_hat > 0) TC_CUDA_TRY(cudaMemsetAsync(per_edge, 0, sizeof(uint32_t) * g->m_hat, s));
    if (trace) TC_CUDA_TRY(cudaEventRecord(ev[1], s));

    CountArgs a;
    a.off = g->off;
    a.cols = g->cols;
    a.tasks = g->trec;
    a.deg = g->deg;
    a.P = w.prefix;
    a.trace_sched = w.sched;
    a.total = total_dev;
    a.t_v = t_v;
    a.per_edge = per_edge;
    a.trace_chunks = trace ? trace->chunks : nullptr;
    a.trace_cap = trace ? trace->cap : 0;
    a.trace_busy = trace ? trace->workers_busy : nullptr;
    a.status = g->status;
    a.retry_limit = opt.retry_limit > 0 ? opt.retry_limit : (1ll << 24);
    a.own_first = g->own_first;
    a.n_owners = g->owners_big;
    a.n_sub = g->n_sub;
    const bool count_streamed = trace && trace->count_streamed;
    a.packs = nullptr;
    a.n_packs = 0;
    a.tbase = nullptr;
    a.cbase = nullptr;
    // small class
    a.cnt_off = t_v ? wpb * slots_s : 0;
    a.hits_off = wpb * slots_s * tab;
    a.gtask = g->sub_task;
    a.streamed = count_streamed ? &w.sched[0].streamed : nullptr;
    a.t_begin = 0;
    a.t_end = Ts;
    a.sched = w.sched;
    a.W = W_s;
    a.cls = 0;
    a.piece = piece;
    a.table_slots = slots_s;
    a.warps_per_block = wpb;
    a.busy_offset = 0;
    if (Ts > 0) {
        if (extra) k_count_small<true, false><<<blocks_s, wpb * 32, smem_s_x, s>>>(a);
        else k_count_small<false, false><<<blocks_s, wpb * 32, smem_s, s>>>(a);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
    }
    if (trace) TC_CUDA_TRY(cudaEventRecord(ev[2], s));
    // big class
    a.cnt_off = t_v ? slots_b : 0;
    a.hits_off = slots_b * tab;
    a.gtask = g->sub_task ? g->sub_task + (g->n_sub + 1) : nullptr;
    a.streamed = count_streamed ? &w.sched[1].streamed : nullptr;
    a.t_begin = Ts;
    a.t_end = T;
    a.sched = w.sched + 1;
    a.W = W_b;
    a.cls = 1;
    a.table_slots = slots_b;
    a.warps_per_block = opt.big_warps;
    a.busy_offset = W_s;
    if (T > Ts) {
        if (extra) k_count_big<true, false><<<blocks_b, threads_b, smem_b_x, s>>>(a);
        else k_count_big<false, false><<<blocks_b, threads_b, smem_b, s>>>(a);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
    }
    if (trace) {
        TC_CUDA_TRY(cudaEventRecord(ev[3], s));
        Sched hs[2];
        TC_CUDA_TRY(cudaMemcpyAsync(hs, w.sched, sizeof(hs), cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        trace->n_chunks = (int64_t)hs[0].n_chunks;
        trace->n_workers[0] = W_s;
        trace->n_workers[1] = W_b;
        for (int c = 0; c < 2; ++c) {
            trace->total_cost[c] = hs[c].C;
            trace->min_chunk[c] = hs[c].min_chunk;
            trace->streamed[c] = count_streamed ? (int64_t)hs[c].streamed : -1;
        }
        trace->tasks_small = Ts;
        float ms = 0.f;
        TC_CUDA_TRY(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        trace->prefix_ms = ms;
        TC_CUDA_TRY(cudaEventElapsedTime(&ms, ev[1], ev[2]));
        trace->kernel_small_ms = ms;
        TC_CUDA_TRY(cudaEventElapsedTime(&ms, ev[2], ev[3]));
        trace->kernel_big_ms = ms;
        for (auto& e : ev) cudaEventDestroy(e);
    }
    return TC_OK;
}

// --------------------------------------------------------------------------- multi-pack count
//
// A batch's packs counted together: one cost prefix over all packs' tasks (pack after pack),
// then per class one schedule over the packs' concatenated costs and one launch of the class
// kernel, whose workers count each chunk pack piece by pack piece.

// The multi-pack cost prefix.  Each pack's tasks start a new scan tile, so every tile lies in
// one pack: a block finds its pack once and evaluates that pack's task costs.  Tile sums, a
// scan of them (scan_exclusive), the downsweep into each pack's P, and each pack's end value
// P[T] = the prefix at the start of the next pack's first tile.
__device__ __forceinline__ int pack_of_tile(const PackDev* __restrict__ packs, int np, long long tile) {
    int lo = 0, hi = np - 1;  // the last pack whose first tile is at or before `tile`
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (packs[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct MultiCostArgs {
    const PackDev* packs;
    int np;
    int model;
    uint32_t piece, small_max, c_task, c_owner;
};

__device__ __forceinline__ TaskCost block_pack_cost(const MultiCostArgs& m, const PackDev*& pk, int64_t& first) {
    __shared__ int s_p;
    if (threadIdx.x == 0) s_p = pack_of_tile(m.packs, m.np, (long long)blockIdx.x);
    __syncthreads();
    pk = m.packs + s_p;
    first = (int64_t)(blockIdx.x - pk->tile_base) * kScanTile;  // the block's first task in its pack
    return TaskCost{pk->tasks, pk->T, pk->off, pk->fcost, m.model, m.piece, m.small_max, m.c_task, m.c_owner};
}

__global__ void __launch_bounds__(kScanBlock) k_multi_tile_sums(MultiCostArgs m, uint64_t* tile_sums) {
    const PackDev* pk;
    int64_t first;
    const TaskCost f = block_pack_cost(m, pk, first);
    const int64_t n = pk->T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = first + (int64_t)warp * 32 * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k * 32 + lane;
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

__global__ void __launch_bounds__(kScanBlock) k_multi_downsweep(MultiCostArgs m, const uint64_t* tile_prefix) {
    const PackDev* pk;
    int64_t first;
    const TaskCost f = block_pack_cost(m, pk, first);
    const int64_t n = pk->T;
    uint64_t* __restrict__ out = pk->P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = first + (int64_t)warp * 32 * kScanItems;
    uint64_t ex[kScanItems];
    uint64_t carry = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k * 32 + lane;
        const uint64_t v = i < n ? f(i) : 0;
        const uint64_t incl = warp_inclusive_scan(v, lane);
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
        const int64_t i = base + k * 32 + lane;
        if (i < n) out[i] = woff + ex[k];
    }
}

// P[T] of every pack: the prefix at the start of the next pack's first tile (the last pack: the
// total).  Padding past a pack's last task costs nothing, so that is the sum through the pack.
__global__ void k_multi_pack_ends(const PackDev* packs, int np, long long tiles, const uint64_t* tile_prefix) {
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const PackDev& pk = packs[p];
        if (pk.T == 0) continue;
        const long long next = p + 1 < np ? packs[p + 1].tile_base : tiles;
        pk.P[pk.T] = tile_prefix[next];
    }
}

// Per class: each pack's first task and cost base in the class's concatenated order, and the
// class's schedule (Eq. 1 share and Eq. 2 floor over the total, as k_sched_init).
__global__ void k_multi_sched_init(const PackDev* packs, int np, long long* tb0, long long* tb1, unsigned long long* cb0,
                                   unsigned long long* cb1, Sched* sc, long long W0, long long W1, int static_percent,
                                   long long min_chunk) {
    long long t0 = 0, t1 = 0;
    unsigned long long c0 = 0, c1 = 0;
    for (int p = 0; p < np; ++p) {
        tb0[p] = t0;
        tb1[p] = t1;
        cb0[p] = c0;
        cb1[p] = c1;
        const PackDev& pk = packs[p];
        if (pk.T > 0) {
            c0 += pk.P[pk.Ts] - pk.P[0];
            c1 += pk.P[pk.T] - pk.P[pk.Ts];
        }
        t0 += pk.Ts;
        t1 += pk.T - pk.Ts;
    }
    tb0[np] = t0;
    tb1[np] = t1;
    cb0[np] = c0;
    cb1[np] = c1;
    const unsigned long long sp = (unsigned long long)static_percent;
    for (int c = 0; c < 2; ++c) {
        const unsigned long long C = c == 0 ? c0 : c1;
        const unsigned long long W = (unsigned long long)(c == 0 ? W0 : W1);
        unsigned long long minc = (unsigned long long)min_chunk;
        if (min_chunk <= 0) {
            minc = C / (W * 128ull);
            if (minc < 32ull) minc = 32ull;
        }
        sc[c].C = C;
        sc[c].H = (C / 100ull) * sp + ((C % 100ull) * sp) / 100ull;
        sc[c].min_chunk = minc;
        sc[c].head = sc[c].H;
        sc[c].n_chunks = 0;
        sc[c].base = 0;
        sc[c].streamed = 0;
        sc[c].at_start = 1;
        sc[c].at_end = 1;
    }
}

static int64_t multi_fixed_words(int n_packs) {
    return 4 * ((int64_t)n_packs + 1) + (int64_t)((2 * sizeof(Sched) + 7) / 8);
}

int64_t multi_scratch_words(int64_t total_tasks, int n_packs) {
    // each pack starts a new scan tile: at most n_packs tiles more than the tasks need
    return multi_fixed_words(n_packs) + scan_scratch_words(total_tasks + (int64_t)n_packs * kScanTile);
}

tc_status count_enqueue_multi(const std::vector<tc_graph*>& packs, const PackDev* packs_dev, uint64_t* scratch,
                              const tc_options& opt, unsigned long long* totals, int32_t k, cudaStream_t s) {
    const int np = (int)packs.size();
    if (np == 0) return TC_OK;
    int64_t total_tasks = 0, small_tasks = 0;
    for (tc_graph* g : packs) {
        total_tasks += g->tasks;
        small_tasks += g->tasks_small;
    }
    long long* tb0 = reinterpret_cast<long long*>(scratch);
    long long* tb1 = tb0 + np + 1;
    unsigned long long* cb0 = reinterpret_cast<unsigned long long*>(tb1 + np + 1);
    unsigned long long* cb1 = cb0 + np + 1;
    Sched* sc = reinterpret_cast<Sched*>(cb1 + np + 1);
    uint64_t* scan_scr = scratch + multi_fixed_words(np);

    const int wpb = opt.warps_per_block;
    const int slots_s = small_table_slots(packs[0]->opt.small_max);
    const size_t smem_s = (size_t)wpb * slots_s * sizeof(uint32_t);
    const int threads_b = opt.big_warps * 32;
    const int slots_b = 8 * opt.piece;
    const size_t smem_b = (size_t)slots_b * sizeof(uint32_t);
    int blocks_s = 0, blocks_b = 0;
    TC_TRY(grid_for_kernel(k_count_small<false, true>, wpb * 32, smem_s, opt.blocks_per_sm, &blocks_s));
    TC_TRY(grid_for_kernel(k_count_big<false, true>, threads_b, smem_b, opt.blocks_per_sm, &blocks_b));

    // a6 over every pack at once
    if (opt.cost_model >= TC_COST_ONE) {
        const int fn = opt.cost_model - TC_COST_ONE;
        for (tc_graph* g : packs) TC_TRY(vertex_cost_enqueue(g, fn, s, g->work.fcost));
    }
    if (total_tasks > 0) {
        long long tiles = 0;
        for (tc_graph* g : packs) tiles += ceil_div(g->tasks, kScanTile);
        const MultiCostArgs m{packs_dev, np, opt.cost_model, (uint32_t)opt.piece, (uint32_t)packs[0]->opt.small_max,
                              (uint32_t)opt.c_task, (uint32_t)opt.c_owner};
        uint64_t* tile = scan_scr;  // tiles + 1
        k_multi_tile_sums<<<(unsigned)tiles, kScanBlock, 0, s>>>(m, tile);
        note_launch();
        if (tiles <= 4096) {
            k_scan_single_block<<<1, 1024, 0, s>>>(tile, tiles);
            note_launch();
        } else {
            uint64_t* tmp = scan_scr + tiles + 1;
            TC_CUDA_TRY(scan_exclusive(IdentityU64{tile}, tiles, tmp, tmp + tiles + 1, s));
            TC_CUDA_TRY(cudaMemcpyAsync(tile, tmp, (tiles + 1) * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        }
        k_multi_downsweep<<<(unsigned)tiles, kScanBlock, 0, s>>>(m, tile);
        note_launch();
        k_multi_pack_ends<<<1, 256, 0, s>>>(packs_dev, np, tiles, tile);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
    }
    k_multi_sched_init<<<1, 1, 0, s>>>(packs_dev, np, tb0, tb1, cb0, cb1, sc, blocks_s, blocks_b, opt.static_percent,
                                       opt.min_chunk);
    note_launch();
    TC_CUDA_TRY(cudaGetLastError());
    TC_CUDA_TRY(cudaMemsetAsync(totals, 0, sizeof(unsigned long long) * (k > 0 ? k : 1), s));

    CountArgs a;
    a.off = nullptr;
    a.cols = nullptr;
    a.tasks = nullptr;
    a.deg = nullptr;
    a.P = nullptr;
    a.trace_sched = sc;
    a.total = totals;
    a.t_v = nullptr;
    a.per_edge = nullptr;
    a.trace_chunks = nullptr;
    a.trace_cap = 0;
    a.trace_busy = nullptr;
    a.busy_offset = 0;
    a.status = packs[0]->status;
    a.retry_limit = opt.retry_limit > 0 ? opt.retry_limit : (1ll << 24);
    a.own_first = nullptr;
    a.n_owners = 0;
    a.gtask = nullptr;
    a.n_sub = 0;
    a.streamed = nullptr;
    a.cnt_off = 0;
    a.hits_off = 0;
    a.packs = packs_dev;
    a.n_packs = np;
    a.piece = opt.piece;
    // small class
    a.tbase = tb0;
    a.cbase = cb0;
    a.t_begin = 0;
    a.t_end = small_tasks;
    a.sched = sc;
    a.W = blocks_s;
    a.cls = 0;
    a.table_slots = slots_s;
    a.warps_per_block = wpb;
    if (small_tasks > 0) {
        k_count_small<false, true><<<blocks_s, wpb * 32, smem_s, s>>>(a);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
    }
    // big class
    a.tbase = tb1;
    a.cbase = cb1;
    a.t_begin = 0;
    a.t_end = total_tasks - small_tasks;
    a.sched = sc + 1;
    a.W = blocks_b;
    a.cls = 1;
    a.table_slots = slots_b;
    a.warps_per_block = opt.big_warps;
    if (total_tasks > small_tasks) {
        k_count_big<false, true><<<blocks_b, threads_b, smem_b, s>>>(a);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
    }
    return TC_OK;
}

}  // namespace tcg

// --------------------------------------------------------------------------- count without allocation
//
// tc_count_static: the same count (cost prefix, Eq. 1 / Eq. 2 schedule, both count kernels)
// with its scratch -- the cost prefix, the scan's tile sums and the two schedule records --
// in one file-scope device array instead of memory allocated for the handle.  Host code
// never uses the array's name as an address: the address is asked of the runtime once per
// device (cudaGetSymbolAddress) and passed to the kernels.

namespace tcg {

constexpr long long kStaticMaxTasks = TC_COUNT_STATIC_MAX_TASKS;  // a 4 MiB cost prefix
constexpr long long kStaticPrefixWords = kStaticMaxTasks + 1;
constexpr long long kStaticScanWords = 512;  // the scan's tile sums; each call checks its need against this
constexpr long long kStaticSchedWords = (2 * sizeof(Sched) + 7) / 8;
constexpr long long kStaticWords = kStaticPrefixWords + kStaticScanWords + kStaticSchedWords;

static __device__ __align__(256) unsigned long long g_static_scratch[kStaticWords];

static std::mutex g_static_mu;
static unsigned long long* g_static_ptr[64] = {nullptr};

// Device address of g_static_scratch on the current device (looked up on first use).
static tc_status static_scratch(unsigned long long** out) {
    int dev = 0;
    TC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return TC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        TC_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_ptr[dev] = (unsigned long long*)p;
    }
    *out = g_static_ptr[dev];
    return TC_OK;
}

static tc_status count_enqueue_static(tc_graph* g, cudaStream_t s, unsigned long long* total_dev) {
    const tc_options& opt = g->opt;
    if (opt.cost_model != TC_COST_EDGE && opt.cost_model != TC_COST_MERGE) return TC_ERR_INVALID_ARG;
    const long long T = g->tasks, Ts = g->tasks_small;
    if (T > kStaticMaxTasks) return TC_ERR_UNSUPPORTED;
    // the scan's scratch must fit its region, or it would run into the schedule records
    if (scan_scratch_words(T) > kStaticScanWords) return TC_ERR_UNSUPPORTED;
    unsigned long long* base = nullptr;
    TC_TRY(static_scratch(&base));
    uint64_t* prefix = (uint64_t*)base;
    uint64_t* scan_scr = (uint64_t*)(base + kStaticPrefixWords);
    Sched* sched = (Sched*)(base + kStaticPrefixWords + kStaticScanWords);

    const int wpb = opt.warps_per_block;
    const int slots_s = small_table_slots(opt.small_max);
    const size_t smem_s = (size_t)wpb * slots_s * sizeof(uint32_t);
    const int threads_b = opt.big_warps * 32;
    const int slots_b = 8 * opt.piece;
    const size_t smem_b = (size_t)slots_b * sizeof(uint32_t);
    int blocks_s = 0, blocks_b = 0;
    TC_TRY(grid_for_kernel(k_count_small<false, false>, wpb * 32, smem_s, opt.blocks_per_sm, &blocks_s));
    TC_TRY(grid_for_kernel(k_count_big<false, false>, threads_b, smem_b, opt.blocks_per_sm, &blocks_b));
    const long long W_s = blocks_s, W_b = blocks_b;

    TaskCost tcf{g->trec, T, g->off, nullptr, opt.cost_model, (uint32_t)opt.piece, (uint32_t)opt.small_max,
                 (uint32_t)opt.c_task, (uint32_t)opt.c_owner};
    TC_CUDA_TRY(scan_exclusive(tcf, T, prefix, scan_scr, s));
    k_sched_init<<<1, 1, 0, s>>>(sched, prefix, Ts, T, W_s, W_b, opt.static_percent, opt.min_chunk, 0, 1);
    note_launch();
    TC_CUDA_TRY(cudaGetLastError());
    TC_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(unsigned long long), s));

    CountArgs a;
    a.off = g->off;
    a.cols = g->cols;
    a.tasks = g->trec;
    a.deg = g->deg;
    a.P = prefix;
    a.trace_sched = sched;
    a.total = total_dev;
    a.t_v = nullptr;
    a.per_edge = nullptr;
    a.trace_chunks = nullptr;
    a.trace_cap = 0;
    a.trace_busy = nullptr;
    a.status = g->status;
    a.retry_limit = opt.retry_limit > 0 ? opt.retry_limit : (1ll << 24);
    a.own_first = g->own_first;
    a.n_owners = g->owners_big;
    a.gtask = nullptr;
    a.streamed = nullptr;
    a.cnt_off = 0;
    a.hits_off = 0;
    a.packs = nullptr;
    a.n_packs = 0;
    a.tbase = nullptr;
    a.cbase = nullptr;
    a.n_sub = 0;
    a.t_begin = 0;
    a.t_end = Ts;
    a.sched = sched;
    a.W = W_s;
    a.cls = 0;
    a.piece = opt.piece;
    a.table_slots = slots_s;
    a.warps_per_block = wpb;
    a.busy_offset = 0;
    if (Ts > 0) {
        k_count_small<false, false><<<blocks_s, wpb * 32, smem_s, s>>>(a);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
    }
    a.t_begin = Ts;
    a.t_end = T;
    a.sched = sched + 1;
    a.W = W_b;
    a.cls = 1;
    a.table_slots = slots_b;
    a.warps_per_block = opt.big_warps;
    a.busy_offset = W_s;
    if (T > Ts) {
        k_count_big<false, false><<<blocks_b, threads_b, smem_b, s>>>(a);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
    }
    return TC_OK;
}

}  // namespace tcg

extern "C" tc_status tc_count_static(tc_graph_t g, tc_stream_t stream, uint64_t* total_dev) {
    if (!g || !total_dev) return TC_ERR_INVALID_ARG;
    g->last_stream = (cudaStream_t)stream;
    return tcg::count_enqueue_static(g, (cudaStream_t)stream, (unsigned long long*)total_dev);
}


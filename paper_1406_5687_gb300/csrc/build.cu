// build.cu -- steps a1-a5 of the path plus the task array.
//
//   a1  canonical keys (min << b) | max, ids range-checked, self-loops to a sentinel (Sec. II)
//   a2  LSD radix sort, drop repeated keys -> the m_hat distinct edges (Sec. II)
//   a3  degrees d_v
//   a4  orientation by the order of Sec. III-A: u < v iff d_u < d_v or (d_u = d_v and u < v)
//   a5  N+ lists (Fig. 1): sort the oriented keys, effective degrees, offsets, columns
//   tasks: each oriented edge owned by the endpoint with the longer list; tasks whose
//       partner list is empty are dropped; sorted by (class, owner, position of the oriented
//       edge in the lists); 16-byte records.
#include <climits>

#include "graph.cuh"
#include "primitives.cuh"
#include "scan.cuh"

namespace tcg {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int threads = kThreads) {
    int64_t g = ceil_div(n > 0 ? n : 1, threads);
    return (unsigned)(g > 0x7FFFFFFF ? 0x7FFFFFFF : g);
}

// --------------------------------------------------------------------------- compaction
constexpr int kCpItems = 8;
constexpr int kCpBlock = 256;
constexpr int64_t kCpTile = (int64_t)kCpBlock * kCpItems;

template <class Pred>
__global__ void __launch_bounds__(kCpBlock) k_compact_counts(Pred p, int64_t n, uint32_t* tile_counts) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kCpTile + (int64_t)warp * 32 * kCpItems;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kCpItems; ++k) {
        int64_t i = base + k * 32 + lane;
        c += __popc(__ballot_sync(kFull, i < n && p(i)));
    }
    __shared__ uint32_t ws[kCpBlock / 32];
    if (lane == 0) ws[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kCpBlock / 32; ++w) t += ws[w];
        tile_counts[blockIdx.x] = t;
    }
}

template <class Pred, class Val, class OutT>
__global__ void __launch_bounds__(kCpBlock) k_compact_write(Pred p, Val v, int64_t n, const uint64_t* tile_prefix,
                                                            OutT* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kCpTile + (int64_t)warp * 32 * kCpItems;
    unsigned bal[kCpItems];
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kCpItems; ++k) {
        int64_t i = base + k * 32 + lane;
        bal[k] = __ballot_sync(kFull, i < n && p(i));
        c += __popc(bal[k]);
    }
    __shared__ uint32_t ws[kCpBlock / 32];
    if (lane == 0) ws[warp] = c;
    __syncthreads();
    uint64_t pos = tile_prefix[blockIdx.x];
    for (int w = 0; w < warp; ++w) pos += ws[w];
#pragma unroll
    for (int k = 0; k < kCpItems; ++k) {
        int64_t i = base + k * 32 + lane;
        if ((bal[k] >> lane) & 1u) out[pos + __popc(bal[k] & lanemask_lt())] = v(i);
        pos += __popc(bal[k]);
    }
}

struct IdentityU32Scan {
    const uint32_t* v;
    __device__ uint64_t operator()(int64_t i) const { return v[i]; }
};

// Compacts {v(i) : p(i)} in index order into out.  *count_dev receives the count (device,
// inside `prefix_out` at [ntiles]); returns the device address of that count.
template <class Pred, class Val, class OutT>
tc_status compact(Pred p, Val v, int64_t n, OutT* out, Allocator* al, cudaStream_t s, uint64_t* count_host) {
    const int64_t tiles = ceil_div(n > 0 ? n : 1, kCpTile);
    DevBuf<uint32_t> tc;
    DevBuf<uint64_t> tp, scr;
    TC_TRY(tc.alloc(al, tiles, s));
    TC_TRY(tp.alloc(al, tiles + 1, s));
    TC_TRY(scr.alloc(al, scan_scratch_words(tiles), s));
    if (n > 0) {
        k_compact_counts<<<(unsigned)tiles, kCpBlock, 0, s>>>(p, n, tc.ptr);
        note_launch();
        TC_CUDA_TRY(scan_exclusive(IdentityU32Scan{tc.ptr}, tiles, tp.ptr, scr.ptr, s));
        k_compact_write<<<(unsigned)tiles, kCpBlock, 0, s>>>(p, v, n, tp.ptr, out);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
        TC_CUDA_TRY(cudaMemcpyAsync(count_host, tp.ptr + tiles, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        *count_host = 0;
    }
    return TC_OK;
}

// --------------------------------------------------------------------------- a1: canonical keys
__global__ void k_canon(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m, int32_t n,
                        int b, uint64_t sent, uint64_t* __restrict__ keys, BuildCounters* cnt, DigitCounts dc) {
    extern __shared__ unsigned dc_sh[];
    digit_counts_init(dc, dc_sh);
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i - lane < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        bool in = i < m;
        int32_t a = in ? src[i] : 0, c = in ? dst[i] : 0;
        bool bad = in && (a < 0 || a >= n || c < 0 || c >= n);
        bool loop = in && !bad && a == c;
        if (in) {
            uint64_t lo = (uint64_t)(uint32_t)(a < c ? a : c), hi = (uint64_t)(uint32_t)(a < c ? c : a);
            const uint64_t k = (bad || loop) ? sent : ((lo << b) | hi);
            keys[i] = k;
            digit_counts_add(dc, dc_sh, k);
        }
        if (bad) atomicMin(&cnt->bad_index, (long long)i);
        unsigned lb = __ballot_sync(kFull, loop);
        if (lane == 0 && lb) atomicAdd(&cnt->self_loops, (unsigned long long)__popc(lb));
    }
    digit_counts_flush(dc, dc_sh);
}

// --------------------------------------------------------------------------- a2-a4
// Degrees (a3) come in two halves.  The pass of the edge sort that completes the larger
// endpoint's bits leaves the keys ordered by it, and its writer adds one count per run of
// equal larger endpoints (duplicates included).  After the sort one pass over the keys counts
// each tile's distinct keys (a key is kept when it is not the sentinel and differs from the
// key before it), adds the kept keys' runs of equal smaller endpoints, and takes each repeated
// key back from its larger endpoint.  After a scan of the tile counts, a second pass orients
// every kept edge by the finished degrees (a4) and writes it at its compacted position,
// counting the digits of the oriented keys for the next sort.

// The larger-endpoint half one key at a time (only when the sort ran no pass: m <= 1).
__global__ void k_degree_larger(const uint64_t* __restrict__ keys, int64_t n, uint64_t sent, int b,
                                int32_t* __restrict__ deg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (keys[i] != sent) atomicAdd(&deg[(uint32_t)(keys[i] & ((1ull << b) - 1))], 1);
}

// Keys of a warp's rows and, for each, the key before it.
__device__ __forceinline__ void load_rows(const uint64_t* __restrict__ keys, int64_t base, int64_t n, uint64_t sent,
                                          int lane, uint64_t (&x)[kCpItems], uint64_t (&xp)[kCpItems]) {
#pragma unroll
    for (int k = 0; k < kCpItems; ++k) {
        const int64_t i = base + k * 32 + lane;
        x[k] = i < n ? __ldg(&keys[i]) : sent;
        xp[k] = (i > 0 && i < n) ? __ldg(&keys[i - 1]) : ~x[k];
    }
}

__global__ void __launch_bounds__(kCpBlock) k_dedupe_degree(const uint64_t* __restrict__ keys, int64_t n, uint64_t sent,
                                                            int b, int32_t* __restrict__ deg, uint32_t* tile_counts) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kCpTile + (int64_t)warp * 32 * kCpItems;
    const uint64_t mask = (1ull << b) - 1;
    uint64_t x[kCpItems], xp[kCpItems];
    load_rows(keys, base, n, sent, lane, x, xp);
    uint32_t c = 0;
    // the smaller endpoints of kept keys form runs (keys are sorted).  A hub's run covers many
    // rows, so the run still open at a row's end is carried into the next row (cv, cc, the same
    // in every lane) and added once when it closes: one atomic per run per warp, not per row.
    uint32_t cv = 0xFFFFFFFFu;
    int cc = 0;
#pragma unroll
    for (int k = 0; k < kCpItems; ++k) {
        const bool real = x[k] != sent;  // past the end, x is the sentinel
        const bool keep = real && x[k] != xp[k];
        const unsigned kb = __ballot_sync(kFull, keep);
        c += __popc(kb);
        const uint32_t a = keep ? (uint32_t)(x[k] >> b) : 0xFFFFFFFFu;
        const uint32_t pa = __shfl_up_sync(kFull, a, 1);
        const bool edge = lane == 0 || a != pa;
        const unsigned after = __ballot_sync(kFull, edge) & ~lanemask_le();
        const int end = after ? __ffs(after) - 1 : 32;
        const uint32_t a0 = __shfl_sync(kFull, a, 0), a31 = __shfl_sync(kFull, a, 31);
        const bool continues = (kb & 1u) && a0 == cv;  // lane 0's run extends the carried one
        if (!continues && cc > 0 && lane == 0) atomicAdd(&deg[cv], cc);
        const bool open = (kb >> 31) & 1u;             // the row ends inside a run of kept keys
        const unsigned heads = __ballot_sync(kFull, keep && edge);
        const int h = open ? 31 - __clz(heads) : 32;   // head of the run reaching lane 31
        if (keep && edge && lane != h) atomicAdd(&deg[a], end - lane + ((lane == 0 && continues) ? cc : 0));
        cc = open ? 32 - h + ((h == 0 && continues) ? cc : 0) : 0;
        cv = open ? a31 : 0xFFFFFFFFu;
        // repeats, counted by the sort: a run of them in the row is one key repeated (each equals
        // the key before it), taken back from its larger endpoint with one atomic per run
        const unsigned rb = __ballot_sync(kFull, real && !keep);
        if (((rb >> lane) & 1u) && (lane == 0 || !((rb >> (lane - 1)) & 1u))) {
            const unsigned rafter = ~rb & ~lanemask_le();
            const int rend = rafter ? __ffs(rafter) - 1 : 32;
            atomicSub(&deg[(uint32_t)(x[k] & mask)], rend - lane);
        }
    }
    if (cc > 0 && lane == 0) atomicAdd(&deg[cv], cc);
    __shared__ uint32_t ws[kCpBlock / 32];
    if (lane == 0) ws[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kCpBlock / 32; ++w) t += ws[w];
        tile_counts[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kCpBlock) k_orient_compact(const uint64_t* __restrict__ keys, int64_t n, uint64_t sent,
                                                             int b, const int32_t* __restrict__ deg,
                                                             const uint64_t* __restrict__ tile_prefix,
                                                             uint64_t* __restrict__ okeys, DigitCounts dc) {
    extern __shared__ unsigned dc_sh[];
    digit_counts_init(dc, dc_sh);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kCpTile + (int64_t)warp * 32 * kCpItems;
    const uint64_t mask = (1ull << b) - 1;
    uint64_t x[kCpItems], xp[kCpItems];
    load_rows(keys, base, n, sent, lane, x, xp);
    unsigned bal[kCpItems];
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kCpItems; ++k) {
        bal[k] = __ballot_sync(kFull, x[k] != sent && x[k] != xp[k]);
        c += __popc(bal[k]);
    }
    __shared__ uint32_t ws[kCpBlock / 32];
    if (lane == 0) ws[warp] = c;
    // the degrees of both endpoints of every kept key, gathered before any write
    int32_t da[kCpItems], dcn[kCpItems];
#pragma unroll
    for (int k = 0; k < kCpItems; ++k) {
        const bool keep = (bal[k] >> lane) & 1u;
        da[k] = keep ? __ldg(&deg[(uint32_t)(x[k] >> b)]) : 0;
        dcn[k] = keep ? __ldg(&deg[(uint32_t)(x[k] & mask)]) : 0;
    }
    __syncthreads();
    uint64_t pos = tile_prefix[blockIdx.x];
    for (int w = 0; w < warp; ++w) pos += ws[w];
#pragma unroll
    for (int k = 0; k < kCpItems; ++k) {
        if ((bal[k] >> lane) & 1u) {
            const uint32_t a = (uint32_t)(x[k] >> b), cc = (uint32_t)(x[k] & mask);
            // u < v iff d_u < d_v or (d_u = d_v and u < v): a < cc, so a comes first unless
            // its degree is larger
            const uint64_t o = da[k] <= dcn[k] ? x[k] : (((uint64_t)cc << b) | a);
            okeys[pos + __popc(bal[k] & lanemask_lt())] = o;
            digit_counts_add(dc, dc_sh, o);
        }
        pos += __popc(bal[k]);
    }
    digit_counts_flush(dc, dc_sh);
}

// --------------------------------------------------------------------------- a5: N+ lists
// One pass over the oriented keys, sorted by owner: the lists are the keys' low bits in this
// order (cols[i] is the partner of key i), and d_hat counts each owner's run of keys (the
// first lane of each run within a warp adds the run's length).
__global__ void k_lists(const uint64_t* __restrict__ okeys, int64_t mh, int b, int32_t* __restrict__ dhat,
                        int32_t* __restrict__ cols) {
    const uint64_t mask = (1ull << b) - 1;
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i - lane < mh;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool in = i < mh;
        const uint64_t k = in ? okeys[i] : 0ull;
        const uint32_t v = in ? (uint32_t)(k >> b) : 0xFFFFFFFFu;
        if (in) cols[i] = (int32_t)(k & mask);
        const uint32_t prev = __shfl_up_sync(kFull, v, 1);
        const bool head = in && (lane == 0 || v != prev);
        const unsigned heads = __ballot_sync(kFull, head);
        const int n_in = __popc(__ballot_sync(kFull, in));  // valid lanes are 0 .. n_in - 1
        const unsigned after = heads & ~lanemask_le();
        const int run_end = after ? __ffs(after) - 1 : n_in;
        if (head) atomicAdd(&dhat[v], run_end - lane);
    }
}

struct DhatVal {
    const int32_t* d;
    __device__ uint64_t operator()(int64_t i) const { return (uint64_t)d[i]; }
};

__global__ void k_max_deg(const int32_t* __restrict__ deg, const int32_t* __restrict__ dhat, int32_t n,
                          BuildCounters* cnt) {
    int md = 0, mh = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        md = max(md, deg[i]);
        mh = max(mh, dhat[i]);
    }
    md = warp_max(md);
    mh = warp_max(mh);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&cnt->max_degree, md);
        atomicMax(&cnt->max_dhat, mh);
    }
}

// --------------------------------------------------------------------------- tasks
// Owners are renumbered so that the task order (class, owner, position) becomes an order on
// one number: small-class vertices (list of at most small_max entries) first, then the big
// ones, each in id order; a dropped task (partner list empty) gets n and sorts last.  With
// n <= 2^24 the sort key is 24 bits (three digit passes).
struct BigVal {
    const int32_t* dhat;
    int small_max;
    __device__ uint64_t operator()(int64_t v) const { return dhat[v] > small_max ? 1ull : 0ull; }
};

// rid[v] = v's number; inv[rid[v]] = v.  big_excl: exclusive prefix of the big flags (n + 1).
__global__ void k_renumber(const int32_t* __restrict__ dhat, int small_max, const uint64_t* __restrict__ big_excl,
                           int32_t n, uint32_t* __restrict__ rid, uint32_t* __restrict__ inv) {
    const uint32_t ns = (uint32_t)((uint64_t)n - big_excl[n]);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t be = (uint32_t)big_excl[v];
        const uint32_t r = dhat[v] > small_max ? ns + be : (uint32_t)v - be;
        rid[v] = r;
        inv[r] = (uint32_t)v;
    }
}

// Task key: partner in the low 32 bits, the owner's number above.  The stable sort on the
// number alone keeps each owner's tasks in the order of their oriented edges in the lists.
__global__ void k_task_keys(const uint64_t* __restrict__ okeys, int64_t mh, int b,
                            const int32_t* __restrict__ dhat, int small_max, const uint32_t* __restrict__ rid,
                            int32_t n, uint64_t* __restrict__ tkeys, BuildCounters* cnt, DigitCounts dcn) {
    extern __shared__ unsigned dc_sh[];
    digit_counts_init(dcn, dc_sh);
    const int lane = threadIdx.x & 31;
    unsigned long long sv = 0, su = 0, ss = 0, nt = 0, nsm = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < mh; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ok = okeys[i];
        const uint32_t v = (uint32_t)(ok >> b);
        const uint32_t u = (uint32_t)(ok & ((1ull << b) - 1ull));
        int32_t dv = dhat[v], du = dhat[u];
        uint32_t o = dv >= du ? v : u, p = dv >= du ? u : v;
        int32_t dp = dv >= du ? du : dv;
        sv += (unsigned long long)dv;
        su += (unsigned long long)du;
        const int32_t dop = dv >= du ? dv : du;
        const bool big = dop > small_max;
        uint64_t num = (uint64_t)(uint32_t)n;
        if (dp > 0) {
            ss += (unsigned long long)dp;
            nt += 1;
            nsm += big ? 0ull : 1ull;
            num = rid[o];
        }
        const uint64_t key = (num << 32) | p;
        tkeys[i] = key;
        digit_counts_add(dcn, dc_sh, key);
    }
    digit_counts_flush(dcn, dc_sh);
    sv = warp_sum(sv);
    su = warp_sum(su);
    ss = warp_sum(ss);
    nt = warp_sum(nt);
    nsm = warp_sum(nsm);
    if (lane == 0) {
        if (sv) atomicAdd(&cnt->sum_dhat_v, sv);
        if (su) atomicAdd(&cnt->sum_dhat_u, su);
        if (ss) atomicAdd(&cnt->sum_stream, ss);
        if (nt) atomicAdd(&cnt->tasks, nt);
        if (nsm) atomicAdd(&cnt->tasks_small, nsm);
    }
}

// First task of each big-class owner.  The records kernel writes it at the owner's number
// (start[num] = t where the owner number changes, t >= Ts); the numbers that got one are then
// compacted in number order, which is the big class's task order.
struct OwnerStartPred {
    const uint32_t* start;
    __device__ bool operator()(int64_t i) const { return start[i] != 0xFFFFFFFFu; }
};
struct OwnerStartVal {
    const uint32_t* start;
    __device__ uint32_t operator()(int64_t i) const { return start[i]; }
};

__global__ void k_task_records(const uint64_t* __restrict__ tkeys, int64_t T, int64_t Ts,
                               const uint32_t* __restrict__ inv, const int64_t* __restrict__ off,
                               TaskRec* __restrict__ rec, uint32_t* __restrict__ start) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = tkeys[t];
        const uint32_t num = (uint32_t)(k >> 32);
        if (t >= Ts && (t == Ts || (uint32_t)(tkeys[t - 1] >> 32) != num)) start[num] = (uint32_t)t;
        uint32_t o = inv[num], p = (uint32_t)(k & 0xFFFFFFFFu);
        int64_t s = off[p], e = off[p + 1];
        TaskRec r;
        r.owner = o;
        r.partner = p;
        r.pstart = (uint32_t)s;
        r.plen = (uint32_t)(e - s);
        rec[t] = r;
    }
}

// --------------------------------------------------------------------------- driver

static int bits_for(int32_t n) {
    uint32_t maxid = n > 1 ? (uint32_t)(n - 1) : 1u;
    int b = 32 - __builtin_clz(maxid);
    return b < 1 ? 1 : b;
}

constexpr int kMaxSortPasses = 8;  // 64-bit keys
static int sort_passes(int nbits) { return (nbits + 7) / 8; }

static tc_status zero_counts(const DigitCounts& dc, cudaStream_t s) {
    TC_CUDA_TRY(cudaMemsetAsync(dc.global, 0, sizeof(unsigned long long) * dc.npass * 256, s));
    return TC_OK;
}

static unsigned grid_stride_blocks(int64_t n) {
    int64_t want = ceil_div(n > 0 ? n : 1, kThreads);
    int64_t cap = (int64_t)num_sms() * 16;
    return (unsigned)(want < cap ? want : cap);
}

// Grid of a kernel that also counts its keys' digits: one wave of fully resident blocks, so
// that few blocks add their shared counts to the global ones.
static unsigned count_blocks(int64_t n) {
    int64_t want = ceil_div(n > 0 ? n : 1, kThreads);
    int64_t cap = (int64_t)num_sms() * (2048 / kThreads);
    return (unsigned)(want < cap ? want : cap);
}

// Synchronise and return the handle's device error word (set by a bounded wait that gave up).
static tc_status check_device_error(tc_graph* g, cudaStream_t s) {
    DevStatus h;
    TC_CUDA_TRY(cudaMemcpyAsync(&h, g->status, sizeof(h), cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    return h.code != 0 ? (tc_status)h.code : TC_OK;
}

tc_status build_graph(tc_graph* g, const int32_t* src, const int32_t* dst, int64_t m, int32_t n, cudaStream_t s) {
    Allocator* al = &g->al;
    const long long spin = g->opt.retry_limit > 0 ? g->opt.retry_limit : (1ll << 20);
    const int b = bits_for(n);
    if (b > 30) return TC_ERR_UNSUPPORTED;  // edge keys hold 2b bits, task keys 32 + bits(n)
    const int nbits = 2 * b;
    const uint64_t sent = (nbits >= 64) ? ~0ull : ((1ull << nbits) - 1);
    g->n = n;
    g->id_bits = b;
    g->m_in = m;

    DevBuf<BuildCounters> cnt;
    TC_TRY(cnt.alloc(al, 1, s));
    {
        BuildCounters init{};
        init.bad_index = LLONG_MAX;
        TC_CUDA_TRY(cudaMemcpyAsync(cnt.ptr, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    }
    DevBuf<uint64_t> ka, kb;
    TC_TRY(ka.alloc(al, m > 0 ? m : 1, s));
    TC_TRY(kb.alloc(al, m > 0 ? m : 1, s));

    // digit counts of each sort's keys, gathered by the kernel that writes them
    DevBuf<unsigned long long> counts;
    TC_TRY(counts.alloc(al, (size_t)kMaxSortPasses * 256, s));

    // a1
    unsigned long long* const ucounts = counts.ptr;
    if (m > 0) {
        const DigitCounts dc{ucounts, 0, sort_passes(nbits)};
        TC_TRY(zero_counts(dc, s));
        k_canon<<<count_blocks(m), kThreads, digit_counts_bytes(dc), s>>>(src, dst, m, n, b, sent, ka.ptr, cnt.ptr,
                                                                          dc);
        note_launch();
    }
    TC_CUDA_TRY(cudaGetLastError());
    // a2, with the larger-endpoint half of a3 counted by the pass that completes those bits
    DevBuf<int32_t> deg, dhat;
    TC_TRY(deg.alloc(al, n > 0 ? n : 1, s));
    TC_TRY(dhat.alloc(al, n > 0 ? n : 1, s));
    TC_CUDA_TRY(cudaMemsetAsync(deg.ptr, 0, sizeof(int32_t) * (n > 0 ? n : 1), s));
    TC_CUDA_TRY(cudaMemsetAsync(dhat.ptr, 0, sizeof(int32_t) * (n > 0 ? n : 1), s));
    OsOut larger;
    larger.mode = OS_OUT_RUNS;
    larger.pass = sort_passes(b) - 1;
    larger.fshift = 0;
    larger.fmask = (1ull << b) - 1;
    larger.skip = sent;
    larger.cnt = deg.ptr;
    larger.nvert = (uint32_t)n;
    uint64_t* sorted = nullptr;
    bool larger_done = false;
    TC_TRY(radix_sort_u64(ka.ptr, kb.ptr, m, 0, nbits, al, s, &sorted, g->status, spin, m > 0 ? ucounts : nullptr,
                          &larger, &larger_done));
    TC_TRY(check_device_error(g, s));  // the sorted keys are read only if every wait of the sort ended
    uint64_t* other = sorted == ka.ptr ? kb.ptr : ka.ptr;
    if (m > 0 && !larger_done) {
        k_degree_larger<<<grid_stride_blocks(m), kThreads, 0, s>>>(sorted, m, sent, b, deg.ptr);
        note_launch();
    }
    const int64_t ctiles = ceil_div(m > 0 ? m : 1, kCpTile);
    DevBuf<uint32_t> tcount;
    DevBuf<uint64_t> tprefix, tscr;
    TC_TRY(tcount.alloc(al, ctiles, s));
    TC_TRY(tprefix.alloc(al, ctiles + 1, s));
    TC_TRY(tscr.alloc(al, scan_scratch_words(ctiles), s));
    uint64_t mh64 = 0;
    if (m > 0) {
        k_dedupe_degree<<<(unsigned)ctiles, kCpBlock, 0, s>>>(sorted, m, sent, b, deg.ptr, tcount.ptr);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
        TC_CUDA_TRY(scan_exclusive(IdentityU32Scan{tcount.ptr}, ctiles, tprefix.ptr, tscr.ptr, s));
        TC_CUDA_TRY(cudaMemcpyAsync(&mh64, tprefix.ptr + ctiles, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    }
    BuildCounters hc;
    TC_CUDA_TRY(cudaMemcpyAsync(&hc, cnt.ptr, sizeof(hc), cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    if (hc.bad_index != LLONG_MAX) {
        g->self_loops = (int64_t)hc.self_loops;
        g->bad_index = (int64_t)hc.bad_index;
        return TC_ERR_VERTEX_RANGE;
    }
    const int64_t mh = (int64_t)mh64;
    g->m_hat = mh;
    g->self_loops = (int64_t)hc.self_loops;
    g->duplicates = m - g->self_loops - mh;
    if (g->opt.input_policy == TC_INPUT_STRICT && (g->self_loops > 0 || g->duplicates > 0)) return TC_ERR_INVALID_ARG;
    if (mh >= (int64_t)0xFFFFFFFFll) return TC_ERR_UNSUPPORTED;  // task records index lists with uint32
    // a4: orient the distinct edges into the other key buffer, compacted
    uint64_t* okeys = other;
    uint64_t* spare = sorted;  // free buffer of m keys
    if (mh > 0) {
        const DigitCounts dc{ucounts, b, sort_passes(b)};
        TC_TRY(zero_counts(dc, s));
        k_orient_compact<<<(unsigned)ctiles, kCpBlock, digit_counts_bytes(dc), s>>>(sorted, m, sent, b, deg.ptr,
                                                                                   tprefix.ptr, okeys, dc);
        note_launch();
    }
    TC_CUDA_TRY(cudaGetLastError());
    tcount.release();
    tprefix.release();
    tscr.release();
    // a5: group the oriented edges by owner.  The distinct keys arrive sorted by (min, max),
    // so a stable sort on the owner bits alone leaves every list ascending: an owner v's
    // partners below v come from earlier runs (keys (u, v), u ascending), its partners above v
    // from v's own run (keys (v, x), x ascending), in that order.  The last pass also writes
    // the lists (cols) and counts each owner's entries (d^).
    DevBuf<int64_t> off;
    DevBuf<int32_t> cols;
    TC_TRY(off.alloc(al, (size_t)n + 1, s));
    TC_TRY(cols.alloc(al, (size_t)(mh > 0 ? mh : 1) + 4, s));  // +4: 16-byte vector reads may run past the end
    OsOut lists_out;
    lists_out.mode = OS_OUT_LISTS;
    lists_out.b = b;
    lists_out.cols = cols.ptr;
    lists_out.fshift = b;
    lists_out.cnt = dhat.ptr;
    lists_out.nvert = (uint32_t)n;
    uint64_t* osorted = nullptr;
    bool lists_done = false;
    TC_TRY(radix_sort_u64(okeys, spare, mh, b, b, al, s, &osorted, g->status, spin, mh > 0 ? ucounts : nullptr,
                          &lists_out, &lists_done));
    TC_TRY(check_device_error(g, s));
    uint64_t* free_buf = osorted == okeys ? spare : okeys;
    if (mh > 0 && !lists_done) {
        k_lists<<<grid_stride_blocks(mh), kThreads, 0, s>>>(osorted, mh, b, dhat.ptr, cols.ptr);
        note_launch();
    }
    {
        // offsets = exclusive scan of dhat (values < 2^63, so the uint64 scan is the int64 array)
        DevBuf<uint64_t> scr;
        TC_TRY(scr.alloc(al, scan_scratch_words(n), s));
        TC_CUDA_TRY(scan_exclusive(DhatVal{dhat.ptr}, n, reinterpret_cast<uint64_t*>(off.ptr), scr.ptr, s));
    }
    if (n > 0) {
        k_max_deg<<<grid_stride_blocks(n), kThreads, 0, s>>>(deg.ptr, dhat.ptr, n, cnt.ptr);
        note_launch();
    }
    TC_CUDA_TRY(cudaGetLastError());

    // tasks
    DevBuf<uint32_t> rid, inv;
    TC_TRY(rid.alloc(al, (size_t)(n > 0 ? n : 1), s));
    TC_TRY(inv.alloc(al, (size_t)(n > 0 ? n : 1), s));
    if (n > 0) {
        DevBuf<uint64_t> bex, scr;
        TC_TRY(bex.alloc(al, (size_t)n + 1, s));
        TC_TRY(scr.alloc(al, scan_scratch_words(n), s));
        TC_CUDA_TRY(scan_exclusive(BigVal{dhat.ptr, g->opt.small_max}, n, bex.ptr, scr.ptr, s));
        k_renumber<<<grid_stride_blocks(n), kThreads, 0, s>>>(dhat.ptr, g->opt.small_max, bex.ptr, n, rid.ptr, inv.ptr);
        note_launch();
    }
    const int task_bits = bits_for(n + 1);
    if (mh > 0) {
        const DigitCounts dc{ucounts, 32, sort_passes(task_bits)};
        TC_TRY(zero_counts(dc, s));
        k_task_keys<<<count_blocks(mh), kThreads, digit_counts_bytes(dc), s>>>(
            osorted, mh, b, dhat.ptr, g->opt.small_max, rid.ptr, n, free_buf, cnt.ptr, dc);
        note_launch();
    }
    TC_CUDA_TRY(cudaGetLastError());
    TC_CUDA_TRY(cudaMemcpyAsync(&hc, cnt.ptr, sizeof(hc), cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t T = (int64_t)hc.tasks;
    DevBuf<TaskRec> rec;
    TC_TRY(rec.alloc(al, T > 0 ? T : 1, s));
    uint64_t* tsorted = nullptr;
    TC_TRY(radix_sort_u64(free_buf, osorted, mh, 32, task_bits, al, s, &tsorted, g->status, spin,
                          mh > 0 ? ucounts : nullptr));
    TC_TRY(check_device_error(g, s));
    // owner numbers run over [0, n]; start[num] receives the first task of big owner num
    DevBuf<uint32_t> start;
    TC_TRY(start.alloc(al, (size_t)n + 1, s));
    TC_CUDA_TRY(cudaMemsetAsync(start.ptr, 0xFF, sizeof(uint32_t) * ((size_t)n + 1), s));
    if (T > 0) {
        k_task_records<<<grid_stride_blocks(T), kThreads, 0, s>>>(tsorted, T, (int64_t)hc.tasks_small, inv.ptr,
                                                                   off.ptr, rec.ptr, start.ptr);
        note_launch();
    }
    TC_CUDA_TRY(cudaGetLastError());

    g->tasks = T;
    g->tasks_small = (int64_t)hc.tasks_small;
    // first task of every big owner, plus T at the end
    {
        const int64_t nb = T - g->tasks_small;
        DevBuf<uint32_t> of;
        TC_TRY(of.alloc(al, (size_t)(nb + 1), s));
        uint64_t k = 0;
        TC_TRY(compact(OwnerStartPred{start.ptr}, OwnerStartVal{start.ptr}, (int64_t)n + 1, of.ptr, al, s, &k));
        const uint32_t endv = (uint32_t)T;
        TC_CUDA_TRY(cudaMemcpyAsync(of.ptr + k, &endv, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        g->owners_big = (int64_t)k;
        g->own_first_cap = (int64_t)(nb + 1);
        g->own_first = of.detach();
    }
    g->max_degree = hc.max_degree;
    g->max_dhat = hc.max_dhat;
    g->sum_dhat_v = hc.sum_dhat_v;
    g->sum_dhat_u = hc.sum_dhat_u;
    g->sum_stream = hc.sum_stream;
    // hand the arrays to the handle; the key buffers and counters are released here
    g->deg = deg.detach();
    g->off = off.detach();
    g->cols = cols.detach();
    g->trec = rec.detach();
    g->bytes = (int64_t)align_up((size_t)(n > 0 ? n : 1) * 4, 256) + (int64_t)align_up(((size_t)n + 1) * 8, 256) +
               (int64_t)align_up(((size_t)(mh > 0 ? mh : 1) + 4) * 4, 256) +
               (int64_t)align_up((size_t)(T > 0 ? T : 1) * sizeof(TaskRec), 256) +
               (int64_t)align_up((size_t)g->own_first_cap * 4, 256);
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    return TC_OK;
}

}  // namespace tcg

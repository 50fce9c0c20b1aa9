// count.cu -- steps a6-a8: task costs and their prefix, the Eq. 1 / Eq. 2 schedule, the
// persistent intersection kernel and the exact reduction.
//
// Work unit.  Fig. 1 sums |N_v ∩ N_u| over oriented edges (v,u).  Each oriented edge is one
// task owned by the endpoint whose list is longer; the owner's list is staged once into a
// per-warp open-addressing hash table in shared memory, and the partner lists of all the
// owner's tasks are streamed through it, 32 list entries per warp step.  So each edge costs
// min(|N_v|, |N_u|) streamed entries instead of the |N_v| + |N_u| of a merge (Sec. III-A).
//
// Schedule (Sec. V-B).  The persistent grid has W warps ("workers").  Task costs are
// prefix-summed (uint64).  The first H = floor(C * static_percent / 100) cost units (Eq. 1,
// default one half) are split into W equal initial chunks, one per warp, taken without any
// coordination; the rest is handed out by a compare-and-swap on a device head: each pop
// takes max(min_chunk, floor((C - head) / W)) (Eq. 2), so chunks shrink as the work drains.
// A cost boundary maps to the first task whose exclusive prefix reaches it.
//
// Reduction.  Each warp sums its hits in registers, then one uint64 atomicAdd per warp:
// exact and independent of order.
#include "graph.cuh"
#include "scan.cuh"

namespace tcg {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kHashMul = 0x9E3779B1u;  // Knuth's multiplicative constant, 2^32 / golden ratio
constexpr int kUnroll = 4;                   // list windows of 32 entries loaded before probing

struct CountArgs {
    const int64_t* off;
    const int32_t* cols;
    const TaskRec* tasks;
    long long T;
    const int32_t* deg;
    const uint64_t* P;  // T + 1 exclusive prefix of task costs
    Sched* sched;
    long long W;
    int piece;
    int table_slots;
    int warps_per_block;
    unsigned long long* total;
    unsigned long long* t_v;
    uint32_t* per_edge;
    uint64_t* trace_chunks;
    long long trace_cap;
    uint64_t* trace_busy;
    DevStatus* status;
    long long retry_limit;
};

// First t in [0, T] with P[t] >= x, given P[T] >= x.  32-way search: each round every lane
// samples one position and the warp keeps the gap between the last sample below x and the
// first at or above it.
__device__ __forceinline__ long long warp_lower_bound(const uint64_t* __restrict__ P, long long T,
                                                      unsigned long long x, int lane) {
    long long lo = 0, hi = T;  // invariant: P[lo-1] < x (or lo = 0), P[hi] >= x
    while (hi - lo > 31) {
        const long long step = (hi - lo + 31) / 32;
        long long q = lo + (long long)lane * step;
        if (q > hi) q = hi;
        const unsigned b = __ballot_sync(kFull, P[q] >= x);
        if (b == 0) {
            long long q31 = lo + 31 * step;
            lo = (q31 > hi ? hi : q31) + 1;
        } else {
            const int f = __ffs(b) - 1;
            if (f == 0) return lo;
            long long qf = lo + (long long)f * step;
            hi = qf > hi ? hi : qf;
            lo = lo + (long long)(f - 1) * step + 1;
        }
    }
    const long long q = lo + lane;
    const unsigned b = __ballot_sync(kFull, q <= hi ? (P[q] >= x) : true);
    return lo + (__ffs(b) - 1);
}

__device__ __forceinline__ long long map_bound(const CountArgs& a, unsigned long long x, unsigned long long C,
                                               int lane) {
    return x >= C ? a.T : warp_lower_bound(a.P, a.T, x, lane);
}

// Position of u in the sorted list N+(v).
__device__ __forceinline__ long long edge_position(const CountArgs& a, uint32_t v, uint32_t u) {
    long long lo = a.off[v], hi = a.off[v + 1];
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if ((uint32_t)a.cols[mid] < u) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <bool EXTRA>
__device__ __forceinline__ void on_hit(const CountArgs& a, uint32_t owner, uint32_t partner, uint32_t w) {
    if (!EXTRA) return;
    if (a.t_v) {
        atomicAdd(&a.t_v[owner], 1ull);
        atomicAdd(&a.t_v[partner], 1ull);
        atomicAdd(&a.t_v[w], 1ull);
    }
    if (a.per_edge) {
        // the oriented edge runs from whichever endpoint comes first in the degree order
        const int32_t dox = a.deg[owner], dpx = a.deg[partner];
        const bool owner_first = dox < dpx || (dox == dpx && owner < partner);
        const uint32_t v = owner_first ? owner : partner, u = owner_first ? partner : owner;
        atomicAdd(&a.per_edge[edge_position(a, v, u)], 1u);
    }
}

// Count the tasks [t0, t1) (uniform across the warp).
template <bool EXTRA>
__device__ void process_range(const CountArgs& a, long long t0, long long t1, uint32_t* __restrict__ tbl, int lane,
                              unsigned long long& acc) {
    long long t = t0;
    while (t < t1) {
        const uint32_t owner = a.tasks[t].owner;
        const long long obase = a.off[owner];
        const uint32_t olen = (uint32_t)(a.off[owner + 1] - obase);
        long long seg_end = -1;  // end of this owner's tasks, found while probing the first piece
        for (uint32_t ps = 0; ps < olen; ps += (uint32_t)a.piece) {
            const uint32_t pl = min((uint32_t)a.piece, olen - ps);
            uint32_t cap = 64;
            while (cap < 2 * pl) cap <<= 1;
            const int shift = 33 - __ffs(cap);  // 32 - log2(cap)
            const uint32_t cmask = cap - 1;
            // stage the piece N+(owner)[ps, ps + pl) into the table
            for (uint32_t i = lane; i < cap; i += 32) tbl[i] = kEmpty;
            __syncwarp();
            for (uint32_t i = lane; i < pl; i += 32) {
                const uint32_t x = (uint32_t)__ldg(&a.cols[obase + ps + i]);
                uint32_t h = (x * kHashMul) >> shift;
                while (atomicCAS(&tbl[h], kEmpty, x) != kEmpty) h = (h + 1) & cmask;
            }
            __syncwarp();
            // stream the partner lists of the owner's tasks, 32 tasks per batch
            long long tt = t;
            for (;;) {
                const long long lim = seg_end >= 0 ? seg_end : t1;
                if (tt >= lim) break;
                const long long j = tt + lane;
                TaskRec r = {0u, 0u, 0u, 0u};
                bool valid = false;
                if (j < lim) {
                    r = a.tasks[j];
                    valid = seg_end >= 0 || r.owner == owner;
                }
                const unsigned vb = __ballot_sync(kFull, valid);
                const int nb = (vb == kFull) ? 32 : __ffs(~vb) - 1;  // leading run of this owner's tasks
                const uint32_t len = lane < nb ? r.plen : 0u;
                const uint32_t start = r.pstart;
                const uint32_t incl = warp_inclusive_scan(len, lane);
                const uint32_t excl = incl - len;
                const uint32_t tot = __shfl_sync(kFull, incl, 31);
                uint32_t before = 0;  // tasks of the batch that start before the current window
                for (uint32_t base = 0; base < tot; base += 32 * kUnroll) {
                    uint32_t wv[kUnroll];
                    bool ok[kUnroll];
                    int qj[kUnroll];
#pragma unroll
                    for (int uu = 0; uu < kUnroll; ++uu) {
                        const uint32_t wb = base + 32u * uu;
                        const uint32_t rel = excl - wb;
                        const uint32_t bit = (len != 0u && rel < 32u) ? (1u << rel) : 0u;
                        const uint32_t starts = __reduce_or_sync(kFull, bit);
                        const int q = ((int)(before + __popc(starts & lanemask_le())) - 1) & 31;
                        const uint32_t sj = __shfl_sync(kFull, start, q);
                        const uint32_t ej = __shfl_sync(kFull, excl, q);
                        const uint32_t g = wb + lane;
                        ok[uu] = g < tot;
                        wv[uu] = ok[uu] ? (uint32_t)__ldg(&a.cols[(long long)sj + (g - ej)]) : 0u;
                        qj[uu] = q;
                        before += __popc(starts);
                    }
#pragma unroll
                    for (int uu = 0; uu < kUnroll; ++uu) {
                        bool hit = false;
                        if (ok[uu]) {
                            const uint32_t w = wv[uu];
                            uint32_t h = (w * kHashMul) >> shift;
                            for (;;) {
                                const uint32_t s = tbl[h];
                                if (s == w) { hit = true; break; }
                                if (s == kEmpty) break;
                                h = (h + 1) & cmask;
                            }
                        }
                        acc += hit ? 1ull : 0ull;
                        if (EXTRA) {
                            const uint32_t pj = __shfl_sync(kFull, r.partner, qj[uu]);
                            if (hit) on_hit<EXTRA>(a, owner, pj, wv[uu]);
                        }
                    }
                }
                if (nb < 32) {
                    seg_end = tt + nb;
                    break;
                }
                tt += 32;
            }
            if (seg_end < 0) seg_end = t1;
            __syncwarp();
        }
        t = seg_end;
    }
}

template <bool EXTRA>
__global__ void __launch_bounds__(512) k_count(CountArgs a) {
    extern __shared__ uint32_t smem_tbl[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long wid = (long long)blockIdx.x * a.warps_per_block + wib;
    uint32_t* tbl = smem_tbl + (size_t)wib * a.table_slots;
    const unsigned long long C = a.sched->C, H = a.sched->H, minc = a.sched->min_chunk;
    const unsigned long long W = (unsigned long long)a.W;
    unsigned long long acc = 0;
    long long busy = 0, nch = 0;
    if (wid < a.W) {
        // Eq. 1: the initial share split into W parts of equal cost
        const unsigned long long q = H / W, r = H % W, w0 = (unsigned long long)wid;
        const unsigned long long lo = w0 * q + (w0 < r ? w0 : r);
        const unsigned long long hi = (w0 + 1) * q + (w0 + 1 < r ? w0 + 1 : r);
        long long t0 = wid == 0 ? 0 : map_bound(a, lo, C, lane);
        long long t1 = map_bound(a, hi, C, lane);
        long long c0 = clock64();
        if (a.trace_chunks && lane == 0) {
            unsigned long long idx = atomicAdd(&a.sched->n_chunks, 1ull);
            if ((long long)idx < a.trace_cap) {
                a.trace_chunks[4 * idx] = lo;
                a.trace_chunks[4 * idx + 1] = hi;
                a.trace_chunks[4 * idx + 2] = (uint64_t)t0;
                a.trace_chunks[4 * idx + 3] = (uint64_t)t1;
            }
        }
        process_range<EXTRA>(a, t0, t1, tbl, lane, acc);
        busy += clock64() - c0;
        ++nch;
        // Eq. 2: guided chunks of the remaining cost
        for (;;) {
            unsigned long long c = 0, e = 0;
            int got = 0;
            if (lane == 0) {
                c = *(volatile unsigned long long*)&a.sched->head;
                for (long long tries = 0;; ++tries) {
                    if (c >= C) break;
                    unsigned long long sz = (C - c) / W;
                    if (sz < minc) sz = minc;
                    e = (C - c > sz) ? c + sz : C;
                    const unsigned long long old = atomicCAS(&a.sched->head, c, e);
                    if (old == c) {
                        got = 1;
                        break;
                    }
                    c = old;
                    if (tries >= a.retry_limit) {
                        set_error(a.status, TC_ERR_TIMEOUT, tries);
                        break;
                    }
                }
            }
            got = __shfl_sync(kFull, got, 0);
            if (!got) break;
            c = __shfl_sync(kFull, c, 0);
            e = __shfl_sync(kFull, e, 0);
            t0 = map_bound(a, c, C, lane);
            t1 = map_bound(a, e, C, lane);
            c0 = clock64();
            if (a.trace_chunks && lane == 0) {
                unsigned long long idx = atomicAdd(&a.sched->n_chunks, 1ull);
                if ((long long)idx < a.trace_cap) {
                    a.trace_chunks[4 * idx] = c;
                    a.trace_chunks[4 * idx + 1] = e;
                    a.trace_chunks[4 * idx + 2] = (uint64_t)t0;
                    a.trace_chunks[4 * idx + 3] = (uint64_t)t1;
                }
            }
            process_range<EXTRA>(a, t0, t1, tbl, lane, acc);
            busy += clock64() - c0;
            ++nch;
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) {
        if (acc) atomicAdd(a.total, acc);
        if (a.trace_busy && wid < a.W) {
            a.trace_busy[2 * wid] = (uint64_t)busy;
            a.trace_busy[2 * wid + 1] = (uint64_t)nch;
        }
    }
}

// --------------------------------------------------------------------------- costs (a6)

struct TaskCost {
    const TaskRec* tasks;
    long long T;
    const int64_t* off;
    const uint64_t* f;
    int model;
    uint32_t piece, c_task, c_owner;
    __device__ uint64_t operator()(int64_t t) const {
        const TaskRec r = tasks[t];
        const bool last = (t + 1 == T) || tasks[t + 1].owner != r.owner;
        if (model == TC_COST_EDGE) {
            const uint64_t dho = (uint64_t)(off[r.owner + 1] - off[r.owner]);
            const uint64_t pieces = (dho + piece - 1) / piece;
            uint64_t c = pieces * ((uint64_t)r.plen + c_task);
            if (last) c += dho + c_owner;
            return c;
        }
        if (model == TC_COST_MERGE) return (uint64_t)(off[r.owner + 1] - off[r.owner]) + (uint64_t)r.plen;
        return last ? f[r.owner] : 0ull;  // per-vertex models: the owner's cost on its last task
    }
};

__global__ void k_sched_init(Sched* sc, const uint64_t* P, long long T, long long W, int static_percent,
                             long long min_chunk) {
    const unsigned long long C = P[T];
    const unsigned long long sp = (unsigned long long)static_percent;
    const unsigned long long H = (C / 100ull) * sp + ((C % 100ull) * sp) / 100ull;
    unsigned long long minc = (unsigned long long)min_chunk;
    if (min_chunk <= 0) {
        minc = C / ((unsigned long long)W * 128ull);
        if (minc < 32ull) minc = 32ull;
    }
    sc->C = C;
    sc->H = H;
    sc->min_chunk = minc;
    sc->head = H;
    sc->n_chunks = 0;
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
    if (!w.sched) {
        void* p = nullptr;
        TC_TRY(g->al.get(&p, sizeof(Sched) + 64, s));
        w.sched = (Sched*)p;
        g->bytes += (int64_t)align_up(sizeof(Sched) + 64, 256);
    }
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

template <bool EXTRA>
static tc_status launch_count(const CountArgs& a, int blocks, int threads, size_t smem, cudaStream_t s) {
    k_count<EXTRA><<<blocks, threads, smem, s>>>(a);
    note_launch();
    TC_CUDA_TRY(cudaGetLastError());
    return TC_OK;
}

tc_status count_enqueue(tc_graph* g, const tc_options& opt, cudaStream_t s, unsigned long long* total_dev,
                        unsigned long long* t_v, uint32_t* per_edge, tc_count_trace* trace) {
    TC_TRY(ensure_count_work(g, opt, s));
    CountWork& w = g->work;
    const bool extra = t_v != nullptr || per_edge != nullptr;
    const int wpb = opt.warps_per_block;
    const int threads = wpb * 32;
    const int table_slots = 2 * opt.piece;
    const size_t smem = (size_t)wpb * table_slots * sizeof(uint32_t);
    // occupancy decides the persistent grid
    int per_sm = 0;
    if (extra) {
        TC_CUDA_TRY(cudaFuncSetAttribute(k_count<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        TC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count<true>, threads, smem));
    } else {
        TC_CUDA_TRY(cudaFuncSetAttribute(k_count<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        TC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count<false>, threads, smem));
    }
    if (per_sm < 1) return TC_ERR_INVALID_ARG;
    if (opt.blocks_per_sm > 0 && opt.blocks_per_sm < per_sm) per_sm = opt.blocks_per_sm;
    const int blocks = num_sms() * per_sm;
    const long long W = (long long)blocks * wpb;

    // events around the two phases when a trace is requested (on the launching stream)
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (trace) {
        for (auto& e : ev) TC_CUDA_TRY(cudaEventCreate(&e));
        TC_CUDA_TRY(cudaEventRecord(ev[0], s));
    }
    // a6: costs, prefix, schedule state
    if (opt.cost_model >= TC_COST_ONE) {
        const int fn = opt.cost_model - TC_COST_ONE;  // ONE, DEGREE, PATRIC, NEW in enum order
        TC_TRY(vertex_cost_enqueue(g, fn, s, w.fcost));
    }
    TaskCost tcf{g->trec, g->tasks, g->off, w.fcost, opt.cost_model, (uint32_t)opt.piece, (uint32_t)opt.c_task,
                 (uint32_t)opt.c_owner};
    TC_CUDA_TRY(scan_exclusive(tcf, g->tasks, w.prefix, w.scan_scr, s));
    k_sched_init<<<1, 1, 0, s>>>(w.sched, w.prefix, g->tasks, W, opt.static_percent, opt.min_chunk);
    note_launch();
    TC_CUDA_TRY(cudaGetLastError());
    TC_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(unsigned long long), s));
    if (t_v && g->n > 0) TC_CUDA_TRY(cudaMemsetAsync(t_v, 0, sizeof(unsigned long long) * g->n, s));
    if (per_edge && g->m_hat > 0) TC_CUDA_TRY(cudaMemsetAsync(per_edge, 0, sizeof(uint32_t) * g->m_hat, s));

    CountArgs a;
    a.off = g->off;
    a.cols = g->cols;
    a.tasks = g->trec;
    a.T = g->tasks;
    a.deg = g->deg;
    a.P = w.prefix;
    a.sched = w.sched;
    a.W = W;
    a.piece = opt.piece;
    a.table_slots = table_slots;
    a.warps_per_block = wpb;
    a.total = total_dev;
    a.t_v = t_v;
    a.per_edge = per_edge;
    a.trace_chunks = trace ? trace->chunks : nullptr;
    a.trace_cap = trace ? trace->cap : 0;
    a.trace_busy = trace ? trace->workers_busy : nullptr;
    a.status = g->status;
    a.retry_limit = opt.retry_limit > 0 ? opt.retry_limit : (1ll << 24);
    if (trace) TC_CUDA_TRY(cudaEventRecord(ev[1], s));
    if (g->tasks > 0) {
        if (extra) TC_TRY(launch_count<true>(a, blocks, threads, smem, s));
        else TC_TRY(launch_count<false>(a, blocks, threads, smem, s));
    }
    if (trace) {
        TC_CUDA_TRY(cudaEventRecord(ev[2], s));
        Sched hs;
        TC_CUDA_TRY(cudaMemcpyAsync(&hs, w.sched, sizeof(Sched), cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        trace->n_chunks = (int64_t)hs.n_chunks;
        trace->n_workers = W;
        trace->total_cost = hs.C;
        trace->min_chunk = hs.min_chunk;
        float ms = 0.f;
        TC_CUDA_TRY(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        trace->prefix_ms = ms;
        TC_CUDA_TRY(cudaEventElapsedTime(&ms, ev[1], ev[2]));
        trace->kernel_ms = ms;
        for (auto& e : ev) cudaEventDestroy(e);
    }
    return TC_OK;
}

}  // namespace tcg

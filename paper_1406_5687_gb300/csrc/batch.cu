// batch.cu -- batched counting: many graphs packed into disjoint unions ("packs"), each pack
// built by one pass of the single-graph pipeline.  All packs are counted together: one cost
// prefix over every pack's tasks, and per task class one schedule over the packs' concatenated
// costs and one launch of the class kernel; that count is replayed from one captured CUDA
// graph.  The autotuner times the batched count over a grid of hub thresholds and launch shapes.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <new>
#include <vector>

#include "graph.cuh"
#include "scan.cuh"

namespace tcg {

// Graph j of a pack: its edges are [ebase[j], ebase[j+1]) of the pack's edge arrays, read
// from src[j] / dst[j] (device memory, or pinned host memory read over the host link), and
// its vertices [vbase[j], vbase[j+1]) of the pack's vertex range.
struct PackMeta {
    const int64_t* ebase;            // k + 1
    const int32_t* vbase;            // k + 1
    const int32_t* const* src;       // k
    const int32_t* const* dst;       // k
    int32_t k;
};

// Gather every graph's edges into the pack's arrays, checking each id against its own
// graph's n and moving it into the graph's vertex range.  An id outside [0, n_j) records
// TC_ERR_VERTEX_RANGE with the pack-wide edge index (the build is abandoned).
__global__ void k_pack_ids(PackMeta pm, int64_t m, int32_t* __restrict__ out_src, int32_t* __restrict__ out_dst,
                           DevStatus* status) {
    int g = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        // graphs are in edge order and e only grows: step forward, else search from g
        if (pm.ebase[g + 1] <= e) {
            int lo = g, hi = pm.k - 1;  // the last graph whose first edge is at or before e
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pm.ebase[mid] <= e) lo = mid; else hi = mid - 1;
            }
            g = lo;
        }
        const int64_t l = e - pm.ebase[g];
        const int32_t vb = pm.vbase[g];
        const int32_t nj = pm.vbase[g + 1] - vb;
        const int32_t a = pm.src[g][l], b = pm.dst[g][l];
        if (a < 0 || a >= nj || b < 0 || b >= nj) {
            set_error(status, TC_ERR_VERTEX_RANGE, e);
            continue;
        }
        out_src[e] = a + vb;
        out_dst[e] = b + vb;
    }
}

// For each task class and each graph boundary j in [0, k]: the first task of the class whose
// owner is at or above vbase[j] (owners ascend within a class); and off[vbase[j]], from which
// each graph's distinct edge count follows.
__global__ void k_sub_tasks(const TaskRec* __restrict__ tasks, int64_t Ts, int64_t T, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ vbase, int32_t k, int64_t* __restrict__ sub_task,
                            int64_t* __restrict__ sub_off) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * (k + 1)) return;
    const int c = i / (k + 1), j = i % (k + 1);
    const uint32_t v = (uint32_t)vbase[j];
    int64_t lo = c == 0 ? 0 : Ts, hi = c == 0 ? Ts : T;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (tasks[mid].owner < v) lo = mid + 1; else hi = mid;
    }
    sub_task[i] = lo;
    if (c == 0) sub_off[j] = off[v];
}

constexpr int64_t kDefaultPackEdges = 1ll << 30;
constexpr int64_t kMaxPackVertices = 1ll << 30;

}  // namespace tcg

using namespace tcg;

struct tc_batch {
    int device = 0;
    tc_options opt{};
    int32_t k = 0;
    std::vector<tc_graph*> packs;
    std::vector<int32_t> first;       // first graph of each pack, then k
    std::vector<int64_t> m_hat;       // per graph
    int64_t m_in = 0;
    Allocator al;                     // the batch's own buffers
    unsigned long long* totals = nullptr;  // device, k
    cudaStream_t cap_stream = nullptr;     // the stream captures are recorded on
    PackDev* packs_dev = nullptr;          // device: one descriptor per pack
    uint64_t* mscratch = nullptr;          // device: the multi-pack count's bases, schedule and scan scratch
    int64_t mscratch_words = 0;
    cudaGraphExec_t exec = nullptr;
    int kernels_per_run = 0;               // kernel nodes in the captured graph
    cudaStream_t last_stream = nullptr;
};

namespace tcg {

static void drop_capture(tc_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

static void destroy_batch(tc_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->last_stream);
    drop_capture(b);
    if (b->packs_dev) b->al.put(b->packs_dev, b->packs.size() * sizeof(PackDev), b->last_stream);
    if (b->mscratch) b->al.put(b->mscratch, (size_t)b->mscratch_words * 8, b->last_stream);
    for (tc_graph* g : b->packs) free_graph(g);
    if (b->totals) b->al.put(b->totals, (size_t)(b->k > 0 ? b->k : 1) * 8, b->last_stream);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaStreamSynchronize(b->last_stream);
    delete b;
}

// Build graphs [j0, j1) into one pack.
static tc_status build_pack(const int32_t* const* src, const int32_t* const* dst, const int64_t* m, const int32_t* n,
                            int32_t j0, int32_t j1, const tc_options& o, cudaStream_t s, tc_graph** out,
                            int64_t* m_hat_out) {
    *out = nullptr;
    const int32_t k = j1 - j0;
    std::vector<int64_t> ebase(k + 1, 0);
    std::vector<int32_t> vbase(k + 1, 0);
    for (int32_t j = 0; j < k; ++j) {
        ebase[j + 1] = ebase[j] + m[j0 + j];
        vbase[j + 1] = vbase[j] + n[j0 + j];
    }
    const int64_t mp = ebase[k];
    const int32_t np = vbase[k];
    tc_graph* g = nullptr;
    TC_TRY(new_graph(o, s, &g));
    tc_status st = TC_OK;
    {
        DevBuf<int32_t> ss, dd;
        DevBuf<int64_t> eb;
        DevBuf<int32_t> vb;
        DevBuf<const int32_t*> sp, dp;
        st = ss.alloc(&g->al, (size_t)(mp > 0 ? mp : 1), s);
        if (st == TC_OK) st = dd.alloc(&g->al, (size_t)(mp > 0 ? mp : 1), s);
        if (st == TC_OK) st = eb.alloc(&g->al, (size_t)k + 1, s);
        if (st == TC_OK) st = vb.alloc(&g->al, (size_t)k + 1, s);
        if (st == TC_OK) st = sp.alloc(&g->al, (size_t)k, s);
        if (st == TC_OK) st = dp.alloc(&g->al, (size_t)k, s);
        // where the gather kernel reads each graph: device memory and pinned host memory in
        // place; pageable host memory is first copied into the graph's part of the pack arrays
        std::vector<const int32_t*> sv(k, nullptr), dv(k, nullptr);
        for (int32_t j = 0; j < k && st == TC_OK; ++j) {
            const int64_t mj = m[j0 + j];
            if (mj == 0) continue;
            const int32_t* a = src[j0 + j];
            const int32_t* b = dst[j0 + j];
            const int32_t* av = is_device_pointer(a) ? a : (const int32_t*)pinned_device_view(a);
            const int32_t* bv = is_device_pointer(b) ? b : (const int32_t*)pinned_device_view(b);
            if (!av) {
                if (cudaMemcpyAsync(ss.ptr + ebase[j], a, (size_t)mj * 4, cudaMemcpyDefault, s) != cudaSuccess) st = TC_ERR_CUDA;
                av = ss.ptr + ebase[j];
            }
            if (!bv) {
                if (cudaMemcpyAsync(dd.ptr + ebase[j], b, (size_t)mj * 4, cudaMemcpyDefault, s) != cudaSuccess) st = TC_ERR_CUDA;
                bv = dd.ptr + ebase[j];
            }
            sv[j] = av;
            dv[j] = bv;
        }
        if (st == TC_OK && (cudaMemcpyAsync(eb.ptr, ebase.data(), (size_t)(k + 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                            cudaMemcpyAsync(vb.ptr, vbase.data(), (size_t)(k + 1) * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                            cudaMemcpyAsync(sp.ptr, sv.data(), (size_t)k * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                            cudaMemcpyAsync(dp.ptr, dv.data(), (size_t)k * 8, cudaMemcpyHostToDevice, s) != cudaSuccess))
            st = TC_ERR_CUDA;
        if (st == TC_OK && mp > 0) {
            const int64_t want = (mp + 255) / 256;
            const unsigned blocks = (unsigned)std::min<int64_t>(want, (int64_t)num_sms() * 8);
            k_pack_ids<<<blocks, 256, 0, s>>>(PackMeta{eb.ptr, vb.ptr, sp.ptr, dp.ptr, k}, mp, ss.ptr, dd.ptr, g->status);
            note_launch();
            if (cudaGetLastError() != cudaSuccess) st = TC_ERR_CUDA;
            if (st == TC_OK) st = read_status(g, s, nullptr);
        }
        if (st == TC_OK) st = build_graph(g, ss.ptr, dd.ptr, mp, np, s);
        ss.release();
        dd.release();
        if (st == TC_OK) {
            void* p = nullptr;
            st = g->al.get(&p, 2 * ((size_t)k + 1) * 8, s);
            if (st == TC_OK) {
                g->sub_task = (int64_t*)p;
                g->n_sub = k;
                g->bytes += (int64_t)align_up(2 * ((size_t)k + 1) * 8, 256);
            }
        }
        DevBuf<int64_t> so;
        if (st == TC_OK) st = so.alloc(&g->al, (size_t)k + 1, s);
        if (st == TC_OK) {
            const int threads = 2 * (k + 1);
            k_sub_tasks<<<(threads + 255) / 256, 256, 0, s>>>(g->trec, g->tasks_small, g->tasks, g->off, vb.ptr, k,
                                                               g->sub_task, so.ptr);
            note_launch();
            if (cudaGetLastError() != cudaSuccess) st = TC_ERR_CUDA;
        }
        if (st == TC_OK) {
            std::vector<int64_t> hoff(k + 1);
            if (cudaMemcpyAsync(hoff.data(), so.ptr, (size_t)(k + 1) * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                st = TC_ERR_CUDA;
            for (int32_t j = 0; j < k && st == TC_OK; ++j) m_hat_out[j] = hoff[j + 1] - hoff[j];
        }
    }
    if (st != TC_OK) {
        (void)cudaGetLastError();
        free_graph(g);
        return st;
    }
    *out = g;
    return TC_OK;
}

// Record the count of every pack into one CUDA graph (work buffers and the pack descriptors
// set up beforehand).
static tc_status capture_batch(tc_batch* b) {
    drop_capture(b);
    const size_t np = b->packs.size();
    int64_t total_tasks = 0, tiles = 0;
    std::vector<PackDev> hp(np);
    for (size_t p = 0; p < np; ++p) {
        tc_graph* g = b->packs[p];
        TC_TRY(ensure_count_work(g, b->opt, b->cap_stream));
        PackDev& d = hp[p];
        d.off = g->off;
        d.cols = g->cols;
        d.tasks = g->trec;
        d.deg = g->deg;
        d.P = g->work.prefix;
        d.fcost = g->work.fcost;
        d.own_first = g->own_first;
        d.n_owners = g->owners_big;
        d.sub_task = g->sub_task;
        d.n_sub = g->n_sub;
        d.Ts = g->tasks_small;
        d.T = g->tasks;
        d.task_base = total_tasks;
        d.tile_base = tiles;  // each pack's cost prefix starts a new scan tile
        d.total = b->totals + b->first[p];
        total_tasks += g->tasks;
        tiles += ceil_div(g->tasks, kScanTile);
    }
    if (!b->packs_dev && np > 0) {
        void* q = nullptr;
        TC_TRY(b->al.get(&q, np * sizeof(PackDev), b->cap_stream));
        b->packs_dev = (PackDev*)q;
    }
    if (!b->mscratch && np > 0) {
        void* q = nullptr;
        b->mscratch_words = multi_scratch_words(total_tasks, (int)np);
        TC_TRY(b->al.get(&q, (size_t)b->mscratch_words * 8, b->cap_stream));
        b->mscratch = (uint64_t*)q;
    }
    if (np > 0)
        TC_CUDA_TRY(cudaMemcpyAsync(b->packs_dev, hp.data(), np * sizeof(PackDev), cudaMemcpyHostToDevice, b->cap_stream));
    TC_CUDA_TRY(cudaStreamSynchronize(b->cap_stream));
    TC_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    tc_status st = TC_OK;
    // kernels are counted when they run, not when they are recorded
    const int64_t l0 = tc_kernel_launches();
    st = count_enqueue_multi(b->packs, b->packs_dev, b->mscratch, b->opt, b->totals, b->k, b->cap_stream);
    b->kernels_per_run = (int)(tc_kernel_launches() - l0);
    note_launch(-b->kernels_per_run);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (st == TC_OK && e != cudaSuccess) st = TC_ERR_CUDA;
    if (st == TC_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) st = TC_ERR_CUDA;
    if (graph) cudaGraphDestroy(graph);
    if (st != TC_OK) {
        (void)cudaGetLastError();
        b->exec = nullptr;
    }
    return st;
}

static tc_status batch_check(tc_batch* b, cudaStream_t s) {
    tc_status first = TC_OK;
    for (tc_graph* g : b->packs) {
        const tc_status st = read_status(g, s, nullptr);
        if (first == TC_OK) first = st;
    }
    return first;
}

}  // namespace tcg

extern "C" {

tc_status tc_batch_build(const int32_t* const* src, const int32_t* const* dst, const int64_t* m, const int32_t* n,
                         int32_t k, int64_t pack_edges, const tc_options* opt, tc_stream_t stream, tc_batch_t* out) {
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    if (k < 0 || (k > 0 && (!m || !n || !src || !dst)) || pack_edges < 0) return TC_ERR_INVALID_ARG;
    for (int32_t j = 0; j < k; ++j) {
        if (m[j] < 0 || n[j] < 0) return TC_ERR_INVALID_ARG;
        if (m[j] > 0 && (!src[j] || !dst[j])) return TC_ERR_INVALID_ARG;
        if ((int64_t)n[j] > kMaxPackVertices) return TC_ERR_UNSUPPORTED;
    }
    tc_options o;
    tc_options_default(&o);
    if (opt) o = *opt;
    TC_TRY(check_options(o));
    const int64_t cap = pack_edges > 0 ? pack_edges : kDefaultPackEdges;
    cudaStream_t s = (cudaStream_t)stream;

    tc_batch* b = new (std::nothrow) tc_batch();
    if (!b) return TC_ERR_OOM;
    b->opt = o;
    b->k = k;
    b->al.alloc = o.alloc;
    b->al.release = o.release;
    b->al.ctx = o.alloc_ctx;
    b->last_stream = s;
    cudaGetDevice(&b->device);
    tc_status st = TC_OK;
    try {
        b->m_hat.assign((size_t)k, 0);
    } catch (...) {
        delete b;
        return TC_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) st = TC_ERR_CUDA;
    if (st == TC_OK) {
        void* p = nullptr;
        st = b->al.get(&p, (size_t)(k > 0 ? k : 1) * 8, s);
        b->totals = (unsigned long long*)p;
    }
    // greedy packing in graph order: a pack takes graphs while its edges stay within the cap
    // and its vertices within 2^30; a graph above the cap forms a pack of its own
    int32_t j = 0;
    while (st == TC_OK && j < k) {
        int32_t j1 = j + 1;
        int64_t me = m[j], nv = n[j];
        while (j1 < k && me + m[j1] <= cap && nv + n[j1] <= kMaxPackVertices) {
            me += m[j1];
            nv += n[j1];
            ++j1;
        }
        tc_graph* g = nullptr;
        st = build_pack(src, dst, m, n, j, j1, o, s, &g, b->m_hat.data() + j);
        if (st == TC_OK) {
            b->packs.push_back(g);
            b->first.push_back(j);
            b->m_in += me;
        }
        j = j1;
    }
    b->first.push_back(k);
    if (st != TC_OK) {
        destroy_batch(b);
        return st;
    }
    *out = b;
    return TC_OK;
}

tc_status tc_batch_run(tc_batch_t b, tc_stream_t stream, uint64_t* totals_dev) {
    if (!b || (!totals_dev && b->k > 0)) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    b->last_stream = s;
    for (tc_graph* g : b->packs) g->last_stream = s;
    if (b->k == 0) return TC_OK;
    if (!b->exec) TC_TRY(capture_batch(b));
    TC_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    note_launch(b->kernels_per_run);
    if ((void*)totals_dev != (void*)b->totals)
        TC_CUDA_TRY(cudaMemcpyAsync(totals_dev, b->totals, (size_t)b->k * 8, cudaMemcpyDeviceToDevice, s));
    return TC_OK;
}

tc_status tc_batch_check(tc_batch_t b, tc_stream_t stream) {
    if (!b) return TC_ERR_INVALID_ARG;
    return batch_check(b, (cudaStream_t)stream);
}

tc_status tc_batch_count(tc_batch_t b, tc_stream_t stream, uint64_t* totals) {
    if (!b || (!totals && b->k > 0)) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (b->k == 0) return TC_OK;
    TC_TRY(tc_batch_run(b, stream, (uint64_t*)b->totals));
    TC_CUDA_TRY(cudaMemcpyAsync(totals, b->totals, (size_t)b->k * 8, cudaMemcpyDeviceToHost, s));
    return batch_check(b, s);  // synchronises s
}

tc_status tc_batch_get_info(tc_batch_t b, tc_batch_info* info) {
    if (!b || !info) return TC_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->k = b->k;
    info->packs = (int32_t)b->packs.size();
    info->m_in = b->m_in;
    for (tc_graph* g : b->packs) {
        info->m_hat += g->m_hat;
        info->tasks += g->tasks;
        info->tasks_small += g->tasks_small;
        info->device_bytes += g->bytes;
        if (g->max_dhat > info->max_dhat) info->max_dhat = g->max_dhat;
    }
    info->device_bytes += (int64_t)align_up((size_t)(b->k > 0 ? b->k : 1) * 8, 256);
    return TC_OK;
}

tc_status tc_batch_graph_edges(tc_batch_t b, int64_t* m_hat) {
    if (!b || (!m_hat && b->k > 0)) return TC_ERR_INVALID_ARG;
    if (b->k > 0) std::memcpy(m_hat, b->m_hat.data(), (size_t)b->k * 8);
    return TC_OK;
}

tc_status tc_batch_set_options(tc_batch_t b, const tc_options* opt) {
    if (!b || !opt) return TC_ERR_INVALID_ARG;
    TC_TRY(check_options(*opt));
    const tc_options& o = b->opt;
    if (opt->input_policy != o.input_policy || opt->small_max != o.small_max || opt->alloc != o.alloc ||
        opt->release != o.release || opt->alloc_ctx != o.alloc_ctx || opt->hbm_budget_bytes != o.hbm_budget_bytes)
        return TC_ERR_INVALID_ARG;
    cudaStreamSynchronize(b->last_stream);
    b->opt = *opt;
    for (tc_graph* g : b->packs) {
        if (opt->cost_model >= TC_COST_ONE) TC_TRY(ensure_count_work(g, b->opt, b->cap_stream));
        g->opt = *opt;
    }
    drop_capture(b);
    return TC_OK;
}

void tc_batch_free(tc_batch_t b) { destroy_batch(b); }

tc_status tc_batch_autotune(const int32_t* const* src, const int32_t* const* dst, const int64_t* m, const int32_t* n,
                            int32_t k, const tc_options* opt, int32_t reps, tc_stream_t stream, tc_options* best,
                            tc_tune_report* report) {
    if (!best || reps < 1 || (report && report->cap > 0 && !report->entries)) return TC_ERR_INVALID_ARG;
    tc_options base;
    tc_options_default(&base);
    if (opt) base = *opt;
    TC_TRY(check_options(base));
    cudaStream_t s = (cudaStream_t)stream;
    static const int kSmallMax[] = {32, 64, 128};
    static const int kWarps[] = {4, 8, 16};
    static const int kBigWarps[] = {8, 16};
    static const int kPiece[] = {1024, 2048};
    float best_ms = -1.f, default_ms = -1.f;
    tc_options chosen = base;
    int32_t tried = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TC_CUDA_TRY(cudaEventCreate(&e0));
    TC_CUDA_TRY(cudaEventCreate(&e1));
    DevBuf<uint64_t> out;
    Allocator al;
    tc_status st = out.alloc(&al, (size_t)(k > 0 ? k : 1), s);
    for (int sm : kSmallMax) {
        if (st != TC_OK) break;
        tc_options bo = base;
        bo.small_max = sm;
        tc_batch* b = nullptr;
        st = tc_batch_build(src, dst, m, n, k, 0, &bo, stream, &b);
        if (st != TC_OK) break;
        for (int w : kWarps)
            for (int bw : kBigWarps)
                for (int pc : kPiece) {
                    if (st != TC_OK) break;
                    tc_options c = bo;
                    c.warps_per_block = w;
                    c.big_warps = bw;
                    c.piece = pc;
                    if (check_options(c) != TC_OK) continue;
                    st = tc_batch_set_options(b, &c);
                    float ms_min = -1.f;
                    for (int r = 0; r <= reps && st == TC_OK; ++r) {  // run 0 captures and warms up
                        if (cudaEventRecord(e0, s) != cudaSuccess) st = TC_ERR_CUDA;
                        if (st == TC_OK) st = tc_batch_run(b, stream, out.ptr);
                        if (st == TC_OK && cudaEventRecord(e1, s) != cudaSuccess) st = TC_ERR_CUDA;
                        if (st == TC_OK) st = batch_check(b, s);
                        float ms = 0.f;
                        if (st == TC_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = TC_ERR_CUDA;
                        if (st == TC_OK && r > 0 && (ms_min < 0.f || ms < ms_min)) ms_min = ms;
                    }
                    if (st != TC_OK) break;
                    if (report && tried < report->cap)
                        report->entries[tried] = tc_tune_entry{sm, w, bw, pc, c.static_percent, ms_min};
                    ++tried;
                    if (best_ms < 0.f || ms_min < best_ms) {
                        best_ms = ms_min;
                        chosen = c;
                    }
                    if (sm == base.small_max && w == base.warps_per_block && bw == base.big_warps && pc == base.piece)
                        default_ms = ms_min;
                }
        destroy_batch(b);
    }
    out.release();
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (report) {
        report->n = tried;
        report->best_ms = best_ms;
        report->default_ms = default_ms;
    }
    if (st != TC_OK) return st;
    *best = chosen;
    return TC_OK;
}

}  // extern "C"

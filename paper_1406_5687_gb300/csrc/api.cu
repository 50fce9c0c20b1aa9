// api.cu -- the extern "C" entry points for single graphs declared in include/tc.h.
#include <algorithm>
#include <climits>
#include <cstring>
#include <new>

#include "graph.cuh"
#include "primitives.cuh"

namespace tcg {

// Small per-handle device block: error word, last result, schedule state.
struct HandleDev {
    DevStatus status;
    unsigned long long result;
    long long pad;
    Sched sched[2];
};

tc_status check_options(const tc_options& o) {
    if (o.input_policy != TC_INPUT_SANITIZE && o.input_policy != TC_INPUT_STRICT) return TC_ERR_INVALID_ARG;
    if (o.cost_model < TC_COST_EDGE || o.cost_model > TC_COST_NEW) return TC_ERR_INVALID_ARG;
    if (o.piece != 256 && o.piece != 512 && o.piece != 1024 && o.piece != 2048 && o.piece != 4096)
        return TC_ERR_INVALID_ARG;
    if (o.warps_per_block != 1 && o.warps_per_block != 2 && o.warps_per_block != 4 && o.warps_per_block != 8 &&
        o.warps_per_block != 16)
        return TC_ERR_INVALID_ARG;
    if (o.big_warps != 4 && o.big_warps != 8 && o.big_warps != 16) return TC_ERR_INVALID_ARG;
    if (o.small_max != 0 && o.small_max != 16 && o.small_max != 32 && o.small_max != 64 && o.small_max != 128 &&
        o.small_max != 256)
        return TC_ERR_INVALID_ARG;
    // shared memory: the small kernel's per-warp tables, the big kernel's block table
    if ((size_t)o.warps_per_block * small_table_slots(o.small_max) * 4 > 200 * 1024) return TC_ERR_INVALID_ARG;
    if (o.blocks_per_sm < 0 || o.static_percent < 0 || o.static_percent > 100) return TC_ERR_INVALID_ARG;
    if (o.min_chunk < 0 || o.c_task < 0 || o.c_owner < 0 || o.hbm_budget_bytes < 0 || o.retry_limit < 0)
        return TC_ERR_INVALID_ARG;
    if ((o.alloc == nullptr) != (o.release == nullptr)) return TC_ERR_INVALID_ARG;
    return TC_OK;
}

// The device address of pinned (page-locked, mapped) host memory, or null for any other
// memory.  Kernels read such memory directly over the host link.
const void* pinned_device_view(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

bool is_device_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device bytes a build of (m, n) holds at its peak (keys, sort scratch, arrays, staging).
int64_t build_peak_bytes(int64_t m, int32_t n, bool host_input) {
    int64_t mm = m > 0 ? m : 1;
    int64_t b = 16 * mm + radix_sort_scratch_bytes(mm) + 8 * (int64_t)n * 2 + 8 * ((int64_t)n + 1) + 4 * mm +
                16 * mm + (1 << 20);
    if (host_input) b += 8 * mm;
    return b;
}

// Device bytes a built graph keeps, including the count workspace.
int64_t graph_resident_bytes(int64_t m_hat, int64_t tasks, int32_t n) {
    return 4 * (int64_t)n + 8 * ((int64_t)n + 1) + 4 * m_hat + 16 * tasks + 8 * (tasks + 1) +
           8 * (tasks / 2048 + 64) + 8 * (int64_t)n + (1 << 16);
}

void free_graph(tc_graph* g) {
    if (!g) return;
    cudaStream_t s = g->last_stream;
    cudaStreamSynchronize(s);
    auto put = [&](void* p, size_t bytes) {
        if (p) g->al.put(p, bytes, s);
    };
    put(g->deg, (size_t)(g->n > 0 ? g->n : 1) * 4);
    put(g->off, ((size_t)g->n + 1) * 8);
    put(g->cols, ((size_t)(g->m_hat > 0 ? g->m_hat : 1) + 4) * 4);
    put(g->trec, (size_t)(g->tasks > 0 ? g->tasks : 1) * sizeof(TaskRec));
    put(g->own_first, (size_t)g->own_first_cap * 4);
    put(g->work.prefix, (size_t)(g->tasks + 1) * 8);
    put(g->work.scan_scr, (size_t)g->work.scan_words * 8);
    put(g->work.fcost, (size_t)(g->n > 0 ? g->n : 1) * 8);
    put(g->sub_task, (size_t)(g->n_sub > 0 ? 2 * ((size_t)g->n_sub + 1) : 0) * 8);
    put(g->status, sizeof(HandleDev));
    cudaStreamSynchronize(s);
    delete g;
}

// A new empty handle with its device status block, on stream s (options already checked).
tc_status new_graph(const tc_options& o, cudaStream_t s, tc_graph** out) {
    *out = nullptr;
    retain_pool_memory();
    tc_graph* g = new (std::nothrow) tc_graph();
    if (!g) return TC_ERR_OOM;
    g->opt = o;
    g->al.alloc = o.alloc;
    g->al.release = o.release;
    g->al.ctx = o.alloc_ctx;
    g->al.budget = o.hbm_budget_bytes;
    g->last_stream = s;
    cudaGetDevice(&g->device);
    void* p = nullptr;
    tc_status st = g->al.get(&p, sizeof(HandleDev), s);
    if (st == TC_OK) {
        g->status = (DevStatus*)p;
        HandleDev* hd = (HandleDev*)p;
        g->work.result = &hd->result;
        g->work.sched = hd->sched;
        if (cudaMemsetAsync(p, 0, sizeof(HandleDev), s) != cudaSuccess) st = TC_ERR_CUDA;
    }
    if (st != TC_OK) {
        (void)cudaGetLastError();
        free_graph(g);
        return st;
    }
    *out = g;
    return TC_OK;
}

tc_status read_status(tc_graph* g, cudaStream_t s, unsigned long long* result) {
    HandleDev h;
    TC_CUDA_TRY(cudaMemcpyAsync(&h, g->status, offsetof(HandleDev, pad), cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    if (result) *result = h.result;
    if (h.status.code != 0) {
        TC_CUDA_TRY(cudaMemsetAsync(g->status, 0, sizeof(DevStatus), s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        return (tc_status)h.status.code;
    }
    return TC_OK;
}

}  // namespace tcg

using namespace tcg;

extern "C" {

const char* tc_status_str(tc_status s) {
    switch (s) {
        case TC_OK: return "ok";
        case TC_ERR_INVALID_ARG: return "invalid argument";
        case TC_ERR_VERTEX_RANGE: return "vertex id outside [0, n)";
        case TC_ERR_OOM: return "out of memory";
        case TC_ERR_CUDA: return "CUDA runtime error";
        case TC_ERR_TIMEOUT: return "bounded device wait gave up";
        case TC_ERR_BUDGET: return "device memory budget exceeded";
        case TC_ERR_UNSUPPORTED: return "input exceeds a limit of this build";
        case TC_ERR_CANCELLED: return "request withdrawn before it ran";
    }
    return "unknown status";
}

const char* tc_version(void) { return "1.0.0 sm_103a"; }

void tc_options_default(tc_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->input_policy = TC_INPUT_SANITIZE;
    o->cost_model = TC_COST_EDGE;
    o->piece = 2048;
    o->warps_per_block = 16;
    o->big_warps = 16;
    o->small_max = 64;
    o->blocks_per_sm = 0;
    o->static_percent = 50;
    o->min_chunk = 0;
    o->c_task = 4;
    o->c_owner = 32;
    o->hbm_budget_bytes = 0;
    o->retry_limit = 0;
}

tc_status tc_build(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, const tc_options* opt,
                   tc_stream_t stream, tc_graph_t* out) {
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    if (m < 0 || n < 0 || n == INT32_MAX) return m < 0 || n < 0 ? TC_ERR_INVALID_ARG : TC_ERR_UNSUPPORTED;
    if (m > 0 && (!src || !dst)) return TC_ERR_INVALID_ARG;
    tc_options o;
    tc_options_default(&o);
    if (opt) o = *opt;
    TC_TRY(check_options(o));
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev_in = m > 0 && is_device_pointer(src) && is_device_pointer(dst);
    const bool mixed = m > 0 && (is_device_pointer(src) != is_device_pointer(dst));
    if (mixed) return TC_ERR_INVALID_ARG;
    if (o.hbm_budget_bytes > 0 && build_peak_bytes(m, n, !dev_in) > o.hbm_budget_bytes) return TC_ERR_BUDGET;

    tc_graph* g = nullptr;
    TC_TRY(new_graph(o, s, &g));
    tc_status st = TC_OK;
    {
        const int32_t* s_d = src;
        const int32_t* d_d = dst;
        DevBuf<int32_t> ss, dd;
        // pinned host lists are read in place by the canonicalize kernel (one pass over the
        // host link, no staging copy); pageable ones are staged in device memory first
        const int32_t* s_pin = m > 0 && !dev_in ? (const int32_t*)pinned_device_view(src) : nullptr;
        const int32_t* d_pin = m > 0 && !dev_in ? (const int32_t*)pinned_device_view(dst) : nullptr;
        if (s_pin && d_pin) {
            s_d = s_pin;
            d_d = d_pin;
        } else if (m > 0 && !dev_in) {
            st = ss.alloc(&g->al, (size_t)m, s);
            if (st == TC_OK) st = dd.alloc(&g->al, (size_t)m, s);
            if (st == TC_OK && (cudaMemcpyAsync(ss.ptr, src, (size_t)m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                                cudaMemcpyAsync(dd.ptr, dst, (size_t)m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess))
                st = TC_ERR_CUDA;
            s_d = ss.ptr;
            d_d = dd.ptr;
        }
        if (st == TC_OK) st = build_graph(g, s_d, d_d, m, n, s);
    }
    if (st != TC_OK) {
        (void)cudaGetLastError();
        free_graph(g);
        return st;
    }
    *out = g;
    return TC_OK;
}

// Split interleaved pairs into the two device arrays tc_build takes.
__global__ void k_split_pairs(const int32_t* __restrict__ pairs, int64_t m, int32_t* __restrict__ src,
                              int32_t* __restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        src[i] = pairs[2 * i];
        dst[i] = pairs[2 * i + 1];
    }
}

tc_status tc_build_pairs(const int32_t* edges, int64_t m, int32_t n, const tc_options* opt, tc_stream_t stream,
                         tc_graph_t* out) {
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    if (m < 0 || n < 0) return TC_ERR_INVALID_ARG;
    if (m > 0 && !edges) return TC_ERR_INVALID_ARG;
    if (m == 0) return tc_build(nullptr, nullptr, 0, n, opt, stream, out);
    tc_options o;
    tc_options_default(&o);
    if (opt) o = *opt;
    TC_TRY(check_options(o));
    cudaStream_t s = (cudaStream_t)stream;
    retain_pool_memory();
    Allocator al;
    al.alloc = o.alloc;
    al.release = o.release;
    al.ctx = o.alloc_ctx;
    tc_status st = TC_OK;
    {
        DevBuf<int32_t> sd, dd, staged;
        TC_TRY(sd.alloc(&al, (size_t)m, s));
        TC_TRY(dd.alloc(&al, (size_t)m, s));
        const int32_t* pairs = is_device_pointer(edges) ? edges : (const int32_t*)pinned_device_view(edges);
        if (!pairs) {  // pageable host pairs: one copy to the device first
            TC_TRY(staged.alloc(&al, (size_t)(2 * m), s));
            TC_CUDA_TRY(cudaMemcpyAsync(staged.ptr, edges, (size_t)m * 8, cudaMemcpyHostToDevice, s));
            pairs = staged.ptr;
        }
        const int grid = (int)std::min<int64_t>(ceil_div(m, 256), (int64_t)num_sms() * 8);
        k_split_pairs<<<grid, 256, 0, s>>>(pairs, m, sd.ptr, dd.ptr);
        note_launch();
        TC_CUDA_TRY(cudaGetLastError());
        staged.release();
        // the build's budget covers its own peak; the split arrays are held beside it
        if (o.hbm_budget_bytes > 0) {
            if (o.hbm_budget_bytes <= 8 * m) return TC_ERR_BUDGET;
            o.hbm_budget_bytes -= 8 * m;
        }
        st = tc_build(sd.ptr, dd.ptr, m, n, &o, stream, out);
        cudaStreamSynchronize(s);
    }
    return st;
}

void tc_free(tc_graph_t g) { free_graph(g); }

tc_status tc_count(tc_graph_t g, tc_stream_t stream, uint64_t* total) {
    if (!g || !total) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    TC_TRY(count_enqueue(g, g->opt, s, g->work.result, nullptr, nullptr, nullptr));
    unsigned long long r = 0;
    TC_TRY(read_status(g, s, &r));
    *total = r;
    return TC_OK;
}

tc_status tc_count_async(tc_graph_t g, tc_stream_t stream, uint64_t* total_dev) {
    if (!g || !total_dev) return TC_ERR_INVALID_ARG;
    g->last_stream = (cudaStream_t)stream;
    return count_enqueue(g, g->opt, (cudaStream_t)stream, (unsigned long long*)total_dev, nullptr, nullptr, nullptr);
}

tc_status tc_count_graphs(const tc_graph_t* gs, int32_t k, tc_stream_t stream, uint64_t* totals) {
    if (k < 0 || (k > 0 && (!gs || !totals))) return TC_ERR_INVALID_ARG;
    for (int32_t j = 0; j < k; ++j)
        if (!gs[j]) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (int32_t j = 0; j < k; ++j) {
        tc_graph* g = gs[j];
        g->last_stream = s;
        TC_TRY(count_enqueue(g, g->opt, s, g->work.result, nullptr, nullptr, nullptr));
        // a repeated handle keeps its result word: take each total as soon as it is written
        TC_CUDA_TRY(cudaMemcpyAsync(&totals[j], g->work.result, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    }
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    for (int32_t j = 0; j < k; ++j) TC_TRY(read_status(gs[j], s, nullptr));
    return TC_OK;
}

tc_status tc_count_partition(tc_graph_t g, int32_t part, int32_t nparts, tc_stream_t stream, uint64_t* partial) {
    if (!g || !partial || nparts < 1 || part < 0 || part >= nparts) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    TC_TRY(count_enqueue(g, g->opt, s, g->work.result, nullptr, nullptr, nullptr, part, nparts));
    unsigned long long r = 0;
    TC_TRY(read_status(g, s, &r));
    *partial = r;
    return TC_OK;
}

tc_status tc_graph_check(tc_graph_t g, tc_stream_t stream) {
    if (!g) return TC_ERR_INVALID_ARG;
    return read_status(g, (cudaStream_t)stream, nullptr);
}

tc_status tc_count_per_vertex(tc_graph_t g, tc_stream_t stream, uint64_t* t_v, uint64_t* total) {
    if (!g || (!t_v && g->n > 0)) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    unsigned long long* tv = (unsigned long long*)t_v;
    if (g->n > 0) TC_CUDA_TRY(cudaMemsetAsync(tv, 0, sizeof(uint64_t) * g->n, s));
    TC_TRY(count_enqueue(g, g->opt, s, g->work.result, tv ? tv : nullptr, nullptr, nullptr));
    unsigned long long r = 0;
    TC_TRY(read_status(g, s, &r));
    if (total) *total = r;
    return TC_OK;
}

tc_status tc_count_per_edge(tc_graph_t g, tc_stream_t stream, uint32_t* c, uint64_t* total) {
    if (!g || (!c && g->m_hat > 0)) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    if (g->m_hat > 0) TC_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(uint32_t) * g->m_hat, s));
    TC_TRY(count_enqueue(g, g->opt, s, g->work.result, nullptr, c, nullptr));
    unsigned long long r = 0;
    TC_TRY(read_status(g, s, &r));
    if (total) *total = r;
    return TC_OK;
}

tc_status tc_clustering(tc_graph_t g, const uint64_t* t_v, double* cc, tc_stream_t stream) {
    if (!g || ((!t_v || !cc) && g->n > 0)) return TC_ERR_INVALID_ARG;
    g->last_stream = (cudaStream_t)stream;
    return clustering_enqueue(g, t_v, cc, (cudaStream_t)stream);
}

tc_status tc_graph_get_info(tc_graph_t g, tc_graph_info* info) {
    if (!g || !info) return TC_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n = g->n;
    info->max_degree = g->max_degree;
    info->max_dhat = g->max_dhat;
    info->id_bits = g->id_bits;
    info->m_in = g->m_in;
    info->self_loops = g->self_loops;
    info->duplicates = g->duplicates;
    info->m_hat = g->m_hat;
    info->tasks = g->tasks;
    info->tasks_small = g->tasks_small;
    info->sum_dhat_v = g->sum_dhat_v;
    info->sum_dhat_u = g->sum_dhat_u;
    info->sum_stream = g->sum_stream;
    info->device_bytes = g->bytes;
    return TC_OK;
}

tc_status tc_graph_csr(tc_graph_t g, const int32_t** deg, const int64_t** off, const int32_t** cols,
                       const uint32_t** tasks) {
    if (!g) return TC_ERR_INVALID_ARG;
    if (deg) *deg = g->deg;
    if (off) *off = g->off;
    if (cols) *cols = g->cols;
    if (tasks) *tasks = (const uint32_t*)g->trec;
    return TC_OK;
}

tc_status tc_vertex_cost(tc_graph_t g, int32_t fn, tc_stream_t stream, uint64_t* f) {
    if (!g || (!f && g->n > 0)) return TC_ERR_INVALID_ARG;
    g->last_stream = (cudaStream_t)stream;
    return vertex_cost_enqueue(g, fn, (cudaStream_t)stream, f);
}

tc_status tc_count_ex(tc_graph_t g, const tc_options* opt, tc_stream_t stream, uint64_t* total,
                      tc_count_trace* trace) {
    if (!g || !total) return TC_ERR_INVALID_ARG;
    tc_options o = opt ? *opt : g->opt;
    TC_TRY(check_options(o));
    if (trace && trace->cap < 0) return TC_ERR_INVALID_ARG;
    if (trace && trace->cap > 0 && !trace->chunks) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    TC_TRY(count_enqueue(g, o, s, g->work.result, nullptr, nullptr, trace));
    unsigned long long r = 0;
    TC_TRY(read_status(g, s, &r));
    *total = r;
    return TC_OK;
}

}  // extern "C"

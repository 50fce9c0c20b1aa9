// server.cu -- serving with continuous batching: a FIFO of borrowed edge lists, slot threads
// that each own a CUDA stream and take, whenever they are free, the requests at the head of
// the queue that fit the group size and the device-memory budget.  One request goes through
// the single-graph path, several through one batch pack; the slots' work overlaps on the GPU.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "graph.cuh"

namespace tcg {

struct Request {
    const int32_t* src;
    const int32_t* dst;
    int64_t m;
    int32_t n;
    uint64_t tag;
    double t_submit;
    int64_t bytes;  // estimated device bytes of this request alone
};

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Device bytes a build + count of (m, n) may hold at once: the build's peak plus what the
// built graph keeps (tasks <= m).
static int64_t request_bytes(int64_t m, int64_t n) {
    const int32_t nn = n > INT32_MAX ? INT32_MAX : (int32_t)n;
    return build_peak_bytes(m, nn, true) + graph_resident_bytes(m, m, nn);
}

constexpr int64_t kDefaultGroupEdges = 1ll << 26;
constexpr int64_t kMaxGroupVertices = 1ll << 30;

}  // namespace tcg

using namespace tcg;

struct tc_server {
    int device = 0;
    tc_options opt{};
    int64_t budget = 0;
    int64_t group_edges = 0;
    std::mutex mu;
    std::condition_variable cv_work;  // a request or memory became available, or stop
    std::condition_variable cv_done;  // results were produced
    std::deque<Request> queue;
    std::deque<tc_result> results;
    std::vector<std::thread> threads;
    bool stopping = false;
    int64_t submitted = 0, finished = 0, groups = 0, grouped = 0;
    int64_t in_flight = 0, peak_in_flight = 0;
    int busy = 0, peak_busy = 0;
};

namespace tcg {

// Count one request through the single-graph path on stream s.
static tc_status count_alone(const tc_options& opt, const Request& r, cudaStream_t s, uint64_t* total) {
    tc_graph_t g = nullptr;
    TC_TRY(tc_build(r.src, r.dst, r.m, r.n, &opt, (tc_stream_t)s, &g));
    const tc_status st = tc_count(g, (tc_stream_t)s, total);
    tc_free(g);
    return st;
}

// Count a group as one batch pack; on a failure of the whole batch, count each request
// alone so that every request gets its own status.
static void count_group(const tc_options& opt, const std::vector<Request>& grp, cudaStream_t s,
                        std::vector<uint64_t>& total, std::vector<tc_status>& status) {
    const size_t k = grp.size();
    total.assign(k, 0);
    status.assign(k, TC_OK);
    if (k == 1) {
        status[0] = count_alone(opt, grp[0], s, &total[0]);
        return;
    }
    std::vector<const int32_t*> src(k), dst(k);
    std::vector<int64_t> m(k);
    std::vector<int32_t> n(k);
    for (size_t j = 0; j < k; ++j) {
        src[j] = grp[j].src;
        dst[j] = grp[j].dst;
        m[j] = grp[j].m;
        n[j] = grp[j].n;
    }
    tc_batch_t b = nullptr;
    tc_status st = tc_batch_build(src.data(), dst.data(), m.data(), n.data(), (int32_t)k, INT64_MAX, &opt,
                                  (tc_stream_t)s, &b);
    if (st == TC_OK) st = tc_batch_count(b, (tc_stream_t)s, total.data());
    tc_batch_free(b);
    if (st == TC_OK) return;
    for (size_t j = 0; j < k; ++j) status[j] = count_alone(opt, grp[j], s, &total[j]);
}

static void slot_loop(tc_server* sv, int slot) {
    cudaSetDevice(sv->device);
    cudaStream_t s = nullptr;
    const bool have_stream = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    std::vector<Request> grp;
    std::vector<uint64_t> total;
    std::vector<tc_status> status;
    for (;;) {
        int64_t bytes = 0;
        grp.clear();
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] {
                return sv->stopping || (!sv->queue.empty() && sv->in_flight + sv->queue.front().bytes <= sv->budget);
            });
            if (sv->stopping) break;
            // the head always fits here; more requests join while the group stays within
            // its edge and vertex limits and the budget
            int64_t edges = 0, verts = 0;
            while (!sv->queue.empty()) {
                const Request& r = sv->queue.front();
                const int64_t e2 = edges + r.m, v2 = verts + r.n;
                const int64_t b2 = grp.empty() ? r.bytes : request_bytes(e2, v2);
                if (!grp.empty() && (e2 > sv->group_edges || v2 > kMaxGroupVertices || sv->in_flight + b2 > sv->budget))
                    break;
                grp.push_back(r);
                sv->queue.pop_front();
                edges = e2;
                verts = v2;
                bytes = b2;
            }
            sv->in_flight += bytes;
            if (sv->in_flight > sv->peak_in_flight) sv->peak_in_flight = sv->in_flight;
            ++sv->busy;
            if (sv->busy > sv->peak_busy) sv->peak_busy = sv->busy;
            ++sv->groups;
            if (grp.size() > 1) sv->grouped += (int64_t)grp.size();
        }
        const double t_start = now_s();
        if (have_stream) {
            count_group(sv->opt, grp, s, total, status);
        } else {
            total.assign(grp.size(), 0);
            status.assign(grp.size(), TC_ERR_CUDA);
        }
        const double t_done = now_s();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (size_t j = 0; j < grp.size(); ++j) {
                tc_result r;
                std::memset(&r, 0, sizeof(r));
                r.tag = grp[j].tag;
                r.status = status[j];
                r.total = status[j] == TC_OK ? total[j] : 0;
                r.slot = slot;
                r.group = (int32_t)grp.size();
                r.t_submit = grp[j].t_submit;
                r.t_start = t_start;
                r.t_done = t_done;
                sv->results.push_back(r);
            }
            sv->in_flight -= bytes;
            --sv->busy;
            sv->finished += (int64_t)grp.size();
        }
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
    if (have_stream) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
}

}  // namespace tcg

extern "C" {

tc_status tc_server_create(int64_t hbm_budget_bytes, int32_t slots, int64_t group_edges, const tc_options* opt,
                           tc_server_t* out) {
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || slots < 1 || slots > 64 || group_edges < 0) return TC_ERR_INVALID_ARG;
    tc_options o;
    tc_options_default(&o);
    if (opt) o = *opt;
    TC_TRY(check_options(o));
    tc_server* sv = new (std::nothrow) tc_server();
    if (!sv) return TC_ERR_OOM;
    sv->opt = o;
    sv->budget = hbm_budget_bytes;
    sv->group_edges = group_edges > 0 ? group_edges : kDefaultGroupEdges;
    cudaGetDevice(&sv->device);
    retain_pool_memory();
    (void)num_sms();
    try {
        for (int i = 0; i < slots; ++i) sv->threads.emplace_back(slot_loop, sv, i);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stopping = true;
        }
        sv->cv_work.notify_all();
        for (auto& t : sv->threads) t.join();
        delete sv;
        return TC_ERR_OOM;
    }
    *out = sv;
    return TC_OK;
}

tc_status tc_server_submit(tc_server_t sv, const int32_t* src, const int32_t* dst, int64_t m, int32_t n,
                           uint64_t tag) {
    if (!sv || m < 0 || n < 0 || (m > 0 && (!src || !dst))) return TC_ERR_INVALID_ARG;
    const int64_t bytes = request_bytes(m, n);
    if (bytes > sv->budget) return TC_ERR_BUDGET;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) return TC_ERR_INVALID_ARG;
        sv->queue.push_back(Request{src, dst, m, n, tag, now_s(), bytes});
        ++sv->submitted;
    }
    sv->cv_work.notify_one();
    return TC_OK;
}

tc_status tc_server_cancel(tc_server_t sv, uint64_t tag, int64_t* n_cancelled) {
    if (!sv) return TC_ERR_INVALID_ARG;
    int64_t k = 0;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        const double t = now_s();
        for (auto it = sv->queue.begin(); it != sv->queue.end();) {
            if (it->tag != tag) {
                ++it;
                continue;
            }
            tc_result r;
            std::memset(&r, 0, sizeof(r));
            r.tag = it->tag;
            r.status = TC_ERR_CANCELLED;
            r.slot = -1;
            r.group = 0;
            r.t_submit = it->t_submit;
            r.t_start = t;
            r.t_done = t;
            sv->results.push_back(r);
            it = sv->queue.erase(it);
            ++sv->finished;
            ++k;
        }
    }
    if (k) {
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
    if (n_cancelled) *n_cancelled = k;
    return TC_OK;
}

tc_status tc_server_poll(tc_server_t sv, tc_result* out, int32_t max, int32_t* n_out) {
    if (!sv || !n_out || max < 0 || (max > 0 && !out)) return TC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    int32_t k = 0;
    while (k < max && !sv->results.empty()) {
        out[k++] = sv->results.front();
        sv->results.pop_front();
    }
    *n_out = k;
    return TC_OK;
}

tc_status tc_server_drain(tc_server_t sv, int64_t timeout_ms) {
    if (!sv) return TC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto done = [&] { return sv->finished >= sv->submitted; };
    if (timeout_ms < 0) {
        sv->cv_done.wait(lk, done);
        return TC_OK;
    }
    return sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done) ? TC_OK : TC_ERR_TIMEOUT;
}

tc_status tc_server_get_stats(tc_server_t sv, tc_server_stats* st) {
    if (!sv || !st) return TC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = sv->submitted;
    st->finished = sv->finished;
    st->queued = (int64_t)sv->queue.size();
    st->groups = sv->groups;
    st->grouped = sv->grouped;
    st->bytes_in_flight = sv->in_flight;
    st->peak_bytes_in_flight = sv->peak_in_flight;
    st->peak_slots_busy = sv->peak_busy;
    return TC_OK;
}

void tc_server_destroy(tc_server_t sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->threads) t.join();
    delete sv;
}

}  // extern "C"

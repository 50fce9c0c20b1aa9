// graph.cuh -- the device representation behind a tc_graph_t handle.
#pragma once

#include "common.cuh"

namespace tcg {

// One task = one oriented edge, owned by the endpoint with the longer N+ list.  The owner's
// list is staged in shared memory; the partner's list N+(partner) = cols[pstart, pstart+plen)
// is streamed through it.  16 bytes, so a warp reads its tasks with one vector load each.
struct __align__(16) TaskRec {
    uint32_t owner;
    uint32_t partner;
    uint32_t pstart;
    uint32_t plen;
};

// Device-side scheduling state of one count (Sec. V-B): total cost C, the initial share H
// (Eq. 1), the Eq. 2 floor, and the head of the dynamic queue.
struct Sched {
    unsigned long long C;
    unsigned long long H;
    unsigned long long min_chunk;
    unsigned long long head;
    unsigned long long n_chunks;
    unsigned long long base;  // exclusive prefix at the class's first task
    unsigned long long streamed;  // partner-list entries the class's kernel read (traced counts only)
    unsigned long long at_start;  // 1: this schedule starts at the class's first task (not a later part)
    unsigned long long at_end;    // 1: it ends at the class's last task
};

// Device counters written by the build kernels.
struct BuildCounters {
    unsigned long long self_loops;
    unsigned long long unique;
    unsigned long long tasks;
    unsigned long long sum_dhat_v;
    unsigned long long sum_dhat_u;
    unsigned long long sum_stream;
    unsigned long long tasks_small;
    long long bad_index;
    int max_degree;
    int max_dhat;
};

// Workspace of the count, allocated on the handle's first count and reused.
struct CountWork {
    uint64_t* prefix = nullptr;   // T + 1
    int64_t prefix_len = 0;
    uint64_t* scan_scr = nullptr;
    int64_t scan_words = 0;
    uint64_t* fcost = nullptr;    // n, per-vertex cost models only
    Sched* sched = nullptr;       // two: the small and the big class
    unsigned long long* result = nullptr;  // device copy of the last total
};

}  // namespace tcg

struct tc_graph {
    int device = 0;
    tc_options opt{};
    tcg::Allocator al;
    int32_t n = 0;
    int id_bits = 1;
    int64_t m_in = 0, self_loops = 0, duplicates = 0, m_hat = 0, tasks = 0, bad_index = -1;
    int64_t tasks_small = 0;       // tasks [0, tasks_small) have owners with at most opt.small_max entries
    int32_t max_degree = 0, max_dhat = 0;
    uint64_t sum_dhat_v = 0, sum_dhat_u = 0, sum_stream = 0;
    // device arrays owned by the handle
    int32_t* deg = nullptr;        // n
    int64_t* off = nullptr;        // n + 1
    int32_t* cols = nullptr;       // m_hat
    tcg::TaskRec* trec = nullptr;  // tasks
    uint32_t* own_first = nullptr; // first task of each big owner, then `tasks` (owners_big + 1 used)
    int64_t owners_big = 0, own_first_cap = 0;
    tcg::DevStatus* status = nullptr;
    tcg::CountWork work;
    int64_t bytes = 0;             // device bytes held
    // A pack (batched counting): the handle holds n_sub graphs as one disjoint union, graph j's
    // vertex v being vertex vbase[j] + v.  sub_task (device, 2 (n_sub + 1)) holds, per task
    // class, the first task of each graph and then the class's end; a count writes n_sub totals.
    int32_t n_sub = 0;
    int64_t* sub_task = nullptr;
    cudaStream_t last_stream = nullptr;  // stream of the last call; tc_free waits for it
};

namespace tcg {

// The count pipeline (count.cu): cost prefix, schedule init, persistent count kernel.
// Results: total into *total_dev (device uint64), optional t_v (device, n) and per-edge
// counts (device, m_hat), optional trace.  Enqueue only (no synchronisation).
// With nparts > 1 only part `part` is counted: per class, the tasks whose exclusive cost
// prefix lies in [C part / nparts, C (part + 1) / nparts).
tc_status count_enqueue(tc_graph* g, const tc_options& opt, cudaStream_t s, unsigned long long* total_dev,
                        unsigned long long* t_v, uint32_t* per_edge, tc_count_trace* trace, int part = 0,
                        int nparts = 1);

tc_status ensure_count_work(tc_graph* g, const tc_options& opt, cudaStream_t s);

tc_status vertex_cost_enqueue(tc_graph* g, int fn, cudaStream_t s, uint64_t* f);

tc_status clustering_enqueue(tc_graph* g, const uint64_t* t_v, double* cc, cudaStream_t s);

// One pack of a batch as the multi-pack count sees it (device memory, one per pack).  A pack's
// cost prefix P holds running sums over the whole batch (pack after pack); only differences
// within a pack are used.
struct PackDev {
    const int64_t* off;
    const int32_t* cols;
    const TaskRec* tasks;
    const int32_t* deg;
    uint64_t* P;                 // T + 1
    const uint64_t* fcost;       // per-vertex cost models only
    const uint32_t* own_first;
    long long n_owners;
    const int64_t* sub_task;     // per class: first task of each graph, then the class end
    long long n_sub;
    long long Ts, T;
    long long task_base;         // first task of this pack in the batch's pack-after-pack order
    long long tile_base;         // first scan tile of this pack (each pack starts a new tile)
    unsigned long long* total;   // the totals of the pack's graphs
};

// Count every pack of a batch with one cost prefix over all packs and one launch of each
// class kernel: per class, one Eq. 1 + Eq. 2 schedule over the packs' concatenated costs.
// `packs_dev`: n_packs PackDev entries (device), followed by scratch the call lays out itself
// (multi_scratch_words(...) uint64 words at `scratch`).  totals: device, the batch's k totals.
int64_t multi_scratch_words(int64_t total_tasks, int n_packs);
tc_status count_enqueue_multi(const std::vector<tc_graph*>& packs, const PackDev* packs_dev, uint64_t* scratch,
                              const tc_options& opt, unsigned long long* totals, int32_t k, cudaStream_t s);

// Build (build.cu).  src/dst are device pointers here.
tc_status build_graph(tc_graph* g, const int32_t* src_d, const int32_t* dst_d, int64_t m, int32_t n,
                      cudaStream_t s);

tc_status check_options(const tc_options& o);

// Handle life cycle (api.cu): an empty handle with its status block; release everything;
// read (and clear) the device error word after synchronising s, optionally the last total.
tc_status new_graph(const tc_options& o, cudaStream_t s, tc_graph** out);
void free_graph(tc_graph* g);
tc_status read_status(tc_graph* g, cudaStream_t s, unsigned long long* result);

// Memory kinds (api.cu): device (or managed) memory; the device address of pinned host
// memory (null for anything else).
bool is_device_pointer(const void* p);
const void* pinned_device_view(const void* p);

// Device bytes a build of (m, n) holds at its peak, and a built graph keeps (api.cu).
int64_t build_peak_bytes(int64_t m, int32_t n, bool host_input);
int64_t graph_resident_bytes(int64_t m_hat, int64_t tasks, int32_t n);

// Slots of one small-class warp table: room for one owner of small_max entries at a load of
// at most 1/8, and at least 1024 so that a window of tiny owners fits at once.  Region
// offsets are packed in 16 bits, so at most 32768.
inline int small_table_slots(int small_max) {
    int p = 4;
    while (p < small_max) p <<= 1;
    return 8 * p > 1024 ? 8 * p : 1024;
}

}  // namespace tcg

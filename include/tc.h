/*
 * tc.h -- C ABI of the GB300 exact triangle counter.
 *
 * Method: the degree-ordered node-iterator of Arifuzzaman, Khan and Marathe,
 * "Parallel Algorithms for Counting Triangles in Networks with Large Degrees"
 * (arXiv 1406.5687), Fig. 1, with the cost-balanced dynamic load balancing of
 * Sec. V (Eq. 1 and Eq. 2), run as CUDA kernels on one sm_103a GPU.
 *
 * Steps of the path, as the comments below name them:
 *   a1 canonical edge keys (ids checked, self-loops dropped)   a2 sort + dedupe
 *   a3 degrees d_v          a4 orientation by the order of Sec. III-A
 *   a5 the N+ lists of Fig. 1 (offsets, ascending lists)
 *   a6 task costs, their prefix and the Eq. 1 / Eq. 2 schedule
 *   a7 |N+(v) ∩ N+(u)| for every oriented edge (Fig. 1's last loop)
 *   a8 the exact reduction to T (and optional T_v, per-edge counts)
 *
 * Conventions for every call:
 *   - Vertex ids are int32 in [0, n).  Counts are exact uint64.
 *   - Pointers marked "host or device" may point to either; the library asks the
 *     CUDA runtime which.  Pointers marked "device" must be device memory of the
 *     current device.  Pointers marked "host" must be host memory.
 *   - The caller owns every buffer it passes in; the library never frees or keeps
 *     it after the call returns (unless stated).  The library owns the opaque
 *     handles it returns and all device memory behind them until the matching
 *     *_free / *_destroy call.
 *   - Work is enqueued on `stream` (NULL = the legacy default stream).  Calls
 *     that return results into host memory synchronise that stream.
 *   - Errors are returned as tc_status, never thrown or printed.  When a kernel
 *     detects a problem it sets a device error word; the first error wins and is
 *     returned by the next call that synchronises.  No kernel traps or asserts.
 *   - The device used is the current CUDA device at the call.
 */
#ifndef TC_H_
#define TC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared without the CUDA headers. */
typedef struct CUstream_st* tc_stream_t;

typedef enum tc_status {
    TC_OK = 0,
    TC_ERR_INVALID_ARG = 1,   /* NULL/negative argument, bad option, or strict input policy saw a loop or repeat */
    TC_ERR_VERTEX_RANGE = 2,  /* an input id outside [0, n) */
    TC_ERR_OOM = 3,           /* a device or pinned-host allocation failed */
    TC_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    TC_ERR_TIMEOUT = 5,       /* a bounded device wait or retry loop gave up */
    TC_ERR_BUDGET = 6,        /* the request needs more device memory than the configured budget */
    TC_ERR_UNSUPPORTED = 7,   /* the input exceeds a limit of this build (e.g. n >= 2^31 - 1) */
    TC_ERR_CANCELLED = 8      /* a queued serving request withdrawn by tc_server_cancel */
} tc_status;

/* Static text for a status code (never NULL). */
const char* tc_status_str(tc_status s);

/* Library version string, e.g. "1.0.0 sm_103a". */
const char* tc_version(void);

/* ------------------------------------------------------------------ options */

/*
 * Cost of a task, used for the partition (step a6).  A task is one oriented edge,
 * owned by the endpoint with the longer list.
 *   TC_COST_EDGE    this build's model of its own work: pieces(owner) *
 *                   (d^_partner + c_task), plus d^_owner + c_owner on the owner's
 *                   last task (default);
 *   TC_COST_MERGE   the paper's merge cost d^_v + d^_u of one edge (Sec. III-A);
 *   TC_COST_ONE     f(v) = 1 (Sec. V-A), per owner vertex;
 *   TC_COST_DEGREE  f(v) = d_v (Sec. V-A), per owner vertex;
 *   TC_COST_PATRIC  f(v) = sum_{u in N_v} (d^_v + d^_u) (Sec. IV-B), per owner vertex;
 *   TC_COST_NEW     f(v) = sum_{u in Nfull_v - N_v} (d^_v + d^_u) (Sec. IV-F), per owner.
 * Per-vertex costs sit on the owner's last task, so a chunk never splits a vertex
 * (the paper's atomic task <v,1>, Sec. V-A).  The cost changes speed, never the count.
 */
typedef enum tc_cost_model {
    TC_COST_EDGE = 0,
    TC_COST_MERGE = 1,
    TC_COST_ONE = 2,
    TC_COST_DEGREE = 3,
    TC_COST_PATRIC = 4,
    TC_COST_NEW = 5
} tc_cost_model;

/* Per-vertex cost functions for tc_vertex_cost (Sec. IV-B, IV-F, V-A).  TC_FN_LIST, f(v) = |N_v|
 * (the entries of v's list, so parts of equal cost hold about m / P entries each, Sec. IV), is for
 * tc_surrogate_plan only. */
typedef enum tc_cost_fn { TC_FN_ONE = 0, TC_FN_DEGREE = 1, TC_FN_PATRIC = 2, TC_FN_NEW = 3, TC_FN_LIST = 4 } tc_cost_fn;

/* Sec. II assumes a simple graph.  SANITIZE drops self-loops and merges repeated
 * or reversed pairs; STRICT returns TC_ERR_INVALID_ARG if it sees any. */
typedef enum tc_input_policy { TC_INPUT_SANITIZE = 0, TC_INPUT_STRICT = 1 } tc_input_policy;

/*
 * Optional device allocator.  alloc returns NULL on failure (the library then
 * returns TC_ERR_OOM); release frees what alloc returned.  Both get the stream
 * the memory is used on.  NULL hooks select cudaMallocAsync / cudaFreeAsync.
 */
typedef void* (*tc_alloc_fn)(void* ctx, size_t bytes, tc_stream_t stream);
typedef void (*tc_release_fn)(void* ctx, void* ptr, tc_stream_t stream);

/*
 * Tasks fall in two classes by the length of the owner's list.  Small owners (at most
 * small_max entries) are counted with per-warp hash tables, several owners at a time;
 * big owners one at a time by a whole block, whose warps share one table of 8 * piece
 * slots (lists longer than `piece` are staged in pieces, each partner list streamed
 * once per piece).  In both classes one block is one worker of the schedule.
 */
typedef struct tc_options {
    int32_t input_policy;      /* tc_input_policy */
    int32_t cost_model;        /* tc_cost_model */
    int32_t piece;             /* big owners: list entries staged per block table: 256..4096, power of 2 (default 2048) */
    int32_t warps_per_block;   /* small-class kernel: warps per block: 1..16, power of 2 (default 16) */
    int32_t blocks_per_sm;     /* cap on resident blocks per SM of both count kernels (0 = as many as fit) */
    int32_t big_warps;         /* big-class kernel: warps per block (one worker): 4, 8 or 16 (default 16) */
    int32_t small_max;         /* build option: owners with at most this many list entries are small:
                                  0, 16, 32, 64, 128 or 256 (default 64) */
    int32_t static_percent;    /* share of the total cost handed out as initial tasks (Eq. 1); default 50 */
    int64_t min_chunk;         /* floor of an Eq. 2 chunk, in cost units (0 = automatic) */
    int32_t c_task;            /* TC_COST_EDGE per-task constant (default 4) */
    int32_t c_owner;           /* TC_COST_EDGE per-owner constant (default 32) */
    int32_t reserved;
    int64_t hbm_budget_bytes;  /* device memory a build may hold at its peak (0 = no limit) */
    int64_t retry_limit;       /* bound on any device retry loop before TC_ERR_TIMEOUT (0 = default 1<<24) */
    tc_alloc_fn alloc;         /* optional allocator hooks (both or neither) */
    tc_release_fn release;
    void* alloc_ctx;
} tc_options;

/* Fill *opt with the defaults listed above. */
void tc_options_default(tc_options* opt);

/* -------------------------------------------------------------- single graph */

typedef struct tc_graph* tc_graph_t;

/*
 * Build the device representation of a graph (steps a1-a5 and the task array):
 * canonical keys, radix sort, dedupe, degrees, orientation by the order of
 * Sec. III-A, the N+ lists of Fig. 1 (sorted ascending), and the owner-grouped
 * task array.
 *   src, dst  host or device, m int32 each: edge i is (src[i], dst[i]); never modified.
 *             Pinned (page-locked) host lists are read in place by the first kernel;
 *             pageable ones are copied to device memory first.
 *   m         number of input pairs (>= 0).
 *   n         number of vertices, 0 <= n <= 2^30 (TC_ERR_UNSUPPORTED beyond);
 *             at most 2^32 - 2 distinct edges.
 *   opt       NULL for defaults; copied into the handle.
 *   out       receives the handle; NULL on error.
 * Errors: TC_ERR_INVALID_ARG (NULL pointers with m > 0, negative sizes, bad
 * options, strict policy violated), TC_ERR_VERTEX_RANGE, TC_ERR_OOM,
 * TC_ERR_BUDGET, TC_ERR_CUDA.  Synchronises `stream`.
 */
tc_status tc_build(const int32_t* src, const int32_t* dst, int64_t m, int32_t n,
                   const tc_options* opt, tc_stream_t stream, tc_graph_t* out);

/*
 * tc_build for an edge list stored as interleaved pairs: edge i is (edges[2i], edges[2i+1]).
 *   edges     host or device, 2 m int32; never modified.  A kernel splits the pairs into two
 *             device arrays (page-locked host pairs are read in place, pageable ones copied
 *             first), which then go through tc_build; they hold 8 m bytes more than tc_build's
 *             peak while it runs, counted against opt->hbm_budget_bytes.
 * Other arguments, results and errors as for tc_build.
 */
tc_status tc_build_pairs(const int32_t* edges, int64_t m, int32_t n, const tc_options* opt,
                         tc_stream_t stream, tc_graph_t* out);

/* Release a handle and its device memory (NULL-safe).  Waits for the stream of the
 * handle's last call; the handle must not be in use on any other stream. */
void tc_free(tc_graph_t g);

/*
 * Exact triangle count T = sum over oriented edges (v,u) of |N+(v) ∩ N+(u)|
 * (Fig. 1; Sec. V's schedule; steps a6-a8).
 *   total  host; receives T.
 * Synchronises `stream`.  Errors: TC_ERR_INVALID_ARG, TC_ERR_CUDA, TC_ERR_TIMEOUT, TC_ERR_OOM.
 */
tc_status tc_count(tc_graph_t g, tc_stream_t stream, uint64_t* total);

/*
 * Same count, enqueued only: total_dev (device, one uint64) receives T when the
 * stream reaches it.  Nothing is allocated after the handle's first count, so
 * the call can be captured into a CUDA graph after one warm-up call.  Device-side
 * errors are reported by tc_graph_check.
 */
tc_status tc_count_async(tc_graph_t g, tc_stream_t stream, uint64_t* total_dev);

/*
 * Count k graphs already built (each as tc_count), enqueued back to back on `stream`, with one
 * synchronisation for all of them.  For many graphs not yet built, tc_batch_build packs them
 * into disjoint unions that build and count in one pass each.
 *   gs      host, k handles of the current device (a handle may repeat; none may be in use on
 *           another stream).
 *   totals  host, k uint64: totals[j] = T of gs[j].
 * Errors: TC_ERR_INVALID_ARG (k < 0, NULL pointers), and the first error of any graph's count,
 * in the order of gs.  Synchronises `stream`.
 */
tc_status tc_count_graphs(const tc_graph_t* gs, int32_t k, tc_stream_t stream, uint64_t* totals);

/*
 * Count one part of the graph's tasks, for a count split over several GPUs (each holding a
 * replica of the graph) or several calls.  Per task class, part p of P takes the tasks whose
 * exclusive cost prefix lies in [C p / P, C (p + 1) / P) -- Sec. IV-B's cost-balanced
 * partition, applied to the task costs of a6 -- and schedules them by Eq. 1 + Eq. 2 among
 * this GPU's workers.  Every task lies in exactly one part, so the sum of the P partial
 * counts (one uint64 reduction, the MPI_Reduce of Fig. 11) is T.
 *   part, nparts  0 <= part < nparts.
 *   partial       host; receives this part's count.
 * Synchronises `stream`.
 */
tc_status tc_count_partition(tc_graph_t g, int32_t part, int32_t nparts, tc_stream_t stream,
                             uint64_t* partial);

/* Synchronise `stream` and return (and clear) the handle's device error word. */
tc_status tc_graph_check(tc_graph_t g, tc_stream_t stream);

/*
 * Per-vertex counts T_v (Sec. II): each triangle adds one to each of its three
 * vertices, so sum T_v = 3T.
 *   t_v    device, n uint64 (overwritten).
 *   total  host (nullable); receives T.
 */
tc_status tc_count_per_vertex(tc_graph_t g, tc_stream_t stream, uint64_t* t_v, uint64_t* total);

/*
 * Per-oriented-edge counts: c[i] = |N+(v) ∩ N+(u)| for the oriented edge stored at
 * position i of the N+ lists (tc_graph_csr); by Theorem 1 each triangle is counted
 * on exactly one edge: the one joining its lowest and middle vertex.
 *   c      device, m_hat uint32 (overwritten).
 *   total  host (nullable); receives T.
 */
tc_status tc_count_per_edge(tc_graph_t g, tc_stream_t stream, uint32_t* c, uint64_t* total);

/* Local clustering coefficients C_v = 2 T_v / (d_v (d_v - 1)), 0 when d_v < 2
 * (the use named in Sec. I).  t_v: device, n uint64 from tc_count_per_vertex;
 * cc: device, n double (overwritten). */
tc_status tc_clustering(tc_graph_t g, const uint64_t* t_v, double* cc, tc_stream_t stream);

/* ----------------------------------------------------------- introspection */

typedef struct tc_graph_info {
    int32_t n;
    int32_t max_degree;    /* max d_v */
    int32_t max_dhat;      /* max |N+(v)| (effective degree, Sec. III-A) */
    int32_t id_bits;       /* bits per vertex id in the sort keys */
    int64_t m_in;          /* input pairs */
    int64_t self_loops;    /* dropped (sanitize) */
    int64_t duplicates;    /* merged repeats, either orientation (sanitize) */
    int64_t m_hat;         /* distinct undirected edges = oriented edges */
    int64_t tasks;         /* oriented edges whose partner list is non-empty */
    int64_t tasks_small;   /* of which owned by small owners (they come first in the task array) */
    uint64_t sum_dhat_v;   /* sum over oriented edges (v,u) of d^_v */
    uint64_t sum_dhat_u;   /* sum over oriented edges (v,u) of d^_u */
    uint64_t sum_stream;   /* sum over tasks of d^_partner: list entries the count kernel streams (piece 1024) */
    int64_t device_bytes;  /* device memory held by the handle */
} tc_graph_info;

tc_status tc_graph_get_info(tc_graph_t g, tc_graph_info* info);

/*
 * Device pointers to the handle's arrays (valid until tc_free; read-only):
 *   deg   n int32          d_v
 *   off   n+1 int64        N+(v) = cols[off[v] .. off[v+1])
 *   cols  m_hat int32      ascending within each list
 *   tasks 4*tasks uint32   one record per task: owner, partner, start of N+(partner) in
 *                          cols, |N+(partner)|; the small class first, then by owner, and
 *                          an owner's tasks in the order of their oriented edges in cols
 * Any output pointer may be NULL.
 */
tc_status tc_graph_csr(tc_graph_t g, const int32_t** deg, const int64_t** off, const int32_t** cols,
                       const uint32_t** tasks);

/*
 * Per-vertex cost f(v) (step a6): fn is a tc_cost_fn.
 *   f  device, n uint64 (overwritten).
 */
tc_status tc_vertex_cost(tc_graph_t g, int32_t fn, tc_stream_t stream, uint64_t* f);

/*
 * Count with explicit options and a record of the schedule (steps a6-a8).  Each task
 * class is scheduled on its own (Eq. 1 + Eq. 2 over its own costs, class c in cost
 * units counted from 0) by its own kernel.
 *   opt      NULL = the handle's options; the build-time small_max is always the handle's.
 *   total    host; receives T.
 *   trace    NULL, or a record the count fills in:
 *              chunks  device, 4*cap uint64 or NULL: one record per chunk a worker
 *                      took, ((class << 56) | cost_lo, cost_hi, task_lo, task_hi),
 *                      task indices into the whole task array, in no particular
 *                      order; records beyond cap are dropped;
 *              workers_busy device, 2*(n_workers[0] + n_workers[1]) uint64 or
 *                      NULL: per worker (a worker is one block; small-class blocks
 *                      first, then big-class blocks), (clock64 cycles spent on
 *                      tasks, chunks taken) -- the per-worker idle time of Sec. V-E;
 *            and on return: n_chunks (records produced), and per class c:
 *            n_workers[c] (W), total_cost[c] (C), min_chunk[c] (the Eq. 2 floor
 *            used); tasks_small; the CUDA-event times of the cost prefix and
 *            schedule set-up (prefix_ms) and of each class's kernel; with
 *            count_streamed set, streamed[c]: the partner-list entries class c's kernel
 *            read (big owners read only the part of each partner list inside the owner
 *            list's [first, last] range).  Counting adds one atomic per warp batch.
 * With trace != NULL the call synchronises `stream` before returning.
 */
/* Partner lists of big owners with at least this many entries are trimmed to the owner
 * list's [first, last] range before they are probed; shorter ones are probed whole. */
#define TC_TRIM_MIN_ENTRIES 16

typedef struct tc_count_trace {
    uint64_t* chunks;
    int64_t cap;
    uint64_t* workers_busy;
    int64_t n_chunks;
    int64_t n_workers[2];
    uint64_t total_cost[2];
    uint64_t min_chunk[2];
    int64_t tasks_small;
    float prefix_ms;        /* a6: task costs, prefix, schedule set-up */
    float kernel_small_ms;  /* a7-a8, small-owner kernel */
    float kernel_big_ms;    /* a7-a8, big-owner kernel */
    int32_t count_streamed; /* in: nonzero = count the partner-list entries each kernel reads */
    int64_t streamed[2];    /* out: those entries per class (after trimming), or -1 */
} tc_count_trace;

tc_status tc_count_ex(tc_graph_t g, const tc_options* opt, tc_stream_t stream, uint64_t* total,
                      tc_count_trace* trace);

/* Number of kernels this library has launched in this process so far (all devices,
 * all handles); differences around a region count the launches inside it. */
int64_t tc_kernel_launches(void);

/*
 * Count without allocating.  The paper has no counterpart: this exists for callers that
 * must not allocate device memory at count time -- code that owns all device memory
 * through its own pool, runs where an allocation could block or is not permitted, or
 * has no room left to give.  It is tc_count_async with the count's scratch (the cost
 * prefix of at most TC_COUNT_STATIC_MAX_TASKS + 1 entries, the scan's partial sums and
 * the two schedule records, about 4 MiB) held in one fixed device array that the library
 * declares statically; every GPU that loads the library keeps that array until the
 * process exits.  It never calls cudaMalloc, cudaFree or any other allocating routine.
 *   g          a built graph (its arrays are the inputs); its options must use
 *              TC_COST_EDGE or TC_COST_MERGE (per-vertex cost models need a per-vertex
 *              array: TC_ERR_INVALID_ARG).
 *   total_dev  device, one uint64; receives T when the stream reaches it (output).
 * Errors: TC_ERR_UNSUPPORTED when the graph has more than TC_COUNT_STATIC_MAX_TASKS
 * tasks (tc_graph_info.tasks); TC_ERR_INVALID_ARG; TC_ERR_CUDA.  Device-side errors are
 * reported by tc_graph_check.
 * The first call on a device looks up the array's device address on that device; make
 * that first call before any stream capture.  Every call shares the one array and
 * leaves its contents behind (each call rewrites what it reads), so calls whose work
 * overlaps on the GPU -- on different streams, or on the same graph from several
 * threads -- race and give wrong totals: serialise them.
 */
#define TC_COUNT_STATIC_MAX_TASKS (1ll << 19)
tc_status tc_count_static(tc_graph_t g, tc_stream_t stream, uint64_t* total_dev);

/*
 * Self-test of the library's bounded device waits (the paper has no counterpart).  One
 * thread waits, through the same wait routine the radix sort's look-back uses, on a device
 * flag that nothing sets.  It must give up after spin_limit polls (>= 1) and return
 * TC_ERR_TIMEOUT; the CUDA context stays usable.  Synchronises `stream`.
 */
tc_status tc_wait_selftest(int64_t spin_limit, tc_stream_t stream);

/* ------------------------------------------------- non-overlapping partition (Sec. IV) */

/*
 * Count over a non-overlapping partition, for N+ lists that need not fit in device memory
 * (Sec. IV, the space-efficient algorithm).  The input is the oriented graph itself, in the
 * layout of tc_graph_csr: N_v = cols[off[v] .. off[v+1]), each list strictly ascending, every
 * triangle appearing as (v, u, w) with u, w in N_v and w in N_u (Fig. 1's orientation).
 *
 * The vertices are split into the sets of consecutive ids V_j = [cuts[j], cuts[j+1]) of Def. 1;
 * part j's partition G_j is the lists N_u, u in V_j, one contiguous slice of cols.  Parts
 * part_lo .. part_hi-1 are counted one after another on this GPU: part j's slice is copied to
 * device memory (the copy of the next part overlapping the count of this one), and every list
 * N_v holding an entry in V_j is a data message to part j, sent once (the surrogate approach of
 * Sec. IV-C), which adds SurrogateCount(N_v, j) = sum over u in N_v ∩ V_j of |N_u ∩ N_v|
 * (Fig. 2).  Messages are read in place.  Device memory holds the offsets, two per-vertex
 * cursors (8 n bytes), the work items (16 (n + m / 256) bytes) and two part slices, never all
 * of cols.
 *   off        host or device, n + 1 int64: off[0] = 0, non-decreasing, off[n] = m.
 *   cols       host or device, m int32.  Host lists are read over the host link; page-locked
 *              memory is read in place, pageable memory is page-locked for the call.
 *   n, m       vertices (0 <= n < 2^31 - 1) and list entries.
 *   cuts       host, nparts + 1 int32: cuts[0] = 0, cuts[nparts] = n, non-decreasing (empty
 *              sets allowed); 1 <= nparts <= TC_SURROGATE_MAX_PARTS.
 *   part_lo, part_hi  the receiving parts counted: 0 <= part_lo <= part_hi <= nparts.  Disjoint
 *              ranges counted separately (on several GPUs, or calls) add up to the full count.
 *   opt        NULL for defaults; only the allocator hooks and hbm_budget_bytes are used.
 *   table      host, nparts * nparts uint64, or NULL: table[i * nparts + j] = the sum over v in
 *              V_i of SurrogateCount(N_v, j), the triangles whose two lowest vertices (in the
 *              orientation's order) lie in V_i and V_j; columns outside [part_lo, part_hi) are 0.
 *   total      host; the sum of the table: T when the range covers every part.
 *   stats      host, or NULL: filled with the work done (counting it adds one atomic per warp
 *              batch, and CUDA events around every kernel).
 * Errors: TC_ERR_INVALID_ARG (bad sizes or cuts, off not as stated, a list not strictly
 * ascending, pageable host lists that partly overlap lists another call has page-locked),
 * TC_ERR_VERTEX_RANGE (a list entry outside [0, n), found when the range covers the lists'
 * entries), TC_ERR_UNSUPPORTED (a part slice of 2^32 - 8 or more entries), TC_ERR_OOM,
 * TC_ERR_BUDGET, TC_ERR_CUDA.  Synchronises `stream`.  Calls may run at once on other streams
 * and threads, on the same lists.
 */
#define TC_SURROGATE_MAX_PARTS 1024
/* Messages longer than this are staged a piece of this many entries at a time, each resident list
 * streamed once per piece (trimmed to the piece's [first, last] range). */
#define TC_SURROGATE_PIECE 256
typedef struct tc_surrogate_stats {
    int64_t items;         /* work items: runs of at most 256 entries of one message in one part */
    int64_t staged;        /* message entries staged into shared memory (X of Fig. 2) */
    int64_t streamed;      /* resident list entries streamed through them, after trimming each
                              N_u to its message's [first, last] range */
    int64_t copied_bytes;  /* part slices copied into device memory */
    float route_ms;        /* CUDA-event time of the routing kernels, all parts */
    float count_ms;        /* CUDA-event time of the count kernels, all parts */
} tc_surrogate_stats;
tc_status tc_count_surrogate(const int64_t* off, const int32_t* cols, int32_t n, int64_t m, const int32_t* cuts,
                             int32_t nparts, int32_t part_lo, int32_t part_hi, const tc_options* opt,
                             tc_stream_t stream, uint64_t* table, uint64_t* total, tc_surrogate_stats* stats);

/*
 * Cuts for tc_count_surrogate (Sec. IV-B): with a per-vertex cost f, cuts[k] is the first vertex q
 * whose exclusive prefix F[q] = f(0) + ... + f(q-1) reaches ceil(k F[n] / P); cuts[0] = 0 and
 * cuts[P] = n.  Every part then holds about 1 / P of the cost.
 *   off, cols, n, m  as for tc_count_surrogate (cols is read only for DEGREE, PATRIC and NEW).
 *   fn         a tc_cost_fn.  TC_FN_NEW (Sec. IV-F): f(u) = sum over the lists N_v holding u of
 *              (|N_u| + |N_v|), the work u's part does for u: parts of equal work, for parts
 *              counted on several GPUs.  TC_FN_LIST: f(v) = |N_v|: parts of equal size, the
 *              fewest parts within a memory bound.  ONE, DEGREE (d_v) and PATRIC (Sec. IV-B)
 *              as for tc_vertex_cost.
 *   nparts     > 0: P = nparts.  0: the smallest P in [ceil(4 m / part_bytes), max_parts] whose
 *              cuts keep every part's slice within part_bytes.
 *   part_bytes bytes of one part's slice (4 per entry); 0 = no limit (needs nparts > 0).
 *   max_parts  upper bound on P when nparts = 0 (<= TC_SURROGATE_MAX_PARTS).
 *   cuts       host, receives P + 1 int32 (capacity nparts + 1, or max_parts + 1).
 *   nparts_out host; receives P.
 * Errors: TC_ERR_BUDGET (no P within the bounds fits; the last cuts tried are written),
 * TC_ERR_INVALID_ARG, TC_ERR_VERTEX_RANGE, TC_ERR_OOM, TC_ERR_CUDA.  Synchronises `stream`.
 */
tc_status tc_surrogate_plan(const int64_t* off, const int32_t* cols, int32_t n, int64_t m, int32_t fn,
                            int32_t nparts, int64_t part_bytes, int32_t max_parts, tc_stream_t stream, int32_t* cuts,
                            int32_t* nparts_out);

/*
 * Cuts bounded in work and in size at once (Sec. IV-B with the cost of Sec. IV-F, and Sec. IV's
 * memory bound): the union of the cuts of work_parts parts of equal cost `fn` (as
 * tc_surrogate_plan with nparts = work_parts) and the cuts of the fewest parts of equal size whose
 * slices fit part_bytes (as tc_surrogate_plan with TC_FN_LIST and nparts = 0).  Every part lies
 * inside one part of each, so its cost is at most 1 / work_parts of the total plus one vertex's
 * cost, and its slice at most part_bytes.  Equal-size cuts alone can leave most of the work in
 * one part (the part holding the hubs); equal-work cuts alone can make one slice large.
 *   fn, off, cols, n, m  as for tc_surrogate_plan.
 *   work_parts  1 .. TC_SURROGATE_MAX_PARTS.
 *   part_bytes  > 0; max_parts bounds the equal-size part count (1 .. TC_SURROGATE_MAX_PARTS).
 *   cuts        host, receives P + 1 int32, strictly increasing except for n = 0 (capacity
 *               work_parts + max_parts + 1).
 *   nparts_out  host; receives P (at most work_parts + the equal-size part count).
 * Errors: as tc_surrogate_plan; TC_ERR_BUDGET also when P would exceed TC_SURROGATE_MAX_PARTS.
 * Synchronises `stream`.
 */
tc_status tc_surrogate_plan_both(const int64_t* off, const int32_t* cols, int32_t n, int64_t m, int32_t fn,
                                 int32_t work_parts, int64_t part_bytes, int32_t max_parts, tc_stream_t stream,
                                 int32_t* cuts, int32_t* nparts_out);

/* ------------------------------------------------------------------ batch */

/*
 * Batched counting.  The paper counts one graph at a time; counting many independent graphs
 * in one pass is this library's own addition.  k graphs are packed, as disjoint unions with
 * each graph's vertex ids moved into a range of their own, into as few packs as the limits
 * allow: at most pack_edges input edges and 2^30 vertices per pack, a graph with more edges
 * than pack_edges forming a pack of its own.  Each pack goes once through the single-graph
 * build (steps a1-a5 and the task decomposition), so a pack's sort, degree, orientation and
 * list kernels serve all of its graphs.  Degrees, the order of Sec. III-A and every list are
 * those of each graph alone: the union has no edge between graphs.
 */
typedef struct tc_batch* tc_batch_t;

/*
 * Build a batch.
 *   src, dst    host arrays of k pointers: graph j's edges are src[j][0..m[j]) and
 *               dst[j][0..m[j]) (int32, host or device memory, never modified).
 *   m, n        host arrays of k sizes, m[j] >= 0, 0 <= n[j] <= 2^30.
 *   pack_edges  input edges per pack at most (0 = 2^30).
 *   opt         NULL = defaults; input policy, hub threshold (small_max) and count options
 *               of every graph.
 *   out         receives the batch (free with tc_batch_free).
 * Errors: TC_ERR_INVALID_ARG; TC_ERR_VERTEX_RANGE (an id outside [0, n[j]) in graph j);
 * TC_ERR_OOM / TC_ERR_BUDGET; TC_ERR_UNSUPPORTED (a graph beyond the single-graph limits).
 * Synchronises `stream`.
 */
tc_status tc_batch_build(const int32_t* const* src, const int32_t* const* dst, const int64_t* m,
                         const int32_t* n, int32_t k, int64_t pack_edges, const tc_options* opt,
                         tc_stream_t stream, tc_batch_t* out);

/*
 * Count every graph of the batch.  Per pack: the task costs and their prefix (step a6),
 * one Eq. 1 + Eq. 2 schedule over all of the pack's tasks, and one launch of each count
 * kernel, whose chunks are cut at graph boundaries so that each graph's hits go to its own
 * total.  The launches of all packs are captured into one CUDA graph on the first run (and
 * again after tc_batch_set_options) and replayed.
 *   totals_dev  device, k uint64, overwritten: graph j's exact triangle count at index j.
 * Enqueue only: check errors with tc_batch_check.  Runs of one batch must not overlap on
 * the device (they share its work buffers).
 */
tc_status tc_batch_run(tc_batch_t b, tc_stream_t stream, uint64_t* totals_dev);

/* Synchronise `stream`; return (and clear) the first device error of any pack. */
tc_status tc_batch_check(tc_batch_t b, tc_stream_t stream);

/* tc_batch_run, then copy the k totals to host memory `totals` and check. */
tc_status tc_batch_count(tc_batch_t b, tc_stream_t stream, uint64_t* totals);

typedef struct tc_batch_info {
    int32_t k;             /* graphs */
    int32_t packs;
    int32_t max_dhat;      /* longest N+ list of any graph */
    int32_t reserved;
    int64_t m_in;          /* input edges, all graphs */
    int64_t m_hat;         /* distinct edges, all graphs */
    int64_t tasks;
    int64_t tasks_small;
    int64_t device_bytes;  /* device memory held by the batch */
} tc_batch_info;

tc_status tc_batch_get_info(tc_batch_t b, tc_batch_info* info);

/* Each graph's distinct edge count m_hat[j] (host, k int64). */
tc_status tc_batch_graph_edges(tc_batch_t b, int64_t* m_hat);

/*
 * Replace the count-time options (piece, warps_per_block, big_warps, blocks_per_sm,
 * static_percent, min_chunk, c_task, c_owner, cost_model, retry_limit).  The build-time
 * fields (input_policy, small_max, allocator hooks, budget) must equal the build's:
 * TC_ERR_INVALID_ARG otherwise.  Waits for the batch's last stream.
 */
tc_status tc_batch_set_options(tc_batch_t b, const tc_options* opt);

/* Release the batch (NULL-safe; waits for its last stream). */
void tc_batch_free(tc_batch_t b);

/*
 * Autotuner for the batched count.  The given graphs (a sample of a workload) are built as a
 * batch once per hub threshold small_max in {32, 64, 128}, and each build is counted with
 * every launch shape warps_per_block in {4, 8, 16} (small-owner kernel) x big_warps in
 * {8, 16} x piece in {1024, 2048} (big-owner table of 8 x piece slots).  Each candidate is
 * timed with CUDA events on `stream` and keeps the fastest of `reps` runs after one warm-up.
 *   opt     base options (NULL = defaults); the other fields are kept.
 *   best    receives the fastest candidate's options.
 *   report  optional: entries[0..cap) receive the candidates in the order tried; n, the
 *           fastest time and the time of the base options' own shape (-1 if not in the grid).
 */
typedef struct tc_tune_entry {
    int32_t small_max;
    int32_t warps_per_block;
    int32_t big_warps;
    int32_t piece;
    int32_t static_percent;
    float ms;
} tc_tune_entry;

typedef struct tc_tune_report {
    tc_tune_entry* entries;
    int32_t cap;
    int32_t n;
    float best_ms;
    float default_ms;
} tc_tune_report;

tc_status tc_batch_autotune(const int32_t* const* src, const int32_t* const* dst, const int64_t* m,
                            const int32_t* n, int32_t k, const tc_options* opt, int32_t reps,
                            tc_stream_t stream, tc_options* best, tc_tune_report* report);

/* ---------------------------------------------------------------- serving */

/*
 * Serving with continuous batching (this library's own addition; the paper counts one
 * graph at a time).  Submitted graphs wait in a FIFO host queue.  Each of `slots` slot
 * threads owns a CUDA stream; whenever a slot is free it takes the requests at the head of
 * the queue -- as many as fit within group_edges input edges and within what is left of the
 * device-memory budget -- and counts them: one request through the single-graph path
 * (tc_build + tc_count), several as one batch (tc_batch_build + tc_batch_count, one pack).
 * Requests that arrive while others run are admitted as soon as a slot and memory free up,
 * and the work of different slots overlaps on the device.  A request's device memory
 * (its CSR, tasks and build scratch) is held from admission until its result has been read
 * back, then released.  Every total is exact and the same as the graph's count alone.
 */
typedef struct tc_server* tc_server_t;

typedef struct tc_result {
    uint64_t tag;       /* the caller's tag from tc_server_submit */
    uint64_t total;     /* T (0 if status != TC_OK) */
    int32_t status;     /* tc_status of this request */
    int32_t slot;       /* the slot that ran it */
    int32_t group;      /* requests counted together with it, itself included */
    int32_t reserved;
    double t_submit;    /* seconds on the steady clock when submitted */
    double t_start;     /* when a slot admitted it */
    double t_done;      /* when its result was known on the host */
} tc_result;

/*
 * Create a server on the current device.
 *   hbm_budget_bytes  > 0: device memory the requests in flight may hold together, by the
 *                     library's estimate of each build's peak.
 *   slots             1..64 slot threads (and streams).
 *   group_edges       input edges one slot takes at once at most (0 = 2^26; 1 = every
 *                     request alone).
 *   opt               NULL = defaults; options of every request.
 */
tc_status tc_server_create(int64_t hbm_budget_bytes, int32_t slots, int64_t group_edges,
                           const tc_options* opt, tc_server_t* out);

/*
 * Queue one graph.  src/dst: m int32 each, host (pinned for full copy speed) or device
 * memory.  The server BORROWS them: they must stay valid and unchanged until this request's
 * result has been returned by tc_server_poll.  tag: any value, returned with the result.
 * Errors: TC_ERR_INVALID_ARG; TC_ERR_BUDGET (the graph alone needs more than the budget).
 * A graph's own errors (e.g. TC_ERR_VERTEX_RANGE) come back in its result.
 */
tc_status tc_server_submit(tc_server_t s, const int32_t* src, const int32_t* dst, int64_t m,
                           int32_t n, uint64_t tag);

/*
 * Withdraw the requests with this tag that are still waiting in the queue.  Their results
 * come back from tc_server_poll with status TC_ERR_CANCELLED (and the server no longer
 * borrows their arrays); requests already admitted to a slot run to the end.
 *   n_cancelled  optional (host); receives how many requests were withdrawn.
 */
tc_status tc_server_cancel(tc_server_t s, uint64_t tag, int64_t* n_cancelled);

/* Move up to max finished results into out (host, oldest first); *n_out: how many. */
tc_status tc_server_poll(tc_server_t s, tc_result* out, int32_t max, int32_t* n_out);

/* Block until every submitted request has a result, or timeout_ms passes (TC_ERR_TIMEOUT;
 * timeout_ms < 0 waits without limit). */
tc_status tc_server_drain(tc_server_t s, int64_t timeout_ms);

typedef struct tc_server_stats {
    int64_t submitted;
    int64_t finished;      /* results produced (polled or not) */
    int64_t queued;        /* waiting for a slot */
    int64_t groups;        /* slot admissions */
    int64_t grouped;       /* requests admitted together with others */
    int64_t bytes_in_flight;
    int64_t peak_bytes_in_flight;  /* never above the budget */
    int32_t peak_slots_busy;
    int32_t reserved;
} tc_server_stats;

tc_status tc_server_get_stats(tc_server_t s, tc_server_stats* st);

/* Stop taking requests, finish those in flight, drop those still queued, release
 * everything (NULL-safe). */
void tc_server_destroy(tc_server_t s);

#ifdef __cplusplus
}
#endif

#endif /* TC_H_ */

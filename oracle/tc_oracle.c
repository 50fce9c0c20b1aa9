/*
 * tc_oracle.c -- CPU oracle for exact triangle counting.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It shares
 * no code with the CUDA path: no headers, helpers or tables.
 *
 * Plain, slow, obviously correct C written from the paper (Arifuzzaman, Khan,
 * Marathe, "Parallel Algorithms for Counting Triangles in Networks with Large
 * Degrees", arXiv 1406.5687).  Every function names the passage it follows.
 *
 *   or_simple_graph   Sec. II: the input is a simple undirected graph on
 *                     vertices 0..n-1.  Input policy (the paper is silent on
 *                     dirty input): ids outside [0,n) are an error; "sanitize"
 *                     drops self-loops and merges repeated or reversed pairs;
 *                     "strict" rejects them.
 *   or_oriented_csr   Fig. 1, first two loops: the order u < v iff d_u < d_v or
 *                     (d_u = d_v and u < v) (Sec. III-A); each edge is stored
 *                     once, in the list of its lower endpoint; every list N_v is
 *                     sorted ascending.  An optional rank array replaces the
 *                     order (Sec. III-A: any total order counts each triangle
 *                     once), which the tests use to check order invariance.
 *   or_count          Fig. 1, last loop: T = sum over v, u in N_v of
 *                     |N_v intersect N_u|, by a two-pointer merge of the sorted
 *                     lists.  Optional outputs: the per-oriented-edge counts and
 *                     the per-vertex counts T_v (Sec. II), attributing each
 *                     triangle found at (v,u,w) to v, u and w (Theorem 1: it is
 *                     found exactly once).
 *   or_vertex_cost    Cost functions f(v): f = 1 and f = d_v (Sec. V-A), the
 *                     PATRIC estimate sum_{u in N_v}(dh_v + dh_u) (Sec. IV-B) and
 *                     the new estimate sum_{u in Nfull_v - N_v}(dh_v + dh_u)
 *                     (Sec. IV-F), dh = effective degree |N_v|.
 *   or_count_parts    Sec. IV-A and IV-C: V split into P sets of consecutive
 *                     vertices (Def. 1); processor i sends N_v (v in V_i) once
 *                     to every processor j that owns some u in N_v (the
 *                     surrogate approach, with its LastProc variable), and j
 *                     adds SurrogateCount(N_v, j) = sum over u in N_v with u in
 *                     V_j of |N_u intersect N_v|.  The result is the P x P table
 *                     of those sums by (sender i, counter j), whose total is T.
 *   or_balanced_cuts  Sec. IV-B: cut V into P sets of consecutive vertices whose
 *                     costs each come to about 1/P of the total: cut k is the
 *                     first vertex q whose cost prefix f(0) + ... + f(q-1)
 *                     reaches k/P of the total (cut 0 = 0, cut P = n).
 *   or_schedule       Sec. V-B: the chunk table of the dynamic load balancing
 *                     scheme over a sequence of task costs -- the first half
 *                     of the total cost split into W equal initial tasks (Eq. 1)
 *                     and the rest handed out in chunks of remaining/W (Eq. 2)
 *                     with a floor.  Which tasks there are, and what each costs,
 *                     is the caller's input: the paper's per-vertex costs come
 *                     from or_vertex_cost.
 *
 * Parity of every function is pinned by the tests against brute force,
 * trace(A^3)/6, closed forms and invariants; none is "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    OR_OK = 0,
    OR_ERR_INVALID_ARG = 1,   /* bad sizes, or strict policy saw a loop/duplicate */
    OR_ERR_VERTEX_RANGE = 2,  /* an id outside [0, n) */
    OR_ERR_OOM = 3
};

typedef struct {
    int64_t m_in;        /* input pairs */
    int64_t self_loops;  /* pairs (v, v) */
    int64_t duplicates;  /* extra copies of a pair, in either orientation */
    int64_t m_hat;       /* distinct undirected edges */
    int64_t bad_index;   /* first input index with an id outside [0, n), else -1 */
} or_input_stats;

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Sec. II: reduce the input pairs to the simple undirected graph.
 * Writes the m_hat distinct edges as (ea[i], eb[i]) with ea < eb, sorted by
 * (ea, eb).  ea/eb need capacity m.  Returns an OR_* code.
 */
int or_simple_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, int strict,
                    int32_t* ea, int32_t* eb, or_input_stats* st) {
    st->m_in = m;
    st->self_loops = 0;
    st->duplicates = 0;
    st->m_hat = 0;
    st->bad_index = -1;
    if (n < 0 || m < 0) return OR_ERR_INVALID_ARG;
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) {
            st->bad_index = i;
            return OR_ERR_VERTEX_RANGE;
        }
    }
    /* bucket every non-loop pair under its smaller endpoint */
    int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* bucket = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!start || !fill || !bucket) { free(start); free(fill); free(bucket); return OR_ERR_OOM; }
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] == dst[i]) { st->self_loops++; continue; }
        int32_t a = src[i] < dst[i] ? src[i] : dst[i];
        start[a + 1]++;
    }
    for (int32_t v = 0; v < n; ++v) start[v + 1] += start[v];
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] == dst[i]) continue;
        int32_t a = src[i] < dst[i] ? src[i] : dst[i];
        int32_t b = src[i] < dst[i] ? dst[i] : src[i];
        bucket[start[a] + fill[a]++] = b;
    }
    /* sort each bucket and keep one copy of each pair */
    int64_t out = 0;
    for (int32_t a = 0; a < n; ++a) {
        int64_t lo = start[a], hi = start[a + 1];
        qsort(bucket + lo, (size_t)(hi - lo), sizeof(int32_t), cmp_i32);
        for (int64_t j = lo; j < hi; ++j) {
            if (j > lo && bucket[j] == bucket[j - 1]) { st->duplicates++; continue; }
            ea[out] = a;
            eb[out] = bucket[j];
            ++out;
        }
    }
    st->m_hat = out;
    free(start); free(fill); free(bucket);
    if (strict && (st->self_loops > 0 || st->duplicates > 0)) return OR_ERR_INVALID_ARG;
    return OR_OK;
}

/* The order of Sec. III-A: u < v iff d_u < d_v, or d_u = d_v and u < v. */
static int precedes(int32_t u, int32_t v, const int32_t* deg, const int64_t* rank) {
    if (rank) return rank[u] < rank[v];
    return deg[u] < deg[v] || (deg[u] == deg[v] && u < v);
}

/*
 * Fig. 1, first two loops.  Input: the simple graph (ea, eb), m_hat edges.
 * Output: deg[n] (d_v), off[n+1], cols[m_hat] -- N_v = cols[off[v] .. off[v+1])
 * sorted ascending.  rank == NULL selects the degree order.
 */
int or_oriented_csr(int32_t n, int64_t mh, const int32_t* ea, const int32_t* eb, const int64_t* rank,
                    int32_t* deg, int64_t* off, int32_t* cols) {
    if (n < 0 || mh < 0) return OR_ERR_INVALID_ARG;
    memset(deg, 0, (size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < mh; ++i) { deg[ea[i]]++; deg[eb[i]]++; }
    int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!fill) return OR_ERR_OOM;
    memset(off, 0, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < mh; ++i) {
        int32_t u = ea[i], v = eb[i];
        if (precedes(u, v, deg, rank)) off[u + 1]++; else off[v + 1]++;
    }
    for (int32_t v = 0; v < n; ++v) off[v + 1] += off[v];
    for (int64_t i = 0; i < mh; ++i) {
        int32_t u = ea[i], v = eb[i];
        if (precedes(u, v, deg, rank)) cols[off[u] + fill[u]++] = v;  /* store v in N_u */
        else                           cols[off[v] + fill[v]++] = u;  /* store u in N_v */
    }
    for (int32_t v = 0; v < n; ++v)
        qsort(cols + off[v], (size_t)(off[v + 1] - off[v]), sizeof(int32_t), cmp_i32);
    free(fill);
    return OR_OK;
}

/* |A intersect B| of two ascending lists by a two-pointer merge; if t_v is given, each
 * common element w adds one to t_v[v], t_v[u] and t_v[w]. */
static uint64_t merge_count(const int32_t* a, int64_t na, const int32_t* b, int64_t nb,
                            int32_t v, int32_t u, uint64_t* t_v) {
    uint64_t s = 0;
    int64_t i = 0, j = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else {
            if (t_v) { t_v[v]++; t_v[u]++; t_v[a[i]]++; }
            ++s; ++i; ++j;
        }
    }
    return s;
}

/*
 * Fig. 1, last loop: T = sum_v sum_{u in N_v} |N_v intersect N_u|.
 * per_edge (nullable, length m_hat): the count of oriented edge at CSR position i.
 * t_v (nullable, length n, zeroed here): triangles incident on each vertex.
 * nthreads > 1 splits the outer loop over OpenMP threads (only when t_v is NULL);
 * the integer sum is exact in any order.
 */
uint64_t or_count(int32_t n, const int64_t* off, const int32_t* cols, uint32_t* per_edge,
                  uint64_t* t_v, int nthreads) {
    uint64_t T = 0;
    if (t_v) memset(t_v, 0, (size_t)n * sizeof(uint64_t));
    if (t_v || nthreads <= 1) {
        for (int32_t v = 0; v < n; ++v) {
            for (int64_t i = off[v]; i < off[v + 1]; ++i) {
                int32_t u = cols[i];
                uint64_t s = merge_count(cols + off[v], off[v + 1] - off[v],
                                         cols + off[u], off[u + 1] - off[u], v, u, t_v);
                if (per_edge) per_edge[i] = (uint32_t)s;
                T += s;
            }
        }
        return T;
    }
    #pragma omp parallel for schedule(dynamic, 256) reduction(+ : T) num_threads(nthreads)
    for (int32_t v = 0; v < n; ++v) {
        for (int64_t i = off[v]; i < off[v + 1]; ++i) {
            int32_t u = cols[i];
            uint64_t s = merge_count(cols + off[v], off[v + 1] - off[v],
                                     cols + off[u], off[u + 1] - off[u], v, u, NULL);
            if (per_edge) per_edge[i] = (uint32_t)s;
            T += s;
        }
    }
    return T;
}

/* The processor (part) that holds vertex u: cuts[j] <= u < cuts[j + 1]. */
static int32_t part_of(int32_t u, int32_t nparts, const int32_t* cuts) {
    int32_t j = 0;
    while (j + 1 < nparts && u >= cuts[j + 1]) ++j;
    return j;
}

/* SurrogateCount (Sec. IV-C): processor j receives X = N_v and, for every u in X that it
 * owns, counts |N_u intersect X|. */
static uint64_t surrogate_count(const int32_t* X, int64_t nx, int32_t j, int32_t nparts, const int32_t* cuts,
                                const int64_t* off, const int32_t* cols) {
    uint64_t T = 0;
    for (int64_t k = 0; k < nx; ++k) {
        const int32_t u = X[k];
        if (part_of(u, nparts, cuts) != j) continue;
        T += merge_count(cols + off[u], off[u + 1] - off[u], X, nx, u, u, NULL);
    }
    return T;
}

/*
 * Sec. IV-A and IV-C: the count over a non-overlapping partition (Def. 1) of the vertices
 * into nparts sets of consecutive vertices, V_j = [cuts[j], cuts[j+1]) (cuts[0] = 0,
 * cuts[nparts] = n, non-decreasing; empty sets allowed).  For every v in V_i, N_v is sent
 * to processor j when a u in N_v with u in V_j is met and j differs from the last processor
 * N_v went to (LastProc; N_v is sorted and the V_j are consecutive, so that is once per
 * j); j adds SurrogateCount(N_v, j) to out[i * nparts + j] (zeroed here).
 */
int or_count_parts(int32_t n, const int64_t* off, const int32_t* cols, int32_t nparts, const int32_t* cuts,
                   uint64_t* out) {
    if (n < 0 || nparts < 1 || cuts[0] != 0 || cuts[nparts] != n) return OR_ERR_INVALID_ARG;
    for (int32_t j = 0; j < nparts; ++j)
        if (cuts[j] > cuts[j + 1]) return OR_ERR_INVALID_ARG;
    memset(out, 0, sizeof(uint64_t) * (size_t)nparts * (size_t)nparts);
    for (int32_t i = 0; i < nparts; ++i) {
        for (int32_t v = cuts[i]; v < cuts[i + 1]; ++v) {
            int32_t last_proc = -1;
            for (int64_t k = off[v]; k < off[v + 1]; ++k) {
                const int32_t j = part_of(cols[k], nparts, cuts);
                if (j == last_proc) continue;
                out[(size_t)i * nparts + j] +=
                    surrogate_count(cols + off[v], off[v + 1] - off[v], j, nparts, cuts, off, cols);
                last_proc = j;
            }
        }
    }
    return OR_OK;
}

/*
 * Sec. IV-B: sum over v in V_k of f(v) ~ (1/P) sum over v of f(v).  With the exclusive prefix
 * F(q) = f(0) + ... + f(q-1), cut k (0 < k < P) is the first q in [0, n] with
 * F(q) * P >= k * F(n), i.e. F(q) >= k F(n) / P; cuts[0] = 0 and cuts[P] = n.  The products are
 * taken in 128 bits.  cuts needs P + 1 entries.
 */
int or_balanced_cuts(int32_t n, const uint64_t* f, int32_t P, int32_t* cuts) {
    if (n < 0 || P < 1) return OR_ERR_INVALID_ARG;
    unsigned __int128 total = 0;
    for (int32_t v = 0; v < n; ++v) total += f[v];
    cuts[0] = 0;
    cuts[P] = n;
    for (int32_t k = 1; k < P; ++k) {
        unsigned __int128 F = 0;  /* F(q), recomputed from 0 for every cut */
        int32_t q = 0;
        while (q < n && F * (unsigned)P < total * (unsigned)k) F += f[q++];
        cuts[k] = q;
    }
    return OR_OK;
}

enum { OR_COST_ONE = 0, OR_COST_DEGREE = 1, OR_COST_PATRIC = 2, OR_COST_NEW = 3 };

/* Per-vertex cost f(v) (Sec. IV-B, IV-F, V-A).  dh_v = off[v+1] - off[v]. */
int or_vertex_cost(int fn, int32_t n, const int32_t* deg, const int64_t* off, const int32_t* cols,
                   uint64_t* f) {
    for (int32_t v = 0; v < n; ++v) f[v] = 0;
    for (int32_t v = 0; v < n; ++v) {
        uint64_t dv = (uint64_t)(off[v + 1] - off[v]);
        if (fn == OR_COST_ONE) f[v] = 1;
        else if (fn == OR_COST_DEGREE) f[v] = (uint64_t)deg[v];
        else if (fn == OR_COST_PATRIC) {
            for (int64_t i = off[v]; i < off[v + 1]; ++i) {
                int32_t u = cols[i];
                f[v] += dv + (uint64_t)(off[u + 1] - off[u]);
            }
        } else if (fn == OR_COST_NEW) {
            /* u in Nfull_v - N_v  <=>  v in N_u: charge (dh_v + dh_u) of every
             * oriented edge (u, v) to its higher endpoint v */
            for (int64_t i = off[v]; i < off[v + 1]; ++i) {
                int32_t w = cols[i];
                f[w] += (uint64_t)(off[w + 1] - off[w]) + dv;
            }
        } else {
            return OR_ERR_INVALID_ARG;
        }
    }
    return OR_OK;
}

/*
 * Chunk table of the dynamic load balancing scheme over tasks 0..T-1 with
 * costs cost[t] and W workers.
 *   C = total cost, H = floor(C / 2): the initial half (Sec. V-B).
 *   Eq. 1: chunks 0..W-1 split [0, H) into W parts of equal cost,
 *          part w = [w*(H/W) + min(w, H%W), ...).
 *   Eq. 2: then, from c = H while c < C, the next chunk takes
 *          max(min_chunk, floor((C - c) / W)) of the remaining cost.
 * A cost boundary x maps to the first task whose exclusive cost prefix is >= x;
 * the first boundary maps to task 0 and a boundary >= C maps to T.
 * Writes chunk k as cost range [cb[k], cb[k+1]) and task range [tb[k], tb[k+1]);
 * cb and tb need room for (#chunks + 1) entries, at most cap.
 * Returns the number of chunks, or -1 if cap is too small / bad arguments.
 */
int64_t or_schedule(int64_t T, const uint64_t* cost, int64_t W, uint64_t min_chunk,
                    uint64_t* cb, int64_t* tb, int64_t cap) {
    if (W < 1 || min_chunk < 1 || T < 0) return -1;
    uint64_t* prefix = (uint64_t*)malloc((size_t)(T + 1) * sizeof(uint64_t));
    if (!prefix) return -1;
    prefix[0] = 0;
    for (int64_t t = 0; t < T; ++t) prefix[t + 1] = prefix[t] + cost[t];
    const uint64_t C = prefix[T];
    const uint64_t H = C / 2;
    int64_t k = 0;
    /* Eq. 1 */
    for (int64_t w = 0; w <= W; ++w) {
        if (k >= cap) { free(prefix); return -1; }
        uint64_t ww = (uint64_t)w;
        cb[k++] = ww * (H / (uint64_t)W) + (ww < H % (uint64_t)W ? ww : H % (uint64_t)W);
    }
    /* Eq. 2 */
    uint64_t c = H;
    while (c < C) {
        uint64_t s = (C - c) / (uint64_t)W;
        if (s < min_chunk) s = min_chunk;
        uint64_t e = (C - c > s) ? c + s : C;
        if (k >= cap) { free(prefix); return -1; }
        cb[k++] = e;
        c = e;
    }
    /* cost boundaries -> task boundaries (the boundaries never decrease, so one
     * forward scan finds each first t with prefix[t] >= cb[j]) */
    int64_t t = 0;
    for (int64_t j = 0; j < k; ++j) {
        if (j == 0) { tb[j] = 0; continue; }
        if (cb[j] >= C) { tb[j] = T; continue; }
        while (t < T && prefix[t] < cb[j]) ++t;
        tb[j] = t;
    }
    free(prefix);
    return k - 1;
}

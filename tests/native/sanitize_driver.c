/*
 * Test driver for tests/test_sanitizers.py: the oracle (oracle/tc_oracle.c) and the input
 * generators (graphgen/graphgen.c), compiled with AddressSanitizer and UndefinedBehaviorSanitizer,
 * run through every entry point on seeded graphs of each family.  Any memory error or undefined
 * behaviour aborts with a nonzero status; the driver also checks the results against each other
 * (the partition table and the task decomposition sum to T, the per-vertex counts to 3T).
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t m_in, self_loops, duplicates, m_hat, bad_index;
} or_input_stats;

int64_t gg_er(int32_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst);
int64_t gg_ba(int32_t n, int32_t k, uint64_t seed, int32_t* src, int32_t* dst);
int64_t gg_chung_lu(int32_t n, double gamma, double avg_deg, double w_max, int64_t draws, uint64_t seed,
                    int32_t* src, int32_t* dst);
int or_simple_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, int strict, int32_t* ea,
                    int32_t* eb, or_input_stats* st);
int or_oriented_csr(int32_t n, int64_t mh, const int32_t* ea, const int32_t* eb, const int64_t* rank, int32_t* deg,
                    int64_t* off, int32_t* cols);
uint64_t or_count(int32_t n, const int64_t* off, const int32_t* cols, uint32_t* per_edge, uint64_t* t_v,
                  int nthreads);
int or_count_parts(int32_t n, const int64_t* off, const int32_t* cols, int32_t nparts, const int32_t* cuts,
                   uint64_t* out);
int or_balanced_cuts(int32_t n, const uint64_t* f, int32_t P, int32_t* cuts);
int or_vertex_cost(int fn, int32_t n, const int32_t* deg, const int64_t* off, const int32_t* cols, uint64_t* f);
int64_t or_schedule(int64_t T, const uint64_t* cost, int64_t W, uint64_t min_chunk, uint64_t* cb, int64_t* tb,
                    int64_t cap);

#define CHECK(c)                                                   \
    do {                                                           \
        if (!(c)) {                                                \
            fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
            exit(3);                                               \
        }                                                          \
    } while (0)

static void run(const char* name, int32_t n, int64_t m, const int32_t* src, const int32_t* dst) {
    int32_t* ea = malloc((size_t)(m > 0 ? m : 1) * 4);
    int32_t* eb = malloc((size_t)(m > 0 ? m : 1) * 4);
    or_input_stats st;
    CHECK(or_simple_graph(n, m, src, dst, 0, ea, eb, &st) == 0);
    const int64_t mh = st.m_hat;
    int32_t* deg = malloc((size_t)(n > 0 ? n : 1) * 4);
    int64_t* off = malloc((size_t)(n + 1) * 8);
    int32_t* cols = malloc((size_t)(mh > 0 ? mh : 1) * 4);
    CHECK(or_oriented_csr(n, mh, ea, eb, NULL, deg, off, cols) == 0);
    uint32_t* pe = calloc((size_t)(mh > 0 ? mh : 1), 4);
    uint64_t* tv = calloc((size_t)(n > 0 ? n : 1), 8);
    const uint64_t T = or_count(n, off, cols, pe, tv, 1);
    CHECK(or_count(n, off, cols, NULL, NULL, 4) == T);
    uint64_t s3 = 0, se = 0;
    for (int32_t v = 0; v < n; ++v) s3 += tv[v];
    for (int64_t i = 0; i < mh; ++i) se += pe[i];
    CHECK(s3 == 3 * T && se == T);
    /* costs, balanced cuts and the partition table */
    uint64_t* f = malloc((size_t)(n > 0 ? n : 1) * 8);
    for (int fn = 0; fn < 4; ++fn) CHECK(or_vertex_cost(fn, n, deg, off, cols, f) == 0);
    for (int32_t P = 1; P <= 9; P += 4) {
        int32_t cuts[10];
        CHECK(or_balanced_cuts(n, f, P, cuts) == 0);
        uint64_t* tab = malloc((size_t)P * P * 8);
        CHECK(or_count_parts(n, off, cols, P, cuts, tab) == 0);
        uint64_t s = 0;
        for (int32_t k = 0; k < P * P; ++k) s += tab[k];
        CHECK(s == T);
        free(tab);
    }
    /* the Eq. 1 / Eq. 2 chunk table over the merge cost d^_v + d^_u of every oriented edge */
    uint64_t* cost = malloc((size_t)(mh > 0 ? mh : 1) * 8);
    for (int32_t v = 0; v < n; ++v)
        for (int64_t i = off[v]; i < off[v + 1]; ++i)
            cost[i] = (uint64_t)(off[v + 1] - off[v]) + (uint64_t)(off[cols[i] + 1] - off[cols[i]]);
    const int64_t cap = 1 << 16;
    uint64_t* cb = malloc((size_t)cap * 8);
    int64_t* tb = malloc((size_t)cap * 8);
    CHECK(or_schedule(mh, cost, 7, 32, cb, tb, cap) >= 0);
    printf("%s: n=%d m=%lld m_hat=%lld T=%llu\n", name, n, (long long)m, (long long)mh, (unsigned long long)T);
    free(ea); free(eb); free(deg); free(off); free(cols); free(pe); free(tv); free(f);
    free(cost); free(cb); free(tb);
}

int main(void) {
    const int32_t n = 3000;
    const int64_t m = 30000;
    int32_t* s = malloc(8 * m * 4);
    int32_t* d = malloc(8 * m * 4);
    CHECK(gg_er(n, m, 7, s, d) == m);
    run("erdos_renyi", n, m, s, d);
    const int64_t mb = gg_ba(n, 8, 8, s, d);
    CHECK(mb == (int64_t)8 * (n - 8));
    run("barabasi_albert", n, mb, s, d);
    CHECK(gg_chung_lu(n, 2.1, 20.0, 600.0, 8 * m, 9, s, d) == 8 * m);
    run("chung_lu", n, 8 * m, s, d);
    run("empty", 5, 0, s, d);
    free(s);
    free(d);
    return 0;
}

/*
 * graphgen.c -- seeded synthetic edge-list generators.
 *
 * This module only produces inputs: COO edge lists of int32 vertex ids.  It
 * holds none of the triangle-counting arithmetic and is shared by the CPU
 * oracle's tests and by the GPU path's tests and benchmark, so that both sides
 * see the same graphs.
 *
 * Random numbers come from a counter-based generator: draw i of stream key k is
 * the SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) applied to k + (i+1)*gamma with
 * gamma = 0x9E3779B97F4A7C15.  A draw therefore depends only on (seed, i), not
 * on the thread that makes it, and the parallel generators are deterministic.
 *
 * Families (the paper's PA(n,d) model of Sec. II is the BA generator):
 *   gg_er          Erdos-Renyi G(n,m): m distinct non-loop pairs by rejection.
 *   gg_ba          Barabasi-Albert preferential attachment, k edges per new
 *                  vertex to distinct targets chosen with probability
 *                  proportional to degree; m = k(n-k).
 *   gg_chung_lu    Chung-Lu expected-degree graph: `draws` edges whose two
 *                  endpoints are drawn independently with probability
 *                  proportional to w_i = c (i+i0)^(-1/(gamma-1)); self-loops
 *                  and repeated pairs are left in the output on purpose (the
 *                  counter's input policy removes them).
 *
 * Floating point appears only in the Chung-Lu weights (libm pow).  The build
 * uses -ffp-contract=off so that the remaining double arithmetic is plain IEEE
 * and gives the same bits on x86_64 and aarch64; pow itself may differ in the
 * last place between C libraries, so a Chung-Lu graph is reproducible on one
 * platform but is not promised to be bit-identical across platforms.  ER and
 * BA use integer arithmetic only and are identical everywhere.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Stream key for (seed, stream tag). */
uint64_t gg_key(uint64_t seed, uint64_t tag) {
    return gg_mix(gg_mix(seed + GG_GAMMA) ^ (tag * 0xD1B54A32D192ED03ULL + 0x8CB92BA72F3D8DD7ULL));
}

/* Draw i of stream `key`. */
uint64_t gg_draw(uint64_t key, uint64_t i) { return gg_mix(key + (i + 1) * GG_GAMMA); }

/* Uniform integer in [0, n) from a 64-bit draw (multiply-high; bias < n / 2^64). */
static inline uint64_t gg_below(uint64_t r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
}

/* ------------------------------------------------------------------------ */
/* Erdos-Renyi G(n, m): m distinct unordered pairs {a,b}, a != b, uniform.     */
/* Pairs are emitted in draw order with the orientation they were drawn in.    */
/* Returns m on success, -1 if m > n(n-1)/2 or n < 2 with m > 0, -2 on OOM.    */
/* ------------------------------------------------------------------------ */
int64_t gg_er(int32_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst) {
    if (m == 0) return 0;
    if (n < 2) return -1;
    if ((unsigned __int128)m * 2 > (unsigned __int128)n * (uint64_t)(n - 1)) return -1;
    uint64_t cap = 16;
    while (cap < (uint64_t)m * 2) cap <<= 1;
    uint64_t* set = (uint64_t*)malloc(cap * sizeof(uint64_t));
    if (!set) return -2;
    memset(set, 0xFF, cap * sizeof(uint64_t));
    const uint64_t key = gg_key(seed, 1);
    uint64_t i = 0;
    int64_t got = 0;
    while (got < m) {
        uint32_t a = (uint32_t)gg_below(gg_draw(key, i), (uint64_t)n);
        uint32_t b = (uint32_t)gg_below(gg_draw(key, i + 1), (uint64_t)n);
        i += 2;
        if (a == b) continue;
        uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
        uint64_t k = (lo << 32) | hi;
        uint64_t h = gg_mix(k) & (cap - 1);
        int seen = 0;
        while (set[h] != UINT64_MAX) {
            if (set[h] == k) { seen = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (seen) continue;
        set[h] = k;
        src[got] = (int32_t)a;
        dst[got] = (int32_t)b;
        ++got;
    }
    free(set);
    return got;
}

/* ------------------------------------------------------------------------ */
/* Barabasi-Albert: vertices 0..k-1 start isolated, vertex k links to all of   */
/* them, then every vertex t = k+1..n-1 links to k distinct earlier vertices,  */
/* each drawn with probability proportional to its current degree (a uniform  */
/* pick from the list of edge endpoints).  Output: m = k(n-k) edges (t, target)*/
/* Returns m, or -1 on bad arguments, -2 on OOM.                               */
/* ------------------------------------------------------------------------ */
int64_t gg_ba(int32_t n, int32_t k, uint64_t seed, int32_t* src, int32_t* dst) {
    if (k < 1 || n <= k) return -1;
    const int64_t m = (int64_t)k * (int64_t)(n - k);
    int32_t* ends = (int32_t*)malloc((size_t)(2 * m) * sizeof(int32_t));
    int32_t* pick = (int32_t*)malloc((size_t)k * sizeof(int32_t));
    if (!ends || !pick) { free(ends); free(pick); return -2; }
    const uint64_t key = gg_key(seed, 2);
    uint64_t draw = 0;
    int64_t e = 0;
    for (int32_t j = 0; j < k; ++j) {
        src[e] = k; dst[e] = j;
        ends[2 * e] = k; ends[2 * e + 1] = j;
        ++e;
    }
    for (int32_t t = k + 1; t < n; ++t) {
        const uint64_t len = (uint64_t)(2 * e);
        int32_t chosen = 0;
        while (chosen < k) {
            int32_t cand = ends[gg_below(gg_draw(key, draw++), len)];
            int dup = 0;
            for (int32_t q = 0; q < chosen; ++q)
                if (pick[q] == cand) { dup = 1; break; }
            if (!dup) pick[chosen++] = cand;
        }
        for (int32_t q = 0; q < k; ++q) {
            src[e] = t; dst[e] = pick[q];
            ends[2 * e] = t; ends[2 * e + 1] = pick[q];
            ++e;
        }
    }
    free(ends);
    free(pick);
    return e;
}

/* ------------------------------------------------------------------------ */
/* Chung-Lu.                                                                   */
/* ------------------------------------------------------------------------ */

/* Integral approximation of sum_{i=0}^{n-1} (i+i0)^(-a), a != 1. */
static double cl_sum_approx(double n, double i0, double a) {
    double lo = i0 - 0.5, hi = n + i0 - 0.5;
    if (lo < 1e-9) lo = 1e-9;
    return (pow(hi, 1.0 - a) - pow(lo, 1.0 - a)) / (1.0 - a);
}

/* Offset i0 such that w_0 / mean(w) = w_max / avg_deg, by bisection. */
double gg_chung_lu_i0(int32_t n, double gamma, double avg_deg, double w_max) {
    const double a = 1.0 / (gamma - 1.0);
    const double target = w_max / avg_deg;
    double lo = 1e-6, hi = (double)n * 1e3;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        double ratio = (double)n * pow(mid, -a) / cl_sum_approx((double)n, mid, a);
        if (ratio > target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/*
 * Expected-degree weights w[0..n) (descending, mean avg_deg, w[0] ~ w_max).
 * Returns 0, or -1 on bad arguments.
 */
int gg_chung_lu_weights(int32_t n, double gamma, double avg_deg, double w_max, double* w) {
    if (n < 2 || !(gamma > 1.0) || gamma == 2.0 || !(avg_deg > 0) || !(w_max > 0)) return -1;
    const double a = 1.0 / (gamma - 1.0);
    const double i0 = gg_chung_lu_i0(n, gamma, avg_deg, w_max);
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) { w[i] = pow((double)i + i0, -a); s += w[i]; }
    const double c = (double)n * avg_deg / s;
    for (int32_t i = 0; i < n; ++i) w[i] *= c;
    return 0;
}

/*
 * `draws` edges, both endpoints i.i.d. with P(i) = w_i / sum w, sampled with
 * Vose's alias method (integer coin thresholds).  Self-loops and repeated
 * pairs are kept.  Returns draws, -1 on bad arguments, -2 on OOM.
 */
int64_t gg_chung_lu(int32_t n, double gamma, double avg_deg, double w_max, int64_t draws,
                    uint64_t seed, int32_t* src, int32_t* dst) {
    if (draws < 0) return -1;
    double* w = (double*)malloc((size_t)n * sizeof(double));
    double* q = (double*)malloc((size_t)n * sizeof(double));
    uint32_t* thr = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    int32_t* alias = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* small = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* large = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int64_t rc = draws;
    if (!w || !q || !thr || !alias || !small || !large) { rc = -2; goto done; }
    if (gg_chung_lu_weights(n, gamma, avg_deg, w_max, w) != 0) { rc = -1; goto done; }
    {
        double s = 0.0;
        for (int32_t i = 0; i < n; ++i) s += w[i];
        int32_t ns = 0, nl = 0;
        for (int32_t i = 0; i < n; ++i) {
            q[i] = w[i] * (double)n / s;
            alias[i] = i;
            if (q[i] < 1.0) small[ns++] = i; else large[nl++] = i;
        }
        while (ns > 0 && nl > 0) {
            int32_t l = small[--ns], g = large[--nl];
            alias[l] = g;
            double t = q[l] * 4294967296.0;
            thr[l] = t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
            q[g] = (q[g] + q[l]) - 1.0;
            if (q[g] < 1.0) small[ns++] = g; else large[nl++] = g;
        }
        while (nl > 0) thr[large[--nl]] = 0xFFFFFFFFu;
        while (ns > 0) thr[small[--ns]] = 0xFFFFFFFFu;
    }
    {
        const uint64_t key = gg_key(seed, 3);
        #pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < draws; ++e) {
            int32_t ends[2];
            for (int s2 = 0; s2 < 2; ++s2) {
                uint64_t r1 = gg_draw(key, (uint64_t)(4 * e + 2 * s2));
                uint64_t r2 = gg_draw(key, (uint64_t)(4 * e + 2 * s2 + 1));
                int32_t col = (int32_t)gg_below(r1, (uint64_t)n);
                uint32_t coin = (uint32_t)(r2 >> 32);
                ends[s2] = coin < thr[col] ? col : alias[col];
            }
            src[e] = ends[0];
            dst[e] = ends[1];
        }
    }
done:
    free(w); free(q); free(thr); free(alias); free(small); free(large);
    return rc;
}

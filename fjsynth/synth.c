/*
 * Seeded synthetic inputs for the Friedkin-Johnsen solver: graph edge lists
 * (R-MAT, Barabasi-Albert, stochastic block model) and innate-opinion vectors.
 *
 * This module holds no part of the FJ method: it only draws random numbers and
 * turns them into edges and opinions.  Both the FP64 CPU oracle and the CUDA
 * path consume its output, so it is the single source of every test input.
 *
 * Random numbers come from a counter-based generator built on the SplitMix64
 * finaliser (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): value(seed, stream, i) = mix(key(seed, stream) +
 * (i+1)*gamma).  Every draw is addressed by (seed, stream, counter), so edge e
 * of an R-MAT graph is the same no matter which thread or machine makes it.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FJS_GAMMA 0x9E3779B97F4A7C15ULL

enum {
    FJS_STREAM_RMAT = 1,
    FJS_STREAM_WEIGHT = 2,
    FJS_STREAM_OPINION = 3,
    FJS_STREAM_BA = 4,
    FJS_STREAM_SBM = 5,
    FJS_STREAM_SIZE = 6
};

static inline uint64_t fjs_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t fjs_key(uint64_t seed, uint64_t stream)
{
    return fjs_mix64(seed + FJS_GAMMA * (stream + 1));
}

static inline uint64_t fjs_draw(uint64_t key, uint64_t ctr)
{
    return fjs_mix64(key + FJS_GAMMA * (ctr + 1));
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double fjs_u01(uint64_t key, uint64_t ctr)
{
    return (double)(fjs_draw(key, ctr) >> 11) * 0x1.0p-53;
}

uint64_t fjs_raw(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return fjs_draw(fjs_key(seed, stream), ctr);
}

double fjs_uniform(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return fjs_u01(fjs_key(seed, stream), ctr);
}

/* out[i] = U(seed, stream, ctr0 + i) for i < n. */
void fjs_uniform_fill(uint64_t seed, uint64_t stream, uint64_t ctr0, int64_t n, double *out)
{
    uint64_t key = fjs_key(seed, stream);
    for (int64_t i = 0; i < n; ++i) out[i] = fjs_u01(key, ctr0 + (uint64_t)i);
}

/* ------------------------------------------------------------------ R-MAT */

typedef struct {
    int scale;
    int64_t e0, e1;
    double a, ab, abc;
    uint64_t key_edge, key_w;
    int32_t *src, *dst;
    float *w;
} rmat_job;

static void *rmat_worker(void *arg)
{
    rmat_job *j = (rmat_job *)arg;
    for (int64_t e = j->e0; e < j->e1; ++e) {
        uint32_t u = 0, v = 0;
        for (int l = 0; l < j->scale; ++l) {
            double x = fjs_u01(j->key_edge, (uint64_t)e * 64u + (uint64_t)l);
            uint32_t bu, bv;
            if (x < j->a) { bu = 0; bv = 0; }
            else if (x < j->ab) { bu = 0; bv = 1; }
            else if (x < j->abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        j->src[e] = (int32_t)u;
        j->dst[e] = (int32_t)v;
        if (j->w) j->w[e] = (float)(0.5 + fjs_u01(j->key_w, (uint64_t)e));
    }
    return NULL;
}

/*
 * R-MAT edge e (0 <= e < n_edges): at each of `scale` levels, from the most
 * significant bit down, one uniform picks a quadrant with probabilities
 * a, b, c, 1-a-b-c.  No noise, no vertex relabelling.  Optional weight
 * w_e = float(0.5 + U) lies in [0.5, 1.5].
 */
int fjs_rmat(int scale, int64_t n_edges, double a, double b, double c, uint64_t seed,
             int32_t *src, int32_t *dst, float *w, int nthreads)
{
    if (scale < 1 || scale > 30 || n_edges < 0 || !src || !dst) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    rmat_job jobs[64];
    pthread_t th[64];
    int64_t per = (n_edges + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].scale = scale;
        jobs[t].e0 = (int64_t)t * per < n_edges ? (int64_t)t * per : n_edges;
        jobs[t].e1 = (int64_t)(t + 1) * per < n_edges ? (int64_t)(t + 1) * per : n_edges;
        jobs[t].a = a;
        jobs[t].ab = a + b;
        jobs[t].abc = a + b + c;
        jobs[t].key_edge = fjs_key(seed, FJS_STREAM_RMAT);
        jobs[t].key_w = fjs_key(seed, FJS_STREAM_WEIGHT);
        jobs[t].src = src;
        jobs[t].dst = dst;
        jobs[t].w = w;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, rmat_worker, &jobs[t]) != 0) break;
        started = t;
    }
    rmat_worker(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    for (int t = started + 1; t < nthreads; ++t) rmat_worker(&jobs[t]);
    return 0;
}

/* ------------------------------------------------------ Barabasi-Albert */

int64_t fjs_ba_num_edges(int64_t n, int m)
{
    if (n <= m) return n * (n - 1) / 2;
    return (int64_t)m * (m + 1) / 2 + (n - m - 1) * (int64_t)m;
}

/*
 * Preferential attachment: a clique on nodes 0..m, then node v = m+1..n-1
 * attaches to m distinct earlier nodes, each drawn with probability
 * proportional to its current degree (uniform over the list of edge
 * endpoints; repeats are redrawn).  Edges are written in creation order.
 * Returns the number of edges, or -1.
 */
int64_t fjs_ba(int64_t n, int m, uint64_t seed, int32_t *src, int32_t *dst)
{
    if (n < 1 || m < 1 || !src || !dst) return -1;
    int64_t ne = fjs_ba_num_edges(n, m);
    int32_t *ends = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * ne + 2));
    if (!ends) return -1;
    int64_t nends = 0, k = 0;
    int64_t clique = n < m + 1 ? n : m + 1;
    for (int64_t i = 0; i < clique; ++i)
        for (int64_t j = i + 1; j < clique; ++j) {
            src[k] = (int32_t)i; dst[k] = (int32_t)j; ++k;
            ends[nends++] = (int32_t)i; ends[nends++] = (int32_t)j;
        }
    uint64_t key = fjs_key(seed, FJS_STREAM_BA);
    int32_t pick[64];
    for (int64_t v = m + 1; v < n; ++v) {
        int got = 0;
        uint64_t attempt = 0;
        while (got < m) {
            double x = fjs_u01(key, (uint64_t)v * 4096u + attempt);
            ++attempt;
            int64_t idx = (int64_t)(x * (double)nends);
            if (idx >= nends) idx = nends - 1;
            int32_t t = ends[idx];
            int dup = 0;
            for (int q = 0; q < got; ++q) dup |= (pick[q] == t);
            if (!dup) pick[got++] = t;
            if (attempt >= 4096) break; /* cannot happen for m <= 64 in practice */
        }
        for (int q = 0; q < got; ++q) {
            src[k] = (int32_t)v; dst[k] = pick[q]; ++k;
            ends[nends++] = (int32_t)v; ends[nends++] = pick[q];
        }
    }
    free(ends);
    return k;
}

/* ----------------------------------------------- stochastic block model */

/*
 * Undirected SBM with `nblocks` near-equal blocks (block of v = v*nblocks/n).
 * Each node has expected `deg_in` neighbours inside its block and `deg_out`
 * outside.  For every block pair the number of edges is fixed to the rounded
 * expectation and the endpoints are drawn uniformly inside the two blocks, so
 * repeats and self-pairs can occur (graph ingest drops them).
 * With src == NULL only the edge count is returned.
 */
static int64_t block_lo(int64_t n, int nb, int b) { return (int64_t)(((__int128)n * b + nb - 1) / nb); }

int64_t fjs_sbm(int64_t n, int nblocks, double deg_in, double deg_out, uint64_t seed,
                int32_t *src, int32_t *dst)
{
    if (n < 2 || nblocks < 1) return -1;
    uint64_t key = fjs_key(seed, FJS_STREAM_SBM);
    int64_t k = 0;
    for (int a = 0; a < nblocks; ++a) {
        int64_t a0 = block_lo(n, nblocks, a), a1 = block_lo(n, nblocks, a + 1);
        int64_t na = a1 - a0;
        for (int b = a; b < nblocks; ++b) {
            int64_t b0 = block_lo(n, nblocks, b), b1 = block_lo(n, nblocks, b + 1);
            int64_t nbk = b1 - b0;
            double expect;
            if (a == b) expect = 0.5 * (double)na * deg_in;
            else expect = (double)na * (double)nbk * deg_out / (double)(n - na > 0 ? n - na : 1);
            int64_t mab = (int64_t)llround(expect);
            uint64_t pair = (uint64_t)a * 1024u + (uint64_t)b;
            for (int64_t e = 0; e < mab; ++e) {
                if (src) {
                    uint64_t c = (pair << 40) + (uint64_t)e * 2u;
                    int64_t u = a0 + (int64_t)(fjs_u01(key, c) * (double)na);
                    int64_t v = b0 + (int64_t)(fjs_u01(key, c + 1) * (double)nbk);
                    if (u >= a1) u = a1 - 1;
                    if (v >= b1) v = b1 - 1;
                    src[k] = (int32_t)u;
                    dst[k] = (int32_t)v;
                }
                ++k;
            }
        }
    }
    return k;
}

/* ---------------------------------------------------------- opinions */

enum {
    FJS_OP_UNIFORM = 0,   /* U[0,1) */
    FJS_OP_BETA_MIX = 1,  /* Beta(2,5) on even ids, Beta(5,2) on odd ids */
    FJS_OP_ARCSINE = 2,   /* Beta(1/2,1/2) */
    FJS_OP_SIGN = 3,      /* +1 / -1 labels */
    FJS_OP_EXP = 4,       /* exponential, x_min = 1, divided by the sample max */
    FJS_OP_PARETO = 5     /* Pareto alpha = 2.5, x_min = 1, divided by the sample max */
};

/* k-th smallest (1-based) of six uniforms drawn at counters base..base+5. */
static double order_stat6(uint64_t key, uint64_t base, int k)
{
    double x[6];
    for (int i = 0; i < 6; ++i) x[i] = fjs_u01(key, base + (uint64_t)i);
    for (int i = 1; i < 6; ++i) {
        double t = x[i];
        int j = i - 1;
        while (j >= 0 && x[j] > t) { x[j + 1] = x[j]; --j; }
        x[j + 1] = t;
    }
    return x[k - 1];
}

/*
 * Innate opinions for vector number `vec` (several vectors per graph use
 * vec = 0, 1, 2, ...).  Beta(k, 7-k) is the k-th order statistic of six
 * uniforms; the arcsine law is sin^2(pi U / 2).
 */
int fjs_opinions(int64_t n, int kind, uint64_t seed, uint64_t vec, double *s)
{
    if (n < 0 || !s) return -1;
    uint64_t key = fjs_key(seed ^ (vec * 0xD1B54A32D192ED03ULL), FJS_STREAM_OPINION);
    const double pi = 3.14159265358979323846;
    double mx = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        double x;
        switch (kind) {
        case FJS_OP_UNIFORM: x = fjs_u01(key, (uint64_t)v); break;
        case FJS_OP_BETA_MIX:
            x = order_stat6(key, (uint64_t)v * 8u, (v & 1) ? 5 : 2);
            break;
        case FJS_OP_ARCSINE: {
            double sn = sin(0.5 * pi * fjs_u01(key, (uint64_t)v));
            x = sn * sn;
            break;
        }
        case FJS_OP_SIGN: x = (fjs_draw(key, (uint64_t)v) >> 63) ? 1.0 : -1.0; break;
        case FJS_OP_EXP: x = 1.0 - log1p(-fjs_u01(key, (uint64_t)v)); break;
        case FJS_OP_PARETO: x = pow(1.0 - fjs_u01(key, (uint64_t)v), -1.0 / 1.5); break;
        default: return -1;
        }
        s[v] = x;
        if (x > mx) mx = x;
    }
    if ((kind == FJS_OP_EXP || kind == FJS_OP_PARETO) && mx > 0.0)
        for (int64_t v = 0; v < n; ++v) s[v] /= mx;
    return 0;
}

/* Log-uniform integer sizes in [lo, hi] for ragged batches. */
int fjs_loguniform_sizes(int64_t count, int64_t lo, int64_t hi, uint64_t seed, int64_t *out)
{
    if (count < 0 || lo < 1 || hi < lo || !out) return -1;
    uint64_t key = fjs_key(seed, FJS_STREAM_SIZE);
    double l0 = log((double)lo), l1 = log((double)hi);
    for (int64_t i = 0; i < count; ++i) {
        int64_t v = (int64_t)floor(exp(l0 + (l1 - l0) * fjs_u01(key, (uint64_t)i)));
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        out[i] = v;
    }
    return 0;
}

/*
 * FP64 CPU oracle for the Friedkin-Johnsen (FJ) equilibrium and its metrics.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: only the test suite, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code with the CUDA library.
 *
 * Conventions (graph stored as CSR; row u lists the nodes u listens to):
 *   a_uj = w[k] for k in row u (unit weight when w == NULL),
 *   d_u  = sum_j a_uj (weighted out-degree, the row sum of A),
 *   L    = D - A, and the FJ equilibrium is z = (I + L)^{-1} s  (Lemma 1).
 * A push at node v moves delta = omega * r_v / (1 + d_v) into zhat_v and adds
 * a_uv * delta to r_u for every u with a_uv > 0, i.e. every in-neighbour of v
 * (Eqs. sor1-sor3 of Section 5.2; Alg. 1 is the omega = 1 case).
 *
 * Everything is sequential, scalar and in FP64, except
 * oracle_push_rounds_threads, which runs the rounds of oracle_push_rounds on
 * several host threads (the all-core CPU baseline) with the same arithmetic.
 */
#define _POSIX_C_SOURCE 200809L /* pthread barriers */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/*
 * Simple-graph CSR from an arc list (Section 3.2: simple graphs): self-loops
 * dropped, arcs ordered by (src, dst), the first arc in generation order kept
 * of every repeated (src, dst).  Arcs are bucketed by src in generation order
 * (a stable counting sort), each row is sorted by (dst, arc index), and runs of
 * equal dst keep their first element.  row_ptr has n + 1 entries; col and
 * w_out (NULL when w is NULL) room for m.  Returns nnz, or -1 on a bad node id
 * or allocation failure.
 */
typedef struct {
    int32_t dst;
    int64_t e;
} arc_key;

static int arc_cmp(const void *a, const void *b)
{
    const arc_key *x = (const arc_key *)a, *y = (const arc_key *)b;
    if (x->dst != y->dst) return x->dst < y->dst ? -1 : 1;
    return x->e < y->e ? -1 : (x->e > y->e ? 1 : 0);
}

int64_t oracle_csr_build(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const float *w,
                         int64_t *row_ptr, int32_t *col, float *w_out)
{
    int64_t *start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    arc_key *keys = (arc_key *)malloc(sizeof(arc_key) * (size_t)(m > 0 ? m : 1));
    if (!start || !keys) {
        free(start);
        free(keys);
        return -1;
    }
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) {
            free(start);
            free(keys);
            return -1;
        }
        if (src[e] != dst[e]) start[src[e] + 1] += 1;
    }
    for (int64_t u = 0; u < n; ++u) start[u + 1] += start[u];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!fill) {
        free(start);
        free(keys);
        return -1;
    }
    for (int64_t u = 0; u < n; ++u) fill[u] = start[u];
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] == dst[e]) continue;
        arc_key k;
        k.dst = dst[e];
        k.e = e;
        keys[fill[src[e]]++] = k;
    }
    free(fill);
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int64_t u = 0; u < n; ++u) {
        arc_key *row = keys + start[u];
        int64_t len = start[u + 1] - start[u];
        if (len > 1) qsort(row, (size_t)len, sizeof(arc_key), arc_cmp);
        for (int64_t i = 0; i < len; ++i) {
            if (i > 0 && row[i].dst == row[i - 1].dst) continue;
            col[nnz] = row[i].dst;
            if (w && w_out) w_out[nnz] = w[row[i].e];
            ++nnz;
        }
        row_ptr[u + 1] = nnz;
    }
    free(start);
    free(keys);
    return nnz;
}

/* Weighted out-degree d_u = sum of row u, summed in CSR order. */
static void out_degree(int64_t n, const int64_t *row_ptr, const double *w, double *d)
{
    for (int64_t u = 0; u < n; ++u) {
        double acc = 0.0;
        for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) acc += w ? w[k] : 1.0;
        d[u] = acc;
    }
}

/*
 * In-neighbour lists (the transpose of the CSR): for node v, every u with
 * a_uv > 0, in ascending u, with weight a_uv.  Counting sort over rows taken in
 * ascending order, so each list comes out sorted.
 */
static int transpose(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                     int64_t **tptr_out, int32_t **tcol_out, double **tw_out)
{
    int64_t nnz = row_ptr[n];
    int64_t *tptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *tcol = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nnz + 1));
    double *tw = (double *)malloc(sizeof(double) * ((size_t)nnz + 1));
    if (!tptr || !fill || !tcol || !tw) {
        free(tptr); free(fill); free(tcol); free(tw);
        return -1;
    }
    for (int64_t k = 0; k < nnz; ++k) tptr[col[k] + 1]++;
    for (int64_t v = 0; v < n; ++v) tptr[v + 1] += tptr[v];
    memcpy(fill, tptr, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t u = 0; u < n; ++u)
        for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
            int64_t pos = fill[col[k]]++;
            tcol[pos] = (int32_t)u;
            tw[pos] = w ? w[k] : 1.0;
        }
    free(fill);
    *tptr_out = tptr;
    *tcol_out = tcol;
    *tw_out = tw;
    return 0;
}

/*
 * Shift of the robust variant (Alg. 2): c_eff = c + max(0, -min s) makes every
 * shifted opinion s' = s + c_eff at least c > 0; eps' = sigma * eps / (c + sigma).
 * For s >= 0 this is exactly the paper's s + c.
 */
static double shift_of(int64_t n, const double *s, double c)
{
    double mn = 0.0;
    for (int64_t v = 0; v < n; ++v)
        if (s[v] < mn) mn = s[v];
    return c - mn;
}

/*
 * ImprovedBLISOR: Alg. 3 run on s' = s + c_eff with error parameter eps',
 * followed by the unshift of Alg. 2.  omega = 1 is ImprovedBLI (Alg. 1 inside
 * Alg. 2).  The queue starts as 0..n-1; a popped node is always pushed; a node
 * is appended when |r| exceeds eps' s' and it is not already queued.
 *
 * single_pass != 0 disables every append (one pass over the initial queue),
 * which is the setting of the Gauss-Seidel equivalence of Theorem 2.
 *
 * Outputs z (unshifted estimate), r (residual of the shifted system), and
 * stats[0] = pushes, stats[1] = residual updates (sum of in-degrees of pushed
 * nodes, the paper's "number of updates").  Returns 0, or 1 when max_pops
 * pushes were made before the queue emptied, or -1 on allocation failure.
 */
int oracle_blisor_fifo(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                       const double *s, double eps, double omega, double c, double sigma,
                       int single_pass, int64_t max_pops, double *z_out, double *r_out,
                       int64_t *stats)
{
    int64_t *tptr;
    int32_t *tcol;
    double *tw;
    if (transpose(n, row_ptr, col, w, &tptr, &tcol, &tw) != 0) return -1;
    double *d = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *sp = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    unsigned char *inq = (unsigned char *)malloc((size_t)n + 1);
    if (!d || !sp || !queue || !inq) {
        free(tptr); free(tcol); free(tw); free(d); free(sp); free(queue); free(inq);
        return -1;
    }
    out_degree(n, row_ptr, w, d);
    double c_eff = shift_of(n, s, c);
    double epsp = sigma * eps / (c + sigma);
    for (int64_t v = 0; v < n; ++v) {
        sp[v] = s[v] + c_eff;
        r_out[v] = sp[v];
        z_out[v] = 0.0;
        queue[v] = v;
        inq[v] = 1;
    }
    /* ring buffer: each node is queued at most once, so n slots suffice */
    int64_t head = 0, count = n, pops = 0, updates = 0;
    int rc = 0;
    while (count > 0) {
        if (pops >= max_pops) { rc = 1; break; }
        int64_t v = queue[head];
        head = (head + 1 == n) ? 0 : head + 1;
        --count;
        inq[v] = 0;
        double rv = r_out[v];
        double delta = omega * rv / (1.0 + d[v]);
        z_out[v] += delta;
        for (int64_t k = tptr[v]; k < tptr[v + 1]; ++k) {
            int64_t u = tcol[k];
            r_out[u] += tw[k] * delta;
            if (!single_pass && fabs(r_out[u]) > epsp * sp[u] && !inq[u]) {
                int64_t tail = head + count;
                if (tail >= n) tail -= n;
                queue[tail] = u;
                inq[u] = 1;
                ++count;
            }
        }
        r_out[v] = (1.0 - omega) * rv;
        if (!single_pass && fabs(r_out[v]) > epsp * sp[v] && !inq[v]) {
            int64_t tail = head + count;
            if (tail >= n) tail -= n;
            queue[tail] = v;
            inq[v] = 1;
            ++count;
        }
        ++pops;
        updates += tptr[v + 1] - tptr[v];
    }
    for (int64_t v = 0; v < n; ++v) z_out[v] -= c_eff;
    if (stats) { stats[0] = pops; stats[1] = updates; }
    free(tptr); free(tcol); free(tw); free(d); free(sp); free(queue); free(inq);
    return rc;
}

/*
 * Synchronous push rounds (the round view of Theorem 1's proof, with every
 * node above threshold pushed at once): F = {v : |r_v| > eps' s'_v}; each
 * v in F pushes delta_v computed from the round-start residuals.  Valid for
 * omega <= 1.  Stops when F is empty or after max_rounds rounds.
 * stats[0] = pushes, stats[1] = residual updates, stats[2] = rounds.
 */
int oracle_push_rounds(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                       const double *s, double eps, double omega, double c, double sigma,
                       int64_t max_rounds, double *z_out, double *r_out, int64_t *stats)
{
    double *d = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *sp = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *delta = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    int64_t *indeg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!d || !sp || !delta || !indeg) { free(d); free(sp); free(delta); free(indeg); return -1; }
    out_degree(n, row_ptr, w, d);
    for (int64_t k = 0; k < row_ptr[n]; ++k) indeg[col[k]]++;
    double c_eff = shift_of(n, s, c);
    double epsp = sigma * eps / (c + sigma);
    for (int64_t v = 0; v < n; ++v) {
        sp[v] = s[v] + c_eff;
        r_out[v] = sp[v];
        z_out[v] = 0.0;
    }
    int64_t rounds = 0, pushes = 0, updates = 0;
    int rc = 0;
    for (;;) {
        int64_t active = 0;
        for (int64_t v = 0; v < n; ++v) {
            delta[v] = 0.0;
            if (fabs(r_out[v]) > epsp * sp[v]) {
                delta[v] = omega * r_out[v] / (1.0 + d[v]);
                z_out[v] += delta[v];
                r_out[v] = (1.0 - omega) * r_out[v];
                ++active;
                updates += indeg[v];
            }
        }
        if (active == 0) break;
        pushes += active;
        ++rounds;
        /* pull form of the same update: r_u += sum over row u of a_uj delta_j */
        for (int64_t u = 0; u < n; ++u) {
            double acc = 0.0;
            for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k)
                acc += (w ? w[k] : 1.0) * delta[col[k]];
            r_out[u] += acc;
        }
        if (rounds >= max_rounds) { rc = 1; break; }
    }
    if (stats) { stats[0] = pushes; stats[1] = updates; stats[2] = rounds; }
    for (int64_t v = 0; v < n; ++v) z_out[v] -= c_eff;
    free(d); free(sp); free(delta); free(indeg);
    return rc;
}

/*
 * The same synchronous rounds as oracle_push_rounds on nthreads host threads,
 * for the all-core CPU baseline.  Threads own contiguous row ranges of about
 * equal nonzeros; a round is the two loops of oracle_push_rounds, each thread
 * over its own rows, with a barrier after each, so every row's arithmetic is
 * the sequential one (results are bit for bit those of oracle_push_rounds).
 * Workers wait for a start signal, given once every thread exists, with the
 * number of threads that did start.  Returns 0, 1 at max_rounds, or -1 on
 * allocation failure.
 */
typedef struct {
    int64_t n;
    const int64_t *row_ptr;
    const int32_t *col;
    const double *w;
    const double *d, *sp;
    const int64_t *indeg;
    double *delta, *z, *r;
    double epsp, omega;
    int64_t max_rounds;
    int nth;                /* threads taking part (set before the start signal) */
    int64_t *lo;            /* nth + 1 row boundaries */
    int64_t *active, *upd;  /* per thread, per round */
    pthread_barrier_t bar;
    pthread_mutex_t mu;
    pthread_cond_t cv;
    int go;
    int64_t rounds, pushes, updates;
    int rc;
} rounds_ctx;

typedef struct {
    rounds_ctx *c;
    int t;
} rounds_arg;

static void rounds_run(rounds_ctx *c, int t)
{
    const int64_t v0 = c->lo[t], v1 = c->lo[t + 1];
    int64_t rounds = 0;
    for (;;) {
        int64_t act = 0, up = 0;
        for (int64_t v = v0; v < v1; ++v) {
            c->delta[v] = 0.0;
            if (fabs(c->r[v]) > c->epsp * c->sp[v]) {
                c->delta[v] = c->omega * c->r[v] / (1.0 + c->d[v]);
                c->z[v] += c->delta[v];
                c->r[v] = (1.0 - c->omega) * c->r[v];
                ++act;
                up += c->indeg[v];
            }
        }
        c->active[t] = act;
        c->upd[t] = up;
        pthread_barrier_wait(&c->bar);
        int64_t total = 0;
        for (int i = 0; i < c->nth; ++i) total += c->active[i];
        if (total == 0) break;
        if (t == 0) {
            c->pushes += total;
            for (int i = 0; i < c->nth; ++i) c->updates += c->upd[i];
        }
        ++rounds;
        for (int64_t u = v0; u < v1; ++u) {
            double acc = 0.0;
            for (int64_t k = c->row_ptr[u]; k < c->row_ptr[u + 1]; ++k)
                acc += (c->w ? c->w[k] : 1.0) * c->delta[c->col[k]];
            c->r[u] += acc;
        }
        pthread_barrier_wait(&c->bar);
        if (rounds >= c->max_rounds) {
            if (t == 0) c->rc = 1;
            break;
        }
    }
    if (t == 0) c->rounds = rounds;
}

static void *rounds_worker(void *p)
{
    rounds_arg *a = (rounds_arg *)p;
    rounds_ctx *c = a->c;
    pthread_mutex_lock(&c->mu);
    while (!c->go) pthread_cond_wait(&c->cv, &c->mu);
    pthread_mutex_unlock(&c->mu);
    if (a->t < c->nth) rounds_run(c, a->t);
    return NULL;
}

int oracle_push_rounds_threads(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                               const double *s, double eps, double omega, double c, double sigma,
                               int64_t max_rounds, int nthreads, double *z_out, double *r_out, int64_t *stats)
{
    if (nthreads < 1) nthreads = 1;
    rounds_ctx *ctx = (rounds_ctx *)calloc(1, sizeof(rounds_ctx));
    double *d = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *sp = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *delta = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    int64_t *indeg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *lo = (int64_t *)malloc(sizeof(int64_t) * ((size_t)nthreads + 1));
    int64_t *cnt = (int64_t *)calloc(2 * (size_t)nthreads, sizeof(int64_t));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    rounds_arg *args = (rounds_arg *)malloc(sizeof(rounds_arg) * (size_t)nthreads);
    int rc = -1;
    if (!ctx || !d || !sp || !delta || !indeg || !lo || !cnt || !th || !args) goto out;
    out_degree(n, row_ptr, w, d);
    for (int64_t k = 0; k < row_ptr[n]; ++k) indeg[col[k]]++;
    const double c_eff = shift_of(n, s, c);
    for (int64_t v = 0; v < n; ++v) {
        sp[v] = s[v] + c_eff;
        r_out[v] = sp[v];
        z_out[v] = 0.0;
    }
    ctx->n = n; ctx->row_ptr = row_ptr; ctx->col = col; ctx->w = w; ctx->d = d; ctx->sp = sp;
    ctx->indeg = indeg; ctx->delta = delta; ctx->z = z_out; ctx->r = r_out;
    ctx->epsp = sigma * eps / (c + sigma); ctx->omega = omega; ctx->max_rounds = max_rounds;
    ctx->lo = lo; ctx->active = cnt; ctx->upd = cnt + nthreads;
    pthread_mutex_init(&ctx->mu, NULL);
    pthread_cond_init(&ctx->cv, NULL);
    int started = 1;  /* this thread is thread 0 */
    for (int t = 1; t < nthreads; ++t) {
        args[t].c = ctx;
        args[t].t = t;
        if (pthread_create(&th[t], NULL, rounds_worker, &args[t]) != 0) break;
        ++started;
    }
    /* row ranges of about (nnz + n) / started nonzeros plus rows each */
    {
        const double per = (double)(row_ptr[n] + n) / started;
        int64_t v = 0;
        lo[0] = 0;
        for (int t = 1; t < started; ++t) {
            while (v < n && (double)(row_ptr[v] + v) < per * t) ++v;
            lo[t] = v;
        }
        lo[started] = n;
    }
    ctx->nth = started;
    pthread_barrier_init(&ctx->bar, NULL, (unsigned)started);
    pthread_mutex_lock(&ctx->mu);
    ctx->go = 1;
    pthread_cond_broadcast(&ctx->cv);
    pthread_mutex_unlock(&ctx->mu);
    rounds_run(ctx, 0);
    for (int t = 1; t < started; ++t) pthread_join(th[t], NULL);
    pthread_barrier_destroy(&ctx->bar);
    pthread_cond_destroy(&ctx->cv);
    pthread_mutex_destroy(&ctx->mu);
    rc = ctx->rc;
    if (stats) { stats[0] = ctx->pushes; stats[1] = ctx->updates; stats[2] = ctx->rounds; stats[3] = started; }
    for (int64_t u = 0; u < n; ++u) z_out[u] -= c_eff;
out:
    free(ctx); free(d); free(sp); free(delta); free(indeg); free(lo); free(cnt); free(th); free(args);
    return rc;
}

/*
 * Sequential successive over-relaxation in node order on (I + L) z = s, the
 * z-form of Eq. (gauss) with relaxation omega:
 *   z_v <- (1 - omega) z_v + omega (s_v + sum_j a_vj z_j) / (1 + d_v).
 * Runs sweeps until the FP64 residual max_v |s_v - ((I+L) z)_v| <= tol, or
 * max_sweeps.  Because (I+L)^{-1} is nonnegative and row-stochastic, the
 * returned z is within that residual of the exact equilibrium in max-norm.
 * Returns the number of sweeps (negative when max_sweeps was hit); the final
 * residual max-norm is written to *resid.
 */
int64_t oracle_sor_truth(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                         const double *s, double omega, double tol, int64_t max_sweeps,
                         double *z, double *resid)
{
    double *d = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    if (!d) return 0;
    out_degree(n, row_ptr, w, d);
    int64_t sweep = 0;
    double res = INFINITY;
    while (sweep < max_sweeps) {
        for (int64_t v = 0; v < n; ++v) {
            double acc = s[v];
            for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k)
                acc += (w ? w[k] : 1.0) * z[col[k]];
            z[v] = (1.0 - omega) * z[v] + omega * acc / (1.0 + d[v]);
        }
        ++sweep;
        res = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double acc = s[v] - (1.0 + d[v]) * z[v];
            for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k)
                acc += (w ? w[k] : 1.0) * z[col[k]];
            if (fabs(acc) > res) res = fabs(acc);
        }
        if (res <= tol) break;
    }
    *resid = res;
    free(d);
    return res <= tol ? sweep : -sweep;
}

/*
 * One Gauss-Seidel sweep in node order from z = 0 (z-form, omega = 1); the
 * reference side of the Theorem 2 equivalence.
 */
void oracle_gs_sweep_from_zero(int64_t n, const int64_t *row_ptr, const int32_t *col,
                               const double *w, const double *s, double *z)
{
    for (int64_t v = 0; v < n; ++v) z[v] = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        double acc = s[v];
        double dv = 0.0;
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
            acc += (w ? w[k] : 1.0) * z[col[k]];
            dv += w ? w[k] : 1.0;
        }
        z[v] = acc / (1.0 + dv);
    }
}

/*
 * Ordered residual-push SOR: sweeps over the nodes in the given order; each
 * node with |r_v| > eps' s'_v is pushed as in Alg. 3.  Stops after a sweep
 * with no push.  This is the SOR of Section 5.2 with the Gauss-Seidel order
 * fixed to `order` (for a colouring, classes in turn).
 * stats[0] = pushes, stats[1] = residual updates, stats[2] = sweeps.
 */
int oracle_sor_ordered(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                       const double *s, const int32_t *order, double eps, double omega,
                       double c, double sigma, int64_t max_sweeps, double *z_out, double *r_out,
                       int64_t *stats)
{
    int64_t *tptr;
    int32_t *tcol;
    double *tw;
    if (transpose(n, row_ptr, col, w, &tptr, &tcol, &tw) != 0) return -1;
    double *d = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    double *sp = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    if (!d || !sp) { free(tptr); free(tcol); free(tw); free(d); free(sp); return -1; }
    out_degree(n, row_ptr, w, d);
    double c_eff = shift_of(n, s, c);
    double epsp = sigma * eps / (c + sigma);
    for (int64_t v = 0; v < n; ++v) {
        sp[v] = s[v] + c_eff;
        r_out[v] = sp[v];
        z_out[v] = 0.0;
    }
    int64_t sweeps = 0, pushes = 0, updates = 0;
    int rc = 0;
    for (;;) {
        int64_t active = 0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t v = order[i];
            double rv = r_out[v];
            if (!(fabs(rv) > epsp * sp[v])) continue;
            double delta = omega * rv / (1.0 + d[v]);
            z_out[v] += delta;
            for (int64_t k = tptr[v]; k < tptr[v + 1]; ++k) r_out[tcol[k]] += tw[k] * delta;
            r_out[v] = (1.0 - omega) * rv;
            ++active;
            updates += tptr[v + 1] - tptr[v];
        }
        pushes += active;
        if (active == 0) break;
        ++sweeps;
        if (sweeps >= max_sweeps) { rc = 1; break; }
    }
    for (int64_t v = 0; v < n; ++v) z_out[v] -= c_eff;
    if (stats) { stats[0] = pushes; stats[1] = updates; stats[2] = sweeps; }
    free(tptr); free(tcol); free(tw); free(d); free(sp);
    return rc;
}

/* FP64 residual of the FJ system: r_v = s_v - (1 + d_v) z_v + sum_j a_vj z_j. */
void oracle_residual(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                     const double *s, const double *z, double *r)
{
    for (int64_t v = 0; v < n; ++v) {
        double dv = 0.0, acc = 0.0;
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
            double a = w ? w[k] : 1.0;
            dv += a;
            acc += a * z[col[k]];
        }
        r[v] = s[v] - (1.0 + dv) * z[v] + acc;
    }
}

/*
 * The same residual r = s - (I + L) z, evaluated as if in twice the working
 * precision and then rounded: the dot product of row v's terms
 * (s_v, -(1 + d_v) z_v, a_vj z_j ...) is accumulated by Ogita, Rump and
 * Oishi's Dot2 (SIAM J. Sci. Comput. 26, 2005), i.e. Knuth's error-free sum
 * of each term into the running total and fma's exact product error, with
 * the errors summed on the side.  d_v is summed the same way.  Used where a
 * plain FP64 row sum would lose the residual to cancellation (rows whose
 * terms are many orders of magnitude larger than the residual).
 */
static void dot2_add(double *hi, double *lo, double x)
{
    double s = *hi + x;
    double bp = s - *hi;
    double e = (*hi - (s - bp)) + (x - bp);
    *hi = s;
    *lo += e;
}

static void dot2_mul_add(double *hi, double *lo, double a, double b)
{
    double p = a * b;
    double pe = fma(a, b, -p);
    dot2_add(hi, lo, p);
    *lo += pe;
}

void oracle_residual_dot2(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                          const double *s, const double *z, double *r)
{
    for (int64_t v = 0; v < n; ++v) {
        double dh = 1.0, dl = 0.0; /* 1 + d_v */
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) dot2_add(&dh, &dl, w ? w[k] : 1.0);
        double hi = s[v], lo = 0.0;
        /* -(1 + d_v) z_v with 1 + d_v = dh + dl */
        dot2_mul_add(&hi, &lo, -dh, z[v]);
        dot2_mul_add(&hi, &lo, -dl, z[v]);
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) dot2_mul_add(&hi, &lo, w ? w[k] : 1.0, z[col[k]]);
        r[v] = hi + lo;
    }
}

/*
 * Dense LU with partial pivoting (Doolittle, row interchanges), then forward
 * and back substitution: solves M x = b for a dense row-major n x n M, which
 * is overwritten.  Returns 0, or 1 for an exactly singular pivot.
 */
int oracle_lu_solve(int64_t n, double *M, const double *b, double *x)
{
    int64_t *piv = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!piv) return -1;
    for (int64_t i = 0; i < n; ++i) piv[i] = i;
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        double best = fabs(M[k * n + k]);
        for (int64_t i = k + 1; i < n; ++i)
            if (fabs(M[i * n + k]) > best) { best = fabs(M[i * n + k]); p = i; }
        if (best == 0.0) { free(piv); return 1; }
        if (p != k) {
            for (int64_t j = 0; j < n; ++j) {
                double t = M[k * n + j]; M[k * n + j] = M[p * n + j]; M[p * n + j] = t;
            }
            int64_t t = piv[k]; piv[k] = piv[p]; piv[p] = t;
        }
        for (int64_t i = k + 1; i < n; ++i) {
            double l = M[i * n + k] / M[k * n + k];
            M[i * n + k] = l;
            if (l != 0.0)
                for (int64_t j = k + 1; j < n; ++j) M[i * n + j] -= l * M[k * n + j];
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        double acc = b[piv[i]];
        for (int64_t j = 0; j < i; ++j) acc -= M[i * n + j] * x[j];
        x[i] = acc;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double acc = x[i];
        for (int64_t j = i + 1; j < n; ++j) acc -= M[i * n + j] * x[j];
        x[i] = acc / M[i * n + i];
    }
    free(piv);
    return 0;
}

/*
 * The four measures of Table 1 plus the mean:
 *   out[0] = mean z, out[1] = C = sum z^2, out[2] = P = sum (z - mean)^2,
 *   out[3] = I = sum (z - s)^2, out[4] = D = sum over edges a_ij (z_i - z_j)^2.
 * For an undirected graph given as a symmetric CSR every edge appears twice,
 * so the arc sum is halved; a directed graph counts every arc once.
 */
void oracle_metrics(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                    const double *s, const double *z, int undirected, double *out)
{
    double sum = 0.0;
    for (int64_t v = 0; v < n; ++v) sum += z[v];
    double mean = n > 0 ? sum / (double)n : 0.0;
    double C = 0.0, P = 0.0, I = 0.0, D = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        C += z[v] * z[v];
        P += (z[v] - mean) * (z[v] - mean);
        I += (z[v] - s[v]) * (z[v] - s[v]);
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
            double diff = z[v] - z[col[k]];
            D += (w ? w[k] : 1.0) * diff * diff;
        }
    }
    out[0] = mean;
    out[1] = C;
    out[2] = P;
    out[3] = I;
    out[4] = undirected ? 0.5 * D : D;
}

/*
 * Sequential greedy colouring in a given priority order: each node, taken in
 * `order`, gets the smallest colour not held by an already coloured neighbour
 * in the symmetric adjacency (sym_ptr, sym_col).  Returns the colour count.
 */
int64_t oracle_greedy_colour(int64_t n, const int64_t *sym_ptr, const int32_t *sym_col,
                             const int32_t *order, int32_t *colour)
{
    for (int64_t v = 0; v < n; ++v) colour[v] = -1;
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; ++v)
        if (sym_ptr[v + 1] - sym_ptr[v] > maxdeg) maxdeg = sym_ptr[v + 1] - sym_ptr[v];
    int64_t *seen = (int64_t *)malloc(sizeof(int64_t) * ((size_t)maxdeg + 2));
    if (!seen) return -1;
    for (int64_t i = 0; i < maxdeg + 2; ++i) seen[i] = -1;
    int64_t ncol = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = order[i];
        for (int64_t k = sym_ptr[v]; k < sym_ptr[v + 1]; ++k) {
            int32_t cu = colour[sym_col[k]];
            if (cu >= 0 && cu <= maxdeg) seen[cu] = v;
        }
        int64_t c = 0;
        while (seen[c] == v) ++c;
        colour[v] = (int32_t)c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(seen);
    return ncol;
}

/*
 * Greedy colouring with a palette of K colours, in a given priority order,
 * on a symmetric adjacency (sym_ptr, sym_col) whose pair weights sym_q are
 * integers (the arc weights in 32.32 fixed point, summed over both arcs of a
 * pair).  Each node, in `order`, sums the weights of its already coloured
 * neighbours per colour and takes the smallest colour whose sum is zero, or,
 * when every colour of the palette is taken, the colour of least weight
 * (smallest index on ties).  With K at least the greedy colour count this is
 * the plain greedy colouring.  Returns the number of colours used.
 */
int64_t oracle_palette_colour(int64_t n, const int64_t *sym_ptr, const int32_t *sym_col, const int64_t *sym_q,
                              const int32_t *order, int K, int32_t *colour)
{
    int64_t *conf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
    if (!conf) return -1;
    for (int64_t v = 0; v < n; ++v) colour[v] = -1;
    int64_t used = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = order[i];
        for (int c = 0; c < K; ++c) conf[c] = 0;
        for (int64_t k = sym_ptr[v]; k < sym_ptr[v + 1]; ++k) {
            int32_t cu = colour[sym_col[k]];
            if (cu >= 0) conf[cu] += sym_q[k];
        }
        int best = -1;
        for (int c = 0; c < K && best < 0; ++c)
            if (conf[c] == 0) best = c;
        if (best < 0) {
            best = 0;
            for (int c = 1; c < K; ++c)
                if (conf[c] < conf[best]) best = c;
        }
        colour[v] = best;
        if (best + 1 > used) used = best + 1;
    }
    free(conf);
    return used;
}

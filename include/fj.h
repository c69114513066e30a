/*
 * fj.h - C ABI of the GB300 Friedkin-Johnsen solver.
 *
 * The library computes the Friedkin-Johnsen equilibrium z = (I + L)^{-1} s
 * (Lemma 1; Eq. 1 of Section 3.3) with the deterministic local residual push
 * of Section 5 (Alg. 1-3: BoundLocalIter, ImprovedBLI, BoundLocalIterSOR),
 * certifies it with an FP64 residual (Lemmas 3-5), and evaluates the four
 * measures of Table 1.  Every step runs in CUDA kernels on one GPU.
 *
 * Graph convention.  A graph is a CSR matrix A with n rows: row u lists the
 * nodes u listens to, a_uj = w[k] > 0 (1 when w == NULL).  d_u = sum_j a_uj is
 * the weighted out-degree and L = D - A, so node u's FJ update is
 * z_u <- (s_u + sum_j a_uj z_j) / (1 + d_u) (Eq. 1).  An undirected graph is
 * passed as a symmetric CSR (both arcs of every edge, equal weights).  Graphs
 * are simple (Section 3.2): no self-loops, no repeated (u, j) in a row.
 *
 * Memory.  Every array argument is a plain pointer; `mem` says whether the
 * pointers of that call are host (FJ_MEM_HOST) or device (FJ_MEM_DEVICE)
 * memory.  The caller owns all arrays it passes; the library never keeps a
 * caller pointer after a call returns.  A graph handle owns its device copy
 * of the CSR and every derived array and scratch buffer; fj_graph_destroy
 * frees them.  Work is issued on the CUDA stream given (NULL = legacy default
 * stream); calls return after their work is complete on that stream unless
 * stated otherwise.
 *
 * Errors.  Every call returns an fj_status.  Arguments are checked before any
 * work; a bad argument returns FJ_ERR_INVALID_ARG and leaves outputs
 * untouched.  A CUDA failure returns FJ_ERR_CUDA.  fj_last_error() gives a
 * one-line description of the last failure on the calling thread.  No call
 * aborts the process, traps on the device or waits without a bound.
 *
 * A handle is not thread-safe: calls on one handle must not overlap.
 * Separate handles are independent.
 *
 * Environment.  FJ_FRONTIER_LONG=<m> (read at each FP64 frontier cleanup of
 * a solve): in-neighbour lists longer than m are scattered by a block each
 * rather than a warp (default 4096; 0 sends every entry to the block path).
 * It changes the schedule of the cleanup's atomic updates, not its result
 * beyond their order.
 */
#ifndef FJ_H
#define FJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fj_graph fj_graph;

typedef enum {
    FJ_OK = 0,
    FJ_ERR_INVALID_ARG = 1,   /* an argument or the CSR failed validation */
    FJ_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    FJ_ERR_OOM = 3,           /* device allocation failed */
    FJ_ERR_NOT_CONVERGED = 4, /* sweep or refinement cap reached; outputs hold the partial result */
    FJ_ERR_DIVERGED = 5,      /* residual became non-finite (over-relaxation on a directed graph) */
    FJ_ERR_UNSUPPORTED = 6,   /* valid request this build does not serve */
    FJ_ERR_TIMEOUT = 7        /* a bounded device-side wait gave up; the result is not valid */
} fj_status;

enum { FJ_MEM_HOST = 0, FJ_MEM_DEVICE = 1 };

/* Arithmetic of the bulk push.  FP64: residual, increments and estimate in
 * FP64.  FP32: residual, thresholds, increments and all gathered values in
 * FP32; the estimate accumulates in FP64 and the certificate (and any
 * refinement restart) is computed in FP64. */
enum { FJ_PREC_FP64 = 0, FJ_PREC_FP32 = 1 };

/* Order in which pushes are applied.
 *  JACOBI      : synchronous rounds - every node above threshold pushes at
 *                once from the round-start residuals (the round view of the
 *                proof of Theorem 1).  Requires omega <= 1.
 *  MULTICOLOUR : Gauss-Seidel/SOR order (Theorem 2, Eqs. sor1-sor3) realised
 *                as colour classes of the symmetrised graph taken in turn;
 *                each class is an independent set, so its nodes push
 *                concurrently.  One launch per sweep: a node waits only for
 *                its own neighbours in earlier classes.  Any omega in (0, 2)
 *                (convergence for omega > 1 is guaranteed on undirected
 *                graphs only; directed graphs report FJ_ERR_DIVERGED if the
 *                residual blows up).
 *  AUTO        : MULTICOLOUR. */
enum { FJ_SCHED_AUTO = 0, FJ_SCHED_JACOBI = 1, FJ_SCHED_MULTICOLOUR = 2 };

typedef struct {
    double eps;          /* relative error parameter epsilon, in (0, 1) */
    double omega;        /* relaxation factor, in (0, 2); 1 = BoundLocalIter */
    double c;            /* shift constant c of Alg. 2 (default 1e-5) */
    double sigma;        /* threshold sigma of Alg. 2 (default 1e-5) */
    int precision;       /* FJ_PREC_* */
    int schedule;        /* FJ_SCHED_* */
    int64_t max_sweeps;  /* cap on rounds/sweeps per pass (default 100000; FP32 passes also stop
                            after 48): a pass that reaches it is certified and restarted from
                            its FP64 residual like one that stopped pushing */
    int max_refine;      /* cap on FP64 certify-and-restart passes that did not halve the
                            certified relative residual (default 8) */
    int palette;         /* MULTICOLOUR: colours allowed (default 16; 0 = as many as greedy
                            colouring needs).  When the palette runs out a node joins the
                            class where its neighbours' weight is least; those same-class
                            neighbours are coupled as in a synchronous round, and the node's
                            relaxation is lowered to omega_v <= 0.98 * 2(1+d_v)/(1+d_v+w_v)
                            (w_v: its weight to same-class neighbours), which keeps the
                            sweep convergent on undirected graphs (Gershgorin on M+M^T-A) */
    int check_every;     /* sweeps between host checks of the stop flag (0 = default 8) */
    int profile;         /* 1: time every launch of the push kernel with CUDA events on `stream`
                            and report it in fj_solve_info (adds event overhead; off by default) */
    void *stream;        /* cudaStream_t to run on; NULL = default stream */
} fj_solve_opts;

/* Per-solve report (per graph for a ragged handle, per vector for a batch). */
typedef struct {
    int64_t sweeps;          /* rounds (JACOBI) or sweeps (MULTICOLOUR), all passes */
    int64_t pushes;          /* node pushes */
    int64_t edges;           /* residual updates: sum of in-degrees of pushed nodes */
    int32_t refine_passes;   /* FP64 certify passes that restarted the push */
    int32_t converged;       /* 1 when the certificate below holds */
    double c_eff;            /* shift used: c + max(0, -min s) */
    double eps_prime;        /* sigma * eps / (c + sigma) (Alg. 2) */
    double resid_inf;        /* max_v |r_v|, r = s' - (I + L) zhat' in FP64 */
    double resid_rel_max;    /* max_v |r_v| / s'_v; <= eps_prime unless the FP64 resolution
                                term of the certificate (see fj_solve) binds somewhere */
    double z_inf;            /* max_v |z_v| */
    double err_bound;        /* max_v |z_v - z*_v| <= resid_inf (Lemma 5 with a
                                row-stochastic nonnegative (I + L)^{-1}) */
    int64_t launches;        /* kernels this call launched (all kinds) */
    int64_t push_launches;   /* launches of the push (pull-round) kernel */
    double push_ms;          /* profile = 1: summed CUDA-event time of the push launches */
    double push_bytes;       /* algorithmic bytes of the push launches: per nonzero the column,
                                weight and gathered increment; per row the offsets, residual
                                read/write, threshold, 1/(1+d) and increment write; per push
                                the in-degree and the FP64 estimate read/write */
    int64_t frontier_rounds; /* FP64 frontier push rounds (scatter form) run on the few
                                entries the certificate left above threshold */
    int64_t frontier_pushes; /* entries pushed by those rounds */
    double omega_used;       /* relaxation factor of the reported solve: opts.omega, or 1
                                after the FJ_SCHED_AUTO divergence fallback */
    int64_t frontier_edges;  /* residual updates of those frontier rounds (included in edges) */
    double method_bytes;     /* the push's own bytes: per residual update of the sweeps the
                                column, weight (weighted graphs) and increment (4 + 4 + sizeof
                                push precision), plus 32 per push (offsets, residual, estimate,
                                threshold, 1/(1+d)); a batch counts columns and weights once per
                                sweep and nonzero, since one load serves all k vectors */
    double seconds;          /* host wall time of the call */
    double cert_rel_err;     /* resid_inf / (z_inf - resid_inf): a bound on
                                max_v |z_v - zhat_v| / max_v |z*_v| (infinite when
                                resid_inf >= z_inf) */
    int32_t warm_start;      /* start of the push: -1 zero start (no z0 given), 1 the caller's
                                z0, 0 the zero start after z0 lost to it (fj_solve_warm) */
    int32_t reserved;        /* 0 */
} fj_solve_info;

/* The measures of Table 1 (Section 3.4). */
typedef struct {
    double P;       /* polarization  sum_i (z_i - mean z)^2 */
    double D;       /* disagreement  sum over edges a_ij (z_i - z_j)^2; undirected edges once */
    double I;       /* internal conflict sum_i (z_i - s_i)^2 */
    double C;       /* controversy   sum_i z_i^2 */
    double mean_z;  /* (1/n) sum_i z_i */
} fj_metrics_out;

/* Defaults: eps 1e-6, omega 1, c = sigma = 1e-5 (Section 6 settings), FP64,
 * AUTO, max_sweeps 100000, max_refine 8, stream NULL. */
void fj_solve_opts_default(fj_solve_opts *opts);

const char *fj_status_string(fj_status s);
const char *fj_last_error(void);

/*
 * fj_graph_create - device graph from a CSR (Section 3.2 matrices A, D, L).
 * n >= 1 rows; row_ptr[n+1] (int64, row_ptr[0] = 0, nondecreasing), col[nnz]
 * (int32 in [0, n)), w[nnz] (float32 > 0, finite) or NULL for unit weights.
 * directed = 0 declares a symmetric CSR.  Each row must be strictly
 * increasing (sorted, no repeats) and hold no self-loop.  The CSR is copied;
 * validation runs on the GPU and a violation returns FJ_ERR_INVALID_ARG.
 * Derived on the device: FP64 out-degrees, 1/(1+d) in FP32 and FP64,
 * in-degrees and, for directed graphs, the transposed CSR.  nnz < 2^31.
 */
fj_status fj_graph_create(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *w,
                          int directed, int mem, void *stream, fj_graph **out);

/*
 * fj_graph_create_from_arcs - graph ingest from an arc list (src[m], dst[m],
 * optional w[m]); arc e means src[e] listens to dst[e].  Self-loops are
 * dropped; of repeated (src, dst) arcs the first in array order is kept
 * (Section 3.2: simple graphs).  The rows come out sorted.  For an undirected
 * graph pass both arcs of every edge and directed = 0.
 */
fj_status fj_graph_create_from_arcs(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                    const float *w, int directed, int mem, void *stream,
                                    fj_graph **out);

/*
 * fj_graph_create_ragged - a batch of `ngraphs` independent graphs held as
 * one block-diagonal CSR.  node_offsets[ngraphs+1] (int64, starts at 0,
 * strictly increasing) gives each graph's node range; the CSR uses global
 * node ids and every arc must stay inside its graph.  Solves and metrics on
 * the handle report one fj_solve_info / fj_metrics_out per graph; each graph
 * gets its own shift c_eff.
 */
fj_status fj_graph_create_ragged(int ngraphs, const int64_t *node_offsets, const int64_t *row_ptr,
                                 const int32_t *col, const float *w, int directed, int mem,
                                 void *stream, fj_graph **out);

void fj_graph_destroy(fj_graph *g);

/* Sizes: n, nnz, number of graphs (1 unless ragged), number of colour classes
 * (0 until a MULTICOLOUR solve or fj_graph_colour has built them). */
fj_status fj_graph_info(const fj_graph *g, int64_t *n, int64_t *nnz, int *ngraphs, int *ncolours);

/*
 * fj_graph_export - copy the device CSR back: row_ptr[n+1], col[nnz], w[nnz]
 * (w ignored when the graph is unweighted).  transposed = 1 exports the
 * in-neighbour CSR (row v lists every u with a_uv > 0 in ascending u).
 * Any output pointer may be NULL.  deg64[n] receives the FP64 out-degrees.
 */
fj_status fj_graph_export(const fj_graph *g, int transposed, int64_t *row_ptr, int32_t *col,
                          float *w, double *deg64, int mem, void *stream);

/*
 * fj_graph_colour - greedy colouring of the symmetrised graph (u ~ v when
 * a_uv > 0 or a_vu > 0) in largest-degree-first order (ties: higher 32 bits of
 * SplitMix64(v) first, then lower v), computed by a Jones-Plassmann kernel;
 * the result equals the sequential greedy colouring in that order.  palette
 * = 0 allows any number of colours, so classes are independent sets and
 * sweeping them in turn is a Gauss-Seidel order (Theorem 2).  palette = K > 0
 * allows K colours: a node whose palette is exhausted takes the colour of
 * least conflict weight, the sum over coloured neighbours of round(a * 2^32)
 * for each arc between them (smallest colour on ties).  colour[n] (int32) may
 * be NULL; *ncolours may be NULL.
 */
fj_status fj_graph_colour(fj_graph *g, int palette, int32_t *colour, int *ncolours, int mem, void *stream);

/*
 * fj_graph_order - the row order of the multicolour schedule with this
 * palette (built here if no solve or fj_graph_colour has built it).  Rows are
 * renumbered so that each colour class is contiguous, except for a hub
 * prefix: for one graph and a palette of 1..32 colours, the nodes of largest
 * in-degree (in-degree >= the smallest threshold that admits at most 49,152
 * of them; every node when n <= 49,152) come first, ordered by class.  Inside
 * every range the order is in-degree descending, then caller id.  So class c
 * is rows [hub_row[c], hub_row[c+1]) and [class_row[c], class_row[c+1]), with
 * hub_row[ncolours] = *nhub = class_row[0].  Without a hub prefix (palette 0
 * or a ragged handle) the order is by colour then caller id and *nhub = 0.
 * The order keeps the increments most rows gather together (the sweep stages
 * the hubs' in shared memory); any order is a valid Gauss-Seidel order
 * (Theorem 2), and results are returned in caller order.  perm[i] = the caller
 * id of row i (n entries, per mem; may be NULL); hub_row and class_row are host
 * arrays of ncolours + 1 entries (fj_graph_colour or fj_graph_info give
 * ncolours; either may be NULL); *nhub (host) may be NULL.
 */
fj_status fj_graph_order(fj_graph *g, int palette, int32_t *perm, int64_t *nhub, int64_t *hub_row,
                         int64_t *class_row, int mem, void *stream);

/*
 * fj_solve - ImprovedBLISOR (Alg. 3 with the shift of Alg. 2) on the GPU.
 * Under opts->schedule == FJ_SCHED_AUTO a solve whose residual becomes
 * non-finite with omega > 1 (the multicolour SOR is only proven for
 * symmetric systems, Section 5.2; directed graphs can diverge) is restarted
 * with omega = 1 (Gauss-Seidel on the diagonally dominant I + L, which
 * converges); info.omega_used reports the factor of the returned solve.
 * An explicit schedule returns FJ_ERR_DIVERGED instead.
 * s[n] (FP64) innate opinions; z_out[n] (FP64) receives
 * zhat = (push estimate of (I+L)^{-1}(s + c_eff)) - c_eff.  On FJ_OK every
 * node meets the FP64 certificate |r_v| <= max(eps' s'_v, 2^-51 (1 + d_v)
 * |zhat'_v|), where r = s' - (I + L) zhat' is evaluated with sums good to
 * twice the working precision (FP32-pair sums with an error bound on short
 * rows, re-summed in FP64 Dot2 where the bound cannot decide; 128-bit
 * fixed-point sums on rows over 512 nonzeros, whose truncation bound counts
 * against the row).  The second term is the FP64 resolution of
 * row v (one ulp of zhat'_v moves r_v by (1 + d_v) ulp); it binds only where
 * eps' s'_v is finer than that (high degree, s'_v near c).  Where the first
 * term binds everywhere, |z_v - zhat_v| <= eps' (z_v + c_eff) (Lemma 5); in
 * all cases max_v |z_v - zhat_v| <= max_v |r_v| = info.err_bound, since
 * ||(I + L)^{-1}||_inf <= 1.  info (may be NULL) gets one record per graph.
 * FJ_ERR_NOT_CONVERGED / FJ_ERR_DIVERGED still write z_out and info.
 */
fj_status fj_solve(fj_graph *g, const double *s, const fj_solve_opts *opts, double *z_out,
                   fj_solve_info *info, int mem);

/*
 * fj_solve_warm - as fj_solve, but the push starts from the estimate z0[n]
 * (FP64) instead of zero: the initial residual is r = s' - (I + L)(z0 + c_eff),
 * computed in FP64, and pushes use the |r| test of Alg. 3, so any start
 * converges to the same certificate (Lemmas 3 and 5).  The zero start judges
 * z0 and is its fallback: the push's work falls with the residual sum
 * (Section 5.1.2), so z0 is used only when sum_v |r_v| < sum_v s'_v, the
 * zero start's residual sum (both summed in a fixed order); otherwise the
 * solve starts from zero.  info.warm_start reports which start was used.
 */
fj_status fj_solve_warm(fj_graph *g, const double *s, const double *z0, const fj_solve_opts *opts,
                        double *z_out, fj_solve_info *info, int mem);

/*
 * fj_solve_batch - k opinion vectors on one graph as one multi-right-hand-side
 * push.  S and Z_out are node-major [n][k] FP64 (element (v, j) at v*k + j);
 * 1 <= k <= 64.  Every (node, vector) pair keeps its own shift c_eff,
 * threshold, residual and FP64 certificate, and pushes by the test of Alg. 3
 * on its own residual; the sweeps are shared, so a node's column indices and
 * weights are read once per sweep for all k vectors.  The result of each
 * vector meets the same bound as fj_solve.  info (may be NULL) gets k
 * records (sweeps, pushes and launches are batch totals).  A ragged handle is
 * rejected with FJ_ERR_INVALID_ARG.  S must not alias Z_out.
 */
fj_status fj_solve_batch(fj_graph *g, const double *S, int k, const fj_solve_opts *opts,
                         double *Z_out, fj_solve_info *info, int mem);

/*
 * fj_solve_batch_warm - fj_solve_batch from the starts Z0[n][k] (node-major,
 * FP64): every vector's start is judged against its zero start as in
 * fj_solve_warm, and a vector whose start loses restarts from zero while the
 * others keep theirs (info[j].warm_start).  S, Z0 and Z_out must not alias.
 */
fj_status fj_solve_batch_warm(fj_graph *g, const double *S, const double *Z0, int k, const fj_solve_opts *opts,
                              double *Z_out, fj_solve_info *info, int mem);

/*
 * fj_solve_trace - fj_solve that also records how the push converges, for
 * relative-error-versus-time curves (the shape of the paper's Fig. 1).  After
 * every batch of sweeps between stop checks (opts->check_every, 8 by default)
 * and after every certificate it appends one row of 4 doubles to trace:
 *     [ms since the solve's first sweep, sweeps so far, rel, kind]
 * with rel = max_v |r_v| / s'_v of r = s' - (I + L) zhat, kind 0 after a
 * batch of sweeps (r evaluated afresh in FP64 from the current estimate; the
 * time of that evaluation is left out of the rows' times) and kind 1 for the
 * exact certificate.  By Lemma 5, |z - zhat| <= rel (z + c_eff) elementwise,
 * so rel bounds the relative error.  trace is a host array of 4 * cap
 * doubles; at most cap rows are written and *count receives their number.
 * A kind-0 row costs one FP64 residual evaluation (one pass over the graph).
 * On a divergence fallback (FJ_SCHED_AUTO) the trace restarts with the
 * omega = 1 solve.  Otherwise as fj_solve.
 */
fj_status fj_solve_trace(fj_graph *g, const double *s, const fj_solve_opts *opts, double *z_out,
                         fj_solve_info *info, int mem, double *trace, int cap, int *count);

/*
 * fj_graph_omega_opt - the SOR factor of Section 5.2's optimal-omega equation
 * (Eq. 17),  omega_opt = 1 + (mu / (1 + sqrt(1 - mu^2)))^2,  with
 * mu = rho((I + D)^{-1} A), the spectral radius of the Jacobi iteration matrix
 * of (I + L) z = s (D the weighted out-degrees).  mu is estimated by `iters`
 * steps of power iteration on B = (I + M) / 2, M = (I + D)^{-1} A, from the
 * all-ones vector; B's dominant eigenvalue (1 + mu) / 2 is strictly largest
 * in modulus even when -mu is an eigenvalue of M (bipartite graphs), so the
 * iteration converges there too.  Each step is one FP64 SpMV in a fixed
 * summation order (deterministic).  Eq. 17 is exact for consistently ordered
 * matrices (bipartite graphs in red-black order, Theorem 2 of the SOR
 * literature the paper cites); for other graphs it is the standard estimate.
 * mu_out and omega_out are host pointers, either may be NULL; stream may be
 * NULL.  FJ_ERR_INVALID_ARG for iters outside 1..100000 or an empty graph.
 * fj_graph_tune adds omega_opt (200 steps) to its candidates.
 */
fj_status fj_graph_omega_opt(fj_graph *g, int iters, double *mu_out, double *omega_out, void *stream);

/*
 * fj_graph_tune - autotuner for fj_solve on this graph.  Times complete,
 * certified solves of s (reps timed calls after one untimed call each, CUDA
 * events on base->stream) for every candidate: Jacobi rounds at omega 1, and
 * the multicolour schedule for palette K in {4, 8, 16, 32} x omega in {1.2,
 * 1.5, 1.6, 1.7, 1.8, omega_opt of fj_graph_omega_opt}.  *best receives base
 * with the schedule, palette and omega of the fastest (its colouring is left
 * built on the handle); *best_ms (may be NULL) its mean time.  Costs 200
 * power-iteration steps, one colouring per palette and 25 (reps + 1) solves.
 * FJ_ERR_NOT_CONVERGED when no candidate certifies.
 */
fj_status fj_graph_tune(fj_graph *g, const double *s, const fj_solve_opts *base, int reps,
                        fj_solve_opts *best, double *best_ms, int mem);

/*
 * fj_graph_tune_batch - as fj_graph_tune for fj_solve_batch on S[n][k], with
 * one more dimension: how each warp gathers the neighbours' k-vectors (4 or 8
 * per-lane loads in flight, or, for FP32 with k a multiple of 4, bulk
 * asynchronous copies of whole rows into shared memory, the default).  The
 * best choice stays on the handle for later batch solves.
 */
fj_status fj_graph_tune_batch(fj_graph *g, const double *S, int k, const fj_solve_opts *base, int reps,
                              fj_solve_opts *best, double *best_ms, int mem);

/*
 * fj_metrics - P, D, I, C and mean z of Table 1 for opinions s[n] and
 * equilibrium z[n] (FP64), summed in FP64 in a fixed order (deterministic).
 * out gets one record per graph (ngraphs for a ragged handle).
 */
fj_status fj_metrics(fj_graph *g, const double *s, const double *z, fj_metrics_out *out, int mem,
                     void *stream);

/*
 * fj_metrics_batch - the measures of fj_metrics for k opinion vectors at once:
 * S and Z node-major [n][k] (FP64, element (v, j) at v*k + j), 1 <= k <= 64,
 * out[k] one record per vector.  FP64 sums in a fixed order (deterministic).
 * A ragged handle is rejected (use fj_metrics).
 */
fj_status fj_metrics_batch(fj_graph *g, const double *S, const double *Z, int k, fj_metrics_out *out, int mem,
                           void *stream);

/*
 * fj_frontier - the push frontier F = {v : |r_v| > h_v} (strict test of Alg. 1
 * and Alg. 3) as ascending node ids, by warp-ballot and shared-memory
 * compaction with a decoupled look-back across thread blocks.  precision
 * selects FP64 or FP32 r and h.  r, h, list and count are DEVICE pointers;
 * list must hold n entries; *count (int64, device) receives |F|.
 */
fj_status fj_frontier(int64_t n, const void *r, const void *h, int precision, int32_t *list,
                      int64_t *count, void *stream);

/*
 * fj_frontier_static - the same frontier as fj_frontier, for callers that
 * cannot allocate device memory: a process whose device memory is all handed
 * out up front by its own pool or arena (a serving process that reserves the
 * GPU's memory at start-up, or a framework that owns the allocator), where a
 * cudaMalloc would fail or take memory the pool has promised elsewhere.  It
 * makes no allocation of any kind (no cudaMalloc, cudaFree, stream-ordered or
 * library allocation).  The paper has no counterpart: this is a property of
 * the interface only.
 *
 * The look-back scratch is a file-scope device array sized for n up to 2^26
 * (67,108,864) nodes, about 256 KB, which every GPU that loads the library
 * holds until the process exits; a larger n returns FJ_ERR_INVALID_ARG.  The
 * array is shared by every call: the call clears what must start at zero, and
 * calls whose work overlaps on the GPU (on different streams, or from
 * different threads) race on it and must not be made.  The first call on each
 * device looks up the array's device address with cudaGetSymbolAddress and
 * keeps it for the life of the process; make that first call before any stream
 * capture begins.  After cudaDeviceReset the kept address is stale, like every
 * other handle of this library, so no call may follow a reset.  Each call
 * waits for its stream to finish: it reads the count back to the host to
 * check the look-back's status.  Arguments, layout and errors are those of
 * fj_frontier: r, h, list and count are device pointers, list holds n entries,
 * *count receives |F|.
 */
fj_status fj_frontier_static(int64_t n, const void *r, const void *h, int precision, int32_t *list,
                             int64_t *count, void *stream);

/*
 * fj_residual - FP64 residual r[n] = s' - (I + L) zhat' with s' = s + c_eff,
 * zhat' = z + c_eff, for caller-supplied s, z (FP64) and shift c_eff; the
 * quantity of Lemma 3 used by the certificate.
 */
fj_status fj_residual(fj_graph *g, const double *s, const double *z, double c_eff, double *r,
                      int mem, void *stream);

/* ------------------------------------------------------------------ failure paths
 *
 * Two hooks for testing how the library fails, without faulting the GPU.
 * Neither has a counterpart in the paper.
 *
 * fj_wait_selftest - runs the library's two bounded device waits (the scan
 * look-back's wait on a tile status word, the bulk-copy ring's wait on an
 * mbarrier) on one thread of one block, each on something that nothing
 * completes, with a limit of `polls` polls (1..2^24).  Returns FJ_ERR_TIMEOUT
 * when both gave up, as they must; the context stays usable (later calls
 * work).  FJ_OK means a wait returned although nothing completed it.
 *
 * fj_debug_fail_allocation - makes device allocation number after + 1 of the
 * library, counted from this call, fail as if the device were full (the call
 * that made it returns FJ_ERR_OOM); one allocation fails, then the hook
 * disarms itself.  after < 0 disarms it.  Process-wide; meant for tests, not
 * for use while other threads call the library.
 */
fj_status fj_wait_selftest(int64_t polls, void *stream);
void fj_debug_fail_allocation(int64_t after);

/* ------------------------------------------------------------------ learned warm start
 *
 * A three-layer message-passing network that predicts a start z0 for
 * fj_solve_warm.  It has no counterpart in the paper: a push from any start
 * reaches the same certificate (Lemmas 3 and 5), so the network can only
 * change the work, never the result.  With a_vj the CSR weights, d_v the
 * weighted out-degree and din_v the number of nodes listening to v:
 *   x_v  = [s_v, log(1 + d_v), log(1 + din_v), sum_j a_vj s_j / d_v]
 *   h^l_v = relu(Ws^l^T h^{l-1}_v + Wn^l^T g^{l-1}_v + b^l),
 *   g^{l-1}_v = sum_j a_vj h^{l-1}_j / d_v (0 when d_v = 0), h^0 = x,
 *   l = 1, 2, 3, width 64;  z0_v = b_v + w_o . h^3_v + b_o with
 *   b_v = (s_v + d_v m_v) / (1 + d_v), m_v the weighted mean of s over the
 *   nodes v listens to (one Jacobi step of (I + L) z = s from z = s).
 * The dense products run on the tensor cores in BF16 with FP32 accumulation.
 *
 * Parameters are one FP32 vector of fj_mpnn_param_count() entries, in this
 * order: for l = 1, 2, 3 the matrices Ws^l [F_in][64] and Wn^l [F_in][64]
 * (row-major; F_in = 4 for l = 1, else 64) and b^l [64], then w_o [64], b_o.
 * The handle owns the parameters, the Adam state and the activations of the
 * last graph it saw; it is bound to the device current at creation.
 */
typedef struct fj_mpnn fj_mpnn;

int64_t fj_mpnn_param_count(void);

/* params: host FP32 vector of fj_mpnn_param_count() entries (copied). */
fj_status fj_mpnn_create(const float *params, fj_mpnn **out);
void fj_mpnn_destroy(fj_mpnn *m);
fj_status fj_mpnn_get_params(const fj_mpnn *m, float *params);
fj_status fj_mpnn_set_params(fj_mpnn *m, const float *params);

/*
 * fj_mpnn_predict - z0[n] (FP64) for opinions s[n] (FP64) on graph g: the
 * network's output clamped to [min s, max s] (where z lies, Section 3.2),
 * except that a node with d_v = 0 (it listens to nobody) takes s_v, its exact
 * equilibrium value.  Host or device pointers per mem.  A ragged handle is
 * treated as one graph (clamp to the global range).
 */
fj_status fj_mpnn_predict(fj_mpnn *m, fj_graph *g, const double *s, double *z0, int mem, void *stream);

/*
 * fj_mpnn_grad - forward and backward pass on one (graph, s, z) triple with
 * loss mean_v (z0_v - z_v)^2 (z0 before clamping).  *loss receives the loss
 * (may be NULL); grad (host FP32, fj_mpnn_param_count() entries, may be NULL)
 * receives the gradient, which the handle also keeps for fj_mpnn_adam_step.
 */
fj_status fj_mpnn_grad(fj_mpnn *m, fj_graph *g, const double *s, const double *z, double *loss, float *grad,
                       int mem, void *stream);

/*
 * fj_mpnn_adam_step - one Adam update (beta1 0.9, beta2 0.999, eps 1e-8,
 * bias-corrected; Kingma and Ba 2015) with learning rate lr in (0, 1) from
 * the gradient of the last fj_mpnn_grad.  FJ_ERR_INVALID_ARG without one.
 */
fj_status fj_mpnn_adam_step(fj_mpnn *m, double lr, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FJ_H */

/*
 * ccx.h -- C ABI of a GB300 (sm_103a) solver for convex clustering by the
 * proximal distance (PD) algorithm of Chen, Chi, Ranola and Lange,
 * "Convex Clustering: An Attractive Alternative to Hierarchical Clustering"
 * (arXiv:1409.2065).
 *
 * Problem (Methods, Eq. 1 and, with missing entries, Eq. 6):
 *   minimise_U  1/2 sum_{(i,c) observed} (x_ic - u_ic)^2 + mu sum_{i<j} w_ij ||u_i - u_j||
 * over centroids u_i, one per case (row) x_i of the n x p data matrix X.
 * The library computes, for each penalty mu of a user grid (the paper's
 * mu; this header calls it gamma), the fixed point of the paper's PD/MM map
 * (Methods, "The Proximal Distance Algorithm": the projection onto
 * C = {v_ij = u_i - u_j}, the smoothed distance d_m of Eq. 5, the U update
 * and the block soft-threshold V update; "Missing Data": Y = X on observed
 * entries and the current U elsewhere), warm-starting each gamma from the
 * previous one.  Fused edges are those whose V update returns exactly zero
 * (gamma w_ij d >= rho ||b_ij||); clusters are the connected components of
 * the fused edges, labelled 0.. by the rank of their smallest member.
 *
 * Conventions for every call:
 *  - Every function returns a ccx_status.  On failure nothing the caller
 *    owns is freed; ccx_last_error() returns a thread-local message.
 *  - Arrays are row-major.  "host or device" pointers are classified with
 *    cudaPointerGetAttributes; device pointers must be on the device that
 *    was current when the problem was created.
 *  - The caller owns every array it passes.  The library copies inputs at
 *    the call and never keeps a caller pointer after returning.
 *  - All GPU work of a problem runs on the stream given at creation (NULL =
 *    the legacy default stream); calls that return results synchronise that
 *    stream before returning.
 *  - A ccx_problem may be used by one host thread at a time (a problem
 *    submitted to a server belongs to the server until ccx_wait returns).
 *
 * Beyond one path: ccx_solve_batch (several problems together),
 * ccx_server_* (continuous batching with admission by device memory),
 * ccx_build_knn_composite (genetic + geographic weights),
 * ccx_min_connected_k, ccx_principal_axes / ccx_solve_path_projected,
 * ccx_shard_* (one problem split by columns), and
 * instrumentation calls (ccx_time_iterations, ccx_kernel_launches,
 * ccx_sweep_plan) that have no counterpart in the paper.
 */
#ifndef CCX_H
#define CCX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ccx_problem ccx_problem;
typedef struct ccx_server ccx_server;

typedef enum {
    CCX_OK = 0,
    CCX_EINVAL = 1,       /* invalid argument; message says which */
    CCX_ENOMEM = 2,       /* device or host allocation failed */
    CCX_ECUDA = 3,        /* a CUDA runtime call failed */
    CCX_ENOTCONV = 4,     /* max_iter reached for some gamma; outputs are still written */
    CCX_ETIMEOUT = 5,     /* a bounded wait ran out (server); nothing was lost */
    CCX_ECANCELLED = 6,   /* job cancelled before it ran */
    CCX_EUNSUPPORTED = 7  /* size outside what this build handles; message gives the limit */
} ccx_status;

enum { CCX_FP32 = 0, CCX_FP64 = 1 };

/*
 * k-nearest-neighbour Gaussian-kernel weights (Calibration of Weights,
 * Eq. 8): w_ij = 1{i ~_k j} exp(-phi ||x_i - x_j||^2), where i ~_k j when j
 * is among the k nearest other cases of i or i among those of j (ties go to
 * the smaller index).  Missing entries are filled with their column's
 * observed mean for this purpose only.  phi_auto != 0 takes
 * phi = 1 / median ||x_i - x_j||^2 over the union edges.  normalize != 0
 * scales the weights to sum to 1 over i < j (the paper normalises them;
 * this is equivalent to rescaling gamma).  Edges of weight exactly 0 are dropped.
 */
typedef struct {
    int k;          /* neighbours per case, 1 <= k; k >= n-1 gives all pairs */
    double phi;     /* >= 0, used when phi_auto == 0 */
    int phi_auto;
    int normalize;
    int gram;       /* Gram matrix that selects the candidate neighbours: 0 (default) tensor cores on
                       TF32 operands, 1 tensor cores on BF16 operands (rounded to nearest), 2 FP32 CUDA
                       cores.  Candidates are chosen with a rigorous bound on that Gram's error and get
                       exact distances, so the edge set is the same for every choice; a coarser Gram only
                       gives more candidates to refine.  Unused when k >= n - 1 (all pairs). */
} ccx_knn_rule;

/*
 * Solver options.  The paper fixes neither rho (only that it must exceed a
 * Lipschitz constant of the loss) nor eps (only that it is a small positive
 * number); the library takes rho = rho_scale (||Y_c||_F + gamma ||w||_2) and
 * eps = (eps_rel ||Y_c||_F)^2 with Y_c the column-centred start matrix.
 */
typedef struct {
    double rho_scale;  /* default 2 */
    double eps_rel;    /* default 1e-3 */
    double tol;        /* stop when the estimated error of U is <= tol ||U||_F; default 1e-6 (FP32), 1e-10 (FP64) */
    int max_iter;      /* MM iterations per gamma; default 200000 */
    int accelerate;    /* 1: Nesterov-extrapolated MM with restarts (default); 0: the plain MM iteration */
    int chunk;         /* iterations per captured CUDA graph launch; default 64 */
    int extrapolate;   /* 1 (default): from the third gamma of a call on, start each gamma from the
                          secant prediction A_k + c (A_k - A_(k-1)) of the last two solutions
                          (c from the log-gamma spacing, at most 1); 2: the quadratic through
                          the last three solutions while the last three gammas stopped on the
                          tolerance, the secant otherwise; 0: start from A_k.  The fixed point is
                          the same in every case. */
    int stream_edges;  /* 0 (default): the iteration kernel keeps the per-edge index and accumulator
                          arrays in shared memory when they fit beside the rows of a slice, and in
                          global memory otherwise; 1: always in global memory.  Results are
                          identical either way (same arithmetic in the same order). */
    int slice_variant; /* staging of the iteration kernel's column slices: 0 (default) automatic;
                          1: the next slice is staged while the current one is processed (double
                          buffer) whenever both fit in shared memory; 2: one buffer.  Results are
                          identical in every case. */
    int max_ctas;      /* 0 (default): the iteration kernel runs one CTA per SM, at most one per
                          4-column slice; > 0 caps its grid, so that each CTA processes more slices
                          (or a problem leaves SMs to others).  Results agree within the rounding of
                          the per-CTA float partial sums, which the grid size changes. */
    double fuse_delta; /* the V update returns zero when gamma w_ij d >= rho ||b_ij||; when the two
                          sides differ by at most fuse_delta rho ||b_ij||, ||b_ij|| is recomputed in
                          double from the rows of the projection before the decision, so a fuse
                          decision does not rest on the rounding of float partial sums.  Default
                          1e-5; 0 disables the recompute. */
    int anderson;      /* 0 (default): off.  1..16: while the path has not started fusing (no edge fused at
                          the end of the previous gamma), each gamma starts with Anderson mixing of the
                          MM map over the last `anderson` map outputs (the momentum is off meanwhile);
                          the restart rule takes over when an edge fuses, when the mixed residual stops
                          falling, or after 3000 iterations, and its stopping test decides convergence
                          as usual.  The fixed point is the same; the mixing keeps 2 x anderson + 1
                          float copies of the matrix on the device.  The ccx_shard_* calls ignore it. */
} ccx_opts;

/* Per-gamma statistics. */
typedef struct {
    int iters;         /* MM iterations spent on this gamma */
    int converged;     /* 1: error estimate <= tol; 2: stopped at the rounding level of the arithmetic
                          (steps at the level of their own rounding noise, or a residual that no longer
                          falls while the estimate from its last measured decay rate is <= 100 tol);
                          0: max_iter reached */
    int n_fused;       /* fused edges at the returned iterate */
    int n_clusters;    /* connected components of the fused edges */
    double gamma, rho, eps;
    double d_final;    /* d_m of the last iteration */
    double err_est;    /* estimated relative error of U at stop */
    double seconds;    /* wall time of this gamma, including its output copies */
    int n_recomputed;  /* edges whose fuse decision at the returned iterate was taken from the double
                          recompute of ||b_ij|| (see ccx_opts.fuse_delta) */
    long long recomputes;  /* double recomputes of ||b_ij|| over all iterations of this gamma */
    int mixing_iters;  /* iterations of this gamma spent in the Anderson mixing phase (ccx_opts.anderson) */
} ccx_gamma_stats;

/* Fill *o with the defaults listed above. */
void ccx_opts_default(ccx_opts* o);

/*
 * Create a problem from the n x p data matrix X (Methods: n cases, p
 * predictors; rows are cases).
 *   X     : n rows of p floats, row stride ld >= p floats; host or device.
 *   mask  : NULL (all observed) or n rows of p bytes, stride ld; 1 = observed,
 *           0 = missing (Missing Data, the set Gamma).  Host or device.
 *   n, p  : n >= 1, p >= 1.
 *   stream: cudaStream_t for all work of this problem, or NULL.
 *   precision: CCX_FP32 or CCX_FP64 (FP64 keeps a double copy of X).
 * Errors: CCX_EINVAL for bad sizes, a non-finite observed entry, or a row
 * with no observed entry; CCX_ENOMEM; CCX_ECUDA.
 */
ccx_status ccx_problem_create(const float* X, const uint8_t* mask, int64_t n, int64_t p, int64_t ld,
                              int precision, void* stream, ccx_problem** out);

/*
 * Standardise the predictors (Methods: the predictors are standardised before
 * clustering) on the GPU, using observed entries only: each column is centred
 * on the mean of its observed entries and divided by their standard deviation
 * (divisor = their count), in double and rounded once to the working
 * precision; a column whose observed entries are all equal is centred only,
 * and one with no observed entry stays 0.  Call it right after
 * ccx_problem_create: it replaces the problem's data, so it also clears the
 * edge set, the principal axes and the path state.
 */
ccx_status ccx_standardize(ccx_problem* pr);

/*
 * Copy the start matrix Y_0 out: the data as the solver sees them (after any
 * ccx_standardize), with each missing entry at its column's observed mean
 * (Missing Data: the iteration starts from U = Y_0).  Y0_out: n x p floats,
 * host or device.
 */
ccx_status ccx_get_start(const ccx_problem* pr, float* Y0_out);

/*
 * Set the weighted edge set explicitly (host arrays): edge e joins cases
 * ei[e] < ej[e] with weight w[e] >= 0 (Methods: the set E of pairs with
 * positive weight).  Zero-weight edges are dropped.  Replaces any earlier
 * edge set.  CCX_EINVAL on an index out of range, ei >= ej, a duplicate
 * pair, or a negative or non-finite weight.
 */
ccx_status ccx_set_edges(ccx_problem* pr, int64_t n_edges, const int32_t* ei, const int32_t* ej,
                         const double* w);

/*
 * Build the edge set on the GPU by the kNN Gaussian-kernel rule above
 * (Eq. 8).  Candidate neighbours come from a Gram matrix on the tensor
 * cores; their distances are recomputed exactly (double) before the k
 * nearest are chosen.  Replaces any earlier edge set.
 */
ccx_status ccx_build_knn(ccx_problem* pr, const ccx_knn_rule* rule);

/*
 * The kNN Gaussian-kernel rule above on the composite genetic + geographic
 * distance d_ij = alpha ||y_i - y_j|| + (1 - alpha) g_ij (Calibration of
 * Weights): neighbours, phi (phi_auto: 1 / median d^2 over the union edges),
 * weights exp(-phi d^2) and the normalisation all use d.
 *   coords  : host array of n (latitude, longitude) pairs in degrees,
 *             latitude in [-90, 90].
 *   alpha   : in [0, 1]; 1 gives ccx_build_knn.
 *   geodesic: 0: g = Euclidean norm of the coordinate difference in degrees,
 *             longitude difference taken modulo 360; 1: g = great-circle
 *             angle in degrees.
 * Candidates come from the tensor-core Gram with a bound that covers its
 * rounding; their distances, and g, are then computed exactly in double.
 * Replaces any earlier edge set.
 */
ccx_status ccx_build_knn_composite(ccx_problem* pr, const ccx_knn_rule* rule, const double* coords, double alpha,
                                   int geodesic);

/*
 * Smallest k in [1, k_max] for which the kNN union graph of the rule above
 * (i ~_k j; distances on the rows with missing entries at observed column
 * means, ties to the smaller index) is connected, i.e. for which the path can
 * end in complete coalescence (Calibration of Weights: the paper proposes
 * finding this k by bisection with a graph search).  *k_out = 0 when even
 * k_max (capped at n - 1) leaves the graph disconnected.  The neighbour lists
 * for k_max are built once on the GPU; each bisection probe runs the GPU
 * connected-components pass on their k-prefix.  The problem's edge set is not
 * changed.  CCX_EINVAL for k_max < 1 or n < 2.
 */
ccx_status ccx_min_connected_k(ccx_problem* pr, int k_max, int* k_out);

/*
 * Copy the current edge set out (host arrays, sorted by (ei, ej)).  With
 * ei == NULL only *n_edges is written (size query).  Otherwise *n_edges must
 * hold the capacity on entry and receives the count.
 */
ccx_status ccx_get_edges(const ccx_problem* pr, int64_t* n_edges, int32_t* ei, int32_t* ej, double* w);

/*
 * Median over edges of ||y_i - y_j|| / (2 w_ij) (Y = X with missing entries
 * at column means): the gamma at which an isolated pair would fuse under
 * Eq. 1.  Used to place a gamma grid.  CCX_EINVAL without edges.
 */
ccx_status ccx_fusion_scale(const ccx_problem* pr, double* gamma0);

/*
 * The same value as ccx_fusion_scale, computed without allocating memory: no
 * device memory at all, and no host memory unless the call fails (the error
 * message).  The paper has no counterpart to this call.  It serves callers
 * that may not allocate at the moment they need the gamma scale: a service
 * whose device memory is all reserved by its own pool, where cudaMalloc would
 * fail, or a loop that cannot afford the device-wide synchronisation that
 * cudaFree implies.  ccx_fusion_scale takes a temporary device buffer of 8
 * bytes per edge; this call uses a fixed buffer compiled into the library
 * instead (8 MiB of device memory, plus a host array of the same size).
 *   Limit   : at most 1048576 (2^20) edges; a larger edge set returns
 *             CCX_EINVAL with a message saying so (ccx_fusion_scale still
 *             handles it).
 *   Set-up  : the first call on a device looks up the buffer's address on
 *             that device and keeps it; make that first call before any
 *             stream capture begins on the device.  The kept address belongs
 *             to the device's current context: after cudaDeviceReset (or any
 *             teardown of the primary context) it is no longer valid, and
 *             this call must not be used again in that process.
 *   Sharing : every call in the process uses the same two buffers, which keep
 *             the last call's per-edge ratios.  A call writes every entry it
 *             reads, so nothing has to be cleared first.  Two calls whose GPU
 *             work overlapped would race on the device buffer; a call
 *             therefore holds a process-wide lock until its GPU work has
 *             finished, and calls from several host threads run one after
 *             another.
 * Returns CCX_EINVAL without edges.
 */
ccx_status ccx_fusion_scale_noalloc(const ccx_problem* pr, double* gamma0);

/*
 * Solve the warm-started path over gammas[0..n_gamma-1] in the order given
 * (Evaluation of Clusters: the program minimises over a user-given grid of mu).
 *   gammas    : host array, each finite and >= 0.
 *   opts      : NULL for defaults.
 *   U_out     : NULL, or n_gamma x n x ld floats (ld of the creation call),
 *               host or device; gamma g writes rows [g*n, (g+1)*n).
 *   labels_out: NULL, or n_gamma x n int32, host or device.
 *   stats     : NULL, or n_gamma host structs.
 * The first gamma starts from U = Y_0 (missing entries at their column's
 * observed mean) and V = 0; with a second call the path continues from
 * where the previous call stopped.  Returns CCX_ENOTCONV (outputs written)
 * when some gamma hit max_iter.  CCX_EUNSUPPORTED beyond this build's
 * on-chip limits (the message gives them).
 */
ccx_status ccx_solve_path(ccx_problem* pr, const double* gammas, int n_gamma, const ccx_opts* opts,
                          float* U_out, int32_t* labels_out, ccx_gamma_stats* stats);

/*
 * ccx_solve_path, also writing each gamma's fused flags (the edges whose V
 * update returned exactly zero at the returned iterate, Methods: the block
 * soft-threshold; the labels are the connected components of these edges):
 *   fused_out : NULL, or n_gamma x n_edges bytes (1 = fused), host or device,
 *               edges in the order of ccx_get_edges.
 */
ccx_status ccx_solve_path_fused(ccx_problem* pr, const double* gammas, int n_gamma, const ccx_opts* opts,
                                float* U_out, int32_t* labels_out, uint8_t* fused_out, ccx_gamma_stats* stats);

/*
 * Serving: a background scheduler that runs submitted path solves while the
 * caller keeps submitting (the paper has no serving layer; each job is one
 * ccx_solve_path).  Jobs that arrive while others are on the GPU are admitted
 * as running jobs finish and device memory frees up: a job starts when fewer
 * than max_active jobs run and the estimated iteration buffers of the running
 * jobs plus its own fit in hbm_budget bytes (0: 80 % of the device memory free
 * at creation); the first job always starts.  Running jobs share the GPU as in
 * ccx_solve_batch, and each job's result equals solving it alone.
 *   ccx_server_create : opts as in ccx_solve_path (NULL: defaults), applied to
 *                       every job; max_active <= 0 means 32.  Starts one host
 *                       thread, which makes all CUDA calls for the jobs.
 *   ccx_submit        : queues the path of problem pr over gammas (copied);
 *                       outputs as in ccx_solve_path.  The caller must not use
 *                       pr or the output buffers until ccx_wait has returned
 *                       for the ticket.  One job per problem at a time
 *                       (CCX_EINVAL otherwise).  When the job ends, the
 *                       problem's iteration buffers are released, so its next
 *                       solve starts from U_0 = Y_0.
 *   ccx_wait          : waits up to timeout_ms (< 0: no limit) and returns the
 *                       job's status, or CCX_ETIMEOUT while it still runs (wait
 *                       again later).  Never blocks beyond the limit.  A ticket
 *                       is released by the call that returns its status.
 *   ccx_server_destroy: jobs not yet started end with CCX_ECANCELLED; running
 *                       jobs finish first.  Wait for every ticket before.
 */
ccx_status ccx_server_create(const ccx_opts* opts, size_t hbm_budget, int max_active, ccx_server** out);
ccx_status ccx_submit(ccx_server* srv, ccx_problem* pr, const double* gammas, int n_gamma, float* U_out,
                      int32_t* labels_out, ccx_gamma_stats* stats, uint64_t* ticket);
ccx_status ccx_wait(ccx_server* srv, uint64_t ticket, int64_t timeout_ms);
ccx_status ccx_server_destroy(ccx_server* srv);

/*
 * Leading principal axes of the data (Evaluation of Clusters: the path is
 * displayed on principal components of the original data).  Y_0 (missing
 * entries at observed column means) is centred by its column means; the axes
 * are its leading q right singular vectors, computed on the GPU by subspace
 * iteration with q + 8 vectors and a Rayleigh-Ritz step in double, each signed
 * so that its entry of largest magnitude is positive.
 *   q        : 1 <= q <= 8 and q <= min(n, p).
 *   axes_out : NULL, or host q x p doubles (row c = axis c).
 *   var_out  : NULL, or host q doubles: variance of the data along each axis.
 * The axes are kept with the problem for ccx_solve_path_projected.
 */
ccx_status ccx_principal_axes(ccx_problem* pr, int q, double* axes_out, double* var_out);

/*
 * ccx_solve_path, but each gamma's centroids are projected on the GPU onto
 * the q principal axes above before they leave the device:
 *   scores_out : NULL, or n_gamma x n x q floats, host or device; entry
 *                (g, i, c) = <u_i(gamma_g) - mean of Y_0, axis c>.
 * The paper names the per-gamma transfer of U as its GPU bottleneck; this
 * moves n q instead of n p values per gamma.  Other arguments as in
 * ccx_solve_path (the path continues from the problem's warm-start state).
 */
ccx_status ccx_solve_path_projected(ccx_problem* pr, const double* gammas, int n_gamma, const ccx_opts* opts, int q,
                                    float* scores_out, int32_t* labels_out, ccx_gamma_stats* stats);

/*
 * Solve the paths of several independent problems together (each as
 * ccx_solve_path would, from its own warm-start state; the paper treats one
 * problem at a time, so this adds scheduling only).  Problem i runs its own
 * iterations on its own stream with its own gammas, outputs and stats; up to
 * max_active problems (<= 0: 32) have work queued on the GPU at once, so
 * problems too small to fill the GPU share it.  Results are identical to
 * solving each problem alone.
 *   probs      : n_probs distinct handles.
 *   gammas[i]  : host array of n_gamma[i] values for problem i.
 *   opts       : NULL for defaults, else applied to every problem.
 *   U_out[i], labels_out[i], stats[i] : as in ccx_solve_path for problem i
 *               (the outer arrays themselves may be NULL: no such outputs).
 *   status     : NULL, or n_probs entries receiving each problem's status.
 * Returns the first hard error of any problem (its message names the problem;
 * the other problems still run to the end), else CCX_ENOTCONV if some gamma
 * of some problem hit max_iter, else CCX_OK.  Blocks until all are done.
 */
ccx_status ccx_solve_batch(ccx_problem* const* probs, int n_probs, const double* const* gammas, const int* n_gamma,
                           const ccx_opts* opts, float* const* U_out, int32_t* const* labels_out,
                           ccx_gamma_stats* const* stats, int max_active, ccx_status* status);

/*
 * Feature-sharded iteration: one problem split by columns, e.g. over several
 * GPUs.  The paper's U update and its projection equations act on each column
 * separately (Methods, "The Proximal Distance Algorithm": the U-update display
 * and the stationarity equations of the block descent); only the per-edge
 * ||b_ij||^2 of the V update, the two pieces of d_m (Eq. 5) and the norms of
 * the stopping rule are sums over all columns.  A shard is a problem created
 * from a block of columns of X (and of the mask) and given the whole
 * problem's edge set (ccx_set_edges with the same arrays on every shard).
 *
 *   ccx_shard_norms       : this shard's ||Y_c||_F^2 and ||Y_0||_F^2 (sums over
 *                           its columns).  Sum them over the shards once.
 *   ccx_shard_begin_gamma : start penalty gamma (the shards' gammas must agree);
 *                           yc_sq_total / y0_sq_total are those sums, which fix
 *                           rho, eps and the error scale as for the whole problem.
 *                           The first call continues from the problem's
 *                           warm-start state (U = Y_0, V = 0 for a new problem or
 *                           after ccx_reset_path); later calls continue the path,
 *                           with the predictor of ccx_opts.extrapolate.
 *   ccx_shard_partials    : one MM iteration's column work on this shard, then
 *                           its partial sums in a fixed order into part (device
 *                           memory, *len doubles on entry, at least the size;
 *                           part = NULL: *len receives the size).
 *   exchange (the caller) : row s of an n_shards x len device array holds
 *                           shard s's part (an all-gather in shard order).
 *   ccx_shard_reduce      : the iteration's reduction on the summed partials
 *                           (fixed shard order, so every shard reaches the same
 *                           d_m, fuse decisions and stopping state).  done: NULL,
 *                           or receives whether this gamma has stopped (the host
 *                           then waits for the GPU); all shards stop together.
 *   ccx_shard_end_gamma   : this shard's columns of U (n x p_shard floats, host
 *                           or device), the labels (the same on every shard) and
 *                           the stats, as in ccx_solve_path.
 * With one shard the result is bit-identical to ccx_solve_path with the same
 * options; with several it agrees within the rounding of the partial sums.
 * All calls are ordered on the problem's stream; none blocks the host except
 * ccx_shard_reduce with done != NULL and ccx_shard_end_gamma.
 */
ccx_status ccx_shard_norms(const ccx_problem* pr, double* yc_sq, double* y0_sq);
ccx_status ccx_shard_begin_gamma(ccx_problem* pr, double gamma, const ccx_opts* opts, double yc_sq_total,
                                 double y0_sq_total);
ccx_status ccx_shard_partials(ccx_problem* pr, double* part, int64_t* len);
ccx_status ccx_shard_reduce(ccx_problem* pr, const double* parts, int n_shards, int* done);
ccx_status ccx_shard_end_gamma(ccx_problem* pr, float* U_out, int32_t* labels_out, ccx_gamma_stats* stats);

/*
 * Autotuning of the iteration kernel's grid (no counterpart in the paper).
 * Times 16 MM iterations of this problem at grids of G, G/2, G/4, ... CTAs
 * (G = one per SM, at most one per 4-column slice), down to g_min, and keeps
 * the grid with the least SM time per iteration (grid x iteration time; a
 * smaller grid is taken only when it saves at least 30 %, so work-bound problems
 * keep the whole GPU and only latency-bound ones shrink).  Later solves of the
 * problem whose options leave max_ctas at 0 use that grid, so a small problem
 * leaves SMs to the others in ccx_solve_batch or a server; results agree with
 * the default grid within the rounding of the per-CTA partial sums.  Needs the
 * edge set; must be called before the first solve or after ccx_reset_path (it
 * runs iterations from Y_0 and then resets the path).
 *   g_out : the chosen grid.  ms_out: NULL, or its mean milliseconds per iteration.
 */
ccx_status ccx_tune_grid(ccx_problem* pr, int g_min, int* g_out, double* ms_out);

/* Forget the warm-start state: the next ccx_solve_path starts from Y_0, V = 0. */
ccx_status ccx_reset_path(ccx_problem* pr);

/* Release all device and host memory of the problem (NULL is accepted). */
ccx_status ccx_problem_destroy(ccx_problem* pr);

/*
 * Instrumentation (no counterpart in the paper).  Runs n_iter MM iterations of
 * the problem's current warm-start state at penalty gamma with the stopping
 * test disabled, launching each iteration's two kernels individually and
 * timing them with CUDA events on the stream they run on.  Returns the mean
 * duration in milliseconds of the fused node/edge kernel (slice_ms) and of
 * the reduction kernel (reduce_ms).  The path state advances: a following
 * ccx_solve_path continues from it.  opts as in ccx_solve_path (NULL =
 * defaults).
 */
ccx_status ccx_time_iterations(ccx_problem* pr, double gamma, int n_iter, const ccx_opts* opts, double* slice_ms,
                               double* reduce_ms);

/*
 * Instrumentation: as ccx_time_iterations, with the Anderson mixing kernels
 * (history opts->anderson, which must be >= 1) launched after every
 * iteration; *mix_ms is their mean time per iteration.  Mixing stays on while
 * no edge is fused and for at most 3000 iterations, stagnation aside (it is
 * tested from the 320th iteration on): time it at a gamma below the first
 * fusion with n_iter < 320, or the later iterations measure only the kernels'
 * early exit.  Same errors as ccx_time_iterations; CCX_EINVAL also for a NULL
 * opts or mix_ms.
 */
ccx_status ccx_time_iterations_mixing(ccx_problem* pr, double gamma, int n_iter, const ccx_opts* opts,
                                      double* slice_ms, double* reduce_ms, double* mix_ms);

/*
 * Instrumentation (no counterpart in the paper; host only, needs no GPU): the
 * work layout the iteration kernel uses for a sorted edge set (0 <= ei < ej <
 * n, ordered by (ei, ej), no duplicates; n <= 65535).  The kernel's T threads
 * each walk a run of la node-sweep entries (CSR entries over both directions,
 * row by row) and a run of le edge-sweep entries (edge ids in order); entry k
 * of run t sits at position k * T + t, and inside each row of a run the order
 * is chosen against shared-memory bank conflicts.
 *   sizes    : 4 ints out: T, la, le, number of node-sweep partial slots.
 *   node_row, node_nbr : NULL, or la * T ints: row (case) and neighbour of
 *              each node-sweep position, -1 past the end of a run.
 *   edge_id  : NULL, or le * T ints: edge index of each edge-sweep position,
 *              -1 past the end.
 * Call once with NULL arrays to learn the sizes.  CCX_EINVAL on bad input.
 */
ccx_status ccx_sweep_plan(int64_t n, int64_t n_edges, const int32_t* ei, const int32_t* ej, int precision,
                          int32_t* sizes, int32_t* node_row, int32_t* node_nbr, int32_t* edge_id);

/* Number of GPU kernels this library has launched in the process so far
 * (all problems; kernels inside CUDA-graph launches are counted). */
uint64_t ccx_kernel_launches(void);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* ccx_last_error(void);

/* Library version string. */
const char* ccx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CCX_H */

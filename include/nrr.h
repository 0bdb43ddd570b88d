/*
 * nrr.h - C ABI of the GB300 library for robust non-rigid registration with
 * Welsch's function, majorization-minimization (MM) and Anderson acceleration
 * (Yao, Deng, Xu, Zhang, "Fast and Robust Non-Rigid Registration Using
 * Accelerated Majorization-Minimization", IEEE TPAMI 2023).
 *
 * Problem (Sec. 3): a source point set V = {v_i} (P points) is deformed by an
 * embedded deformation graph with N nodes p_j subset of V; node j carries an
 * affine map X_j = [A_j, t_j]. The library minimises
 *     E(X) = E_align + alpha E_reg + beta E_rot                 (Eq. 2)
 * with Welsch's function psi_nu (Eq. 4) on the closest-point distances to
 * the target set U (T points) and on the regularisation residuals D_ij
 * (Eq. 5), by MM with a convex quadratic surrogate solved as K X = B
 * (Eq. surr_solution), accelerated by Anderson mixing with an
 * energy-decrease safeguard (Sec. 3.3.4, Algorithm 2).
 *
 * Conventions shared by every call
 *  - Transform layout: X is [N][12] row-major doubles; X[j] is the paper's
 *    4x3 block of node j in the stacked X in R^{4N x 3}: X[j][0..8] = A_j^T
 *    row-major (i.e. A_j column-major), X[j][9..11] = t_j.
 *  - Point arrays are [n][3] row-major. Input and output buffers may live in
 *    host or device memory (the library uses unified addressing to tell them
 *    apart); they are caller-owned and only read/written during the call.
 *    The library copies everything it keeps.
 *  - Point indices are the caller's: index i of the arrays passed to
 *    nrr_create. Internally points are reordered; outputs are permuted back.
 *  - Every call runs on the CUDA stream given to nrr_create and returns when
 *    its outputs are ready (calls that return host data synchronise it).
 *  - Errors: every call returns an nrr_status; no exception crosses the ABI.
 *    nrr_last_error() gives a message for the last failure of a context.
 *    A context is not thread-safe; use one context per host thread.
 *  - Determinism: identical inputs and parameters give bitwise identical
 *    outputs (all reductions have a fixed order; no floating-point atomics).
 */
#ifndef NRR_H
#define NRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nrr_ctx nrr_ctx;

typedef enum {
    NRR_OK = 0,
    NRR_E_INVALID = 1,        /* bad argument (null pointer, size, range)   */
    NRR_E_CUDA = 2,           /* a CUDA runtime call failed                 */
    NRR_E_OOM = 3,            /* device or host allocation failed           */
    NRR_E_SINGULAR = 4,       /* the surrogate system could not be solved   */
    NRR_E_TIMEOUT = 5,        /* a bounded device-side wait ran out         */
    NRR_E_NOT_CONVERGED = 6,  /* informational: iteration cap reached       */
    NRR_E_STATE = 7           /* call not valid in the current state        */
} nrr_status;

/* Robust function of the alignment and regularisation terms. The paper's
 * method uses Welsch's function (Eq. 4); Sec. 4.2 compares it with the
 * squared l2 norm (all weights 1) and with l2 whose alignment weight is 0
 * once a distance reaches 3 nu_a (read as the MM weights of the truncated
 * quadratic min(d^2, 9 nu_a^2), the energy the library then reports). For
 * both l2 variants the regularisation term is sum |D_ij|^2 and Eq.
 * (WeightSettings) drops the factors that scale Welsch's curvature at zero:
 * alpha = k_alpha |V|/|E_G|, beta = k_beta |V|/|V_G|; NRR_L2 runs one stage. */
typedef enum {
    NRR_WELSCH = 0,
    NRR_L2 = 1,
    NRR_L2_TRUNCATED = 2
} nrr_robust;

/* Fixed nu instead of the annealing (Sec. 4.2, "Welsch-fmax/fmin/fmed"):
 * one stage at the first stage's (nu_a, nu_r), at the last stage's, or at
 * their means, the stages being those the annealing would run. */
typedef enum {
    NRR_NU_ANNEAL = 0,
    NRR_NU_FIXED_MAX = 1,
    NRR_NU_FIXED_MIN = 2,
    NRR_NU_FIXED_MED = 3
} nrr_nu_schedule;

typedef enum {
    NRR_FP64 = 0,   /* every step in double precision                        */
    NRR_MIXED = 1   /* closest points, weights, assembly and PCG in float;
                       energy sums, safeguard test and the Anderson
                       least-squares problem in double                      */
} nrr_precision;

/* Solver parameters. nrr_params_default() fills the paper's defaults. */
typedef struct {
    double graph_radius;       /* R of Eq. (InfluenceNodes); <= 0: 5 * l-bar
                                  (Sec. 4.1), l-bar = mean distance of a
                                  source point to its 6 nearest neighbours  */
    int    max_influence;      /* cap on |I(v_i)|, the nearest nodes kept;
                                  1..8, default 8                           */
    double nu_a;               /* initial nu_a; <= 0: median closest-point
                                  distance of the undeformed source (Sec.
                                  3.3.3)                                    */
    double nu_r;               /* initial nu_r; <= 0: 3 * l-bar            */
    double nu_a_min;           /* lower bound of nu_a; <= 0: l-bar/sqrt(3) */
    int    anneal;             /* 1: halve nu_a, nu_r per stage (Algorithm
                                  2); 0: a single stage at the initial nu   */
    double k_alpha, k_beta;    /* Eq. (WeightSettings); defaults 100, 1     */
    double alpha, beta;        /* >= 0 overrides the k_* rule; default -1  */
    int    aa_m;               /* Anderson depth m, 0..8; 0 = plain MM;
                                  default 5                                 */
    int    max_iters_per_stage;/* I_max of Algorithm 2 (solves per stage),
                                  default 100                               */
    int    max_total_passes;   /* cap on passes of nrr_solve incl. rejected
                                  ones; default 100000                      */
    double eps;                /* stop when max_i |v_hat_i^(k+1) - v_hat_i^(k)|
                                  < eps; <= 0: 1e-5 x bbox diagonal of
                                  source and target (Sec. 4.1)              */
    double rel_energy_tol;     /* > 0: a stage ends when consecutive kept
                                  energies differ by less than this
                                  relative amount (or at I_max), and the
                                  eps test is not applied; default 0 (off:
                                  the eps test)                             */
    int    precision;          /* nrr_precision; default NRR_MIXED          */
    double pcg_tol;            /* relative residual of the PCG solve of
                                  K X = B; <= 0: 1e-12 (FP64), 1e-6 (MIXED) */
    int    pcg_max_iters;      /* PCG iteration cap; default 500            */
    int    solve_ctas;         /* CTAs of the cluster solve: 0 = the largest
                                  cluster that holds the system (lowest
                                  latency for one pair), -1 = the smallest
                                  (batches; leaves SMs to other pairs),
                                  1..16 = that size if it fits              */
    int    robust;             /* nrr_robust; default NRR_WELSCH            */
    int    nu_schedule;        /* nrr_nu_schedule; default NRR_NU_ANNEAL
                                  (then `anneal` applies)                   */
    int    graph_on_gpu;       /* 1: nrr_create builds the deformation graph
                                  (Algorithm 1) on the GPU, the same graph
                                  as the host construction; default 0       */
    const int32_t* src_faces;  /* NULL (default): the source is a point
                                  cloud and D of Eq. (InfluenceNodes) is the
                                  Euclidean distance. Else the source is a
                                  triangle mesh with these n_src_faces faces
                                  [n][3] (vertex indices into src_xyz, host
                                  or device memory, read during nrr_create):
                                  Algorithm 1 uses exact geodesic distances
                                  on the sub-mesh of each node's ball, and
                                  l-bar is the mean mesh edge length (see
                                  nrr_graph_build_mesh); graph_on_gpu must
                                  then be 0                                 */
    int64_t n_src_faces;
} nrr_params;

/* State after a pass (one execution of the repeat body of Algorithm 2). */
typedef struct {
    double E, E_align, E_reg, E_rot; /* energy terms at the evaluated iterate */
    double nu_a, nu_r, alpha, beta;  /* parameters of the stage of that pass */
    double max_disp;                 /* stop-test quantity of the last solve */
    double pcg_rel_residual;         /* max over the 3 columns               */
    int    kept;                     /* 1: iterate kept; 0: rejected (AA)   */
    int    solved;                   /* 1: the pass ran the solve and mix   */
    int    stage;                    /* 0-based annealing stage              */
    int    done;                     /* 1: Algorithm 2 has returned          */
    int    pcg_iters;
    int    aa_mk;                    /* AA differences used in the mix      */
    int    n_passes, n_solves, n_rejected;
    int    status;                   /* nrr_status of device-side checks    */
    int    warning;                  /* NRR_E_SINGULAR if the last solve's K
                                        was singular (see n_singular), else
                                        NRR_OK; the pass itself succeeded   */
    int    n_singular;               /* connected components of the
                                        deformation graph on which no point
                                        had alignment weight in the last
                                        solve: K does not fix their common
                                        translation, and G keeps the
                                        component's summed translation of
                                        X^(k) (the paper is silent)         */
} nrr_step_info;

void nrr_params_default(nrr_params* params);

/* Creates a registration problem: builds the deformation graph (Sec. 3.1,
 * Algorithm 1 with Euclidean distances), the target search structure and
 * all device buffers, and sets X = identity (Algorithm 2).
 *   src_xyz [P][3], tgt_xyz [T][3]: float32, host or device memory.
 *   src_nrm, tgt_nrm: [P][3]/[T][3] normals or NULL. They are checked to be
 *     finite; the paper's point-to-point energy does not use them.
 *   cuda_stream: cudaStream_t to run on (NULL: the library creates its own
 *     non-blocking stream).
 * Returns NRR_E_INVALID for P < 1, T < 1, P >= 2^25, T >= 2^30, non-finite
 * coordinates or invalid parameters. On success *out owns all resources.
 * The caller's buffers are only read during the call. */
nrr_status nrr_create(nrr_ctx** out,
                      const float* src_xyz, const float* src_nrm, int64_t P,
                      const float* tgt_xyz, const float* tgt_nrm, int64_t T,
                      const nrr_params* params, void* cuda_stream);

void nrr_destroy(nrr_ctx* ctx);

/* One pass of Algorithm 2 at the current iterate X^(k): closest points
 * (Sec. 3.2), rotation projections, energy (Eq. 2), the safeguard test
 * (Sec. 3.3.4); if the iterate is kept: Welsch weights, assembly of K and B
 * (Sec. 3.3.2), the PCG solve of K X = B, and the Anderson mix (Eq.
 * AA_solution). The stopping test and the nu annealing of Algorithm 2 run
 * at the start of the following pass. info (host, may be NULL) receives the
 * pass summary. Returns NRR_E_STATE if the solve has already returned. */
nrr_status nrr_step(nrr_ctx* ctx, nrr_step_info* info);

/* Runs passes until Algorithm 2 returns or max_passes (<= 0: the
 * max_total_passes parameter) passes have run. info (host, may be NULL)
 * receives the final state; NRR_E_NOT_CONVERGED if the cap was hit. The
 * passes repeat on the device inside one graph launch (a conditional loop
 * whose body is the pass and a control kernel that tests the returned
 * flag, the status and the cap); the host reads the state once at the
 * end. With the environment variable NRR_HOST_LOOP set when the context's
 * pass graph is captured, the host launches the passes in groups of four
 * instead (same results). */
nrr_status nrr_solve(nrr_ctx* ctx, int max_passes, nrr_step_info* info);

/* Enqueues n passes (as nrr_step, without the host summary) on the
 * context's stream and returns without waiting for them. Passes after
 * Algorithm 2 has returned do nothing. For timing with events recorded on
 * the same stream; read the outcome afterwards with nrr_get_info. */
nrr_status nrr_enqueue_passes(nrr_ctx* ctx, int n);

/* Runs n passes like nrr_enqueue_passes, launching the steps of a pass
 * one after the other with CUDA events recorded around each on the
 * context's stream, and adds their durations (milliseconds, summed over the
 * n passes) to out_ms[0..5] = {deform + closest points, regularisation and
 * rotation terms, alignment energy + weights + safeguard, assembly of K and
 * B, PCG solve, Anderson mix (two kernels)}. Synchronises. (In the pass
 * graph the second step runs beside the first.) For measuring kernel
 * durations; the result of the passes is the same as with
 * nrr_enqueue_passes. */
nrr_status nrr_time_kernels(nrr_ctx* ctx, int n, double out_ms[6]);

/* Restarts Algorithm 2 from the beginning: X = identity, first stage with
 * the initial nu_a, nu_r, empty Anderson history, counters at zero. The
 * graph and search structures are kept. */
nrr_status nrr_reset(nrr_ctx* ctx);

/* Energy terms of Eq. (2) at X (X [N][12] doubles, host or device; NULL =
 * the current iterate) under the current stage's nu_a, nu_r, alpha, beta.
 * out_terms (host) = {E, E_align, E_reg, E_rot}. Does not change the
 * solver state. */
nrr_status nrr_energy(nrr_ctx* ctx, const double* X, double out_terms[4]);

/* Derivatives (the paper does not differentiate its solver; the readings
 * below are this library's).
 *
 * mode 0 - gradient of E (Eq. 2) at X (NULL = current iterate) with the
 * closest points held fixed at their values at X (rho is piecewise
 * constant):
 *   grad_X   [N][12] doubles (d E / d X, same layout as X), may be NULL;
 *   grad_src [P][3]  doubles (d E / d v_i through Eq. deformed_position,
 *            with node positions p_j held constant), may be NULL.
 *
 * mode 1 - gradient of a loss L(X^(K)) of the last nrr_unroll w.r.t. its
 * X^(0) and the source positions. X is then the cotangent dL/dX^(K)
 * ([N][12] doubles), or NULL for L = E(X^(K)) (closest points held at
 * X^(K)). Each step is differentiated implicitly: with lambda solving
 * K lambda = dL/dX^(k+1) (the same PCG), dL/dB = lambda and dL/dK =
 * -lambda X^(k+1)^T, propagated through the Welsch weights, the rotation
 * targets proj_R(A_j) and the rows of F; closest points, node positions,
 * skinning weights and r_ij are held constant; no gradient flows through
 * the argmin. Closest points, weights and K are recomputed from the
 * checkpoints X^(k). grad_X receives dL/dX^(0) [N][12], grad_src dL/dv
 * [P][3] (caller order); either may be NULL.
 * NRR_E_STATE for mode 1 without a previous nrr_unroll or after the stage
 * parameters changed. Host or device buffers. */
nrr_status nrr_backward(nrr_ctx* ctx, int mode, const double* X,
                        double* grad_X, double* grad_src);

/* The preliminary version's solver, a comparison solver on the same energy
 * (Sec. 3.3.4, the Remark on the preliminary version; Sec. 4.3). Each outer
 * iteration holds the closest points at the current iterate X^k, which
 * turns E into a surrogate that majorises it and equals it at X^k (the
 * Welsch functions and the rotation term are kept, so it is not quadratic),
 * and minimises that surrogate with an inner L-BFGS: the two-loop
 * recursion with m pairs (cleared at every outer iteration; a pair is kept
 * only if y.s > 1e-12 |y| |s|; H0 = gamma I with gamma = s.y / y.y of the
 * newest pair, or 1/|g| without pairs), a backtracking line search from
 * t = 1 that halves t until E(X + t d) <= E(X) + c1 t g.d (at most
 * max_halvings times; no acceptable step ends the inner solve), and the
 * inner solve ends when |g| <= g_tol |g_0| or after max_inner accepted
 * steps. The nu annealing, alpha, beta and the stopping tests (eps or
 * rel_energy_tol, I_max counting outer iterations) are those of Algorithm 2
 * with the context's parameters. */
typedef struct {
    int    m;              /* history pairs, 1..8; default 5                 */
    double c1;             /* sufficient decrease of the line search, (0,1);
                              default 1e-4                                  */
    double g_tol;          /* |g| <= g_tol |g_0| ends the inner solve;
                              default 1e-3                                  */
    int    max_inner;      /* accepted inner steps per outer iteration;
                              default 20                                    */
    int    max_halvings;   /* line-search halvings per step, 0..60; default
                              30                                            */
} nrr_lbfgs_params;

void nrr_lbfgs_params_default(nrr_lbfgs_params* params);

/* Runs outer iterations of the preliminary version's solver from the
 * context's current iterate and stage until the stage loop returns or
 * max_outer (<= 0: the max_total_passes parameter) outer iterations ran.
 * Each outer iteration counts as a pass and a solve in nrr_step_info
 * (n_passes, n_solves); E is the energy at the iterate it started from.
 * params NULL = defaults. info (host, may be NULL) receives the final
 * state; NRR_E_NOT_CONVERGED if the cap was hit; NRR_E_INVALID for
 * parameters out of range. nrr_step / nrr_solve may follow (they start a
 * fresh Anderson history). */
nrr_status nrr_solve_lbfgs(nrr_ctx* ctx, const nrr_lbfgs_params* params, int max_outer, nrr_step_info* info);

/* K plain MM steps from X0 (Sec. 3.3.1-3.3.2): X^(k+1) = K(X^(k))^-1
 * B(X^(k)) of Eq. (surr_solution) at the current stage's nu_a, nu_r, alpha,
 * beta, without the Anderson mix and the safeguard (the accept/reject
 * branch of Algorithm 2 is not differentiable). Keeps X^(0..K) in the
 * context as checkpoints for nrr_backward mode 1 (12 N values per step in
 * the context's precision). X0 [N][12] doubles; XK (may be NULL) receives
 * X^(K). Host or device buffers. The solver state (iterate, stage, Anderson
 * history) is left as it was. K in 0..1024. */
nrr_status nrr_unroll(nrr_ctx* ctx, int K, const double* X0, double* XK);

/* Checkpoint and resume of a solve (the paper has no counterpart). The
 * state is what later passes read and do not rebuild: the stage and
 * safeguard scalars, the iterate X, the last MM results, the Anderson
 * history and the deformed source of the last kept iterate, in the
 * context's precision, behind a header naming the problem's sizes and
 * precision and a 64-bit hash of its inputs (source and target points),
 * deformation graph and parameters. nrr_get_state_size gives its size in bytes; nrr_save_state
 * writes it to buf (host or device, at least that size); nrr_load_state
 * reads it into a context created from the same inputs and parameters, after
 * which the solve continues exactly (bitwise) as the saved one would have.
 * NRR_E_INVALID for a short buffer or a state saved from another problem
 * (other sizes, precision, inputs, graph or parameters). */
nrr_status nrr_get_state_size(nrr_ctx* ctx, size_t* bytes);
nrr_status nrr_save_state(nrr_ctx* ctx, void* buf, size_t bytes);
nrr_status nrr_load_state(nrr_ctx* ctx, const void* buf, size_t bytes);

/* Sets the current iterate X^(k) (X [N][12] doubles) and restarts the
 * current stage (E_prev = +inf, empty Anderson history). */
nrr_status nrr_set_transforms(nrr_ctx* ctx, const double* X);

/* Sets the annealing state: nu_a, nu_r of the current stage (alpha, beta
 * follow Eq. WeightSettings unless fixed in the parameters) and restarts
 * the stage. */
nrr_status nrr_set_stage(nrr_ctx* ctx, double nu_a, double nu_r);

nrr_status nrr_get_transforms(nrr_ctx* ctx, double* X);       /* [N][12]  */
nrr_status nrr_get_deformed(nrr_ctx* ctx, double* v_hat);     /* [P][3] at
                                                                 the last
                                                                 evaluated X */
/* Closest points of the last evaluated iterate: rho [P] (caller target
 * index, ties to the lowest index) and squared distances d2 [P]. */
nrr_status nrr_get_correspondence(nrr_ctx* ctx, int32_t* rho, double* d2);

/* Sizes of the problem. Any pointer may be NULL. */
nrr_status nrr_get_sizes(nrr_ctx* ctx, int64_t* P, int64_t* T, int64_t* N,
                         int64_t* n_edges, int32_t* max_influence);

/* The deformation graph (Algorithm 1): node_src [N] source index of each
 * node; nidx [P][max_influence] node ids of I(v_i) nearest first, -1 padded;
 * w [P][max_influence] weights of Eq. (weight_data); edges [n_edges][2]
 * undirected j<k sorted; r [2 n_edges] r_ij over directed pairs sorted by
 * (i, j) (Sec. 3.2); lbar (mean 6-NN spacing, or NaN if not needed).
 * Host buffers; any pointer may be NULL. */
nrr_status nrr_get_graph(nrr_ctx* ctx, int32_t* node_src, int32_t* nidx,
                         double* w, int32_t* edges, double* r, double* lbar);

/* The deformation graph alone, built on the host without a GPU: the same
 * construction nrr_create performs (Algorithm 1 with Euclidean distances,
 * Sec. 3.1; the weights of Eq. (weight_data) and r_ij of Sec. 3.2).
 * nrr_graph_build: src_xyz [P][3] host float32 source points (copied),
 * radius R (> 0; <= 0: 5 lbar with lbar the mean distance of each point to
 * its 6 nearest others), max_influence 1..8 (<= 0: 8). Errors:
 * NRR_E_INVALID (NULL pointer, P < 1, non-finite coordinate or radius,
 * max_influence > 8, a default radius 5 lbar that is 0, e.g. for identical
 * points), NRR_E_OOM. nrr_graph_sizes: N, n_edges (undirected),
 * max_influence and the radius used. nrr_graph_get: the arrays of
 * nrr_get_graph (same layouts; host buffers, any pointer may be NULL; lbar
 * is always computed here). nrr_graph_destroy accepts NULL. */
typedef struct nrr_graph nrr_graph;
nrr_status nrr_graph_build(nrr_graph** out, const float* src_xyz, int64_t P, double radius,
                           int max_influence);
/* The same graph built on the GPU (Algorithm 1, Sec. 3.1, Euclidean
 * reading): PCA by reductions and a 3x3 Jacobi eigen-solve, the visiting
 * order by a radix sort of the projections, the greedy sampling node by
 * node in that order in one CTA (its threads share the scan for the next
 * uncovered point and the covering of each new node's ball, over a window
 * of the visiting order held in shared memory, or through a uniform grid
 * of cells of size R when a node's R-slab exceeds that window: the
 * sequential decisions exactly), then the influence sets, weights, edges
 * and r_ij; every decision on a distance or projection is taken in double
 * without fused multiply-adds (float tests with proven margins only select
 * the candidates). src_xyz [P][3] float32, host or device; cuda_stream the
 * stream to use (NULL: the legacy default stream); l-bar on the GPU on the
 * graph's grid when the radius is given (points whose six nearest others
 * are not all within R by brute force on the GPU; on the host when the
 * radius defaults to 5 l-bar, or when more than 4,096 points are such).
 * Errors as nrr_graph_build, plus NRR_E_CUDA. The handle is used with
 * nrr_graph_sizes/get/destroy. */
nrr_status nrr_graph_build_gpu(nrr_graph** out, const float* src_xyz, int64_t P, double radius, int max_influence,
                               void* cuda_stream);
/* The deformation graph of a triangle-mesh source (Sec. 3.1, Algorithm 1
 * with the geodesic distance D of Eq. InfluenceNodes). Points are visited in
 * the PCA order of the point-cloud construction; a point with no influencing
 * node becomes a node v, its ball B(v) is found by a breadth-first search
 * along mesh edges through the vertices q with |v - q| < R, and D(v, q) is
 * the exact geodesic distance on the sub-mesh of the faces incident to
 * B(v) (window propagation: straight paths across unfolded faces that bend
 * only at vertices of total angle >= 2 pi or on a boundary; the paper uses
 * the VTP algorithm for the same distances); v influences q when D < R, with
 * the weight of Eq. (weight_data) from D. Influence caps, edges and r_ij as
 * nrr_graph_build. src_xyz [P][3] host float32; faces [n_faces][3] host
 * int32 vertex indices (every edge in at most two faces); radius R (> 0;
 * <= 0: 5 l-bar with l-bar the mean mesh edge length, Sec. 4.1);
 * max_influence 1..8 (<= 0: 8). lbar of nrr_graph_get is the mean edge
 * length. Errors: NRR_E_INVALID (NULL pointer, P < 1, n_faces < 1,
 * non-finite coordinate or radius, max_influence > 8, an index out of
 * range, a face that repeats a vertex or has a zero-length edge, an edge
 * of three or more faces), NRR_E_OOM. Host only; no GPU is used. */
nrr_status nrr_graph_build_mesh(nrr_graph** out, const float* src_xyz, int64_t P, const int32_t* faces,
                                int64_t n_faces, double radius, int max_influence);
nrr_status nrr_graph_sizes(const nrr_graph* g, int64_t* N, int64_t* n_edges, int32_t* max_influence,
                           double* radius);
nrr_status nrr_graph_get(const nrr_graph* g, int32_t* node_src, int32_t* nidx, double* w,
                         int32_t* edges, double* r, double* lbar);
void nrr_graph_destroy(nrr_graph* g);

/* The surrogate system of the last kept pass, in node order: Kdense
 * [4N][4N] (row-major, only the graph's blocks are non-zero) and B [4N][3].
 * Host buffers. For tests of the assembly; N <= 4096. */
nrr_status nrr_get_system(nrr_ctx* ctx, double* Kdense, double* B);

/* The G(X^(k)) of the last solve (the MM minimiser before mixing), [N][12]. */
nrr_status nrr_get_mm_solution(nrr_ctx* ctx, double* G);

/* Per-warp counters of the last closest-point search, for profiling the
 * search: recorded only if the context was created with the environment
 * variable NRR_NN_STATS set (otherwise *n_warps = 0). out [max_warps][4]
 * (host or device) = {SM cycles, super tiles visited, leaves staged, leaves
 * scanned} per warp; *n_warps receives the number of warps of a search.
 * With the tensor-core search the rows are per CTA of 128 queries: {SM
 * cycles, candidate leaves, chunks of 128 candidates (MMAs), queries searched
 * exactly because their window exceeded the kept candidates}. */
nrr_status nrr_get_search_stats(nrr_ctx* ctx, unsigned long long* out, int64_t max_warps,
                                int64_t* n_warps);

/* Phase timestamps (SM clock cycles) of the last cluster solve, recorded by
 * its first CTA, for profiling: only if the context was created with the
 * environment variable NRR_SOLVE_STATS set (otherwise zeros). out[63] holds
 * the number of stamps: start, after setup, before/after the first
 * reduction, before/after each reduction of the first 8 CG iterations,
 * before and after the Anderson mix. */
nrr_status nrr_get_solve_stats(nrr_ctx* ctx, long long out[64]);

/* State of the last pass without running one (host info). */
nrr_status nrr_get_info(nrr_ctx* ctx, nrr_step_info* info);

/* The pass-by-pass record of the last nrr_solve call: the state after each
 * pass of Algorithm 2 (energy terms, nu, kept/rejected, stage, PCG
 * iterations and residual, counters), in pass order, as nrr_step would have
 * reported it; when the call returned, the last record is that of the pass
 * whose stopping test ended Algorithm 2 (done = 1; it is not counted in
 * n_passes). Recorded on the device by the solve's device-side loop (no
 * host round trip per pass), for at most the first 8192 passes of the call;
 * empty when the passes were launched from the host (NRR_HOST_LOOP) or the
 * call ran no pass. out: host array of max_records entries, or NULL to query
 * the count; *n_records (may be NULL): records copied (or available when out
 * is NULL). NRR_E_INVALID for a NULL context or max_records < 0. */
nrr_status nrr_get_history(nrr_ctx* ctx, nrr_step_info* out, int max_records, int* n_records);

/* The alignment term of the energy (the sum of Welsch's function psi_nu_a
 * over the closest-point distances) and the weights of its quadratic
 * surrogate, computed from those distances without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (a preallocated real-time tracking loop, a host
 * framework whose allocator owns all device memory, work issued while a CUDA
 * graph is being captured), who therefore cannot create an nrr context.
 *   d2 [P]    float, device: squared closest-point distances |v_hat_i - u_rho(i)|^2
 *   nu_a      Welsch parameter (> 0)
 *   w_a [P]   float, device, output: exp(-d2_i / (2 nu_a^2)) / (2 nu_a^2)
 *   E_align   one double, device, output: sum_i psi_nu_a(sqrt(d2_i)), summed
 *             per CTA in double and then over CTAs in a fixed order
 *   cuda_stream: stream to run on (NULL = legacy default stream)
 * The call is asynchronous on the stream; it only enqueues work.
 * Scratch: a fixed 64 KiB static device array inside the library (every GPU
 * that loads the library holds it until the process exits), which bounds P
 * to 1..33,423,360 (NRR_E_INVALID beyond, with a message in
 * nrr_last_error(NULL)). The first call on a device looks the array's
 * address up (cudaGetSymbolAddress); make that first call before any stream
 * capture. All calls share the array: calls that overlap on the GPU race and
 * must be serialised by the caller. Allocates nothing, calls no cudaMalloc or
 * cudaFree. */
nrr_status nrr_align_energy_noalloc(const float* d2, int64_t P, double nu_a, float* w_a,
                                    double* E_align, void* cuda_stream);

/* Batches of independent registration problems (pairs). Each pair gets its
 * own context (its own graph, parameters and stream); one CUDA graph runs a
 * pass of every pair as parallel branches, so a batch advances all pairs in
 * one launch. Pairs that have returned do nothing in later passes.
 *   src_xyz[i], tgt_xyz[i]: float32 [P[i]][3], [T[i]][3], host or device.
 *   params: NULL (defaults), one nrr_params for all pairs
 *     (params_per_pair = 0) or an array of n_pairs (params_per_pair = 1).
 *   cuda_stream: the stream the batch graph runs on (NULL: own stream).
 * Errors of pair i are reported with its index in nrr_last_error(NULL). */
typedef struct nrr_batch nrr_batch;

nrr_status nrr_batch_create(nrr_batch** out, int n_pairs, const float* const* src_xyz,
                            const int64_t* P, const float* const* tgt_xyz, const int64_t* T,
                            const nrr_params* params, int params_per_pair, void* cuda_stream);

/* Runs batch passes until every pair's Algorithm 2 has returned or
 * max_passes (<= 0: the largest max_total_passes) passes ran. infos (host,
 * may be NULL) receives n_pairs summaries. NRR_E_NOT_CONVERGED if the cap
 * was hit. One graph launch repeats the pass of every captured pair on the
 * device until every pair has returned, a pair failed, the cap is reached
 * or half of the captured pairs have returned; the host then recaptures
 * the pairs still running (passes of returned pairs launch and do
 * nothing) and launches again. */
nrr_status nrr_batch_solve(nrr_batch* b, int max_passes, nrr_step_info* infos);

/* Restarts every pair (nrr_reset). */
nrr_status nrr_batch_reset(nrr_batch* b);

/* The context of pair i (owned by the batch; valid until nrr_batch_destroy),
 * for the per-pair getters. */
nrr_status nrr_batch_get_context(nrr_batch* b, int i, nrr_ctx** out);

void nrr_batch_destroy(nrr_batch* b);

/* Launch shapes of the two kernels whose best shape depends on the problem
 * (the paper has no counterpart; it runs on a CPU). */
typedef struct {
    int    nn_lanes_per_query; /* lanes that share one closest-point query:
                                  1, 2, 4 or 8 (more lanes shorten the
                                  serial search of the slowest warps)       */
    int    solve_ctas;         /* PCG solve: CTAs of the cluster that keeps
                                  K in shared memory (1..16), or 0 for the
                                  grid-wide solve. For a batch: -1 = each
                                  pair's smallest fitting cluster, 0 = its
                                  largest, -2 = balanced: the smallest
                                  cluster whose CTAs hold at most (all
                                  pairs' nodes / SMs) nodes each            */
    double nn_ms, solve_ms;    /* measured mean kernel durations of the
                                  chosen shapes (nrr_tune; 0 otherwise)     */
    double pass_ms;            /* measured mean batch pass (nrr_batch_tune) */
    int    launches_per_pass;  /* kernels one pass launches                 */
    int    nn_tensor_cores;    /* 1: closest points by the tensor-core
                                  candidate search (mixed path only): BF16
                                  split-precision distance tiles on the
                                  tensor cores choose each query's
                                  candidates, an exact float re-rank picks
                                  the winner; the results are bitwise those
                                  of the exact search (nn_lanes_per_query is
                                  then unused). 0: the exact pruned search   */
} nrr_launch_config;

/* Current launch shapes of a context (ms fields 0). */
nrr_status nrr_get_launch_config(nrr_ctx* ctx, nrr_launch_config* out);

/* Sets the launch shapes (NRR_E_INVALID for lanes not in {1,2,4,8}, a
 * cluster that does not fit this problem or device, or nn_tensor_cores on
 * an FP64 context) and recaptures the pass graph. Results stay within the tolerances of every shape; the
 * floating-point summation order, hence the last bits, depend on it. */
nrr_status nrr_set_launch_config(nrr_ctx* ctx, const nrr_launch_config* cfg);

/* Autotuner: picks the launch shapes by timing them on this context's own
 * problem. It runs the first pass of Algorithm 2 from X = identity, then
 * times reps (<= 0: 5) launches of the closest-point kernel for every
 * lanes-per-query value and of the tensor-core candidate search (mixed path)
 * and of the PCG solve of that pass's system (from the
 * pass's own warm start) for every cluster size that fits (and the
 * grid-wide solve), with CUDA events on the
 * context's stream, keeps the fastest of each and restarts the solve (as
 * nrr_reset). table_path (may be NULL): a text file of earlier results,
 * keyed by precision and the half-octave buckets of P, T and N; a usable
 * entry is applied without timing, a new result is appended. out (host, may
 * be NULL) receives the choice and its timings. */
nrr_status nrr_tune(nrr_ctx* ctx, const char* table_path, int reps, nrr_launch_config* out);

/* Autotuner for a batch: for lanes per query in {4, 8, 2} and each pair's
 * smallest or largest fitting cluster, times reps (<= 0: 3) batch passes
 * from the start (after one untimed pass), keeps the fastest policy for all
 * pairs and restarts every pair. Table as for nrr_tune (keyed by precision,
 * pair count, total points and total nodes). out->pass_ms receives the mean
 * batch pass of the choice. */
nrr_status nrr_batch_tune(nrr_batch* b, const char* table_path, int reps, nrr_launch_config* out);

/* Message describing the last failure on ctx (or a global message if ctx is
 * NULL). The string lives until the next call on ctx. */
const char* nrr_last_error(const nrr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* NRR_H */

/*
 * pdcs.h -- C ABI of the GB300 (sm_103a) restarted primal-dual conic solver.
 *
 * Solves   min c'x   s.t.   K x - h in C,   l <= x <= u
 * (the conic program of Sec. 2, eq. prob_cp, with no primal cone block), where
 * C is a product of zero, nonnegative, second-order, rotated second-order,
 * exponential and dual exponential cones listed in row order (eq. multi_cone_proj).  The dual is
 * eq. dual_conic: y in C*, lambda = c - K'y in Lambda (eq. defn_Lambda1).
 * The method is PDCS, Algorithm 1 of the paper: adaptive-step PDHG (eq. PDHG)
 * on the diagonally rescaled program, reflected Halpern iteration, the
 * step-weighted average, restarts and primal-weight updates, stopped by the
 * relative KKT test of eq. PDCS_terminate_tolerance.
 *
 * Conventions for every entry point:
 *   - all problem arrays passed to pdcs_create are HOST pointers; the library
 *     copies them into device memory it owns, so the caller may free them as
 *     soon as pdcs_create returns;
 *   - result arrays (x: n, y: m, lambda: n) are HOST pointers written by the
 *     library;
 *   - indices are 0-based; the column indices of a row need not be sorted;
 *   - every call returns a pdcs_status; pdcs_last_error() gives the text of the
 *     last failure of a context; no call aborts, traps or prints;
 *   - one context is used by one host thread at a time; all of its GPU work
 *     runs on the CUDA stream given to pdcs_create (NULL: a stream the library
 *     creates).
 */
#ifndef PDCS_H
#define PDCS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Cone kinds (Sec. 1 notation): ZERO {0}^d; NONNEG R_+^d; SOC {(t, x): ||x|| <= t};
 * RSOC {(x, y, z): ||z||^2 <= 2xy, x, y >= 0}; EXP the closure of
 * {(r, s, t): s > 0, t >= s exp(r / s)} (dim must be 3); EXP_DUAL its dual cone K_exp^*,
 * the closure of {(r, s, t): r < 0, -r exp(s / r) <= e t} (dim 3; a dual-cone row block of
 * the problem of Sec. 2, projected through the Remark of App. A.2; y of such a block lies
 * in K_exp). */
typedef enum {
    PDCS_CONE_ZERO = 0,
    PDCS_CONE_NONNEG = 1,
    PDCS_CONE_SOC = 2,
    PDCS_CONE_RSOC = 3,
    PDCS_CONE_EXP = 4,
    PDCS_CONE_EXP_DUAL = 5
} pdcs_cone_type;

typedef struct {
    int32_t type; /* pdcs_cone_type */
    int64_t dim;  /* rows covered; SOC >= 1, RSOC >= 2, EXP and EXP_DUAL == 3; the dims sum to m */
} pdcs_cone;

/* CSR matrix in host memory: row_ptr[m + 1] (row_ptr[0] == 0, nondecreasing),
 * col[nnz] in [0, n), val[nnz] finite.  nnz must be below 2^31. */
typedef struct {
    int64_t m, n, nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const double* val;
} pdcs_csr;

typedef enum {
    PDCS_OK = 0,                 /* call succeeded; for pdcs_solve: converged to tol */
    PDCS_ERR_INVALID = 1,        /* an argument failed validation (nothing changed) */
    PDCS_ERR_CUDA = 2,           /* a CUDA call failed (text in pdcs_last_error) */
    PDCS_ERR_OOM = 3,            /* device allocation failed */
    PDCS_ERR_NUMERIC = 4,        /* a NaN / Inf appeared in the iterates */
    PDCS_ERR_DEVICE_TIMEOUT = 5, /* a bounded device wait gave up: the blocks of the grid-wise SOC
                                    projection (options.soc_grid_dim) wait for one another with an
                                    iteration limit (a few seconds); the solver stops with this
                                    status instead of hanging */
    PDCS_MAX_ITER = 10,          /* max_iter PDHG evaluations done without reaching tol */
    PDCS_TIME_LIMIT = 11         /* options.time_limit seconds passed without reaching tol */
} pdcs_status;

enum { PDCS_RESCALE_NONE = 0, PDCS_RESCALE_COORD = 1, PDCS_RESCALE_BLOCK = 2 };
enum { PDCS_STEP_ADAPTIVE = 0, PDCS_STEP_CONSTANT = 1, PDCS_STEP_PLAIN = 2 };
enum { PDCS_PRECISION_FP64 = 0, PDCS_PRECISION_FP32 = 1 };

typedef struct {
    int32_t rescale;        /* PDCS_RESCALE_*: diagonal rescaling (Sec. 3), default per coordinate */
    int32_t ruiz_iters;     /* Ruiz passes (infinity norm), default 10 */
    int32_t pock_chambolle; /* 1: one Pock-Chambolle pass (alpha = 1) after Ruiz, default 1 */
    int32_t step_mode;      /* PDCS_STEP_*: adaptive (Algorithm 1), constant 0.998/||K||_2,
                               or plain PDHG of App. D (0.9/||K||_2, no Halpern, no restarts) */
    int32_t check_period;   /* restart / termination check every this many PDHG evaluations, default 64 */
    double beta;            /* reflection parameter of ReflectedHalpern (Algorithm 1 step 6), in
                               [0, 1], default 1 (constant: the adaptive rule of Algorithm 1 step 5
                               is not in the paper); 1/2 converges in fewer evaluations on small
                               programs, in more on the 1M-variable and 7,000 x 70,000 Lasso ones */
    int32_t power_iters;    /* power iterations for ||K||_2 (constant / plain modes), default 50 */
    int32_t precision;      /* PDCS_PRECISION_FP64 (default), or PDCS_PRECISION_FP32: SpMV, primal
                               / dual updates and cone projections on FP32 copies of K~, K~', the
                               scaled data and the iterates, while the checks (candidates, their
                               products, KKT residuals, restart and primal-weight decisions) stay
                               FP64; the FP32 phase hands over to FP64 iterations started from the
                               check's candidate (see fp32_switch_tol) */
    double fp32_switch_tol; /* FP32 mode: hand over once the relative KKT error of a check is at
                               most this (or the requested tol), or when its best value has not
                               improved by 10 % over 50 checks; default 1e-4 */
    int32_t use_graphs;     /* 1: replay each check period as one CUDA graph, default 1 */
    int32_t spmv_lanes;     /* lanes per CSR row in SpMV (1..32, power of 2) for every row; 0: rows
                               binned by length, lanes per row matched to each bin */
    double time_limit;      /* seconds for pdcs_solve; 0: none */
    const float* exp_mlp;   /* NULL (default), or PDCS_EXP_MLP_PARAMS weights of the learned starting
                               point of the exponential-cone root search (host array, copied at
                               create); used wherever a cone has no cached root (see below) */
    int32_t spmv_autotune;  /* 1: at create, time the candidate SpMV plans of K and K' (bin shift,
                               unroll) over 20 launches each and keep the fastest; the choice is
                               cached per process by matrix signature (rows, nnz, length histogram).
                               0 (default): the fixed plan (shift 3, unroll 4) */
    int32_t batch_blocks;   /* 0 (default): grids sized per kernel; > 0: every vector / cone kernel
                               of this program runs on exactly this many blocks (needed to join a
                               batch, whose programs share one grid; see pdcs_batch_create) */
    int32_t spmv_format;    /* storage of K~ and K~' for the SpMV: 1 rows binned by length (one to
                               32 lanes per row, see spmv_lanes / spmv_autotune); 2 sliced: rows of
                               at most 256 entries sorted by length in slices of 32, one lane per row
                               reading its entries in pairs by 128-bit loads, longer rows one warp
                               each (spmv_autotune then has no effect); 0 (default): 2 for single
                               programs, 1 when batch_blocks > 0 or spmv_lanes > 0 */
    int32_t soc_lane_entries; /* FP64 dual update of single programs: 0 (default) projects each
                               SOC / RSOC cone with one warp; > 0 stages cones of at most 256 rows
                               in shared memory and projects each with a group of S lanes (S a
                               power of two, the smallest with dim <= S * soc_lane_entries),
                               32 / S cones per warp (measured slower on the 1M-variable mixed-cone
                               program: 182 vs 153 us per dual update at 4) */
    int32_t soc_grid_dim;   /* grid-wise projection of large SOC / RSOC cones (Sec. 4, the grid-wise
                               strategy), single programs with FP64 iterates: several blocks of one
                               cooperative launch share a cone, its sums reduced across them in a
                               fixed order.  0 (default): the cones of at least 4096 rows that hold
                               more than 1 / (number of SMs) of all SOC rows; > 0: every cone of at
                               least this many rows; -1: none (one warp per cone throughout) */
    int32_t fuse_primal;    /* 1: with the sliced SpMV storage (single programs), the K' product of
                               an accepted step also applies the step's update to x and forms the next
                               evaluation's x-hat in its row epilogue (row j of K' is variable j), so
                               the separate primal update runs only after a rejected step or a check;
                               0 (default): separate kernels.  Same arithmetic either way except the
                               order of the ||x-hat - x||^2 sum.  Measured slower on the 1M-variable
                               mixed program (2,729 vs 2,960 evaluations/s): the slices hold the rows
                               sorted by length, so the epilogue's 13 accesses per variable scatter
                               (102.8 us for the fused product against 51.3 + 37.4 us) */
    /* Primal cone blocks x2 in K_p (Sec. 2, eq. prob_cp with n2 > 0): variables
     * primal_cone_start, primal_cone_start + 1, ... taken in order by n_primal_cones cones of
     * the given types (PDCS_CONE_SOC with dim >= 1, PDCS_CONE_RSOC with dim >= 2) and sizes;
     * their bounds must be lb = -inf, ub = +inf.  x-hat projects these blocks onto K_p, the
     * checks project the candidates onto them and the reduced costs lambda = c - K'y of their
     * variables onto K_p^* (both cones are self-dual), with no bound term in the dual
     * objective.  The columns of a block share one scale factor (the largest of their norms in
     * each rescaling pass), so D^{-1} K_p = K_p and the projection is the textbook one.  Host
     * array, copied at create; NULL / 0 (default): none.  Single programs with FP64 iterates
     * and separate primal updates only (PDCS_ERR_INVALID with precision FP32, batch_blocks > 0
     * or fuse_primal). */
    const pdcs_cone* primal_cones;
    int64_t n_primal_cones;
    int64_t primal_cone_start;
} pdcs_options;

typedef struct {
    int64_t attempts;  /* PDHG evaluations (accepted or rejected) so far */
    int64_t accepted;  /* accepted steps so far */
    int64_t restarts;  /* restarts so far */
    double err_p, err_d, err_gap; /* relative KKT errors of the returned solution */
    double pobj, dobj;            /* primal and dual objective values (original scaling) */
    double eta, omega;            /* current step size and primal weight */
    double setup_seconds;         /* time spent in pdcs_create */
    double solve_seconds;         /* time spent in pdcs_solve calls so far */
    int32_t status;               /* pdcs_status of the last pdcs_solve */
    int32_t fp64_phase;           /* 1 once FP32 mode has switched to FP64 polishing */
    int64_t kernel_launches;      /* kernels this context has launched so far (graph nodes included) */
    int32_t spmv_plan[4];         /* SpMV plans in use: bin shift and unroll of K, then of K'
                                     (binned format) */
    int32_t spmv_format;          /* SpMV storage in use: 1 binned, 2 sliced */
    int32_t soc_grid_cones;       /* SOC / RSOC cones projected grid-wise (options.soc_grid_dim) */
    int32_t fuse_primal;          /* 1 when the K' product forms the next primal update (options.fuse_primal) */
} pdcs_info;

typedef struct pdcs_ctx pdcs_ctx;

/* Fills *opt with the defaults listed above. */
void pdcs_default_options(pdcs_options* opt);

/* Builds a solver for one conic program.  K, c (n), h (m), cones are required;
 * lb / ub (n) may be NULL, meaning l = 0 and u = +inf; entries may be -inf / +inf.
 * Copies the data to the device, rescales it (Sec. 3 "diagonal rescaling"),
 * builds K' as a second CSR, groups the rows by cone kind and allocates the
 * iterate state.  cuda_stream: a cudaStream_t or NULL.  opt may be NULL.
 * Errors: PDCS_ERR_INVALID (bad sizes, indices, cone list, NaN data, l > u),
 * PDCS_ERR_OOM, PDCS_ERR_CUDA; *out is NULL then. */
pdcs_status pdcs_create(const pdcs_csr* K, const double* c, const double* h, const double* lb,
                        const double* ub, const pdcs_cone* cones, int64_t n_cones,
                        const pdcs_options* opt, void* cuda_stream, pdcs_ctx** out);

/* Runs Algorithm 1 from the current state until the relative KKT errors of
 * eq. PDCS_terminate_tolerance are all <= tol (checked every check_period
 * evaluations) or max_iter more PDHG evaluations are done.  tol <= 0 disables
 * the test and runs exactly max_iter evaluations.  Calls may be repeated; the
 * state carries over: a solver that converged stays converged, unless the new tol is
 * smaller than the one it met, in which case the iteration continues from where it
 * stopped.  info may be NULL.  Returns PDCS_OK on convergence, PDCS_MAX_ITER /
 * PDCS_TIME_LIMIT otherwise, or an error. */
pdcs_status pdcs_solve(pdcs_ctx* ctx, double tol, int64_t max_iter, pdcs_info* info);

/* Copies the returned solution (projected onto the bounds and the dual cone) in
 * the original scaling: x (n), y (m), lambda = c - K'y (n, may be NULL). */
pdcs_status pdcs_get_solution(pdcs_ctx* ctx, double* x, double* y, double* lambda);

/* Copies the current Halpern iterate z = (x, y) and the last PDHG output
 * zhat = (xhat, yhat), original scaling.  Any pointer may be NULL. */
pdcs_status pdcs_get_iterate(pdcs_ctx* ctx, double* x, double* y, double* xhat, double* yhat);

/* Copies the diagonal scalings: dr (m, rows), dc (n, columns); K~ = diag(dr) K diag(dc). */
pdcs_status pdcs_get_scaling(pdcs_ctx* ctx, double* dr, double* dc);

/* Fills *info with the counters and the errors of the last check. */
pdcs_status pdcs_get_info(pdcs_ctx* ctx, pdcs_info* info);

/* Sets the starting point z^{0,0} = (x, y) (original scaling; NULL means 0) and,
 * when omega > 0, the initial primal weight; resets the counters, the restart state and
 * a NaN / Inf status.  The step size eta is kept (the last one of the previous solve, or
 * 1 / max |K~ij| after pdcs_create), as the oracle's warm start does. */
pdcs_status pdcs_set_warm_start(pdcs_ctx* ctx, const double* x, const double* y, double omega);

/* Scalars of Algorithm 1 carried by pdcs_get_state / pdcs_set_state. */
typedef struct {
    double eta;        /* step size of the next PDHG evaluation */
    double omega;      /* primal weight */
    double wsum;       /* sum of the average's weights (step sizes) since the last restart */
    double phi0;       /* restart metric of the anchor z^{t,0} of the current restart period */
    double phi_prev;   /* restart metric of the previous check's candidate (INFINITY: none yet) */
    double comp0[3];   /* ||r_p||^2, ||r_d||^2 and |gap| of the anchor (rescaled program) */
    int64_t attempts;  /* PDHG evaluations so far (accepted or rejected) */
    int64_t accepted;  /* accepted steps so far */
    int64_t k;         /* accepted steps since the last restart (inner index of Algorithm 1) */
    int64_t restarts;  /* restarts so far */
    int32_t started;   /* 1 once the first anchor has been evaluated; 0: the next pdcs_solve
                          evaluates z^{0,0} first, as after pdcs_create */
    int32_t status;    /* 0 running, 1 converged, 2 NaN / Inf seen */
} pdcs_state;

/* The vectors of the iterate state, in the coordinates of the rescaled program
 * (x~ = x / dc, y~ = y / dr with the scalings of pdcs_get_scaling; rows in the original
 * order).  HOST pointers; any may be NULL. */
typedef struct {
    double *x, *xhat, *x0, *xsum;  /* n each: z^{t,k}, last PDHG output, anchor z^{t,0},
                                      sum of eta_i x^{t,i} (Algorithm 1 steps 6-7) */
    double *y, *yhat, *y0, *ysum;  /* m each: the same for y */
    double *kx, *kx0;              /* m each: cached products K~ x, K~ x0 */
    double *kty, *kty0;            /* n each: cached products K~' y, K~' y0 */
    float* soc_root;               /* one per SOC / RSOC cone (cone-list order): the last root
                                      of Theorem 1's search, the next search's starting point */
    float* exp_root;               /* one per exp cone: the same for Theorem 3's search */
} pdcs_state_arrays;

/* Checkpoint: copies the whole iterate state of Algorithm 1 into the non-NULL arrays of
 * *arr and the scalars into *st (may be NULL).  A pending Halpern update of the last
 * accepted evaluation is applied first (with the arithmetic the next evaluation would use,
 * so the iterates that follow are unchanged).  FP64 phase only: PDCS_ERR_INVALID while an
 * FP32-iterate phase runs. */
pdcs_status pdcs_get_state(pdcs_ctx* ctx, pdcs_state* st, const pdcs_state_arrays* arr);

/* Resume: replaces the iterate state by *st and the arrays of *arr: x, x0, y, y0 are
 * required; xsum / ysum NULL mean 0; xhat, yhat are ignored (the next evaluation forms
 * them); when one of kx, kx0, kty, kty0 is NULL the four cached products are recomputed
 * by the library's SpMV from x, x0, y, y0 (equal to the cached ones up to rounding);
 * soc_root / exp_root NULL leave the searches' starting points as they are (they change
 * results only in the last bits); with the products and both of them given, a state from
 * pdcs_get_state resumes the iteration bit for bit.  The tolerance is set by the next
 * pdcs_solve.  Afterwards the context runs the FP64 iteration, also in FP32 mode.
 * Errors: PDCS_ERR_INVALID (NULL or non-finite required data, status outside 0..2). */
pdcs_status pdcs_set_state(pdcs_ctx* ctx, const pdcs_state* st, const pdcs_state_arrays* arr);

/* Kernel timing for roofline measurements: runs `attempts` more PDHG evaluations
 * (and the checks that fall due) launch by launch, with CUDA events recorded on
 * the context's stream around every kernel, and writes the average duration in
 * milliseconds per launch of each kernel class to ms[0..11]:
 *   [0] primal update, [1] K xhat product, [2] dual update + cone projection,
 *   [3] K' yhat product, [4] one whole restart / termination check, and inside a
 *   check: [5] flush of the pending Halpern update, [6] primal candidates,
 *   [7] dual candidates (cone projections), [8] the four candidate products,
 *   [9] primal-side KKT, [10] dual-side KKT and the controller, [11] restart copy;
 * counts[0..11] (may be NULL) receive the number of launches timed per class.
 * The iterate state advances exactly as in pdcs_solve with tol <= 0. */
pdcs_status pdcs_kernel_times(pdcs_ctx* ctx, int64_t attempts, double* ms, int64_t* counts);

/* Text of the last error of ctx (or of the last failed pdcs_create when ctx is NULL). */
const char* pdcs_last_error(const pdcs_ctx* ctx);

/* Frees every device and host resource of ctx; NULL is a no-op. */
void pdcs_destroy(pdcs_ctx* ctx);

/* Blockwise projection of the DEVICE vector v (m rows) onto D C (dual == 0) or
 * onto (D C)* = D^{-1} C* (dual == 1), D = diag(d) (DEVICE pointer, d > 0; NULL
 * means D = I), written to the DEVICE vector out (may equal v).  The cone list
 * is a HOST array as in pdcs_create; for RSOC blocks d must be equal on their
 * first two rows.  SOC by Theorem 1, exp by Theorem 3, exp* (the dual side of an EXP
 * block, and the primal side of an EXP_DUAL block) by the Remark of App. A.2.  Accuracy: each block within 1e-12 of its exact projection, relative
 * to the block's norm (the root searches run in FP32 and are finished in FP64; an
 * exp point within 1e-14 of its norm from the cone or from the polar cone is
 * returned as itself or as 0).  Runs on cuda_stream and returns once the work is
 * queued.  Errors: PDCS_ERR_INVALID, PDCS_ERR_CUDA. */
pdcs_status pdcs_proj_cones_device(const double* v, const double* d, int64_t m, const pdcs_cone* cones,
                                   int64_t n_cones, int32_t dual, double* out, void* cuda_stream);

/* Projection plan: the cone layout of pdcs_proj_cones_device built once, for repeated
 * projections of vectors with the same cone list.  Each SOC / RSOC cone gets a strategy by
 * its dimension (Sec. 4): up to 4096 rows one warp; beyond, a team of blocks of one
 * cooperative launch (about one block per 32768 rows, at most one per SM), teams packed
 * into waves of at most one block per SM, every sum over a cone reduced across its team's
 * blocks in a fixed order (deterministic).  D = I takes the textbook closed form.
 * pdcs_proj_plan_create copies the HOST cone list (rows in order, sum of dims == m) and
 * allocates the plan's device memory (the lists, 8 bytes per row of FP32 scratch when some
 * SOC cone has more than 129 rows, the teams' barrier words and partials); it synchronises
 * cuda_stream once.  Errors: PDCS_ERR_INVALID (malformed list), PDCS_ERR_OOM, PDCS_ERR_CUDA. */
typedef struct pdcs_proj_plan pdcs_proj_plan;
pdcs_status pdcs_proj_plan_create(int64_t m, const pdcs_cone* cones, int64_t n_cones, void* cuda_stream,
                                  pdcs_proj_plan** out);

/* Enqueues the projection of the DEVICE vector v onto D C (dual == 0) or D^{-1} C*
 * (dual == 1), D = diag(d) (DEVICE pointer, NULL means D = I), into the DEVICE vector
 * out (may equal v): kernel launches on cuda_stream only (no allocation, no copy, no
 * synchronisation).  Same results and accuracy as pdcs_proj_cones_device.  Runs of one
 * plan that overlap on the GPU race on its scratch.  The teams' blocks wait for one
 * another with an iteration limit; a run whose wait gave up leaves out undefined and sets
 * a flag that pdcs_proj_plan_check reports.  Errors: PDCS_ERR_INVALID, PDCS_ERR_CUDA. */
pdcs_status pdcs_proj_plan_run(pdcs_proj_plan* plan, const double* v, const double* d, int32_t dual, double* out,
                               void* cuda_stream);

/* Synchronises cuda_stream and returns PDCS_ERR_DEVICE_TIMEOUT if a run of the plan gave up
 * a wait (the flag stays set), PDCS_OK otherwise. */
pdcs_status pdcs_proj_plan_check(pdcs_proj_plan* plan, void* cuda_stream);

/* Waits for the device and frees the plan; NULL is a no-op. */
void pdcs_proj_plan_destroy(pdcs_proj_plan* plan);

/* Largest cone list pdcs_proj_cones_device_noalloc accepts. */
#define PDCS_NOALLOC_MAX_CONES 262144

/* The same projection as pdcs_proj_cones_device, for callers that cannot allocate
 * device memory: code that runs inside a framework whose allocator owns the whole
 * device (a memory pool sized up front, where a foreign cudaMalloc would fail or
 * fragment the pool), or latency-critical loops that must not pay for an
 * allocation and its implicit synchronisation.  There is no counterpart in the
 * paper; this is a library convenience.
 *   - Scratch: the cone list and one 64-bit row offset per cone are kept in a
 *     file-scope device array of PDCS_NOALLOC_MAX_CONES entries (6 MiB), which every
 *     GPU that loads the library holds until the process exits.  The call performs
 *     no cudaMalloc, cudaFree or other allocating routine.
 *   - The first call on a device looks up that array's device address (once per
 *     device, with the device current); make this first call before any stream
 *     capture.
 *   - The array is shared by all calls and keeps the last call's contents; every
 *     entry a call reads is written by the same call first.  Calls that overlap on
 *     the GPU (different streams, no ordering between them) race on it.
 *   - EXP_DUAL blocks are not accepted (PDCS_ERR_INVALID); the other cone kinds are.
 *   - Arguments and layout as pdcs_proj_cones_device: v, d (may be NULL), out are
 *     DEVICE pointers, cones a HOST array that must stay unchanged until the queued
 *     work has run.  Returns PDCS_ERR_INVALID for a malformed cone list or
 *     n_cones > PDCS_NOALLOC_MAX_CONES, PDCS_ERR_CUDA if a CUDA call fails. */
pdcs_status pdcs_proj_cones_device_noalloc(const double* v, const double* d, int64_t m, const pdcs_cone* cones,
                                           int64_t n_cones, int32_t dual, double* out, void* cuda_stream);

/* ------------------------------------------------------------------------------------
 * Batches: many independent programs solved together, each with its own step size,
 * primal weight, restart state and termination (Algorithm 1 per program), iterated in
 * lockstep by launches whose third grid dimension is the program; one CUDA graph per
 * check period covers the whole batch.  Programs that have converged skip their work.
 * There is no counterpart in the paper (its experiments solve one program at a time).
 * ------------------------------------------------------------------------------------ */
typedef struct pdcs_batch pdcs_batch;

/* Forms a batch of `count` (1..65535) contexts made by pdcs_create with the same
 * options.batch_blocks > 0, FP64, the same check_period, no SpMV autotuning, and not yet
 * solved.  The contexts stay owned by the caller (destroy them after the batch) and give
 * each program's solution and info as usual.  Returns PDCS_ERR_INVALID (text in
 * pdcs_batch_last_error(NULL)) or PDCS_ERR_CUDA / PDCS_ERR_OOM. */
pdcs_status pdcs_batch_create(pdcs_ctx* const* ctxs, int64_t count, pdcs_batch** out);

/* Runs up to max_iter PDHG evaluations of every program (all in lockstep) or until all
 * have met tol.  *n_converged (may be NULL) receives how many have.  Returns PDCS_OK when
 * all converged, PDCS_MAX_ITER otherwise, PDCS_ERR_NUMERIC if a program's iterates hold a
 * NaN / Inf, PDCS_ERR_CUDA on a CUDA failure.  May be called again to continue. */
pdcs_status pdcs_batch_solve(pdcs_batch* b, double tol, int64_t max_iter, int64_t* n_converged);

const char* pdcs_batch_last_error(const pdcs_batch* b);
void pdcs_batch_destroy(pdcs_batch* b);

/* ------------------------------------------------------------------------------------
 * Learned starting point of the exponential-cone root search (case 4 of Theorem 3).
 * A 9 -> 32 -> 32 -> 1 ReLU network (FP32) maps the direction of v0, the log ratios
 * log(ds/dr), log(dt/dr) of the scales and the branch of the search (one-hot: both
 * r0, s0 > 0 searched from a4 or from a3, r0 <= 0, s0 <= 0) to the log-offset L of the
 * root from the branch's endpoint.  It replaces only the cold starting point of the
 * safeguarded Newton search; the bracket and the stopping tests are unchanged, so the
 * projection is the plain search's to its tolerance.  There is no counterpart in the
 * paper.  Parameter layout (PDCS_EXP_MLP_PARAMS floats): W1[32][9], b1[32], W2[32][32],
 * b2[32], w3[32], b3.  All arrays below are HOST arrays; each call allocates and frees
 * its own device memory and synchronises.
 * ------------------------------------------------------------------------------------ */
#define PDCS_EXP_MLP_IN 9
#define PDCS_EXP_MLP_HIDDEN 32
#define PDCS_EXP_MLP_PARAMS (32 * 9 + 32 + 32 * 32 + 32 + 32 + 1)

/* Training pairs from the plain projector: for each of n inputs v0 = v[3i..3i+2] with
 * scales d[3i..3i+2] (> 0) whose projection onto D K_exp falls in case 4 with a root
 * inside its interval and |L| <= 50, the FP64 search (no starting point) gives L; features[9k..9k+8]
 * and target[k] receive the k-th such pair, k < *kept.  Returns PDCS_ERR_INVALID for
 * n < 0 or NULL arrays, PDCS_ERR_CUDA on a CUDA failure. */
pdcs_status pdcs_exp_mlp_dataset(int64_t n, const double* v, const double* d, float* features, float* target,
                                 int64_t* kept);

/* Mean squared error of the network on n pairs and its gradient (same layout as the
 * weights), by the library's forward / backward kernels.  loss and grad are outputs. */
pdcs_status pdcs_exp_mlp_loss_grad(int64_t n, const float* features, const float* target, const float* weights,
                                   float* grad, float* loss);

/* Trains the network in place on the GPU: `steps` Adam steps (beta1 0.9, beta2 0.999,
 * eps 1e-8, learning rate lr) on minibatches of `batch` pairs drawn with replacement by
 * the SplitMix64 generator from `seed`; weights is read as the initial point and
 * overwritten; loss_trace (may be NULL) receives the minibatch loss of every step. */
pdcs_status pdcs_exp_mlp_train(int64_t n, const float* features, const float* target, int32_t steps, int32_t batch,
                               float lr, uint64_t seed, float* weights, float* loss_trace);

/* Projects n vectors onto D K_exp (inputs as in pdcs_exp_mlp_dataset) with the mixed-
 * precision search from a cold start, using the network when weights is not NULL;
 * out[3i..3i+2] is the projection, evals[2i] and evals[2i+1] the FP32 and FP64
 * evaluations of h it took (0 outside case 4). */
pdcs_status pdcs_exp_proj_stats(int64_t n, const double* v, const double* d, const float* weights, double* out,
                                int32_t* evals);

/* ------------------------------------------------------------------------------------
 * A small fully connected network for warm starts of parametric program families (a
 * summary of an instance's data -> initial dual iterate and log primal weight, given to
 * pdcs_set_warm_start).  n_layers weight layers, sizes[0..n_layers] the widths (input
 * first); ReLU after every layer but the last; loss: mean squared error over all outputs.
 * Parameters: for each layer l, W_l (sizes[l+1] x sizes[l], row-major) then b_l.  FP32
 * kernels with sums in a fixed order.  Host arrays; each call allocates its own device
 * memory and synchronises.  There is no counterpart in the paper.
 * ------------------------------------------------------------------------------------ */
#define PDCS_MLP_MAX_LAYERS 8
#define PDCS_MLP_MAX_WIDTH 4096

/* Number of parameters of the network, or -1 for invalid sizes. */
int64_t pdcs_mlp_params(int32_t n_layers, const int32_t* sizes);

/* Outputs Y (n x sizes[n_layers]) of the network with parameters W for the rows X. */
pdcs_status pdcs_mlp_forward(int32_t n_layers, const int32_t* sizes, int64_t n, const float* X, const float* W,
                             float* Y);

/* The same outputs with every layer's product on the tensor cores: the rows and weights are
 * rounded to BF16 as they are loaded and multiplied by mma.sync m16n8k16 tiles with FP32
 * accumulation; bias and ReLU in FP32.  Error against the FP32 forward: about 2^-8 relative
 * to sum |W| |x| per layer (BF16 operands). */
pdcs_status pdcs_mlp_forward_bf16(int32_t n_layers, const int32_t* sizes, int64_t n, const float* X,
                                  const float* W, float* Y);

/* Loss on the n rows (targets T, n x sizes[n_layers]) and its gradient (layout of W). */
pdcs_status pdcs_mlp_loss_grad(int32_t n_layers, const int32_t* sizes, int64_t n, const float* X, const float* T,
                               const float* W, float* grad, float* loss);

/* `steps` Adam steps (0.9, 0.999, 1e-8, learning rate lr) on minibatches of `batch` rows
 * drawn with replacement by SplitMix64 from `seed`; W is the initial point and is
 * overwritten; loss_trace (may be NULL) receives each minibatch loss. */
pdcs_status pdcs_mlp_train(int32_t n_layers, const int32_t* sizes, int64_t n, const float* X, const float* T,
                           int32_t steps, int32_t batch, float lr, uint64_t seed, float* W, float* loss_trace);

#ifdef __cplusplus
}
#endif
#endif

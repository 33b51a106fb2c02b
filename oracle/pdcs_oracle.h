/*
 * pdcs_oracle.h -- plain, slow FP64 CPU oracle for the restarted PDHG conic
 * solver of "A Practical GPU-Enhanced Matrix-Free Primal-Dual Method for
 * Large-Scale Conic Programs" (PDCS).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the reference that the CUDA library is
 * checked against.  It shares no code, header, helper or constant with the
 * CUDA path; only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it.  Everything is single-threaded plain loops in
 * double precision, written to be checked against the paper by eye.
 *
 * Problem (Sec. 2, eq. prob_cp with n2 = 0):
 *     min c'x   s.t.  K x - h in C,   l <= x <= u,
 * C a product of zero, nonnegative, second-order, rotated second-order and
 * exponential cones in row order.  Dual (eq. dual_conic): y in C*,
 * lambda = c - K'y in Lambda (eq. defn_Lambda1).
 * Optionally (orc_options.n_pc > 0) a contiguous range of variables forms
 * primal cone blocks x2 in K_p (eq. prob_cp with n2 > 0), K_p a product of
 * second-order and rotated second-order cones; their reduced costs then lie
 * in K_p* instead of Lambda.
 */
#ifndef PDCS_ORACLE_H
#define PDCS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_ZERO = 0, ORC_NONNEG = 1, ORC_SOC = 2, ORC_RSOC = 3, ORC_EXP = 4, ORC_EXP_DUAL = 5 };
enum { ORC_RESCALE_NONE = 0, ORC_RESCALE_COORD = 1, ORC_RESCALE_BLOCK = 2 };
enum { ORC_STEP_ADAPTIVE = 0, ORC_STEP_CONSTANT = 1, ORC_STEP_PLAIN = 2 };
enum { ORC_RUNNING = 0, ORC_CONVERGED = 1, ORC_MAX_ITER = 2 };

typedef struct {
    int rescale;        /* ORC_RESCALE_* */
    int ruiz_iters;     /* Ruiz equilibration passes (infinity norm) */
    int pock_chambolle; /* 1: one Pock-Chambolle pass (alpha = 1) after Ruiz */
    int step_mode;      /* ORC_STEP_* */
    int check_period;   /* restart / termination check every this many PDHG evaluations */
    double beta;        /* reflection parameter of the reflected Halpern step */
    int power_iters;    /* power iterations for ||K~||_2 (constant / plain step modes) */
    /* primal cone blocks: variables pc_start, pc_start + 1, ... grouped in order into n_pc
     * cones of types pc_types (ORC_SOC or ORC_RSOC) and sizes pc_dims; their bounds must be
     * (-inf, +inf).  The arrays are copied at create.  n_pc = 0: none. */
    const int32_t* pc_types;
    const int64_t* pc_dims;
    int64_t n_pc;
    int64_t pc_start;
} orc_options;

typedef struct {
    double err_p, err_d, err_gap;  /* relative errors, eq. PDCS_terminate_tolerance */
    double pobj, dobj;             /* primal and dual objective values (unscaled) */
} orc_kkt;

typedef struct orc_solver orc_solver;

void orc_default_options(orc_options* o);

/* ---- cone projections (Sec. 3 Thm 1, App. A Thm 3 and Remark) ---------- */
/* Projection of (t, x[0..n-1]) onto D K_soc^{n+1}; d[0..n] is the diagonal of D. */
void orc_proj_soc(double t, const double* x, const double* d, int64_t n, double* out_t, double* out_x);
/* Projection of (x, y, z[0..n-1]) onto D K_rsoc^{n+2}; requires d[0] == d[1]. */
void orc_proj_rsoc(const double* v, const double* d, int64_t dim, double* out);
/* Projection of v0 = (r0, s0, t0) onto D K_exp, D = diag(d[0], d[1], d[2]). */
void orc_proj_exp(const double* v0, const double* d, double* out);
/* Projection of v0 onto D K_exp^* by the Remark of App. A. */
void orc_proj_exp_dual(const double* v0, const double* d, double* out);
/* Projection of the whole vector v (m rows) onto D C (dual == 0) or D^{-1} C* (dual == 1). */
void orc_proj_cones(const double* v, const double* d, int64_t m, const int32_t* types,
                    const int64_t* dims, int64_t n_cones, int dual, double* out);

/* ---- unscaled KKT errors of (x, y) for the original problem ------------- */
int orc_kkt_eval(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                 const double* c, const double* h, const double* lb, const double* ub,
                 const int32_t* types, const int64_t* dims, int64_t n_cones,
                 const double* x, const double* y, orc_kkt* out);

/* The same with primal cone blocks (see orc_options; n_pc = 0: none). */
int orc_kkt_eval_pc(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                    const double* c, const double* h, const double* lb, const double* ub,
                    const int32_t* types, const int64_t* dims, int64_t n_cones,
                    const int32_t* pc_types, const int64_t* pc_dims, int64_t n_pc, int64_t pc_start,
                    const double* x, const double* y, orc_kkt* out);

/* ---- solver ------------------------------------------------------------- */
/* Copies every input.  lb / ub may be NULL (then l = 0, u = +inf).  Returns NULL on invalid input. */
orc_solver* orc_create(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                       const double* c, const double* h, const double* lb, const double* ub,
                       const int32_t* types, const int64_t* dims, int64_t n_cones, const orc_options* opt);
void orc_destroy(orc_solver* s);
/* Warm start in original coordinates (x: n, y: m, omega <= 0 keeps the default weight). */
void orc_set_start(orc_solver* s, const double* x, const double* y, double omega);
/* Runs PDHG evaluations until tol is met or `attempts` more evaluations are done.
 * tol <= 0 disables termination.  Returns ORC_* status. */
int orc_run(orc_solver* s, double tol, int64_t attempts);
/* Scaling factors: dr (m), dc (n). */
void orc_get_scaling(const orc_solver* s, double* dr, double* dc);
/* Current Halpern iterate z (x: n, y: m) and last PDHG output zhat, in ORIGINAL coordinates. */
void orc_get_iterate(const orc_solver* s, double* x, double* y, double* xhat, double* yhat);
/* Returned solution (projected candidate that met tol, or current projected iterate). */
void orc_get_solution(const orc_solver* s, double* x, double* y);
/* Scalars: [eta, omega, attempts, accepted, restarts, inner_k, status, last err_p, err_d, err_gap, wsum, phi_anchor] */
void orc_get_scalars(const orc_solver* s, double* out12);
/* Full iterate state in the solver's scaled coordinates (x~ = x / dc, y~ = y / dr):
 * the Halpern iterate, the last PDHG output, the anchor of the restart period and the
 * eta-weighted sums (x: n, y: m), and ORC_STATE_SCALARS scalars
 * [eta, omega, wsum, attempts, accepted, k, restarts, phi0, phi_prev, comp0[0..2],
 *  status, started].  NULL arrays are skipped.  orc_set_state restores exactly what
 * orc_get_state returned, so orc_run continues as if never interrupted. */
#define ORC_STATE_SCALARS 14
void orc_get_state(const orc_solver* s, double* x, double* xh, double* x0, double* xsum, double* y, double* yh,
                   double* y0, double* ysum, double* scalars);
void orc_set_state(orc_solver* s, const double* x, const double* xh, const double* x0, const double* xsum,
                   const double* y, const double* yh, const double* y0, const double* ysum, const double* scalars);
/* ||K~||_2 estimate used by the constant / plain step modes. */
double orc_norm2_estimate(const orc_solver* s);

#ifdef __cplusplus
}
#endif
#endif

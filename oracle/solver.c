/*
 * solver.c -- oracle restarted PDHG (PDCS, Algorithm 1) in plain FP64 loops.
 *
 * TEST INFRASTRUCTURE ONLY (see pdcs_oracle.h).
 *
 * Follows, in order:
 *   - the conic program and its dual, Sec. 2 (eqs. prob_cp, dual_conic, defn_Lambda1);
 *   - one PDHG evaluation, eq. PDHG, on the diagonally rescaled program (Sec. 3,
 *     "diagonal rescaling"): tau = eta / omega, sigma = eta * omega;
 *   - Algorithm 1: AdaptiveStepPDHG, ReflectedHalpern, the eta-weighted average,
 *     GetRestartCandidate, PrimalWeightUpdate and the termination test of
 *     eq. PDCS_terminate_tolerance.
 *
 * The paper defers the rules of AdaptiveStepPDHG, AdaptiveReflectionParameter,
 * GetRestartCandidate and PrimalWeightUpdate to a technical report that is not
 * part of it.  The readings used here (parity unpinned against the paper):
 *   step    : eta_max = (omega ||dx||^2 + ||dy||^2 / omega) / (2 |dy' K dx|);
 *             accept iff eta <= eta_max; next eta =
 *             min((1 - (j+1)^-0.3) eta_max, (1 + (j+1)^-0.6) eta), j = 1-based
 *             index of the PDHG evaluation; eta_0 = 1 / max_ij |K~_ij|.
 *   beta    : constant, default 1 (the reflected Halpern step of Sec. 3; the rule of
 *             AdaptiveReflectionParameter, Algorithm 1 step 5, is in the report).
 *   average : weights are the step sizes with which each accepted zhat was made.
 *   check   : every `check_period` PDHG evaluations (accepted or not).
 *   restart : candidates z^{t,k+1} and the average, each projected onto X x Y;
 *             phi = sqrt(omega ||r_p||^2 + ||r_d||^2 / omega + gap^2) on the
 *             scaled program; candidate = argmin phi; restart when
 *             phi_c <= 0.2 phi_0, or phi_c <= 0.8 phi_0 and phi_c > phi_prev,
 *             or k >= 0.36 * (accepted steps in total).
 *   weight  : omega_0 = ||c~|| / ||h~|| (1 if either <= 1e-10); at a restart
 *             log omega <- 0.5 log(||dy|| / ||dx||) + 0.5 log omega when both
 *             moves exceed 1e-10.
 *   scaling : Ruiz (infinity norm) then one Pock-Chambolle pass (alpha = 1);
 *             rows 1-2 of a rotated SOC share one factor; in block mode every
 *             SOC / RSOC / exp block shares one factor.
 *   dual obj: h'y + sum_j (l_j mu_j^+ - u_j mu_j^-) with mu = Proj_Lambda(lambda)
 *             and 0 * inf = 0.
 *   sums    : every sum over a whole vector is compensated (Neumaier), so it is the
 *             exact sum of its rounded terms to about one rounding; sums along a row
 *             of K (the matrix-vector products) are plain left-to-right sums.
 */
#include "pdcs_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_solver {
    int64_t m, n, nnz, n_cones;
    int64_t *rp, *rpT;
    int32_t *ci, *ciT;
    double *val, *valT;       /* scaled K~ and K~' (same patterns as K, K') */
    double *c0, *h0, *l0, *u0; /* original data */
    double *cs, *hs, *ls, *us; /* scaled data */
    int32_t* types;
    int64_t *dims, *offs;
    double *dr, *dc;
    orc_options opt;
    /* iterate state, scaled */
    double *x, *y, *xh, *yh, *x0, *y0, *xsum, *ysum, *solx, *soly;
    double *tm, *tn, *tm2, *tn2, *tm3, *tn3; /* work vectors */
    double wsum, eta, omega, norm2;
    int64_t attempts, accepted, k, restarts;
    double phi0, phi_prev, comp0[3];
    int status, started;
    double last_err[3];
    /* primal cone blocks x2 in K_p: types, sizes, first variable of each, a vector of ones */
    int64_t n_pc, pc_lo, pc_hi; /* the blocks cover variables [pc_lo, pc_hi) */
    int32_t* pct;
    int64_t *pcd, *pco;
    double* ones_n;
};

void orc_default_options(orc_options* o) {
    o->rescale = ORC_RESCALE_COORD;
    o->ruiz_iters = 10;
    o->pock_chambolle = 1;
    o->step_mode = ORC_STEP_ADAPTIVE;
    o->check_period = 64;
    o->beta = 1.0;
    o->power_iters = 50;
    o->pc_types = NULL;
    o->pc_dims = NULL;
    o->n_pc = 0;
    o->pc_start = 0;
}

/* Projection of the variables of the primal cone blocks onto K_p (dual == 0) or K_p^*
 * (dual == 1; the SOC and the rotated SOC are self-dual, so both are the same set).  Their
 * column scales are tied within each block, so Dc^{-1} K_p = K_p and D = I takes the
 * textbook projection.  Entries outside the blocks are left as they are. */
static void proj_pc(const struct orc_solver* S, const double* v, double* out) {
    for (int64_t k = 0; k < S->n_pc; ++k) {
        int64_t o = S->pco[k], d = S->pcd[k];
        if (S->pct[k] == ORC_SOC)
            orc_proj_soc(v[o], v + o + 1, S->ones_n, d - 1, out + o, out + o + 1);
        else
            orc_proj_rsoc(v + o, S->ones_n, d, out + o);
    }
}

static int in_pc(const struct orc_solver* S, int64_t j) { return j >= S->pc_lo && j < S->pc_hi; }

/* ---- small helpers ---------------------------------------------------- */
static double* dalloc(int64_t k) { return (double*)calloc((size_t)(k > 0 ? k : 1), sizeof(double)); }

static void spmv(int64_t rows, const int64_t* rp, const int32_t* ci, const double* v, const double* x, double* out) {
    for (int64_t i = 0; i < rows; ++i) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * x[ci[p]];
        out[i] = s;
    }
}

/* Sums over whole vectors (norms, inner products, the KKT and step-size quantities) are
 * accumulated with Neumaier's compensation (improved Kahan-Babuska summation): the
 * result is within about one rounding of the exact sum of the (rounded) terms, whatever
 * the length, where a plain left-to-right sum of 1e6 terms is off by ~1e-14. */
typedef struct { double s, c; } acc_t;
static void acc_add(acc_t* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static double acc_val(const acc_t* a) { return a->s + a->c; }

static double dot(int64_t k, const double* a, const double* b) {
    acc_t s = {0.0, 0.0};
    for (int64_t i = 0; i < k; ++i) acc_add(&s, a[i] * b[i]);
    return acc_val(&s);
}

/* Proj onto Lambda_j (eq. defn_Lambda1) */
static double proj_lambda(double lam, double l, double u) {
    int lf = isfinite(l), uf = isfinite(u);
    if (!lf && !uf) return 0.0;          /* {0} */
    if (!lf && uf) return lam < 0.0 ? lam : 0.0;  /* R^- */
    if (lf && !uf) return lam > 0.0 ? lam : 0.0;  /* R^+ */
    return lam;                           /* R */
}

static double bound_term(double l, double u, double mu) { /* l mu^+ - u mu^-, 0 * inf = 0 */
    double t = 0.0;
    if (mu > 0.0) t += l * mu;
    if (mu < 0.0) t += u * mu; /* -u * mu^- = u * mu */
    return t;
}

/* ---- KKT quantities --------------------------------------------------- */
typedef struct {
    double rp2, rd2, gap;        /* scaled residual norms^2 and |pobj - dobj| (phi) */
    double err_p, err_d, err_gap, pobj, dobj;
} cand_eval;

/* KKT of the (already projected) scaled pair (xt, yt).  Kx = K~ xt, KTy = K~' yt. */
static void eval_pair(const orc_solver* S, const double* xt, const double* yt, cand_eval* r) {
    int64_t m = S->m, n = S->n;
    double* Kx = dalloc(m);
    double* KTy = dalloc(n);
    double* v = dalloc(m);
    double* p = dalloc(m);
    double* ones = dalloc(m);
    spmv(m, S->rp, S->ci, S->val, xt, Kx);
    spmv(n, S->rpT, S->ciT, S->valT, yt, KTy);
    for (int64_t i = 0; i < m; ++i) ones[i] = 1.0;

    /* scaled primal residual: v - Proj_{Dr C}(v), v = K~x~ - h~ */
    for (int64_t i = 0; i < m; ++i) v[i] = Kx[i] - S->hs[i];
    orc_proj_cones(v, S->dr, m, S->types, S->dims, S->n_cones, 0, p);
    acc_t rp2a = {0.0, 0.0};
    for (int64_t i = 0; i < m; ++i) acc_add(&rp2a, (v[i] - p[i]) * (v[i] - p[i]));
    double rp2 = acc_val(&rp2a);

    /* unscaled primal residual: K x - h = (K~x~ - h~) / dr, projected onto C */
    for (int64_t i = 0; i < m; ++i) v[i] = v[i] / S->dr[i];
    orc_proj_cones(v, ones, m, S->types, S->dims, S->n_cones, 0, p);
    double rmax = 0.0, hmax = 0.0, kxmax = 0.0, pmax = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        rmax = fmax(rmax, fabs(v[i] - p[i]));
        hmax = fmax(hmax, fabs(S->h0[i]));
        kxmax = fmax(kxmax, fabs(Kx[i] / S->dr[i]));
        pmax = fmax(pmax, fabs(p[i]));
    }

    /* dual: lambda = c - K'y; scaled lambda~ = dc * lambda.  Box variables: mu = Proj_Lambda;
     * primal cone blocks: mu = Proj_{K_p^*}(lambda) per block, and no bound term (the infimum
     * of mu'x over x in K_p is 0 for mu in K_p^*). */
    double* lam_s = dalloc(n);
    double* mu_s = dalloc(n);
    double* lam_u = dalloc(n);
    double* mu_u = dalloc(n);
    for (int64_t j = 0; j < n; ++j) {
        lam_s[j] = S->cs[j] - KTy[j];
        lam_u[j] = lam_s[j] / S->dc[j];
        mu_s[j] = proj_lambda(lam_s[j], S->ls[j], S->us[j]);
        mu_u[j] = proj_lambda(lam_u[j], S->l0[j], S->u0[j]);
    }
    proj_pc(S, lam_s, mu_s);
    proj_pc(S, lam_u, mu_u);
    double dmax = 0.0, cmax = 0.0, ktymax = 0.0;
    acc_t rd2a = {0.0, 0.0}, bterma = {0.0, 0.0}, pobja = {0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
        double lam = lam_s[j];
        double mu = mu_s[j];
        acc_add(&rd2a, (lam - mu) * (lam - mu));
        if (!in_pc(S, j)) acc_add(&bterma, bound_term(S->ls[j], S->us[j], mu));
        double lamu = lam_u[j];
        double muu = mu_u[j];
        dmax = fmax(dmax, fabs(lamu - muu));
        cmax = fmax(cmax, fabs(S->c0[j]));
        ktymax = fmax(ktymax, fabs(KTy[j] / S->dc[j]));
        acc_add(&pobja, S->cs[j] * xt[j]);
    }
    double rd2 = acc_val(&rd2a), bterm = acc_val(&bterma), pobj = acc_val(&pobja);
    double dobj = dot(m, S->hs, yt) + bterm;
    double gap = fabs(pobj - dobj);
    r->rp2 = rp2;
    r->rd2 = rd2;
    r->gap = gap;
    r->pobj = pobj;
    r->dobj = dobj;
    r->err_p = rmax / (1.0 + fmax(hmax, fmax(kxmax, pmax)));
    r->err_d = dmax / (1.0 + fmax(cmax, ktymax));
    r->err_gap = gap / (1.0 + fmax(fabs(pobj), fabs(dobj)));
    free(Kx); free(KTy); free(v); free(p); free(ones);
    free(lam_s); free(mu_s); free(lam_u); free(mu_u);
}

static double phi_of(const double comp[3], double omega) {
    return sqrt(omega * comp[0] + comp[1] / omega + comp[2] * comp[2]);
}

/* ---- projections onto X = [l~, u~] and Y = Dr^{-1} C^* ------------------ */
static void proj_X(const orc_solver* S, const double* x, double* out) {
    for (int64_t j = 0; j < S->n; ++j) out[j] = fmin(fmax(x[j], S->ls[j]), S->us[j]);
    proj_pc(S, x, out);
}
static void proj_Y(const orc_solver* S, const double* y, double* out) {
    orc_proj_cones(y, S->dr, S->m, S->types, S->dims, S->n_cones, 1, out);
}

/* ---- setup -------------------------------------------------------------- */
static void tie_rows(const orc_solver* S, double* rn, int use_max) {
    /* groups of rows that must share one scale factor */
    (void)use_max;
    for (int64_t k = 0; k < S->n_cones; ++k) {
        int64_t o = S->offs[k], dim = S->dims[k];
        int64_t g = 0;
        if (S->opt.rescale == ORC_RESCALE_COORD && S->types[k] == ORC_RSOC) g = 2;
        if (S->opt.rescale == ORC_RESCALE_BLOCK &&
            (S->types[k] == ORC_SOC || S->types[k] == ORC_RSOC || S->types[k] == ORC_EXP ||
             S->types[k] == ORC_EXP_DUAL)) g = dim;
        if (g < 2) continue;
        double mx = 0.0;
        for (int64_t i = 0; i < g; ++i) mx = fmax(mx, rn[o + i]);
        for (int64_t i = 0; i < g; ++i) rn[o + i] = mx;
    }
}

static void apply_scale_values(orc_solver* S, const double* val0) {
    /* K~_ij = dr_i * K_ij * dc_j, multiplied in this order */
    for (int64_t i = 0; i < S->m; ++i)
        for (int64_t p = S->rp[i]; p < S->rp[i + 1]; ++p) S->val[p] = (S->dr[i] * val0[p]) * S->dc[S->ci[p]];
}

static void rescale(orc_solver* S, const double* val0) {
    int64_t m = S->m, n = S->n;
    for (int64_t i = 0; i < m; ++i) S->dr[i] = 1.0;
    for (int64_t j = 0; j < n; ++j) S->dc[j] = 1.0;
    apply_scale_values(S, val0);
    if (S->opt.rescale == ORC_RESCALE_NONE) return;
    double* rn = dalloc(m);
    double* cn = dalloc(n);
    int passes = S->opt.ruiz_iters + (S->opt.pock_chambolle ? 1 : 0);
    for (int it = 0; it < passes; ++it) {
        int pc = it >= S->opt.ruiz_iters; /* last pass: Pock-Chambolle, 1-norms */
        for (int64_t i = 0; i < m; ++i) rn[i] = 0.0;
        for (int64_t j = 0; j < n; ++j) cn[j] = 0.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = S->rp[i]; p < S->rp[i + 1]; ++p) {
                double a = fabs(S->val[p]);
                int64_t j = S->ci[p];
                if (pc) { rn[i] += a; cn[j] += a; }
                else { rn[i] = fmax(rn[i], a); cn[j] = fmax(cn[j], a); }
            }
        tie_rows(S, rn, 1);
        for (int64_t k = 0; k < S->n_pc; ++k) { /* one factor per primal cone block */
            double mx = 0.0;
            for (int64_t j = S->pco[k]; j < S->pco[k] + S->pcd[k]; ++j) mx = fmax(mx, cn[j]);
            for (int64_t j = S->pco[k]; j < S->pco[k] + S->pcd[k]; ++j) cn[j] = mx;
        }
        for (int64_t i = 0; i < m; ++i) if (rn[i] > 0.0) S->dr[i] = S->dr[i] / sqrt(rn[i]);
        for (int64_t j = 0; j < n; ++j) if (cn[j] > 0.0) S->dc[j] = S->dc[j] / sqrt(cn[j]);
        apply_scale_values(S, val0);
    }
    free(rn);
    free(cn);
}

static void build_transpose(orc_solver* S) {
    int64_t m = S->m, n = S->n;
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t p = 0; p < S->nnz; ++p) cnt[S->ci[p] + 1]++;
    for (int64_t j = 0; j < n; ++j) cnt[j + 1] += cnt[j];
    memcpy(S->rpT, cnt, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = S->rp[i]; p < S->rp[i + 1]; ++p) {
            int64_t q = cnt[S->ci[p]]++;
            S->ciT[q] = (int32_t)i;
        }
    free(cnt);
}

static void fill_transpose_values(orc_solver* S) {
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S->n + 1));
    memcpy(cnt, S->rpT, sizeof(int64_t) * (size_t)(S->n + 1));
    for (int64_t i = 0; i < S->m; ++i)
        for (int64_t p = S->rp[i]; p < S->rp[i + 1]; ++p) S->valT[cnt[S->ci[p]]++] = S->val[p];
    free(cnt);
}

static double power_norm2(orc_solver* S) {
    int64_t m = S->m, n = S->n;
    double* v = dalloc(n);
    double* w = dalloc(m);
    double* u = dalloc(n);
    for (int64_t j = 0; j < n; ++j) v[j] = 1.0 / sqrt((double)n);
    double est = 0.0;
    for (int it = 0; it < S->opt.power_iters; ++it) {
        spmv(m, S->rp, S->ci, S->val, v, w);
        spmv(n, S->rpT, S->ciT, S->valT, w, u);
        double nu = sqrt(dot(n, u, u));
        if (!(nu > 0.0)) break;
        est = sqrt(nu);
        for (int64_t j = 0; j < n; ++j) v[j] = u[j] / nu;
    }
    free(v); free(w); free(u);
    return est;
}

orc_solver* orc_create(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                       const double* c, const double* h, const double* lb, const double* ub,
                       const int32_t* types, const int64_t* dims, int64_t n_cones, const orc_options* opt) {
    if (m < 0 || n <= 0 || !row_ptr || row_ptr[0] != 0) return NULL;
    int64_t nnz = row_ptr[m];
    for (int64_t i = 0; i < m; ++i) if (row_ptr[i + 1] < row_ptr[i]) return NULL;
    for (int64_t p = 0; p < nnz; ++p) if (col[p] < 0 || col[p] >= n) return NULL;
    int64_t tot = 0;
    for (int64_t k = 0; k < n_cones; ++k) {
        if (dims[k] < 1) return NULL;
        if ((types[k] == ORC_EXP || types[k] == ORC_EXP_DUAL) && dims[k] != 3) return NULL;
        if (types[k] == ORC_RSOC && dims[k] < 2) return NULL;
        if (types[k] < ORC_ZERO || types[k] > ORC_EXP_DUAL) return NULL;
        tot += dims[k];
    }
    if (tot != m) return NULL;
    if (lb && ub) for (int64_t j = 0; j < n; ++j) if (lb[j] > ub[j]) return NULL;
    int64_t npc = opt ? opt->n_pc : 0, pcs = opt ? opt->pc_start : 0, pctot = 0;
    if (npc < 0) return NULL;
    if (npc > 0) {
        if (!opt->pc_types || !opt->pc_dims || pcs < 0) return NULL;
        for (int64_t k = 0; k < npc; ++k) {
            if (opt->pc_types[k] != ORC_SOC && opt->pc_types[k] != ORC_RSOC) return NULL;
            if (opt->pc_dims[k] < (opt->pc_types[k] == ORC_RSOC ? 2 : 1)) return NULL;
            pctot += opt->pc_dims[k];
        }
        if (pcs + pctot > n) return NULL;
        for (int64_t j = pcs; j < pcs + pctot; ++j) /* cone variables carry no bounds */
            if (!lb || !ub || lb[j] != -INFINITY || ub[j] != INFINITY) return NULL;
    }

    orc_solver* S = (orc_solver*)calloc(1, sizeof(orc_solver));
    S->m = m; S->n = n; S->nnz = nnz; S->n_cones = n_cones;
    if (opt) S->opt = *opt; else orc_default_options(&S->opt);
    if (S->opt.check_period < 1) S->opt.check_period = 64;
    S->rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
    memcpy(S->rp, row_ptr, sizeof(int64_t) * (size_t)(m + 1));
    S->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    memcpy(S->ci, col, sizeof(int32_t) * (size_t)nnz);
    S->val = dalloc(nnz);
    S->rpT = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    S->ciT = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    S->valT = dalloc(nnz);
    S->c0 = dalloc(n); S->h0 = dalloc(m); S->l0 = dalloc(n); S->u0 = dalloc(n);
    S->cs = dalloc(n); S->hs = dalloc(m); S->ls = dalloc(n); S->us = dalloc(n);
    memcpy(S->c0, c, sizeof(double) * (size_t)n);
    if (m) memcpy(S->h0, h, sizeof(double) * (size_t)m);
    for (int64_t j = 0; j < n; ++j) {
        S->l0[j] = lb ? lb[j] : 0.0;
        S->u0[j] = ub ? ub[j] : INFINITY;
    }
    S->types = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_cones > 0 ? n_cones : 1));
    S->dims = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_cones > 0 ? n_cones : 1));
    S->offs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_cones > 0 ? n_cones : 1));
    int64_t o = 0;
    for (int64_t k = 0; k < n_cones; ++k) {
        S->types[k] = types[k];
        S->dims[k] = dims[k];
        S->offs[k] = o;
        o += dims[k];
    }
    S->dr = dalloc(m);
    S->dc = dalloc(n);
    S->opt.pc_types = NULL; /* the caller's arrays are copied, not kept */
    S->opt.pc_dims = NULL;
    S->n_pc = npc;
    S->pc_lo = pcs;
    S->pc_hi = pcs + pctot;
    S->pct = (int32_t*)malloc(sizeof(int32_t) * (size_t)(npc > 0 ? npc : 1));
    S->pcd = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npc > 0 ? npc : 1));
    S->pco = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npc > 0 ? npc : 1));
    int64_t maxd = 1;
    for (int64_t k = 0, o2 = pcs; k < npc; ++k) {
        S->pct[k] = opt->pc_types[k];
        S->pcd[k] = opt->pc_dims[k];
        S->pco[k] = o2;
        o2 += opt->pc_dims[k];
        if (opt->pc_dims[k] > maxd) maxd = opt->pc_dims[k];
    }
    S->ones_n = dalloc(maxd);
    for (int64_t i = 0; i < maxd; ++i) S->ones_n[i] = 1.0;

    build_transpose(S);
    rescale(S, val);
    fill_transpose_values(S);
    for (int64_t j = 0; j < n; ++j) {
        S->cs[j] = S->dc[j] * S->c0[j];
        S->ls[j] = S->l0[j] / S->dc[j];
        S->us[j] = S->u0[j] / S->dc[j];
    }
    for (int64_t i = 0; i < m; ++i) S->hs[i] = S->dr[i] * S->h0[i];

    S->x = dalloc(n); S->xh = dalloc(n); S->x0 = dalloc(n); S->xsum = dalloc(n); S->solx = dalloc(n);
    S->y = dalloc(m); S->yh = dalloc(m); S->y0 = dalloc(m); S->ysum = dalloc(m); S->soly = dalloc(m);
    S->tm = dalloc(m); S->tm2 = dalloc(m); S->tm3 = dalloc(m);
    S->tn = dalloc(n); S->tn2 = dalloc(n); S->tn3 = dalloc(n);

    /* primal weight omega_0 */
    double nc = sqrt(dot(n, S->cs, S->cs)), nh = sqrt(dot(m, S->hs, S->hs));
    S->omega = (nc > 1e-10 && nh > 1e-10) ? nc / nh : 1.0;
    /* initial step */
    double amax = 0.0;
    for (int64_t p = 0; p < nnz; ++p) amax = fmax(amax, fabs(S->val[p]));
    S->eta = amax > 0.0 ? 1.0 / amax : 1.0;
    S->norm2 = 0.0;
    if (S->opt.step_mode != ORC_STEP_ADAPTIVE) {
        S->norm2 = power_norm2(S);
        double nn = S->norm2 > 0.0 ? S->norm2 : 1.0;
        S->eta = (S->opt.step_mode == ORC_STEP_PLAIN ? 0.9 : 0.998) / nn;
        if (S->opt.step_mode == ORC_STEP_PLAIN) S->omega = 1.0;
    }
    S->phi_prev = INFINITY;
    S->status = ORC_RUNNING;
    return S;
}

void orc_destroy(orc_solver* S) {
    if (!S) return;
    void* ps[] = {S->rp, S->rpT, S->ci, S->ciT, S->val, S->valT, S->c0, S->h0, S->l0, S->u0,
                  S->cs, S->hs, S->ls, S->us, S->types, S->dims, S->offs, S->dr, S->dc,
                  S->x, S->y, S->xh, S->yh, S->x0, S->y0, S->xsum, S->ysum, S->solx, S->soly,
                  S->tm, S->tn, S->tm2, S->tn2, S->tm3, S->tn3, S->pct, S->pcd, S->pco, S->ones_n};
    for (size_t i = 0; i < sizeof(ps) / sizeof(ps[0]); ++i) free(ps[i]);
    free(S);
}

/* Algorithm 1 "Require": z^{0,0} = zbar^{0,0} = (x, y); a new start also begins a
 * new restart period (empty average, k = 0, counters cleared). */
void orc_set_start(orc_solver* S, const double* x, const double* y, double omega) {
    for (int64_t j = 0; j < S->n; ++j) {
        S->x[j] = S->x0[j] = x ? x[j] / S->dc[j] : 0.0;
        S->xsum[j] = 0.0;
    }
    for (int64_t i = 0; i < S->m; ++i) {
        S->y[i] = S->y0[i] = y ? y[i] / S->dr[i] : 0.0;
        S->ysum[i] = 0.0;
    }
    if (omega > 0.0) S->omega = omega;
    S->wsum = 0.0;
    S->k = 0;
    S->attempts = 0;
    S->accepted = 0;
    S->restarts = 0;
    S->status = ORC_RUNNING;
    S->phi_prev = INFINITY;
    S->started = 0;
}

/* ---- one restart / termination check ------------------------------------ */
static void check(orc_solver* S, double tol) {
    int64_t m = S->m, n = S->n;
    cand_eval ev[2];
    double* cx[2] = {S->tn, S->tn2};
    double* cy[2] = {S->tm, S->tm2};
    int nc = 1;
    /* candidate 0: current Halpern iterate z^{t,k+1}; candidate 1: the average */
    proj_X(S, S->x, cx[0]);
    proj_Y(S, S->y, cy[0]);
    eval_pair(S, cx[0], cy[0], &ev[0]);
    if (S->opt.step_mode != ORC_STEP_PLAIN && S->wsum > 0.0) {
        for (int64_t j = 0; j < n; ++j) S->tn3[j] = S->xsum[j] / S->wsum;
        for (int64_t i = 0; i < m; ++i) S->tm3[i] = S->ysum[i] / S->wsum;
        proj_X(S, S->tn3, cx[1]);
        proj_Y(S, S->tm3, cy[1]);
        eval_pair(S, cx[1], cy[1], &ev[1]);
        nc = 2;
    }
    /* termination, eq. PDCS_terminate_tolerance */
    for (int q = 0; q < nc; ++q) {
        double e = fmax(ev[q].err_p, fmax(ev[q].err_d, ev[q].err_gap));
        if (q == 0 || e < fmax(S->last_err[0], fmax(S->last_err[1], S->last_err[2]))) {
            S->last_err[0] = ev[q].err_p; S->last_err[1] = ev[q].err_d; S->last_err[2] = ev[q].err_gap;
            memcpy(S->solx, cx[q], sizeof(double) * (size_t)n);
            memcpy(S->soly, cy[q], sizeof(double) * (size_t)m);
        }
    }
    for (int q = 0; q < nc; ++q) {
        if (tol > 0.0 && ev[q].err_p <= tol && ev[q].err_d <= tol && ev[q].err_gap <= tol) {
            S->last_err[0] = ev[q].err_p; S->last_err[1] = ev[q].err_d; S->last_err[2] = ev[q].err_gap;
            memcpy(S->solx, cx[q], sizeof(double) * (size_t)n);
            memcpy(S->soly, cy[q], sizeof(double) * (size_t)m);
            S->status = ORC_CONVERGED;
            return;
        }
    }
    if (S->opt.step_mode == ORC_STEP_PLAIN) return; /* no restarts in plain PDHG */
    /* GetRestartCandidate */
    double comp[2][3];
    double phi[2];
    for (int q = 0; q < nc; ++q) {
        comp[q][0] = ev[q].rp2; comp[q][1] = ev[q].rd2; comp[q][2] = ev[q].gap;
        phi[q] = phi_of(comp[q], S->omega);
    }
    int best = (nc == 2 && phi[1] < phi[0]) ? 1 : 0;
    double pc = phi[best];
    int restart = (pc <= 0.2 * S->phi0) || (pc <= 0.8 * S->phi0 && pc > S->phi_prev) ||
                  ((double)S->k >= 0.36 * (double)S->accepted);
    S->phi_prev = pc;
    if (!restart) return;
    /* PrimalWeightUpdate */
    double dx = 0.0, dy = 0.0;
    acc_t dxa = {0.0, 0.0}, dya = {0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) acc_add(&dxa, (cx[best][j] - S->x0[j]) * (cx[best][j] - S->x0[j]));
    for (int64_t i = 0; i < m; ++i) acc_add(&dya, (cy[best][i] - S->y0[i]) * (cy[best][i] - S->y0[i]));
    dx = acc_val(&dxa);
    dy = acc_val(&dya);
    dx = sqrt(dx);
    dy = sqrt(dy);
    if (dx > 1e-10 && dy > 1e-10) S->omega = exp(0.5 * log(dy / dx) + 0.5 * log(S->omega));
    /* z^{t+1,0} <- candidate */
    memcpy(S->x0, cx[best], sizeof(double) * (size_t)n);
    memcpy(S->x, cx[best], sizeof(double) * (size_t)n);
    memcpy(S->y0, cy[best], sizeof(double) * (size_t)m);
    memcpy(S->y, cy[best], sizeof(double) * (size_t)m);
    memset(S->xsum, 0, sizeof(double) * (size_t)n);
    memset(S->ysum, 0, sizeof(double) * (size_t)m);
    S->wsum = 0.0;
    S->k = 0;
    S->restarts++;
    memcpy(S->comp0, comp[best], sizeof(S->comp0));
    S->phi0 = phi_of(S->comp0, S->omega);
    S->phi_prev = INFINITY;
}

/* ---- one PDHG evaluation (eq. PDHG) and Algorithm 1 bookkeeping --------- */
static void attempt(orc_solver* S) {
    int64_t m = S->m, n = S->n;
    double tau = S->eta / S->omega, sigma = S->eta * S->omega;
    double* KTy = S->tn;
    double* dxv = S->tn2;
    double* Kv = S->tm;
    double* Kdx = S->tm2;
    /* xhat = Proj_X(x - tau (c - K'y)) */
    spmv(n, S->rpT, S->ciT, S->valT, S->y, KTy);
    for (int64_t j = 0; j < n; ++j) {
        double g = S->cs[j] - KTy[j];
        S->xh[j] = fmin(fmax(S->x[j] - tau * g, S->ls[j]), S->us[j]);
    }
    proj_pc(S, S->xh, S->xh); /* x2 blocks: Proj_{K_p} of the same gradient step */
    /* yhat = Proj_Y(y + sigma (h - K(2 xhat - x))) */
    for (int64_t j = 0; j < n; ++j) dxv[j] = 2.0 * S->xh[j] - S->x[j];
    spmv(m, S->rp, S->ci, S->val, dxv, Kv);
    for (int64_t i = 0; i < m; ++i) S->tm3[i] = S->y[i] + sigma * (S->hs[i] - Kv[i]);
    proj_Y(S, S->tm3, S->yh);
    S->attempts++;
    if (S->opt.step_mode != ORC_STEP_ADAPTIVE) {
        if (S->opt.step_mode == ORC_STEP_PLAIN) {
            memcpy(S->x, S->xh, sizeof(double) * (size_t)n);
            memcpy(S->y, S->yh, sizeof(double) * (size_t)m);
            S->accepted++;
            S->k++;
            return;
        }
    }
    double eta_used = S->eta;
    int accept = 1;
    if (S->opt.step_mode == ORC_STEP_ADAPTIVE) {
        /* AdaptiveStepPDHG */
        for (int64_t j = 0; j < n; ++j) dxv[j] = S->xh[j] - S->x[j];
        spmv(m, S->rp, S->ci, S->val, dxv, Kdx);
        double nx = dot(n, dxv, dxv);
        acc_t nya = {0.0, 0.0}, intera = {0.0, 0.0};
        for (int64_t i = 0; i < m; ++i) {
            double dy = S->yh[i] - S->y[i];
            acc_add(&nya, dy * dy);
            acc_add(&intera, dy * Kdx[i]);
        }
        double ny = acc_val(&nya), inter = acc_val(&intera);
        inter = fabs(inter);
        double move = S->omega * nx + ny / S->omega;
        double eta_max = inter > 0.0 ? move / (2.0 * inter) : INFINITY;
        double j1 = (double)S->attempts + 1.0; /* (j + 1), j = 1-based evaluation index */
        double t1 = (1.0 - pow(j1, -0.3)) * eta_max;
        double t2 = (1.0 + pow(j1, -0.6)) * S->eta;
        accept = S->eta <= eta_max;
        S->eta = fmin(t1, t2);
    }
    if (!accept) return;
    /* ReflectedHalpern and the eta-weighted average */
    double kk = (double)S->k;
    double a = (kk + 1.0) / (kk + 2.0), b = 1.0 / (kk + 2.0), be = S->opt.beta;
    for (int64_t j = 0; j < n; ++j) {
        S->x[j] = a * ((1.0 + be) * S->xh[j] - be * S->x[j]) + b * S->x0[j];
        S->xsum[j] += eta_used * S->x[j];
    }
    for (int64_t i = 0; i < m; ++i) {
        S->y[i] = a * ((1.0 + be) * S->yh[i] - be * S->y[i]) + b * S->y0[i];
        S->ysum[i] += eta_used * S->y[i];
    }
    S->wsum += eta_used;
    S->k++;
    S->accepted++;
}

int orc_run(orc_solver* S, double tol, int64_t attempts) {
    if (!S->started) {
        /* phi of the initial anchor z^{0,0} (projected) */
        cand_eval ev;
        proj_X(S, S->x0, S->tn);
        proj_Y(S, S->y0, S->tm);
        eval_pair(S, S->tn, S->tm, &ev);
        S->comp0[0] = ev.rp2; S->comp0[1] = ev.rd2; S->comp0[2] = ev.gap;
        S->phi0 = phi_of(S->comp0, S->omega);
        S->phi_prev = INFINITY;
        S->last_err[0] = ev.err_p; S->last_err[1] = ev.err_d; S->last_err[2] = ev.err_gap;
        memcpy(S->solx, S->tn, sizeof(double) * (size_t)S->n);
        memcpy(S->soly, S->tm, sizeof(double) * (size_t)S->m);
        S->started = 1;
    }
    for (int64_t a = 0; a < attempts && S->status == ORC_RUNNING; ++a) {
        attempt(S);
        if (S->attempts % S->opt.check_period == 0) check(S, tol);
    }
    if (S->status == ORC_RUNNING && tol > 0.0) return ORC_MAX_ITER;
    return S->status;
}

void orc_get_scaling(const orc_solver* S, double* dr, double* dc) {
    if (dr) memcpy(dr, S->dr, sizeof(double) * (size_t)S->m);
    if (dc) memcpy(dc, S->dc, sizeof(double) * (size_t)S->n);
}

void orc_get_iterate(const orc_solver* S, double* x, double* y, double* xhat, double* yhat) {
    for (int64_t j = 0; j < S->n; ++j) {
        if (x) x[j] = S->x[j] * S->dc[j];
        if (xhat) xhat[j] = S->xh[j] * S->dc[j];
    }
    for (int64_t i = 0; i < S->m; ++i) {
        if (y) y[i] = S->y[i] * S->dr[i];
        if (yhat) yhat[i] = S->yh[i] * S->dr[i];
    }
}

void orc_get_solution(const orc_solver* S, double* x, double* y) {
    for (int64_t j = 0; j < S->n; ++j) if (x) x[j] = S->solx[j] * S->dc[j];
    for (int64_t i = 0; i < S->m; ++i) if (y) y[i] = S->soly[i] * S->dr[i];
}

void orc_get_scalars(const orc_solver* S, double* o) {
    o[0] = S->eta; o[1] = S->omega; o[2] = (double)S->attempts; o[3] = (double)S->accepted;
    o[4] = (double)S->restarts; o[5] = (double)S->k; o[6] = (double)S->status;
    o[7] = S->last_err[0]; o[8] = S->last_err[1]; o[9] = S->last_err[2];
    o[10] = S->wsum; o[11] = S->phi0;
}

double orc_norm2_estimate(const orc_solver* S) { return S->norm2; }

/* ---- full iterate state (scaled coordinates), for resuming and for parity tests -- */
void orc_get_state(const orc_solver* S, double* x, double* xh, double* x0, double* xsum, double* y, double* yh,
                   double* y0, double* ysum, double* sc) {
    size_t nb = sizeof(double) * (size_t)S->n, mb = sizeof(double) * (size_t)S->m;
    if (x) memcpy(x, S->x, nb);
    if (xh) memcpy(xh, S->xh, nb);
    if (x0) memcpy(x0, S->x0, nb);
    if (xsum) memcpy(xsum, S->xsum, nb);
    if (y) memcpy(y, S->y, mb);
    if (yh) memcpy(yh, S->yh, mb);
    if (y0) memcpy(y0, S->y0, mb);
    if (ysum) memcpy(ysum, S->ysum, mb);
    if (sc) {
        sc[0] = S->eta; sc[1] = S->omega; sc[2] = S->wsum; sc[3] = (double)S->attempts;
        sc[4] = (double)S->accepted; sc[5] = (double)S->k; sc[6] = (double)S->restarts;
        sc[7] = S->phi0; sc[8] = S->phi_prev;
        sc[9] = S->comp0[0]; sc[10] = S->comp0[1]; sc[11] = S->comp0[2];
        sc[12] = (double)S->status; sc[13] = (double)S->started;
    }
}

void orc_set_state(orc_solver* S, const double* x, const double* xh, const double* x0, const double* xsum,
                   const double* y, const double* yh, const double* y0, const double* ysum, const double* sc) {
    size_t nb = sizeof(double) * (size_t)S->n, mb = sizeof(double) * (size_t)S->m;
    if (x) memcpy(S->x, x, nb);
    if (xh) memcpy(S->xh, xh, nb);
    if (x0) memcpy(S->x0, x0, nb);
    if (xsum) memcpy(S->xsum, xsum, nb);
    if (y) memcpy(S->y, y, mb);
    if (yh) memcpy(S->yh, yh, mb);
    if (y0) memcpy(S->y0, y0, mb);
    if (ysum) memcpy(S->ysum, ysum, mb);
    if (sc) {
        S->eta = sc[0]; S->omega = sc[1]; S->wsum = sc[2]; S->attempts = (int64_t)sc[3];
        S->accepted = (int64_t)sc[4]; S->k = (int64_t)sc[5]; S->restarts = (int64_t)sc[6];
        S->phi0 = sc[7]; S->phi_prev = sc[8];
        S->comp0[0] = sc[9]; S->comp0[1] = sc[10]; S->comp0[2] = sc[11];
        S->status = (int)sc[12]; S->started = (int)sc[13];
    }
}


/* ---- KKT of an arbitrary pair for the ORIGINAL program ------------------ */
int orc_kkt_eval(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                 const double* c, const double* h, const double* lb, const double* ub,
                 const int32_t* types, const int64_t* dims, int64_t n_cones,
                 const double* x, const double* y, orc_kkt* out) {
    return orc_kkt_eval_pc(m, n, row_ptr, col, val, c, h, lb, ub, types, dims, n_cones, NULL, NULL, 0, 0,
                           x, y, out);
}

int orc_kkt_eval_pc(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                    const double* c, const double* h, const double* lb, const double* ub,
                    const int32_t* types, const int64_t* dims, int64_t n_cones,
                    const int32_t* pc_types, const int64_t* pc_dims, int64_t n_pc, int64_t pc_start,
                    const double* x, const double* y, orc_kkt* out) {
    orc_options o;
    orc_default_options(&o);
    o.rescale = ORC_RESCALE_NONE;
    o.pc_types = pc_types;
    o.pc_dims = pc_dims;
    o.n_pc = n_pc;
    o.pc_start = pc_start;
    orc_solver* S = orc_create(m, n, row_ptr, col, val, c, h, lb, ub, types, dims, n_cones, &o);
    if (!S) return 1;
    cand_eval ev;
    eval_pair(S, x, y, &ev);
    out->err_p = ev.err_p; out->err_d = ev.err_d; out->err_gap = ev.err_gap;
    out->pobj = ev.pobj; out->dobj = ev.dobj;
    orc_destroy(S);
    return 0;
}

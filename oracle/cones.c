/*
 * cones.c -- oracle projections onto (diagonally rescaled) disciplined cones.
 *
 * TEST INFRASTRUCTURE ONLY (see pdcs_oracle.h).  Plain FP64 loops.
 *
 *  - orc_proj_soc      : Theorem 1 (Sec. 3, eq. bisection-soc; proof App. A.1),
 *                        the four cases in the printed order, case 4 by bisection;
 *                        the first entry of the case-4 result is taken from the
 *                        active constraint ||Dhat^{-1} y|| = s (eq. kkt_sys_fixed_2).
 *  - orc_proj_rsoc     : rotated SOC as an orthogonal transform of the SOC
 *                        (Sec. 2 notes the equivalence; App. B.2 uses the map
 *                        ((w+r)/sqrt2, (w-r)/sqrt2)).
 *  - orc_proj_exp      : Theorem 3 (App. A.2, eqs. h_rho, sp_rd, lrho_urho,
 *                        vpvd_defn), cases 1-3 in closed form, case 4 by
 *                        bisection of h on the interval (l_rho, u_rho).
 *  - orc_proj_exp_dual : Remark after Theorem 3 (dual cone via Moreau).
 *
 * Readings where the paper is silent on floating point:
 *  - membership tests of K_exp / K_exp^* are done in log form
 *    (log t - log s >= r/s, and 1 + log t - log(-r) >= s/r) so they never overflow;
 *  - case 4 of Theorem 3 searches over the logarithm L of the offset of rho from
 *    an endpoint of (l_rho, u_rho): rho = a3 - e^L (interval (-inf, a3)),
 *    rho = a4 + e^L (interval (a4, inf)), and for the finite interval each half
 *    from its own endpoint.  The vanishing factor of s~ = r0 (rho - a4) or
 *    r~ = s0 (a3 - rho) (App. A.2, eq. tilde_defs) enters as log r0 + L or
 *    log s0 + L, the sign of h is decided in log form, and the lower end of the
 *    search grows until h shows its endpoint sign, so roots within 1e-16 |rho| of
 *    an endpoint, offsets below the smallest double and rho > 709 are handled;
 *  - the result takes, per coordinate, the smaller of v_p and v_d from its formula
 *    (eq. vpvd_defn) and the other from v0 = v_p + v_d (eq. diagonal_moreau);
 *  - a3 - a4 and d~ = rho (rho - 1) + tau^2 (App. A.2) are evaluated through exact
 *    identities of their definitions, a3 - a4 = N / (r0 s0), d~(a3) = tau N / s0^2,
 *    d~(a4) = tau N / r0^2 with N = tau (r0^2 + s0^2) - r0 s0 formed by error-free
 *    products and sums, and d~(a + dd) = d~(a) + dd (2 a - 1 + dd) at offset dd from
 *    the anchor a, so that no subtraction cancels where the interval is narrow;
 *  - every bisection runs until the midpoint equals an endpoint (FP64 limit).
 * Accuracy: the bisection settles the root to the last bit of L, so the error of a
 * result is that of evaluating h and v_p / v_d in FP64: within 1e-13 of a high-
 * precision solution (relative to |v0|) on 10,000 case-4 inputs chosen for the
 * cancellation in N (tests/test_oracle_pins.py); the plain differences a3 - a4 and
 * rho (rho - 1) + tau^2 left up to 7.9e-12 there.  Where |rho| is large, e^rho in
 * v_p / v_d amplifies the last-bit quantisation of L: ~1e-13 at |rho| ~ 1e4.
 */
#include "pdcs_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Second-order cone, Theorem 1.                                             */
/* ------------------------------------------------------------------------ */

/* f(lambda) of eq. (bisection-soc) / (kkt_sys_fixed_3):
 *   sum_i ( dhat_i^{-1} x_i / (1 + 2 lambda dhat_i^{-2}) )^2 - t^2 / (1 - 2 lambda)^2 */
static double soc_f(double lam, double t, const double* x, const double* dhat, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double di = dhat[i];
        double q = (x[i] / di) / (1.0 + 2.0 * lam / (di * di));
        s += q * q;
    }
    double w = 1.0 - 2.0 * lam;
    return s - (t * t) / (w * w);
}

void orc_proj_soc(double t, const double* x, const double* d, int64_t n, double* out_t, double* out_x) {
    double* dhat = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) dhat[i] = d[i + 1] / d[0]; /* dhat_i = d_{i+1} / d_1 */
    double nDx = 0.0, nDinvx = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double a = dhat[i] * x[i], b = x[i] / dhat[i];
        nDx += a * a;
        nDinvx += b * b;
    }
    nDx = sqrt(nDx);
    nDinvx = sqrt(nDinvx);

    if (t <= 0.0 && nDx <= -t) { /* case 1: -(t,x) in the polar cone */
        *out_t = 0.0;
        for (int64_t i = 0; i < n; ++i) out_x[i] = 0.0;
    } else if (nDinvx <= t) { /* case 2: already in the cone */
        *out_t = t;
        for (int64_t i = 0; i < n; ++i) out_x[i] = x[i];
    } else if (t == 0.0) { /* case 3: lambda = 1/2 in closed form */
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double di = dhat[i];
            double q = x[i] / (di + 1.0 / di);
            s += q * q;
            out_x[i] = x[i] / (1.0 + 1.0 / (di * di));
        }
        *out_t = sqrt(s);
    } else { /* case 4: root of f on (0, 1/2) for t > 0, on (1/2, inf) for t < 0 */
        double lo, hi;
        int sign_lo;
        if (t > 0.0) {
            lo = 0.0;
            hi = 0.5;
            sign_lo = 1; /* f(0+) > 0 since ||Dhat^{-1} x|| > t */
        } else {
            lo = 0.5;
            hi = 1.0;
            sign_lo = -1; /* f(1/2+) = -inf */
            while (soc_f(hi, t, x, dhat, n) <= 0.0) hi *= 2.0; /* lambda^2 f -> (||Dhat x||^2 - t^2)/4 > 0 */
        }
        for (int it = 0; it < 5000; ++it) {
            double mid = 0.5 * (lo + hi);
            if (!(mid > lo && mid < hi)) break;
            double fm = soc_f(mid, t, x, dhat, n);
            int sm = (fm > 0.0) - (fm < 0.0);
            if (sm == 0) { lo = hi = mid; break; }
            if (sm == sign_lo) lo = mid; else hi = mid;
        }
        double lam = 0.5 * (lo + hi);
        /* y = (I + 2 lambda Dhat^{-2})^{-1} x; s from the active cone constraint
         * ||Dhat^{-1} y|| = s of eq. kkt_sys_fixed_2, which equals t / (1 - 2 lambda)
         * at the root but does not cancel when lambda is close to 1/2. */
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            out_x[i] = x[i] / (1.0 + 2.0 * lam / (dhat[i] * dhat[i]));
            double q = out_x[i] / dhat[i];
            s += q * q;
        }
        *out_t = sqrt(s);
    }
    free(dhat);
}

/* Rotated SOC {(x, y, z): ||z||^2 <= 2 x y, x, y >= 0} = Q K_soc with
 * Q = [[1, 1], [1, -1]] / sqrt2 (+) I, orthogonal and symmetric.  With equal
 * scales on the first two coordinates D Q = Q D, so
 * Proj_{D K_rsoc}(v) = Q Proj_{D K_soc}(Q v). */
void orc_proj_rsoc(const double* v, const double* d, int64_t dim, double* out) {
    double* w = (double*)malloc(sizeof(double) * (size_t)dim);
    double* p = (double*)malloc(sizeof(double) * (size_t)dim);
    w[0] = (v[0] + v[1]) * M_SQRT1_2;
    w[1] = (v[0] - v[1]) * M_SQRT1_2;
    for (int64_t i = 2; i < dim; ++i) w[i] = v[i];
    orc_proj_soc(w[0], w + 1, d, dim - 1, &p[0], p + 1);
    out[0] = (p[0] + p[1]) * M_SQRT1_2;
    out[1] = (p[0] - p[1]) * M_SQRT1_2;
    for (int64_t i = 2; i < dim; ++i) out[i] = p[i];
    free(w);
    free(p);
}

/* ------------------------------------------------------------------------ */
/* Exponential cone, Theorem 3 and the Remark (App. A.2).                     */
/* ------------------------------------------------------------------------ */

/* (r, s, t) in K_exp (eq. exp_cone), tested in log form. */
static int in_kexp(double r, double s, double t) {
    if (s > 0.0) return t > 0.0 && (log(t) - log(s)) >= r / s;
    if (s == 0.0) return t >= 0.0 && r <= 0.0;
    return 0;
}

/* (r, s, t) in K_exp^* (eq. exp_cone_dual), tested in log form. */
static int in_kexp_dual(double r, double s, double t) {
    if (r < 0.0) return t > 0.0 && (1.0 + log(t) - log(-r)) >= s / r;
    if (r == 0.0) return s >= 0.0 && t >= 0.0;
    return 0;
}

static double lse(double a, double b) { /* log(e^a + e^b) */
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double mx = a > b ? a : b, mn = a > b ? b : a;
    return mx + log1p(exp(mn - mx));
}

typedef struct {
    double r0, s0, t0, dr, ds, dt, tau, a3, a4, ldt;
    double a4m1; /* a4 - 1 = -(s0 d_s) / (r0 d_r), exact near a4 = 1 */
    int anchor;  /* 3: rho measured from a3, 4: from a4 */
    double dir;  /* rho = anchor + dir * delta, delta = e^L */
    double w34;  /* a3 - a4 */
    double dt3, dt4; /* d~ = rho (rho - 1) + tau^2 at rho = a3 and at rho = a4 */
    int kind;    /* 1: r0 > 0, s0 > 0;  2: r0 <= 0, s0 > 0;  3: r0 > 0, s0 <= 0 */
} exp_ctx;

/* Error-free transformations (Dekker 1971; Knuth, TAOCP vol. 2): a * b = p + e and
 * a + b = s + e exactly in binary floating point. */
static double two_prod(double a, double b, double* e) {
    double p = a * b;
    *e = fma(a, b, -p);
    return p;
}
static double two_sum(double a, double b, double* e) {
    double s = a + b, bb = s - a;
    *e = (a - (s - bb)) + (b - bb);
    return s;
}

/* Theorem 3's endpoint quantities through exact identities of its definitions
 * (a3 = r0 d_s / (s0 d_r), a4 = 1 - s0 d_s / (r0 d_r), d~(rho) = rho (rho - 1) + tau^2,
 * tau = d_s / d_r).  With N = tau (r0^2 + s0^2) - r0 s0:
 *     a3 - a4 = N / (r0 s0),   d~(a3) = tau N / s0^2,   d~(a4) = tau N / r0^2.
 * When both r0, s0 > 0 the difference in N cancels (the interval (l_rho, u_rho) is then
 * narrow, or d~ is small on it); N is formed from error-free products and sums of r0, s0
 * scaled by one power of two (exact), so it is right to its last bits, where the plain
 * differences a3 - a4 and rho (rho - 1) + tau^2 lose the digits that cancel. */
static void exp_endpoint_terms(exp_ctx* e) {
    double r0 = e->r0, s0 = e->s0, tau = e->tau;
    double mx = fabs(r0) > fabs(s0) ? fabs(r0) : fabs(s0);
    int k = 0;
    frexp(mx, &k);
    double r = ldexp(r0, -k), s = ldexp(s0, -k);
    double e1, e2, eS, eq, e3, eD;
    double p1 = two_prod(r, r, &e1), p2 = two_prod(s, s, &e2);
    double S = two_sum(p1, p2, &eS);
    double q = two_prod(tau, S, &eq);
    double p3 = two_prod(r, s, &e3);
    double D = two_sum(q, -p3, &eD);
    double N = D + (eD + eq + tau * (eS + e1 + e2) - e3); /* N / 2^(2k) */
    e->w34 = (r0 > 0.0 && s0 > 0.0) ? N / (r * s) : e->a3 - e->a4;
    e->dt3 = s0 > 0.0 ? tau * N / (s * s) : 0.0;
    e->dt4 = r0 > 0.0 ? tau * N / (r * r) : 0.0;
}

/* rho and the logarithms of s_p, r_d (eq. sp_rd) at log-offset L from the anchor,
 * using s_p = s~ / (d_r d~), r_d = d_s r~ / d~ (App. A.2, eq. tilde_defs).  The
 * quantity that vanishes at the anchor enters as a logarithm (log r0 + L for
 * s~ = r0 (rho - a4) near a4, log s0 + L for r~ = s0 (a3 - rho) near a3), so an
 * offset below the smallest double still carries its value.  A non-positive
 * s_p or r_d (possible only by rounding at the interval ends) gives -inf. */
static void exp_eval(const exp_ctx* e, double L, double* rho, double* lsp, double* lrd) {
    double delta = exp(L);
    double rh, lst, lrt;
    int sst, srt; /* signs of s~ and r~ */
    if (e->anchor == 4) {
        rh = e->a4 + e->dir * delta;
        lst = log(e->r0) + L;
        sst = e->dir > 0.0 ? 1 : -1;
        double rt = (e->kind == 1) ? e->s0 * (e->w34 - e->dir * delta) : e->tau * e->r0 - rh * e->s0;
        lrt = log(fabs(rt));
        srt = (rt > 0.0) - (rt < 0.0);
    } else {
        rh = e->a3 + e->dir * delta;
        lrt = log(e->s0) + L;
        srt = e->dir < 0.0 ? 1 : -1;
        double st = (e->kind == 1) ? e->r0 * (e->w34 + e->dir * delta) : e->s0 * e->tau - e->r0 + e->r0 * rh;
        lst = log(fabs(st));
        sst = (st > 0.0) - (st < 0.0);
    }
    /* d~ = rho (rho - 1) + tau^2 at rho = a + dd: d~(a) + dd (2 a - 1 + dd) */
    double dd = e->dir * delta;
    double dt_ = e->anchor == 4 ? e->dt4 + dd * ((2.0 * e->a4m1 + 1.0) + dd)
                                : e->dt3 + dd * ((2.0 * e->a3 - 1.0) + dd);
    int sdt = (dt_ > 0.0) - (dt_ < 0.0);
    double ldt_ = log(fabs(dt_));
    *rho = rh;
    *lsp = (sst != 0 && sst == sdt) ? lst - log(e->dr) - ldt_ : -INFINITY;
    *lrd = (srt != 0 && srt == sdt) ? log(e->ds) + lrt - ldt_ : -INFINITY;
}

/* sign of h(rho) = d_t e^rho s_p - d_t^{-1} e^{-rho} r_d - t0 (eq. h_rho), decided in logs. */
static int exp_hsign(const exp_ctx* e, double L) {
    double rho, lsp, lrd;
    exp_eval(e, L, &rho, &lsp, &lrd);
    double A = e->ldt + rho + lsp;  /* log of d_t e^rho s_p */
    double B = -e->ldt - rho + lrd; /* log of d_t^{-1} e^-rho r_d */
    double lhs, rhs;
    if (e->t0 >= 0.0) {
        lhs = A;
        rhs = e->t0 > 0.0 ? lse(B, log(e->t0)) : B;
    } else {
        lhs = lse(A, log(-e->t0));
        rhs = B;
    }
    return (lhs > rhs) - (lhs < rhs);
}

/* bisection over L in (lo, hi) with sign(h) at the lo end equal to sign_lo */
static double exp_bisect(const exp_ctx* e, double lo, double hi, int sign_lo) {
    for (int it = 0; it < 5000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        int s = exp_hsign(e, mid);
        if (s == 0) return mid;
        if (s == sign_lo) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* lower end of the search: h keeps the sign it has at the anchor for small enough
 * offsets; step down from hi by 1, 2, 4, ... until that sign shows. */
static double exp_lower(const exp_ctx* e, double hi, int sign_lo) {
    double step = 1.0;
    for (int it = 0; it < 1100; ++it) {
        double lo = hi - step;
        if (exp_hsign(e, lo) == sign_lo || lo == -INFINITY) return lo;
        step *= 2.0;
    }
    return -INFINITY;
}

void orc_proj_exp(const double* v0, const double* d, double* out) {
    double r0 = v0[0], s0 = v0[1], t0 = v0[2];
    double dr = d[0], ds = d[1], dt = d[2];
    /* case 1: v0 in D K_exp */
    if (in_kexp(r0 / dr, s0 / ds, t0 / dt)) { out[0] = r0; out[1] = s0; out[2] = t0; return; }
    /* case 2: v0 in -D^{-1} K_exp^*, i.e. -D v0 in K_exp^* */
    if (in_kexp_dual(-dr * r0, -ds * s0, -dt * t0)) { out[0] = 0.0; out[1] = 0.0; out[2] = 0.0; return; }
    /* case 3: r0 <= 0 and s0 <= 0 */
    if (r0 <= 0.0 && s0 <= 0.0) { out[0] = r0; out[1] = 0.0; out[2] = t0 > 0.0 ? t0 : 0.0; return; }
    /* case 4: root of h on (l_rho, u_rho), eq. lrho_urho */
    exp_ctx e;
    e.r0 = r0; e.s0 = s0; e.t0 = t0; e.dr = dr; e.ds = ds; e.dt = dt;
    e.tau = ds / dr;
    e.ldt = log(dt);
    e.a3 = (s0 > 0.0) ? (r0 * ds) / (s0 * dr) : 0.0;
    e.a4 = (r0 > 0.0) ? 1.0 - (s0 * ds) / (r0 * dr) : 0.0;
    e.a4m1 = (r0 > 0.0) ? -(s0 * ds) / (r0 * dr) : -1.0;
    exp_endpoint_terms(&e);
    double L;
    if (r0 > 0.0 && s0 > 0.0) {
        e.kind = 1;
        double W = fabs(e.w34);
        if (!(W > 0.0)) { out[0] = 0.0; out[1] = 0.0; out[2] = 0.0; return; }
        double Lh = log(0.5 * W);
        /* sign at the midpoint, measured from a4 */
        e.anchor = 4;
        e.dir = e.w34 > 0.0 ? 1.0 : -1.0;
        int sm = exp_hsign(&e, Lh);
        if (sm == 0) {
            L = Lh;
        } else if (sm > 0) { /* h(a4) < 0 < h(mid): root in the half next to a4 */
            L = exp_bisect(&e, exp_lower(&e, Lh, -1), Lh, -1);
        } else {             /* h(mid) < 0 < h(a3): root in the half next to a3 */
            e.anchor = 3;
            e.dir = -e.dir;
            L = exp_bisect(&e, exp_lower(&e, Lh, +1), Lh, +1);
        }
    } else if (s0 > 0.0) { /* r0 <= 0: interval (-inf, a3), rho = a3 - delta */
        e.kind = 2;
        e.anchor = 3;
        e.dir = -1.0;
        double hi = 0.0;
        while (exp_hsign(&e, hi) > 0 && hi < 60.0) hi = 2.0 * hi + 1.0; /* h -> -inf as rho -> -inf */
        L = exp_bisect(&e, exp_lower(&e, hi, +1), hi, +1);
    } else { /* r0 > 0, s0 <= 0: interval (a4, inf), rho = a4 + delta */
        e.kind = 3;
        e.anchor = 4;
        e.dir = 1.0;
        double hi = 0.0;
        while (exp_hsign(&e, hi) < 0 && hi < 60.0) hi = 2.0 * hi + 1.0; /* h -> +inf as rho -> +inf */
        L = exp_bisect(&e, exp_lower(&e, hi, -1), hi, -1);
    }
    double rho, lsp, lrd;
    exp_eval(&e, L, &rho, &lsp, &lrd);
    /* eq. vpvd_defn: v_p = (d_r rho, d_s, d_t e^rho) s_p and
     * v_d = (d_r^{-1}, (1 - rho) d_s^{-1}, -d_t^{-1} e^-rho) r_d, with v_p + v_d = v0
     * (eq. diagonal_moreau).  Per coordinate the part of smaller magnitude is taken
     * from its formula and v_p from v0 - v_d when v_d is the larger part, so both
     * parts keep an absolute error of a few ulps of |v0|. */
    double sp = exp(lsp), rd = exp(lrd);
    double vp[3] = {dr * rho * sp, ds * sp, exp(e.ldt + rho + lsp)};
    double vd[3] = {rd / dr, (1.0 - rho) * rd / ds, -exp(-e.ldt - rho + lrd)};
    for (int k = 0; k < 2; ++k) out[k] = fabs(vp[k]) <= fabs(vd[k]) ? vp[k] : v0[k] - vd[k];
    /* t entry: h(rho) = 0 says e^A - e^B = t0, so the part of smaller magnitude is
     * v_d (t0 >= 0) or v_p (t0 < 0) whatever the rounding of A and B */
    out[2] = t0 >= 0.0 ? t0 - vd[2] : vp[2];
}

/* Remark (App. A.2): Proj_{D K_exp^*}(v0) = v0 + Proj_{D^{-1} K_exp}(-v0). */
void orc_proj_exp_dual(const double* v0, const double* d, double* out) {
    double nv[3] = {-v0[0], -v0[1], -v0[2]};
    double di[3] = {1.0 / d[0], 1.0 / d[1], 1.0 / d[2]};
    double p[3];
    orc_proj_exp(nv, di, p);
    for (int i = 0; i < 3; ++i) out[i] = v0[i] + p[i];
}

/* Blockwise projection, eq. multi_cone_proj.  dual == 0: onto D C.
 * dual == 1: onto (D C)^* = D^{-1} C^*, where zero^* = R, nonneg, SOC and RSOC
 * are self-dual and exp^* is handled by the Remark.  An EXP_DUAL block is K_exp^*
 * itself (the dual-cone row blocks of the problem of Sec. 2): D K_exp^* by the Remark,
 * its dual D^{-1} K_exp directly. */
void orc_proj_cones(const double* v, const double* d, int64_t m, const int32_t* types,
                    const int64_t* dims, int64_t n_cones, int dual, double* out) {
    (void)m;
    int64_t o = 0;
    for (int64_t k = 0; k < n_cones; ++k) {
        int64_t dim = dims[k];
        const double* vv = v + o;
        const double* dd = d + o;
        double* oo = out + o;
        double* dinv = NULL;
        if ((dual && (types[k] == ORC_SOC || types[k] == ORC_RSOC)) || types[k] == ORC_EXP_DUAL) {
            dinv = (double*)malloc(sizeof(double) * (size_t)dim);
            for (int64_t i = 0; i < dim; ++i) dinv[i] = 1.0 / dd[i];
        }
        switch (types[k]) {
            case ORC_ZERO:
                for (int64_t i = 0; i < dim; ++i) oo[i] = dual ? vv[i] : 0.0;
                break;
            case ORC_NONNEG:
                for (int64_t i = 0; i < dim; ++i) oo[i] = vv[i] > 0.0 ? vv[i] : 0.0;
                break;
            case ORC_SOC:
                orc_proj_soc(vv[0], vv + 1, dual ? dinv : dd, dim - 1, &oo[0], oo + 1);
                break;
            case ORC_RSOC:
                orc_proj_rsoc(vv, dual ? dinv : dd, dim, oo);
                break;
            case ORC_EXP:
                if (dual) { /* Remark with E = D^-1: Proj_{D^-1 K*}(v) = v + Proj_{D K}(-v) */
                    double nv[3] = {-vv[0], -vv[1], -vv[2]}, p[3];
                    orc_proj_exp(nv, dd, p);
                    for (int i = 0; i < 3; ++i) oo[i] = vv[i] + p[i];
                } else {
                    orc_proj_exp(vv, dd, oo);
                }
                break;
            case ORC_EXP_DUAL: /* the block is D K_exp*; its dual cone is D^-1 K_exp */
                if (dual) {
                    orc_proj_exp(vv, dinv, oo);
                } else { /* Remark with E = D: Proj_{D K*}(v) = v + Proj_{D^-1 K}(-v) */
                    double nv[3] = {-vv[0], -vv[1], -vv[2]}, p[3];
                    orc_proj_exp(nv, dinv, p);
                    for (int i = 0; i < 3; ++i) oo[i] = vv[i] + p[i];
                }
                break;
            default:
                break;
        }
        free(dinv);
        o += dim;
    }
}

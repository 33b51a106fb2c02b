// cone_math.cuh -- device projections onto diagonally rescaled cones.
//
// SOC: Theorem 1 (Sec. 3; proof in App. A.1).  Cases 1-3 in closed form; in
//      case 4 the root lambda of eq. (bisection-soc) is found by Newton's method
//      on the equivalent monotone function
//          G(lambda) = (1 - 2 lambda)^2 S(lambda) - t^2,
//          S(lambda) = sum_i w_i x_i^2 / (1 + 2 lambda w_i)^2,   w_i = dhat_i^{-2},
//      (G = (1 - 2 lambda)^2 f(lambda) has the sign of f), safeguarded by the
//      bracket (0, 1/2) for t > 0 and (1/2, hi) for t < 0.  One warp per cone;
//      the last root is kept per cone and used as the next starting point.
//      The first entry of the result is ||Dhat^{-1} y|| (the active constraint of
//      eq. kkt_sys_fixed_2), which equals t / (1 - 2 lambda) at the root.
// EXP: Theorem 3 (App. A.2).  Cases 1-3 in closed form with log-form membership
//      tests; in case 4 the root of h (eq. h_rho) on (l_rho, u_rho) is found by
//      Newton's method on the logarithm L of the offset of rho from an endpoint
//      (rho = a4 + dir e^L or a3 + dir e^L), with h compared in log form, the
//      vanishing factor of s~ or r~ carried as log r0 + L or log s0 + L, and a
//      bracket (grown by doubling at its lower end) as safeguard.  The result takes
//      per coordinate the smaller of v_p, v_d from eq. vpvd_defn and the other from
//      v0 = v_p + v_d.  One thread per cone; the last L of each cone is kept as the
//      next starting point.
// EXP*: the Remark of App. A.2: Proj_{E K*}(v) = v + Proj_{E^{-1} K}(-v).
#pragma once
#include "common.cuh"

namespace pdcs {

// ---------------------------------------------------------------------------
// Second-order cone
// ---------------------------------------------------------------------------
// Weight of entry i (0-based over the x part) for the projection onto E K_soc,
// E = diag(e_0, e_1, ...): dhat_i = e_{i+1} / e_0 and w_i = dhat_i^{-2}.
// kInv selects E = D^{-1} for a given D (dual side): w_i = (d_{i+1} / d_0)^2.
template <bool kInv>
__device__ __forceinline__ double soc_weight(const double* __restrict__ d, double d0, int i) {
    if (d == nullptr) return 1.0;
    double q = kInv ? d[i + 1] / d0 : d0 / d[i + 1];
    return q * q;
}

// Projects the SOC block stored at buf[0..dim) in place onto E K_soc (E as
// above).  Called by all 32 lanes of a warp with identical arguments.
// lam_cache (may be null): last root of this cone, updated.
// Returns the number of Newton / bisection evaluations (for diagnostics).
template <bool kInv>
__device__ int soc_project_warp(double* buf, const double* __restrict__ d, int dim, double* lam_cache) {
    const int lane = threadIdx.x & 31;
    const int nx = dim - 1;
    const double t = buf[0];
    const double d0 = d ? d[0] : 1.0;
    double a = 0.0, b = 0.0;  // a = ||Dhat x||^2, b = ||Dhat^{-1} x||^2
    for (int i = lane; i < nx; i += 32) {
        double x = buf[1 + i], w = soc_weight<kInv>(d, d0, i);
        a += x * x / w;
        b += w * x * x;
    }
    a = warp_sum(a);
    b = warp_sum(b);
    const double nDx = sqrt(a), nDinvx = sqrt(b);
    __syncwarp();
    if (t <= 0.0 && nDx <= -t) {  // case 1: in the polar cone
        for (int i = lane; i < dim; i += 32) buf[i] = 0.0;
        __syncwarp();
        return 0;
    }
    if (nDinvx <= t) return 0;    // case 2: in the cone
    double lam;
    int evals = 0;
    if (t == 0.0) {               // case 3: lambda = 1/2
        lam = 0.5;
    } else {                      // case 4
        double lo, hi;
        int slo;
        auto G = [&](double l, double& g, double& dg) {
            double S = 0.0, S1 = 0.0;
            for (int i = lane; i < nx; i += 32) {
                double x = buf[1 + i], w = soc_weight<kInv>(d, d0, i);
                double r = 1.0 / (1.0 + 2.0 * l * w);
                double term = w * x * x * r * r;
                S += term;
                S1 -= 4.0 * w * term * r;
            }
            S = warp_sum(S);
            S1 = warp_sum(S1);
            double u = 1.0 - 2.0 * l;
            g = u * u * S - t * t;
            dg = -4.0 * u * S + u * u * S1;
        };
        double g, dg;
        if (t > 0.0) {
            lo = 0.0; hi = 0.5; slo = 1;
        } else {
            lo = 0.5; hi = 1.0; slo = -1;
            for (int it = 0; it < 1100; ++it) {  // G(hi) -> ||Dhat x||^2 - t^2 > 0
                G(hi, g, dg);
                ++evals;
                if (g > 0.0) break;
                lo = hi;
                hi *= 2.0;
            }
        }
        double guess = (nDinvx - t) / (2.0 * (nDinvx + t));  // exact root when Dhat = I
        if (lam_cache && *lam_cache > lo && *lam_cache < hi) guess = *lam_cache;
        lam = (guess > lo && guess < hi) ? guess : 0.5 * (lo + hi);
        for (int it = 0; it < 200; ++it) {
            G(lam, g, dg);
            ++evals;
            if (g == 0.0) break;
            int s = g > 0.0 ? 1 : -1;
            if (s == slo) lo = lam; else hi = lam;
            double nl = lam - g / dg;
            // a Newton step below 1e-10 relative leaves an error of order its square
            // (lam itself has just become an end of the bracket, so test this first)
            if (nl >= lo && nl <= hi && fabs(nl - lam) <= 1e-10 * lam) {
                lam = nl;
                break;
            }
            if (!(nl > lo && nl < hi)) nl = 0.5 * (lo + hi);
            const bool done = !(nl > lo && nl < hi) || (hi - lo) <= 4e-16 * hi;
            lam = nl;
            if (done) break;
        }
        if (lam_cache && lane == 0) *lam_cache = lam;
    }
    // y = (I + 2 lambda Dhat^{-2})^{-1} x ;  s = ||Dhat^{-1} y||
    double s = 0.0;
    for (int i = lane; i < nx; i += 32) {
        double x = buf[1 + i], w = soc_weight<kInv>(d, d0, i);
        double y = x / (1.0 + 2.0 * lam * w);
        s += w * y * y;
        buf[1 + i] = y;
    }
    s = warp_sum(s);
    __syncwarp();
    if (lane == 0) buf[0] = sqrt(s);
    __syncwarp();
    return evals;
}

// Rotated SOC as Q K_soc with Q = [[1, 1], [1, -1]] / sqrt2 (+) I: with equal
// scales on the first two rows, Proj_{E K_rsoc}(v) = Q Proj_{E K_soc}(Q v).
template <bool kInv>
__device__ int rsoc_project_warp(double* buf, const double* __restrict__ d, int dim, double* lam_cache) {
    const int lane = threadIdx.x & 31;
    const double r2 = 0.70710678118654752440;
    __syncwarp();
    if (lane == 0) {
        double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
    int ev = soc_project_warp<kInv>(buf, d, dim, lam_cache);
    if (lane == 0) {
        double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
    return ev;
}

// ---------------------------------------------------------------------------
// Exponential cone
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ bool in_kexp(double r, double s, double t) {
    if (s > 0.0) return t > 0.0 && (log(t) - log(s)) >= r / s;
    if (s == 0.0) return t >= 0.0 && r <= 0.0;
    return false;
}

__host__ __device__ __forceinline__ bool in_kexp_dual(double r, double s, double t) {
    if (r < 0.0) return t > 0.0 && (1.0 + log(t) - log(-r)) >= s / r;
    if (r == 0.0) return s >= 0.0 && t >= 0.0;
    return false;
}

__host__ __device__ __forceinline__ double lse2(double a, double b) {  // log(e^a + e^b)
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double mx = fmax(a, b), mn = fmin(a, b);
    return mx + log1p(exp(mn - mx));
}

struct ExpCase4 {
    double r0, s0, t0, dr, ds, tau, a3, a4, a4m1, w34, ldt, dir, lt0, lr0, ls0, ldr, lds;
    int anchor;  // 3 or 4: endpoint rho is measured from
    int kind;    // 1: r0 > 0, s0 > 0;  2: r0 <= 0 < s0;  3: s0 <= 0 < r0
};

// At log-offset L (rho = anchor + dir e^L): rho, log s_p, log r_d (eq. sp_rd via
// eq. tilde_defs, the vanishing factor as log r0 + L or log s0 + L), and
// F(L) = lhs - rhs with the sign of h(rho) (eq. h_rho) decided in logs:
//   t0 >= 0: lhs = A, rhs = log(e^B + t0);  t0 < 0: lhs = log(e^A - t0), rhs = B,
//   A = log(d_t e^rho s_p), B = log(d_t^{-1} e^{-rho} r_d);  dF = dF/dL.
__host__ __device__ __forceinline__ void exp_F(const ExpCase4& e, double L, double& F, double& dF, double& rho_out,
                                               double& lsp_out, double& lrd_out) {
    const double delta = exp(L);
    double rho, rm1, lst, lrt, dlst, dlrt;  // rm1 = rho - 1 from the exact offset; logs of |s~|, |r~|
    int sst, srt;
    if (e.anchor == 4) {
        rho = e.a4 + e.dir * delta;
        rm1 = e.a4m1 + e.dir * delta;
        lst = e.lr0 + L;
        dlst = 1.0;
        sst = e.dir > 0.0 ? 1 : -1;
        const double rt = (e.kind == 1) ? e.s0 * (e.w34 - e.dir * delta) : e.tau * e.r0 - rho * e.s0;
        lrt = log(fabs(rt));
        dlrt = (-e.s0 / rt) * e.dir * delta;
        srt = (rt > 0.0) - (rt < 0.0);
    } else {
        rho = e.a3 + e.dir * delta;
        rm1 = (e.a3 - 1.0) + e.dir * delta;
        lrt = e.ls0 + L;
        dlrt = 1.0;
        srt = e.dir < 0.0 ? 1 : -1;
        const double st = (e.kind == 1) ? e.r0 * (e.w34 + e.dir * delta) : e.s0 * e.tau - e.r0 + e.r0 * rho;
        lst = log(fabs(st));
        dlst = (e.r0 / st) * e.dir * delta;
        sst = (st > 0.0) - (st < 0.0);
    }
    const double dt_ = rho * rm1 + e.tau * e.tau;  // d~ = rho (rho - 1) + tau^2
    const int sdt = (dt_ > 0.0) - (dt_ < 0.0);
    const double ldt_ = log(fabs(dt_));
    const double dldt = ((2.0 * rho - 1.0) / dt_) * e.dir * delta;
    const double lsp = (sst != 0 && sst == sdt) ? lst - e.ldr - ldt_ : -INFINITY;
    const double lrd = (srt != 0 && srt == sdt) ? e.lds + lrt - ldt_ : -INFINITY;
    const double A = e.ldt + rho + lsp;
    const double B = -e.ldt - rho + lrd;
    const double dA = e.dir * delta + dlst - dldt;
    const double dB = -e.dir * delta + dlrt - dldt;
    // log(e^a + e^b) = max + log1p(q), q = e^(min - max); the weight e^(a - lse) of a
    // comes from the same q, so each evaluation needs one exp and one log1p here
    auto lse_w = [](double a, double b, double& wa) {
        if (a == -INFINITY) { wa = 0.0; return b; }
        if (b == -INFINITY) { wa = 1.0; return a; }
        const bool amax = a >= b;
        const double q = exp(amax ? b - a : a - b);
        wa = amax ? 1.0 / (1.0 + q) : q / (1.0 + q);
        return (amax ? a : b) + log1p(q);
    };
    if (e.t0 >= 0.0) {
        double wB = 1.0;
        const double rhs = e.t0 > 0.0 ? lse_w(B, e.lt0, wB) : B;
        if (B == -INFINITY) wB = 0.0;
        F = A - rhs;
        dF = dA - wB * dB;
    } else {
        double wA;
        const double lhs = lse_w(A, e.lt0, wA);
        F = lhs - B;
        dF = wA * dA - dB;
    }
    rho_out = rho;
    lsp_out = lsp;
    lrd_out = lrd;
}

__host__ __device__ __forceinline__ int exp_sign(const ExpCase4& e, double L, int& evals) {
    double F, dF, rho, lsp, lrd;
    exp_F(e, L, F, dF, rho, lsp, lrd);
    ++evals;
    return (F > 0.0) - (F < 0.0);
}

// Lower end of the search: step down from hi by 1, 2, 4, ... until F shows the
// sign it has next to the anchor.
__host__ __device__ __forceinline__ double exp_lower(const ExpCase4& e, double hi, int slo, int& evals) {
    double step = 1.0;
    for (int it = 0; it < 1100; ++it) {
        const double lo = hi - step;
        if (lo == -INFINITY || exp_sign(e, lo, evals) == slo) return lo;
        step *= 2.0;
    }
    return -INFINITY;
}

// Safeguarded Newton for F(L) = 0 on (lo, hi); sign(F) at the lo end is slo.
__host__ __device__ __forceinline__ double exp_newton(const ExpCase4& e, double lo, double hi, int slo, double L,
                                                      int& evals) {
    if (!(L > lo && L < hi)) L = (lo == -INFINITY) ? hi - 1.0 : 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
        double F, dF, rho, lsp, lrd;
        exp_F(e, L, F, dF, rho, lsp, lrd);
        ++evals;
        if (!(F == F)) break;  // NaN: both sides infinite, already at the limit
        if (F == 0.0) break;
        const int s = F > 0.0 ? 1 : -1;
        if (s == slo) lo = L; else hi = L;
        double nl = L - F / dF;
        // a Newton step below 1e-10 relative leaves an error of order its square
        // (L itself has just become an end of the bracket, so test this first)
        if (nl >= lo && nl <= hi && fabs(nl - L) <= 1e-10 * fmax(1.0, fabs(L))) {
            L = nl;
            break;
        }
        if (!(nl > lo && nl < hi)) nl = (lo == -INFINITY) ? hi - 2.0 * fmax(1.0, fabs(hi - L)) : 0.5 * (lo + hi);
        const bool done = !(nl > lo && nl < hi) || (hi - lo) <= 4e-16 * fmax(1.0, fabs(hi));
        L = nl;
        if (done) break;
    }
    return L;
}

// Projection of v0 onto D K_exp, D = diag(dr, ds, dt) (Theorem 3).
// L_cache (may be null): last log-offset of this cone, used as the Newton start and updated.
__host__ __device__ inline void exp_project(double r0, double s0, double t0, double dr, double ds, double dt,
                                            double* out, double* L_cache, int* evals_out) {
    int evals = 0;
    if (evals_out) *evals_out = 0;
    if (in_kexp(r0 / dr, s0 / ds, t0 / dt)) {  // case 1
        out[0] = r0; out[1] = s0; out[2] = t0;
        return;
    }
    if (in_kexp_dual(-dr * r0, -ds * s0, -dt * t0)) {  // case 2
        out[0] = 0.0; out[1] = 0.0; out[2] = 0.0;
        return;
    }
    if (r0 <= 0.0 && s0 <= 0.0) {  // case 3
        out[0] = r0; out[1] = 0.0; out[2] = t0 > 0.0 ? t0 : 0.0;
        return;
    }
    ExpCase4 e;
    e.r0 = r0; e.s0 = s0; e.t0 = t0; e.dr = dr; e.ds = ds;
    e.tau = ds / dr;
    e.ldt = log(dt);
    e.ldr = log(dr);
    e.lds = log(ds);
    e.lr0 = r0 > 0.0 ? log(r0) : -INFINITY;
    e.ls0 = s0 > 0.0 ? log(s0) : -INFINITY;
    e.lt0 = t0 > 0.0 ? log(t0) : (t0 < 0.0 ? log(-t0) : -INFINITY);
    e.a3 = (s0 > 0.0) ? (r0 * ds) / (s0 * dr) : 0.0;
    e.a4 = (r0 > 0.0) ? 1.0 - (s0 * ds) / (r0 * dr) : 0.0;
    e.a4m1 = (r0 > 0.0) ? -(s0 * ds) / (r0 * dr) : -1.0;
    e.w34 = e.a3 - e.a4;
    const double guess = L_cache ? *L_cache : NAN;
    double L;
    if (r0 > 0.0 && s0 > 0.0) {
        e.kind = 1;
        const double W = fabs(e.w34);
        if (!(W > 0.0)) { out[0] = 0.0; out[1] = 0.0; out[2] = 0.0; return; }
        const double Lh = log(0.5 * W);
        e.anchor = 4;
        e.dir = e.w34 > 0.0 ? 1.0 : -1.0;
        const int sm = exp_sign(e, Lh, evals);
        if (sm == 0) {
            L = Lh;
        } else if (sm > 0) {  // root in the half next to a4
            L = exp_newton(e, exp_lower(e, Lh, -1, evals), Lh, -1, guess, evals);
        } else {              // root in the half next to a3
            e.anchor = 3;
            e.dir = -e.dir;
            L = exp_newton(e, exp_lower(e, Lh, +1, evals), Lh, +1, guess, evals);
        }
    } else if (s0 > 0.0) {  // r0 <= 0: (-inf, a3)
        e.kind = 2; e.anchor = 3; e.dir = -1.0;
        double hi = 0.0;
        for (int it = 0; it < 8 && exp_sign(e, hi, evals) > 0 && hi < 60.0; ++it) hi = 2.0 * hi + 1.0;
        L = exp_newton(e, exp_lower(e, hi, +1, evals), hi, +1, guess, evals);
    } else {  // s0 <= 0 < r0: (a4, inf)
        e.kind = 3; e.anchor = 4; e.dir = 1.0;
        double hi = 0.0;
        for (int it = 0; it < 8 && exp_sign(e, hi, evals) < 0 && hi < 60.0; ++it) hi = 2.0 * hi + 1.0;
        L = exp_newton(e, exp_lower(e, hi, -1, evals), hi, -1, guess, evals);
    }
    if (L_cache) *L_cache = L;
    double F, dF, rho, lsp, lrd;
    exp_F(e, L, F, dF, rho, lsp, lrd);
    if (evals_out) *evals_out = evals;
    // eq. vpvd_defn with v0 = v_p + v_d (eq. diagonal_moreau): per coordinate the
    // smaller part from its formula, v_p = v0 - v_d when v_d is the larger one.
    const double sp = exp(lsp), rd = exp(lrd);
    const double vp[3] = {dr * rho * sp, ds * sp, exp(e.ldt + rho + lsp)};
    const double vd[3] = {rd / dr, (1.0 - rho) * rd / ds, -exp(-e.ldt - rho + lrd)};
    const double v0[3] = {r0, s0, t0};
#pragma unroll
    for (int k = 0; k < 2; ++k) out[k] = fabs(vp[k]) <= fabs(vd[k]) ? vp[k] : v0[k] - vd[k];
    // t entry: h(rho) = 0 says e^A - e^B = t0, so v_d is the smaller part when t0 >= 0
    out[2] = t0 >= 0.0 ? t0 - vd[2] : vp[2];
}

// Projection onto D^{-1} K_exp^* (Remark of App. A.2): v + Proj_{D K_exp}(-v).
__host__ __device__ __forceinline__ void exp_dual_project(double r, double s, double t, double dr, double ds, double dt,
                                                 double* out, double* L_cache, int* evals) {
    double p[3];
    exp_project(-r, -s, -t, dr, ds, dt, p, L_cache, evals);
    out[0] = r + p[0];
    out[1] = s + p[1];
    out[2] = t + p[2];
}

}  // namespace pdcs

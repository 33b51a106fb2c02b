// cone_math.cuh -- device projections onto diagonally rescaled cones.
//
// SOC: Theorem 1 (Sec. 3; proof in App. A.1).  Cases 1-3 in closed form; in
//      case 4 the root of eq. (bisection-soc) is found by safeguarded Newton on
//      an equivalent monotone, nearly affine function psi (see below).
//      One warp per cone; the last root is kept per cone and used as the next
//      starting point.  The first entry of the result is ||Dhat^{-1} y|| (the
//      active constraint of eq. kkt_sys_fixed_2), which equals t / (1 - 2 lambda)
//      at the root.
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

// Newton step (relative) below which the SOC root search stops: the error left is of
// order its square.
constexpr double RootTolSoc = 1e-10;

// ---------------------------------------------------------------------------
// Second-order cone
//
// Case 4 of Theorem 1 puts lambda in (0, 1/2) for t > 0 and in (1/2, inf) for
// t < 0.  With mu = 2 lambda and w_i = dhat_i^{-2}, the root of eq. (bisection-soc)
// multiplied by (1 - mu)^2 and square-rooted is the root of
//     |1 - mu| sqrt(S(mu)) = |t|,   S(mu) = sum_i w_i x_i^2 / (1 + mu w_i)^2,
// whose left side moves away from |t| monotonically as mu leaves 1.  The search runs
// on a variable u chosen so that the root is a small u where it needs relative
// precision:
//   t > 0, root at mu >= 1/2:  u = 1 - mu in (0, 1)  (nearly inactive cones: u ~ t)
//   t > 0, root at mu < 1/2:   u = mu in (0, 1)      (v almost in the cone: u ~ 0)
//   t < 0:                     u = mu - 1 in (0, inf)
// (for t > 0 the half is read off the cached root or the sign of psi at mu = 1/2, and
// Newton's relative stopping test uses the smaller of u and 1 - u)
// The equation is solved in the reciprocal form used for trust-region secular
// equations (More and Sorensen, 1983): 1 / sqrt(S(mu)) is affine in mu when one term
// of S dominates, so
//     psi(u) = (u - pm) / |t| + eps / sqrt(S(mu)),
// (pm = 0, eps = -1 for the first and last variable; pm = 1, eps = +1 for the second)
// increases in u, is negative at u = 0, and is nearly affine: safeguarded Newton with
// a relative test on u converges in a few steps even where the poles -1/w_i of S are
// close.  The projection is y = (I + mu Dhat^{-2})^{-1} x, s = ||Dhat^{-1} y|| (the
// active constraint of eq. kkt_sys_fixed_2).
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

// The search variable of case 4 (see above): mu = a0 + a1 u, psi = (u - pm) / |t| + eps / sqrt(S).
// near (t > 0 only): the root has mu < 1/2, decided from the cached root or from the
// sign of psi at mu = 1/2.  The cached value of a cone is u, negated for
// the variable mu next to the cone.
template <typename R>
struct SocVar {
    R a0, a1, pm, iat, eps;
    bool near, tpos;
    __device__ __forceinline__ SocVar(R t, bool near_) {
        tpos = t > R(0);
        near = tpos && near_;
        iat = R(1) / fabs(t);
        eps = near ? R(1) : R(-1);
        if (near) { a0 = R(0); a1 = R(1); pm = R(1); }
        else if (tpos) { a0 = R(1); a1 = R(-1); pm = R(0); }
        else { a0 = R(1); a1 = R(1); pm = R(0); }
    }
    // Start: the cached u (converted between the two t > 0 variables), else the root
    // when Dhat = I.
    __device__ __forceinline__ R guess(R t, R nDinvx, const float* cache) const {
        const R at = fabs(t);
        R u = near ? (nDinvx - at) / (nDinvx + at)
                   : (tpos ? R(2) * at / (nDinvx + at) : (nDinvx > at ? R(2) * at / (nDinvx - at) : R(-1)));
        if (cache) {
            const R cv = (R)*cache;
            R cu = R(-1);
            if (!tpos) cu = cv;
            else if (near) cu = cv < R(0) ? -cv : R(1) - cv;
            else cu = cv > R(0) ? cv : R(1) + cv;
            if (cu > R(0) && (!tpos || cu < R(1))) u = cu;
        }
        return u;
    }
    // the same variable in another precision
    template <typename Q>
    __device__ __forceinline__ explicit SocVar(const SocVar<Q>& o)
        : a0(R(o.a0)), a1(R(o.a1)), pm(R(o.pm)), iat(R(o.iat)), eps(R(o.eps)), near(o.near), tpos(o.tpos) {}
    __device__ __forceinline__ float store(R u) const { return near ? -(float)u : (float)u; }
    __device__ __forceinline__ R mu(R u) const { return a0 + a1 * u; }
    // psi and dpsi/du from sq = sqrt(S) and S2 = sum w_i^2 x_i^2 / (1 + mu w_i)^3 (so
    // dS/dmu = -2 S2); sc is the size of the terms of psi (its rounding error is a few
    // ulps of sc)
    __device__ __forceinline__ void psi(R u, R sq, R S2, R& ph, R& dph, R& sc) const {
        const R p = u - pm, isq = R(1) / sq;
        ph = p * iat + eps * isq;
        dph = iat + eps * a1 * S2 * isq * isq * isq;
        sc = fabs(p) * iat + isq;
    }
};

// For t > 0: whether the cached root (see SocVar) has mu < 1/2; false with known = false
// when the cache holds no usable value.
__device__ __forceinline__ bool soc_cached_near(const float* cache, bool& known) {
    known = false;
    if (!cache) return false;
    const float cv = *cache;
    const float mu = cv < 0.0f ? -cv : 1.0f - cv;
    known = cv == cv && cv != 0.0f && mu > 0.0f && mu < 1.0f;
    return known && mu < 0.5f;
}

// Safeguarded Newton for psi(u) = 0 given an evaluator ev(u, psi, dpsi, sc) (warp-
// uniform results), with psi(0) < 0.  hi: 1 for t > 0; found by doubling for t < 0.
// Stops on a relative Newton step below tol, on a bracket collapsed to collapse
// relative, or on |psi| within 4 collapse of sc (zero to working precision: next to
// the cone u is then fixed only to a few ulps, absolutely).
template <typename R, typename Ev>
__device__ __forceinline__ R soc_root(Ev ev, bool tpos, R guess, R tol, R collapse, int max_it) {
    R lo = R(0), hi = R(1), ph, dph, sc;
    if (!tpos) {
        for (int it = 0; it < 1100; ++it) {
            ev(hi, ph, dph, sc);
            if (ph > R(0) || !(hi < (sizeof(R) == 4 ? R(1e30) : R(1e300)))) break;
            lo = hi;
            hi *= R(2);
        }
    }
    R g = (guess > lo && guess < hi) ? guess : R(0.5) * (lo + hi);
    for (int it = 0; it < max_it; ++it) {
        ev(g, ph, dph, sc);
        if (!(ph == ph) || fabs(ph) <= R(4) * collapse * sc) break;
        if (ph < R(0)) lo = g; else hi = g;
        R ng = g - ph / dph;
        // relative to the smaller of u and 1 - u for t > 0 (both mu and 1 - mu matter)
        if (ng >= lo && ng <= hi && fabs(ng - g) <= tol * (tpos ? fmin(g, R(1) - g) : g)) { g = ng; break; }
        if (!(ng > lo && ng < hi)) ng = R(0.5) * (lo + hi);
        const bool done = !(ng > lo && ng < hi) || (hi - lo) <= collapse * hi;
        g = ng;
        if (done) break;
    }
    return g;
}

// Projects the SOC block stored at buf[0..dim) in place onto E K_soc (E as above),
// entries read from memory (any dim).  Called by all 32 lanes of a warp with
// identical arguments.  cache (may be null): last u of this cone (see SocVar), updated.
template <bool kInv>
__device__ int soc_project_warp(double* buf, const double* __restrict__ d, int dim, float* cache) {
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
    double mu = 1.0;              // 2 lambda; case 3 (t == 0): lambda = 1/2
    int evals = 0;
    if (t != 0.0) {               // case 4
        bool known, near = t > 0.0 && soc_cached_near(cache, known);
        if (t > 0.0 && !known) {  // sign of psi at mu = 1/2
            double S = 0.0;
            for (int i = lane; i < nx; i += 32) {
                const double x = buf[1 + i], w = soc_weight<kInv>(d, d0, i);
                const double r = 1.0 / (1.0 + 0.5 * w);
                S += w * x * x * r * r;
            }
            near = 0.5 * sqrt(warp_sum(S)) < t;
        }
        const SocVar<double> V(t, near);
        auto ev = [&](double u, double& ph, double& dph, double& sc) {
            double S = 0.0, S2 = 0.0;
            const double m = V.mu(u);
            for (int i = lane; i < nx; i += 32) {
                const double x = buf[1 + i], w = soc_weight<kInv>(d, d0, i);
                const double r = 1.0 / (1.0 + m * w);
                const double term = w * x * x * r * r;
                S += term;
                S2 += w * term * r;
            }
            S = warp_sum(S);
            S2 = warp_sum(S2);
            V.psi(u, sqrt(S), S2, ph, dph, sc);
            ++evals;
        };
        const double u = soc_root<double>(ev, V.tpos, V.guess(t, nDinvx, cache), RootTolSoc, 4e-16, 200);
        if (cache && lane == 0) *cache = V.store(u);
        mu = V.mu(u);
    }
    // y = (I + 2 lambda Dhat^{-2})^{-1} x ;  s = ||Dhat^{-1} y||
    double s = 0.0;
    for (int i = lane; i < nx; i += 32) {
        double x = buf[1 + i], w = soc_weight<kInv>(d, d0, i);
        double y = x / (1.0 + mu * w);
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
__device__ int rsoc_project_warp(double* buf, const double* __restrict__ d, int dim, float* cache) {
    const int lane = threadIdx.x & 31;
    const double r2 = 0.70710678118654752440;
    __syncwarp();
    if (lane == 0) {
        double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
    int ev = soc_project_warp<kInv>(buf, d, dim, cache);
    if (lane == 0) {
        double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
    return ev;
}

// ---------------------------------------------------------------------------
// Second-order cone, mixed precision (cones with dim - 1 <= 32 R): the entries
// stay in registers, weights w_i come precomputed, the root of psi is found in
// FP32 and polished by at most three FP64 Newton steps, in which 1 / (1 + mu w) is
// an FP32 reciprocal refined by two Newton-Raphson steps r <- r (2 - a r) in FP64.
// Whatever the FP32 pass cannot settle falls back to the full FP64 search.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp_refined(double a) {
    double r = (double)__frcp_rn((float)a);
    r = r * (2.0 - a * r);
    return r * (2.0 - a * r);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Weights of the SOC entries for the mixed-precision path: precomputed (w[i], or all ones
// when w is null), or formed from the block's scales d as soc_weight<kInv> does.
struct SocWeightsArray {
    const double* w;
    const double* wi;  // 1 / w[i] to rounding (may be null: divided out)
    __device__ __forceinline__ double operator()(int i) const { return w ? w[i] : 1.0; }
    __device__ __forceinline__ double inv(int i) const { return wi ? wi[i] : (w ? 1.0 / w[i] : 1.0); }
    __device__ __forceinline__ bool unit() const { return w == nullptr; }  // Dhat = I
};
template <bool kInv>
struct SocWeightsScales {
    const double* d;
    double d0;
    __device__ __forceinline__ double operator()(int i) const { return soc_weight<kInv>(d, d0, i); }
    __device__ __forceinline__ double inv(int i) const { return soc_weight<!kInv>(d, d0, i); }
    __device__ __forceinline__ bool unit() const { return d == nullptr; }
};

// buf[0..dim): the block, projected in place onto E K_soc where the weight of x entry
// i is wf(i) = dhat_i^{-2}.  cache may be null.
template <int R, typename WF>
__device__ void soc_project_warp_fast(double* buf, WF wf, int dim, float* cache) {
    const int lane = threadIdx.x & 31;
    const int nx = dim - 1;
    const double t = buf[0];
    double xr[R], wr[R], wir[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int i = lane + 32 * k;
        const bool in = i < nx;
        xr[k] = in ? buf[1 + i] : 0.0;
        wr[k] = in ? wf(i) : 1.0;
        wir[k] = in ? wf.inv(i) : 1.0;
    }
    double a = 0.0, b = 0.0;  // ||Dhat x||^2, ||Dhat^{-1} x||^2
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const double x2 = xr[k] * xr[k];
        a += x2 * wir[k];
        b += wr[k] * x2;
    }
    a = warp_sum(a);
    b = warp_sum(b);
    const double nDx = sqrt(a), nDinvx = sqrt(b);
    __syncwarp();
    if (t <= 0.0 && nDx <= -t) {  // case 1
#pragma unroll
        for (int k = 0; k < R; ++k) if (lane + 32 * k < nx) buf[1 + lane + 32 * k] = 0.0;
        if (lane == 0) buf[0] = 0.0;
        __syncwarp();
        return;
    }
    if (nDinvx <= t) return;  // case 2
    double mu = 1.0;          // case 3 (t == 0)
    if (t != 0.0) {           // case 4
        float xf[R], wf[R];
        bool rng = fabs(t) < 1e30 && fabs(t) > 1e-30 && nDinvx < 1e30;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            xf[k] = (float)xr[k];
            wf[k] = (float)wr[k];
            rng = rng && wr[k] < 1e30 && wr[k] > 1e-30;
        }
        rng = __all_sync(0xffffffffu, rng);
        bool known, near = t > 0.0 && soc_cached_near(cache, known);
        if (t > 0.0 && !known) {  // sign of psi at mu = 1/2
            if (rng) {
                float S = 0.0f;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const float r = __frcp_rn(1.0f + 0.5f * wf[k]);
                    S += wf[k] * xf[k] * xf[k] * r * r;
                }
                near = 0.5f * sqrtf(warp_sum_f(S)) < (float)t;
            } else {
                double S = 0.0;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const double r = 1.0 / (1.0 + 0.5 * wr[k]);
                    S += wr[k] * xr[k] * xr[k] * r * r;
                }
                near = 0.5 * sqrt(warp_sum(S)) < t;
            }
        }
        const SocVar<double> V(t, near);
        // ---- FP32 root of psi
        const SocVar<float> Vf(V);
        auto ev32 = [&](float u, float& ph, float& dph, float& sc) {
            float S = 0.0f, S2 = 0.0f;
            const float m = Vf.mu(u);
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const float r = __frcp_rn(1.0f + m * wf[k]);
                const float term = wf[k] * xf[k] * xf[k] * r * r;
                S += term;
                S2 += wf[k] * term * r;
            }
            S = warp_sum_f(S);
            S2 = warp_sum_f(S2);
            Vf.psi(u, sqrtf(S), S2, ph, dph, sc);
        };
        float uf = 0.0f;
        bool ok = rng;
        if (ok) {
            uf = soc_root<float>(ev32, V.tpos, (float)V.guess(t, nDinvx, cache), 2e-6f, 2e-7f, 100);
            ok = uf > 0.0f && isfinite(uf);
        }
        // ---- FP64 polish
        bool conv = false;
        double u = (double)uf;
        if (ok) {
            double x2w[R];
#pragma unroll
            for (int k = 0; k < R; ++k) x2w[k] = wr[k] * xr[k] * xr[k];
            for (int it = 0; it < 3; ++it) {
                double S = 0.0, S2 = 0.0;
                const double m = V.mu(u);
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const double r = rcp_refined(1.0 + m * wr[k]);
                    const double term = x2w[k] * r * r;
                    S += term;
                    S2 += wr[k] * term * r;
                }
                S = warp_sum(S);
                S2 = warp_sum(S2);
                double ph, dph, sc;
                V.psi(u, sqrt(S), S2, ph, dph, sc);
                if (fabs(ph) <= 1.6e-15 * sc) {  // zero to working precision
                    u = fmax(u, 0.0);
                    conv = true;
                    break;
                }
                const double step = ph / dph;
                if (!isfinite(step)) break;
                u -= step;
                // psi is nearly affine: the error after a Newton step is of order its
                // square, so a first step below 1e-7 relative (from the FP32 root) is final
                if (fabs(step) <= (it == 0 ? 1e-7 : RootTolSoc) * (V.tpos ? fmin(u, 1.0 - u) : u)) {
                    conv = true;
                    break;
                }
            }
            conv = conv && u >= 0.0 && (!V.tpos || u < 1.0);
        }
        if (!conv) {  // full FP64 safeguarded search on the registers
            auto ev = [&](double uu, double& ph, double& dph, double& sc) {
                double S = 0.0, S2 = 0.0;
                const double m = V.mu(uu);
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const double r = 1.0 / (1.0 + m * wr[k]);
                    const double term = wr[k] * xr[k] * xr[k] * r * r;
                    S += term;
                    S2 += wr[k] * term * r;
                }
                S = warp_sum(S);
                S2 = warp_sum(S2);
                V.psi(uu, sqrt(S), S2, ph, dph, sc);
            };
            u = soc_root<double>(ev, V.tpos, V.guess(t, nDinvx, nullptr), RootTolSoc, 4e-16, 200);
        }
        if (cache && lane == 0) *cache = V.store(u);
        mu = V.mu(u);
    }
    // y = (I + 2 lambda Dhat^{-2})^{-1} x ;  s = ||Dhat^{-1} y||
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const double y = xr[k] * rcp_refined(1.0 + mu * wr[k]);
        s += wr[k] * y * y;
        if (lane + 32 * k < nx) buf[1 + lane + 32 * k] = y;
    }
    s = warp_sum(s);
    __syncwarp();
    if (lane == 0) buf[0] = sqrt(s);
    __syncwarp();
}

// Rotated SOC through Q (see rsoc_project_warp) on the mixed-precision SOC path.
template <int R, typename WF>
__device__ void rsoc_project_warp_fast(double* buf, WF wf, int dim, float* cache) {
    const int lane = threadIdx.x & 31;
    const double r2 = 0.70710678118654752440;
    __syncwarp();
    if (lane == 0) {
        const double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
    soc_project_warp_fast<R>(buf, wf, dim, cache);
    if (lane == 0) {
        const double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
}

// Large blocks (memory loop), mixed precision: one FP64 pass forms the norms of the
// case tests and an FP32 copy of x and of the weights in scr (2 (dim - 1) floats); the
// root of psi is searched in FP32 over that copy, polished by at most three FP64 Newton
// steps over the block (the first accepted below 1e-7 relative, as in registers), and
// the projection is formed in FP64.  Anything the FP32 pass cannot settle falls back to
// the FP64 search (soc_project_warp).  wf(i): weight of x entry i.
template <bool kInv, typename WF>
__device__ void soc_project_warp_mp(double* buf, WF wf, const double* __restrict__ d, int dim, float* cache,
                                    float* __restrict__ scr) {
    const int lane = threadIdx.x & 31;
    const int nx = dim - 1;
    float* x32 = scr;
    float* w32 = scr + nx;
    const double t = buf[0];
    double a = 0.0, b = 0.0;
    bool rng = fabs(t) < 1e30 && fabs(t) > 1e-30;
    for (int i = lane; i < nx; i += 32) {
        const double x = buf[1 + i], w = wf(i);
        const double x2 = x * x;
        a += x2 / w;
        b += w * x2;
        x32[i] = (float)x;
        w32[i] = (float)w;
        rng = rng && w < 1e30 && w > 1e-30 && fabs(x) < 1e30;
    }
    a = warp_sum(a);
    b = warp_sum(b);
    rng = __all_sync(0xffffffffu, rng) && sqrt(b) < 1e30;
    const double nDx = sqrt(a), nDinvx = sqrt(b);
    __syncwarp();
    if (t <= 0.0 && nDx <= -t) {  // case 1
        for (int i = lane; i < dim; i += 32) buf[i] = 0.0;
        __syncwarp();
        return;
    }
    if (nDinvx <= t) return;  // case 2
    double mu = 1.0;          // case 3 (t == 0)
    if (t != 0.0) {           // case 4
        bool known, near = t > 0.0 && soc_cached_near(cache, known);
        if (t > 0.0 && !known) {  // sign of psi at mu = 1/2 (in FP32 when in range)
            float S = 0.0f;
            for (int i = lane; i < nx; i += 32) {
                const float r = __frcp_rn(1.0f + 0.5f * w32[i]);
                S += w32[i] * x32[i] * x32[i] * r * r;
            }
            near = 0.5f * sqrtf(warp_sum_f(S)) < (float)t;
        }
        const SocVar<double> V(t, near);
        const SocVar<float> Vf(V);
        bool conv = false;
        double u = 0.0;
        if (rng) {
            auto ev32 = [&](float uu, float& ph, float& dph, float& sc) {
                float S = 0.0f, S2 = 0.0f;
                const float m = Vf.mu(uu);
                for (int i = lane; i < nx; i += 32) {
                    const float w = w32[i], x = x32[i];
                    const float r = __frcp_rn(1.0f + m * w);
                    const float term = w * x * x * r * r;
                    S += term;
                    S2 += w * term * r;
                }
                S = warp_sum_f(S);
                S2 = warp_sum_f(S2);
                Vf.psi(uu, sqrtf(S), S2, ph, dph, sc);
            };
            const float uf = soc_root<float>(ev32, V.tpos, (float)V.guess(t, nDinvx, cache), 2e-6f, 2e-7f, 100);
            u = (double)uf;
            if (uf > 0.0f && isfinite(uf)) {
                for (int it = 0; it < 3; ++it) {
                    double S = 0.0, S2 = 0.0;
                    const double m = V.mu(u);
                    for (int i = lane; i < nx; i += 32) {
                        const double x = buf[1 + i], w = wf(i);
                        const double r = rcp_refined(1.0 + m * w);
                        const double term = w * x * x * r * r;
                        S += term;
                        S2 += w * term * r;
                    }
                    S = warp_sum(S);
                    S2 = warp_sum(S2);
                    double ph, dph, sc;
                    V.psi(u, sqrt(S), S2, ph, dph, sc);
                    if (fabs(ph) <= 1.6e-15 * sc) {
                        u = fmax(u, 0.0);
                        conv = true;
                        break;
                    }
                    const double step = ph / dph;
                    if (!isfinite(step)) break;
                    u -= step;
                    if (fabs(step) <= (it == 0 ? 1e-7 : RootTolSoc) * (V.tpos ? fmin(u, 1.0 - u) : u)) {
                        conv = true;
                        break;
                    }
                }
                conv = conv && u >= 0.0 && (!V.tpos || u < 1.0);
            }
        }
        if (!conv) {
            soc_project_warp<kInv>(buf, d, dim, cache);
            return;
        }
        if (cache && lane == 0) *cache = V.store(u);
        mu = V.mu(u);
    }
    double s = 0.0;
    for (int i = lane; i < nx; i += 32) {
        const double w = wf(i);
        const double y = buf[1 + i] * rcp_refined(1.0 + mu * w);
        s += w * y * y;
        buf[1 + i] = y;
    }
    s = warp_sum(s);
    __syncwarp();
    if (lane == 0) buf[0] = sqrt(s);
    __syncwarp();
}

template <bool kInv, typename WF>
__device__ void rsoc_project_warp_mp(double* buf, WF wf, const double* __restrict__ d, int dim, float* cache,
                                     float* __restrict__ scr) {
    const int lane = threadIdx.x & 31;
    const double r2 = 0.70710678118654752440;
    __syncwarp();
    if (lane == 0) {
        const double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
    soc_project_warp_mp<kInv>(buf, wf, d, dim, cache, scr);
    if (lane == 0) {
        const double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Second-order cone by lane groups (segmented warps).  S lanes (a power of two) project
// one cone staged in shared memory, 32 / S cones side by side in a warp; lane g of a group
// takes the x entries i = g, g + S, ...  On this GPU an FP64 warp instruction takes the
// same time whatever lanes are active, so the steps done once per cone (case tests, psi,
// the Newton steps, square roots) cost 32 / S times less per cone than with a warp per
// cone, and the sums need log2 S shuffle levels instead of five.  Same mathematics and
// precision scheme as soc_project_warp_fast: FP32 search, at most three FP64 Newton
// steps with refined reciprocals, FP64 output; FP64 search as fallback.
//   v      : the cone's staged rows (t, x_1 .. x_{dim-1}) in shared memory, projected in place
//   w, wi  : weights of the x entries and their inverses (global memory)
//   xf, wf : dim - 1 floats each of shared-memory scratch
//   gmask  : the group's lanes, g: this lane's index in the group
// ---------------------------------------------------------------------------
template <int S>
__device__ __forceinline__ double seg_sum(double v, unsigned gmask) {
#pragma unroll
    for (int o = S / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o);
    return v;
}
template <int S>
__device__ __forceinline__ float seg_sum_f(float v, unsigned gmask) {
#pragma unroll
    for (int o = S / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o);
    return v;
}

template <int S>
__device__ void soc_seg_project(double* v, const double* __restrict__ w, const double* __restrict__ wi, float* xf,
                                float* wf, int dim, bool rot, float* cache, unsigned gmask, int g) {
    const double r2 = 0.70710678118654752440;
    if (rot) {
        if (g == 0) {
            const double p = v[0], q = v[1];
            v[0] = (p + q) * r2;
            v[1] = (p - q) * r2;
        }
        __syncwarp(gmask);
    }
    const int nx = dim - 1;
    const double t = v[0];
    double a = 0.0, b = 0.0;  // ||Dhat x||^2, ||Dhat^{-1} x||^2
    bool rng = fabs(t) < 1e30 && fabs(t) > 1e-30;
    for (int i = g; i < nx; i += S) {
        const double x = v[1 + i], wv = w[i];
        const double x2 = x * x;
        a += x2 * wi[i];
        b += wv * x2;
        xf[i] = (float)x;
        wf[i] = (float)wv;
        rng = rng && wv < 1e30 && wv > 1e-30 && fabs(x) < 1e30;
    }
    a = seg_sum<S>(a, gmask);
    b = seg_sum<S>(b, gmask);
    if (S > 1) rng = __all_sync(gmask, rng);
    const double nDx = sqrt(a), nDinvx = sqrt(b);
    rng = rng && nDinvx < 1e30;
    double mu = -1.0;  // < 0: v unchanged (case 2)
    if (t <= 0.0 && nDx <= -t) {
        mu = 0.0;  // case 1: zero (marked below)
    } else if (!(nDinvx <= t)) {
        mu = 1.0;  // case 3 (t == 0)
        if (t != 0.0) {  // case 4
            bool known, near = t > 0.0 && soc_cached_near(cache, known);
            if (t > 0.0 && !known) {  // sign of psi at mu = 1/2
                if (rng) {
                    float Sf = 0.0f;
                    for (int i = g; i < nx; i += S) {
                        const float r = __frcp_rn(1.0f + 0.5f * wf[i]);
                        Sf += wf[i] * xf[i] * xf[i] * r * r;
                    }
                    near = 0.5f * sqrtf(seg_sum_f<S>(Sf, gmask)) < (float)t;
                } else {
                    double Sd = 0.0;
                    for (int i = g; i < nx; i += S) {
                        const double x = v[1 + i], r = 1.0 / (1.0 + 0.5 * w[i]);
                        Sd += w[i] * x * x * r * r;
                    }
                    near = 0.5 * sqrt(seg_sum<S>(Sd, gmask)) < t;
                }
            }
            const SocVar<double> V(t, near);
            const SocVar<float> Vf(V);
            bool conv = false;
            double u = 0.0;
            if (rng) {
                auto ev32 = [&](float uu, float& ph, float& dph, float& sc) {
                    float Sf = 0.0f, S2 = 0.0f;
                    const float m = Vf.mu(uu);
                    for (int i = g; i < nx; i += S) {
                        const float r = __frcp_rn(1.0f + m * wf[i]);
                        const float term = wf[i] * xf[i] * xf[i] * r * r;
                        Sf += term;
                        S2 += wf[i] * term * r;
                    }
                    Sf = seg_sum_f<S>(Sf, gmask);
                    S2 = seg_sum_f<S>(S2, gmask);
                    Vf.psi(uu, sqrtf(Sf), S2, ph, dph, sc);
                };
                const float uf = soc_root<float>(ev32, V.tpos, (float)V.guess(t, nDinvx, cache), 2e-6f, 2e-7f, 100);
                u = (double)uf;
                if (uf > 0.0f && isfinite(uf)) {
                    for (int it = 0; it < 3; ++it) {
                        double Sd = 0.0, S2 = 0.0;
                        const double m = V.mu(u);
                        for (int i = g; i < nx; i += S) {
                            const double x = v[1 + i], wv = w[i];
                            const double r = rcp_refined(1.0 + m * wv);
                            const double term = wv * x * x * r * r;
                            Sd += term;
                            S2 += wv * term * r;
                        }
                        Sd = seg_sum<S>(Sd, gmask);
                        S2 = seg_sum<S>(S2, gmask);
                        double ph, dph, sc;
                        V.psi(u, sqrt(Sd), S2, ph, dph, sc);
                        if (fabs(ph) <= 1.6e-15 * sc) {  // zero to working precision
                            u = fmax(u, 0.0);
                            conv = true;
                            break;
                        }
                        const double step = ph / dph;
                        if (!isfinite(step)) break;
                        u -= step;
                        if (fabs(step) <= (it == 0 ? 1e-7 : RootTolSoc) * (V.tpos ? fmin(u, 1.0 - u) : u)) {
                            conv = true;
                            break;
                        }
                    }
                    conv = conv && u >= 0.0 && (!V.tpos || u < 1.0);
                }
            }
            if (!conv) {  // full FP64 safeguarded search
                auto ev = [&](double uu, double& ph, double& dph, double& sc) {
                    double Sd = 0.0, S2 = 0.0;
                    const double m = V.mu(uu);
                    for (int i = g; i < nx; i += S) {
                        const double x = v[1 + i], wv = w[i];
                        const double r = 1.0 / (1.0 + m * wv);
                        const double term = wv * x * x * r * r;
                        Sd += term;
                        S2 += wv * term * r;
                    }
                    Sd = seg_sum<S>(Sd, gmask);
                    S2 = seg_sum<S>(S2, gmask);
                    V.psi(uu, sqrt(Sd), S2, ph, dph, sc);
                };
                u = soc_root<double>(ev, V.tpos, V.guess(t, nDinvx, nullptr), RootTolSoc, 4e-16, 200);
            }
            if (cache && g == 0) *cache = V.store(u);
            mu = V.mu(u);
        }
    }
    if (mu == 0.0) {  // case 1
        for (int i = g; i < nx; i += S) v[1 + i] = 0.0;
        __syncwarp(gmask);
        if (g == 0) v[0] = 0.0;
    } else if (mu > 0.0) {
        // y = (I + 2 lambda Dhat^{-2})^{-1} x ;  s = ||Dhat^{-1} y||
        double s = 0.0;
        for (int i = g; i < nx; i += S) {
            const double wv = w[i];
            const double y = v[1 + i] * rcp_refined(1.0 + mu * wv);
            s += wv * y * y;
            v[1 + i] = y;
        }
        s = seg_sum<S>(s, gmask);
        __syncwarp(gmask);
        if (g == 0) v[0] = sqrt(s);
    }
    __syncwarp(gmask);
    if (rot) {
        if (g == 0) {
            const double p = v[0], q = v[1];
            v[0] = (p + q) * r2;
            v[1] = (p - q) * r2;
        }
        __syncwarp(gmask);
    }
}

// Dhat = I (every weight 1): the textbook projection onto K_soc (Q K_soc for rot),
// (t + ||x||) / 2 (1, x / ||x||) when ||x|| > |t|, by a warp on memory (any dim).
static __device__ __noinline__ void soc_project_warp_unit(double* buf, int dim, bool rot) {
    const int lane = threadIdx.x & 31;
    const double r2 = 0.70710678118654752440;
    __syncwarp();
    if (rot && lane == 0) {
        const double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
    const double t = buf[0];
    double a = 0.0;
    for (int i = 1 + lane; i < dim; i += 32) a += buf[i] * buf[i];
    const double nx = sqrt(warp_sum(a));
    if (nx > fabs(t)) {
        const double top = 0.5 * (t + nx), sc = top / nx;
        for (int i = 1 + lane; i < dim; i += 32) buf[i] *= sc;
        __syncwarp();
        if (lane == 0) buf[0] = top;
    } else if (t <= 0.0) {  // in the polar cone (nx <= -t)
        for (int i = lane; i < dim; i += 32) buf[i] = 0.0;
    }
    __syncwarp();
    if (rot && lane == 0) {
        const double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
}

// Picks the register count for the block (dim - 1 <= 128, weights from wf); larger blocks
// use the FP64 memory-loop projection with weights formed from the scales d (kInv as there).
// Dhat = I takes the closed form.
template <bool kInv, typename WF>
__device__ __forceinline__ void soc_project_wf(double* buf, WF wf, const double* __restrict__ d, int dim, bool rot,
                                               float* cache, float* scr) {
    if (wf.unit()) {
        soc_project_warp_unit(buf, dim, rot);
        return;
    }
    const int nx = dim - 1;
    if (nx > 128) {
        if (scr) {
            if (rot) rsoc_project_warp_mp<kInv>(buf, wf, d, dim, cache, scr);
            else soc_project_warp_mp<kInv>(buf, wf, d, dim, cache, scr);
        } else {
            if (rot) rsoc_project_warp<kInv>(buf, d, dim, cache);
            else soc_project_warp<kInv>(buf, d, dim, cache);
        }
        return;
    }
    const int R = (nx + 31) / 32;
    if (rot) {
        if (R <= 1) rsoc_project_warp_fast<1>(buf, wf, dim, cache);
        else if (R == 2) rsoc_project_warp_fast<2>(buf, wf, dim, cache);
        else if (R == 3) rsoc_project_warp_fast<3>(buf, wf, dim, cache);
        else rsoc_project_warp_fast<4>(buf, wf, dim, cache);
    } else {
        if (R <= 1) soc_project_warp_fast<1>(buf, wf, dim, cache);
        else if (R == 2) soc_project_warp_fast<2>(buf, wf, dim, cache);
        else if (R == 3) soc_project_warp_fast<3>(buf, wf, dim, cache);
        else soc_project_warp_fast<4>(buf, wf, dim, cache);
    }
}

// Precomputed weights w (w[i] for x entry i, or all ones when null).  scr (may be null):
// 2 (dim - 1) floats of scratch for blocks beyond the registers (mixed precision there).
// wi (may be null): precomputed 1 / w[i], saving a division per entry.
template <bool kInv>
__device__ __forceinline__ void soc_project_any(double* buf, const double* __restrict__ w,
                                                const double* __restrict__ d, int dim, bool rot, float* cache,
                                                float* scr = nullptr, const double* __restrict__ wi = nullptr) {
    soc_project_wf<kInv>(buf, SocWeightsArray{w, wi}, d, dim, rot, cache, scr);
}

// Weights formed from the block's scales d (may be null: D = I) on the fly.
template <bool kInv>
__device__ __forceinline__ void soc_project_scaled(double* buf, const double* __restrict__ d, int dim, bool rot,
                                                   float* scr = nullptr) {
    soc_project_wf<kInv>(buf, SocWeightsScales<kInv>{d, d ? d[0] : 1.0}, d, dim, rot, nullptr, scr);
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

// Tolerances of the root search in each precision: the Newton step below which the
// iteration stops (its square is the remaining error) and the bracket collapse.
template <typename R> struct RootTol;
template <> struct RootTol<double> {
    static constexpr double newton = 1e-10, collapse = 4e-16;
};
template <> struct RootTol<float> {
    static constexpr float newton = 2e-6f, collapse = 2e-7f;
};

template <typename R>
struct ExpCase4T {
    R r0, s0, t0, dr, ds, tau, a3, a4, a4m1, w34, ldt, dir, lt0, lr0, ls0, ldr, lds;
    R dt3, dt4;  // d~ = rho (rho - 1) + tau^2 at rho = a3 and at rho = a4
    int anchor;  // 3 or 4: endpoint rho is measured from
    int slo;     // sign of F next to the anchor when the root is inside the interval
    bool dm;     // F finite at the anchor: affine in delta = e^L next to it
    int kind;    // 1: r0 > 0, s0 > 0;  2: r0 <= 0 < s0;  3: s0 <= 0 < r0
};
using ExpCase4 = ExpCase4T<double>;

// Everything known at one log-offset L (see exp_eval).
template <typename R>
struct ExpAt {
    R F, dF, rho, lsp, lrd, Fs;  // F, dF/dL, rho, log s_p, log r_d, size of the terms of F
    R A, B, dA, dB, drho;        // A, B of F and their derivatives, drho/dL
};

// At log-offset L (rho = anchor + dir e^L): rho, log s_p, log r_d (eq. sp_rd via
// eq. tilde_defs, the vanishing factor as log r0 + L or log s0 + L), and
// F(L) = lhs - rhs with the sign of h(rho) (eq. h_rho) decided in logs:
//   t0 >= 0: lhs = A, rhs = log(e^B + t0);  t0 < 0: lhs = log(e^A - t0), rhs = B,
//   A = log(d_t e^rho s_p), B = log(d_t^{-1} e^{-rho} r_d);  dF = dF/dL.
template <typename R>
__host__ __device__ __forceinline__ void exp_eval(const ExpCase4T<R>& e, R L, ExpAt<R>& o) {
    const R one = R(1), zero = R(0);
    const R delta = exp(L);
    R rho, lst, lrt, dlst, dlrt;  // logs of |s~|, |r~| and their derivatives
    int sst, srt;
    if (e.anchor == 4) {
        rho = e.a4 + e.dir * delta;
        lst = e.lr0 + L;
        dlst = one;
        sst = e.dir > zero ? 1 : -1;
        const R rt = (e.kind == 1) ? e.s0 * (e.w34 - e.dir * delta) : e.tau * e.r0 - rho * e.s0;
        lrt = log(fabs(rt));
        dlrt = (-e.s0 / rt) * e.dir * delta;
        srt = (rt > zero) - (rt < zero);
    } else {
        rho = e.a3 + e.dir * delta;
        lrt = e.ls0 + L;
        dlrt = one;
        srt = e.dir < zero ? 1 : -1;
        const R st = (e.kind == 1) ? e.r0 * (e.w34 + e.dir * delta) : e.s0 * e.tau - e.r0 + e.r0 * rho;
        lst = log(fabs(st));
        dlst = (e.r0 / st) * e.dir * delta;
        sst = (st > zero) - (st < zero);
    }
    // d~ = rho (rho - 1) + tau^2 at rho = anchor + dd, as d~(anchor) + dd (2 anchor - 1 + dd)
    const R dd = e.dir * delta;
    const R dt_ = e.anchor == 4 ? e.dt4 + dd * ((R(2) * e.a4m1 + one) + dd) : e.dt3 + dd * ((R(2) * e.a3 - one) + dd);
    const int sdt = (dt_ > zero) - (dt_ < zero);
    const R ldt_ = log(fabs(dt_));
    const R dldt = ((R(2) * rho - one) / dt_) * e.dir * delta;
    const R ninf = -R(INFINITY);
    const R lsp = (sst != 0 && sst == sdt) ? lst - e.ldr - ldt_ : ninf;
    const R lrd = (srt != 0 && srt == sdt) ? e.lds + lrt - ldt_ : ninf;
    const R A = e.ldt + rho + lsp;
    const R B = -e.ldt - rho + lrd;
    const R dA = e.dir * delta + dlst - dldt;
    const R dB = -e.dir * delta + dlrt - dldt;
    // log(e^a + e^b) = max + log1p(q), q = e^(min - max); the weight e^(a - lse) of a
    // comes from the same q, so each evaluation needs one exp and one log1p here
    auto lse_w = [ninf, one](R a, R b, R& wa) {
        if (a == ninf) { wa = R(0); return b; }
        if (b == ninf) { wa = one; return a; }
        const bool amax = a >= b;
        const R q = exp(amax ? b - a : a - b);
        wa = amax ? one / (one + q) : q / (one + q);
        return (amax ? a : b) + log1p(q);
    };
    if (e.t0 >= zero) {
        R wB = one;
        const R rhs = e.t0 > zero ? lse_w(B, e.lt0, wB) : B;
        if (B == ninf) wB = zero;
        o.F = A - rhs;
        o.dF = dA - wB * dB;
        o.Fs = fabs(A) + fabs(rhs);
    } else {
        R wA;
        const R lhs = lse_w(A, e.lt0, wA);
        o.F = lhs - B;
        o.dF = wA * dA - dB;
        o.Fs = fabs(lhs) + fabs(B);
    }
    o.rho = rho;
    o.lsp = lsp;
    o.lrd = lrd;
    o.A = A;
    o.B = B;
    o.dA = dA;
    o.dB = dB;
    o.drho = e.dir * delta;
}

template <typename R>
__host__ __device__ __forceinline__ void exp_F(const ExpCase4T<R>& e, R L, R& F, R& dF, R& rho_out, R& lsp_out,
                                               R& lrd_out, R& Fscale_out) {
    ExpAt<R> o;
    exp_eval(e, L, o);
    F = o.F;
    dF = o.dF;
    rho_out = o.rho;
    lsp_out = o.lsp;
    lrd_out = o.lrd;
    Fscale_out = o.Fs;
}

template <typename R>
__host__ __device__ __forceinline__ int exp_sign(const ExpCase4T<R>& e, R L, int& evals) {
    R F, dF, rho, lsp, lrd, Fs;
    exp_F(e, L, F, dF, rho, lsp, lrd, Fs);
    ++evals;
    return (F > R(0)) - (F < R(0));
}

// Lower end of the search.  First F at the anchor itself (offset 0, L = -inf) is
// evaluated: it is the endpoint value h(a4) or h(a3) of App. A.2 in log form.  When
// it is zero to working precision or has the other sign (v0 on the boundary of the
// polar cone or of the cone, up to rounding), the root is the endpoint: at_end is set
// and -inf returned.  When it is finite, F is analytic in the offset delta = e^L next
// to the anchor: F0 returns it and the search starts unbounded below, the anchor
// itself being the lower end.  Otherwise (F -> +-inf linearly in L; F0 returned
// infinite) step down from hi, doubling the distance (or going twice as far as the
// Newton point in L when that is farther) until F shows the sign it has there.
template <typename R>
__host__ __device__ __forceinline__ R exp_lower(const ExpCase4T<R>& e, R hi, int slo, int& evals, bool& at_end,
                                                R& F0) {
    const R ninf = -R(INFINITY);
    at_end = false;
    {
        R dF, rho, lsp, lrd, Fs;
        exp_F(e, ninf, F0, dF, rho, lsp, lrd, Fs);
        ++evals;
        const int s0 = (F0 > R(0)) - (F0 < R(0));
        const bool finite = fabs(F0) < R(INFINITY);
        const bool tiny = finite && fabs(F0) <= R(16) * RootTol<R>::collapse * Fs;
        if (F0 == F0 && (s0 != slo || tiny)) {
            at_end = true;
            return ninf;
        }
        if (finite) return ninf;
        F0 = R(INFINITY);
    }
    R step = R(1);
    for (int it = 0; it < 1100; ++it) {
        const R lo = hi - step;
        if (lo == ninf) return lo;
        R F, dF, rho, lsp, lrd, Fs;
        exp_F(e, lo, F, dF, rho, lsp, lrd, Fs);
        ++evals;
        const int s = (F > R(0)) - (F < R(0));
        if (s == slo || s == 0) return lo;
        // twice the distance, or past the Newton point by as much again when that is farther
        const R nd = F / dF;
        step = (nd > R(0) && nd < R(INFINITY)) ? fmax(R(2) * step, step + R(2) * nd) : R(2) * step;
    }
    return ninf;
}

// Safeguarded Newton for F(L) = 0 on (lo, hi); sign(F) at the lo end is slo.  F0 is
// F at the anchor (L = -inf) when finite.  Then F is affine in delta = e^L next to
// the anchor, and the first step is Newton's in delta, L <- L + log1p(-F / dF), exact
// for that model; without F0 (F linear in L there) it is Newton's in L.  Later steps
// take whichever of the two models better predicts F at the previous point (far from
// the anchor F can be affine in delta through rho, or linear in L through the logs).
// A step that leaves the bracket is replaced by the other model's step; while no
// lower end is known yet, by the farther of that and the secant in delta between the
// anchor and L (or a doubling downward extension); otherwise by bisection, which
// also replaces steps that fail to halve within a finite bracket.
template <typename R>
__host__ __device__ __forceinline__ R exp_newton(const ExpCase4T<R>& e, R lo, R hi, int slo, R L, R F0, int& evals) {
    const R one = R(1), ninf = -R(INFINITY);
    const bool dmodel = fabs(F0) < R(INFINITY);
    if (!(L > lo && L < hi)) L = (lo == ninf) ? hi - one : R(0.5) * (lo + hi);
    R ext = one, Lp = R(NAN), Fp = R(NAN), dx = R(INFINITY), dxold = R(INFINITY);
    for (int it = 0; it < 400; ++it) {
        R F, dF, rho, lsp, lrd, Fs;
        exp_F(e, L, F, dF, rho, lsp, lrd, Fs);
        ++evals;
        if (!(F == F)) break;  // NaN: both sides infinite, already at the limit
        // F zero to working precision: no other L in reach is a better root
        if (Fs < R(INFINITY) && fabs(F) <= R(4) * RootTol<R>::collapse * Fs) break;
        const int s = F > R(0) ? 1 : -1;
        if (s == slo) lo = L; else hi = L;
        const R st = -F / dF;
        // the model (affine in delta or in L) that better predicts the previous point
        bool dstep = dmodel;
        if (Lp == Lp) {
            const R errL = fabs(F + dF * (Lp - L) - Fp), errD = fabs(F + dF * expm1(Lp - L) - Fp);
            dstep = errD <= errL;
        }
        Lp = L;
        Fp = F;
        const R nD = st > -one ? L + log1p(st) : ninf, nL = L + st;
        R nl = dstep ? nD : nL;
        // a Newton step below RootTol::newton relative leaves an error of order its square
        // (L itself has just become an end of the bracket, so test this first)
        if (nl >= lo && nl <= hi && fabs(nl - L) <= RootTol<R>::newton * fmax(one, fabs(L))) {
            L = nl;
            break;
        }
        if (!(nl > lo && nl < hi)) {
            const R alt = dstep ? nL : nD;  // the other model's step
            if (lo != ninf) {
                nl = (alt > lo && alt < hi) ? alt : R(0.5) * (lo + hi);
            } else {
                // the root is below L: the farther of the other step and, with F0, the
                // secant in delta to the anchor (F0 / (F0 - F) in (0, 1)); else extend
                R cand = (alt > lo && alt < hi) ? alt : R(INFINITY);
                if (dmodel) cand = fmin(cand, L + log(F0 / (F0 - F)));
                if (cand < hi) {
                    nl = cand;
                } else {
                    nl = hi - ext;
                    ext *= R(2);
                }
            }
        }
        // inside a finite bracket, bisect when the steps do not halve (as in rtsafe)
        if (lo != ninf && fabs(nl - L) > R(0.5) * dxold) nl = R(0.5) * (lo + hi);
        dxold = dx;
        dx = fabs(nl - L);
        const bool done = !(nl > lo && nl < hi) || (hi - lo) <= RootTol<R>::collapse * fmax(one, fabs(hi));
        L = nl;
        if (done) break;
    }
    return L;
}

// ---------------------------------------------------------------------------
// Learned starting point of the case-4 search: a 9 -> 32 -> 32 -> 1 ReLU network of the
// direction of v0, the log ratios of the scales and the branch (kind, anchor) predicts
// the log-offset L of the root.  It only replaces the cold starting point: the bracket,
// the safeguarded Newton iteration and its stopping tests are unchanged, so the result
// is the plain search's.  Parameters (kExpMlpParams floats): W1[32][9], b1[32],
// W2[32][32], b2[32], w3[32], b3.
// ---------------------------------------------------------------------------
constexpr int kExpMlpIn = 9, kExpMlpHidden = 32;
constexpr int kExpMlpParams = kExpMlpHidden * kExpMlpIn + kExpMlpHidden + kExpMlpHidden * kExpMlpHidden +
                              kExpMlpHidden + kExpMlpHidden + 1;

template <typename R>
__host__ __device__ __forceinline__ void exp_mlp_features(const ExpCase4T<R>& e, float* f) {
    const float r = (float)e.r0, s = (float)e.s0, t = (float)e.t0;
    const float nv = sqrtf(r * r + s * s + t * t);
    const float inv = nv > 0.0f ? 1.0f / nv : 0.0f;
    f[0] = r * inv;
    f[1] = s * inv;
    f[2] = t * inv;
    f[3] = (float)(e.lds - e.ldr);
    f[4] = (float)(e.ldt - e.ldr);
    f[5] = (e.kind == 1 && e.anchor == 4) ? 1.0f : 0.0f;
    f[6] = (e.kind == 1 && e.anchor == 3) ? 1.0f : 0.0f;
    f[7] = e.kind == 2 ? 1.0f : 0.0f;
    f[8] = e.kind == 3 ? 1.0f : 0.0f;
}

__host__ __device__ __forceinline__ float exp_mlp_eval(const float* __restrict__ W, const float* f) {
    const float* W1 = W;
    const float* b1 = W1 + kExpMlpHidden * kExpMlpIn;
    const float* W2 = b1 + kExpMlpHidden;
    const float* b2 = W2 + kExpMlpHidden * kExpMlpHidden;
    const float* w3 = b2 + kExpMlpHidden;
    const float b3 = w3[kExpMlpHidden];
    float h1[kExpMlpHidden];
#pragma unroll 4
    for (int i = 0; i < kExpMlpHidden; ++i) {
        float a = b1[i];
#pragma unroll
        for (int j = 0; j < kExpMlpIn; ++j) a = fmaf(W1[i * kExpMlpIn + j], f[j], a);
        h1[i] = fmaxf(a, 0.0f);
    }
    float y = b3;
#pragma unroll 2
    for (int i = 0; i < kExpMlpHidden; ++i) {
        float a = b2[i];
#pragma unroll
        for (int j = 0; j < kExpMlpHidden; ++j) a = fmaf(W2[i * kExpMlpHidden + j], h1[j], a);
        y = fmaf(w3[i], fmaxf(a, 0.0f), y);
    }
    return y;
}

template <typename R>
__host__ __device__ __forceinline__ R exp_mlp_guess(const ExpCase4T<R>& e, const float* mlp, R guess) {
    if (!mlp || guess == guess) return guess;  // no network, or a cached root to start from
    float f[kExpMlpIn];
    exp_mlp_features(e, f);
    return (R)exp_mlp_eval(mlp, f);
}

// Case 4 of Theorem 3 for the prepared e (logs and a3, a4 filled in): chooses the
// interval branch of eq. lrho_urho and the anchor, and returns the log-offset L of
// the root of h.  Returns false when the interval is empty by rounding.
template <typename R>
__host__ __device__ __forceinline__ bool exp_case4_solve(ExpCase4T<R>& e, R guess, R& L, int& evals,
                                                         const float* mlp = nullptr) {
    const R zero = R(0), one = R(1);
    if (e.r0 > zero && e.s0 > zero) {
        e.kind = 1;
        const R W = fabs(e.w34);
        if (!(W > zero)) return false;
        const R Lh = log(R(0.5) * W);
        e.anchor = 4;
        e.dir = e.w34 > zero ? one : -one;
        const int sm = exp_sign(e, Lh, evals);
        e.slo = -1;
        e.dm = false;
        if (sm == 0) {
            L = Lh;
            return true;
        }
        if (sm < 0) {  // h(mid) < 0 < h(a3): root in the half next to a3
            e.anchor = 3;
            e.dir = -e.dir;
        }
        const int slo = sm > 0 ? -1 : +1;
        e.slo = slo;
        bool at_end;
        R F0;
        const R lo = exp_lower(e, Lh, slo, evals, at_end, F0);
        e.dm = fabs(F0) < R(INFINITY);
        L = at_end ? lo : exp_newton(e, lo, Lh, slo, exp_mlp_guess(e, mlp, guess), F0, evals);
    } else if (e.s0 > zero) {  // r0 <= 0: (-inf, a3)
        e.kind = 2; e.anchor = 3; e.dir = -one; e.slo = +1;
        R hi = zero;
        for (int it = 0; it < 8 && exp_sign(e, hi, evals) > 0 && hi < R(60); ++it) hi = R(2) * hi + one;
        bool at_end;
        R F0;
        const R lo = exp_lower(e, hi, +1, evals, at_end, F0);
        e.dm = fabs(F0) < R(INFINITY);
        L = at_end ? lo : exp_newton(e, lo, hi, +1, exp_mlp_guess(e, mlp, guess), F0, evals);
    } else {  // s0 <= 0 < r0: (a4, inf)
        e.kind = 3; e.anchor = 4; e.dir = one; e.slo = -1;
        R hi = zero;
        for (int it = 0; it < 8 && exp_sign(e, hi, evals) < 0 && hi < R(60); ++it) hi = R(2) * hi + one;
        bool at_end;
        R F0;
        const R lo = exp_lower(e, hi, -1, evals, at_end, F0);
        e.dm = fabs(F0) < R(INFINITY);
        L = at_end ? lo : exp_newton(e, lo, hi, -1, exp_mlp_guess(e, mlp, guess), F0, evals);
    }
    return true;
}

// Error-free transformations (Dekker 1971; Knuth, TAOCP vol. 2): a * b = p + e and
// a + b = s + e exactly in binary floating point.
__host__ __device__ __forceinline__ double two_prod(double a, double b, double& e) {
    const double p = a * b;
    e = fma(a, b, -p);
    return p;
}
__host__ __device__ __forceinline__ double two_sum(double a, double b, double& e) {
    const double s = a + b, bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

// Theorem 3's quantities at the ends of the case-4 interval (a3, a4 of eq. lrho_urho and
// d~(rho) = rho (rho - 1) + tau^2, tau = ds / dr), in FP64.  With
// N = tau (r0^2 + s0^2) - r0 s0 they satisfy the exact identities
//     a3 - a4 = N / (r0 s0),   d~(a3) = tau N / s0^2,   d~(a4) = tau N / r0^2.
// For r0, s0 > 0 the difference in N cancels exactly where the interval is narrow or d~ is
// small on it; N is formed from error-free products and sums of r0, s0 scaled by one power
// of two (exact), so it keeps the digits that a3 - a4 and rho (rho - 1) + tau^2 would lose.
struct ExpEnds {
    double a3, a4, a4m1, w34, dt3, dt4;
};
__host__ __device__ __forceinline__ ExpEnds exp_ends(double r0, double s0, double dr, double ds) {
    ExpEnds o;
    const double tau = ds / dr;
    o.a3 = (s0 > 0.0) ? (r0 * ds) / (s0 * dr) : 0.0;
    o.a4m1 = (r0 > 0.0) ? -(s0 * ds) / (r0 * dr) : -1.0;
    o.a4 = (r0 > 0.0) ? 1.0 + o.a4m1 : 0.0;
    const double mx = fmax(fabs(r0), fabs(s0));
    int k = 0;
    frexp(mx, &k);
    const double r = ldexp(r0, -k), s = ldexp(s0, -k);
    double e1, e2, eS, eq, e3, eD;
    const double p1 = two_prod(r, r, e1), p2 = two_prod(s, s, e2);
    const double S = two_sum(p1, p2, eS);
    const double q = two_prod(tau, S, eq);
    const double p3 = two_prod(r, s, e3);
    const double Dq = two_sum(q, -p3, eD);
    const double N = Dq + (eD + eq + tau * (eS + e1 + e2) - e3);  // N / 2^(2k)
    o.w34 = (r0 > 0.0 && s0 > 0.0) ? N / (r * s) : o.a3 - o.a4;
    o.dt3 = s0 > 0.0 ? tau * N / (s * s) : 0.0;
    o.dt4 = r0 > 0.0 ? tau * N / (r * r) : 0.0;
    return o;
}

// Fills the case-4 data of v0 = (r0, s0, t0), D = diag(dr, ds, dt), in precision R
// from values given in double (logs of the scales and the endpoint quantities passed in).
// Logarithms of the data used by the log-domain evaluation (exp_eval); anchor 3 or 4 (0:
// both): the evaluation next to that endpoint reads log s0 or log r0 only.
template <typename R>
__host__ __device__ __forceinline__ void exp_case4_logs(ExpCase4T<R>& e, double r0, double s0, double t0, int anchor) {
    const R ninf = -R(INFINITY);
    e.lr0 = (anchor != 3 && r0 > 0.0) ? R(log(R(r0))) : ninf;
    e.ls0 = (anchor != 4 && s0 > 0.0) ? R(log(R(s0))) : ninf;
    e.lt0 = t0 > 0.0 ? R(log(R(t0))) : (t0 < 0.0 ? R(log(R(-t0))) : ninf);
}

// (logs = false: without the logarithms of the data; exp_case4_logs adds them)
template <typename R>
__host__ __device__ __forceinline__ void exp_case4_setup(ExpCase4T<R>& e, double r0, double s0, double t0, double dr,
                                                         double ds, R ldr, R lds, R ldt, const ExpEnds& q,
                                                         int anchor = 0, bool logs = true) {
    e.r0 = R(r0); e.s0 = R(s0); e.t0 = R(t0); e.dr = R(dr); e.ds = R(ds);
    e.tau = R(ds / dr);
    e.ldt = ldt; e.ldr = ldr; e.lds = lds;
    if (logs) exp_case4_logs(e, r0, s0, t0, anchor);
    e.a3 = R(q.a3);
    e.a4 = R(q.a4);
    e.a4m1 = R(q.a4m1);
    e.w34 = R(q.w34);
    e.dt3 = R(q.dt3);
    e.dt4 = R(q.dt4);
}

// Result of case 4 at the root L (eq. vpvd_defn with v0 = v_p + v_d, eq. diagonal_moreau):
// per coordinate the smaller part from its formula, v_p = v0 - v_d when v_d is larger.
__host__ __device__ __forceinline__ void exp_case4_output(const ExpCase4& e, double L, double r0, double s0, double t0,
                                                          double dr, double ds, double* out) {
    double F, dF, rho, lsp, lrd, Fs;
    exp_F(e, L, F, dF, rho, lsp, lrd, Fs);
    const double sp = exp(lsp), rd = exp(lrd);
    const double vp[3] = {dr * rho * sp, ds * sp, exp(e.ldt + rho + lsp)};
    const double vd[3] = {rd / dr, (1.0 - rho) * rd / ds, -exp(-e.ldt - rho + lrd)};
    const double v0[3] = {r0, s0, t0};
#pragma unroll
    for (int k = 0; k < 2; ++k) out[k] = fabs(vp[k]) <= fabs(vd[k]) ? vp[k] : v0[k] - vd[k];
    // t entry: h(rho) = 0 says e^A - e^B = t0, so v_d is the smaller part when t0 >= 0
    out[2] = t0 >= 0.0 ? t0 - vd[2] : vp[2];
}

// The result of case 4 at the root L* = L + s from the values at L (s small): v_p and
// v_d of eq. vpvd_defn to first order in s (the error is of order s^2), then the same
// per-coordinate choice as exp_case4_output.
__host__ __device__ __forceinline__ void exp_case4_output_lin(const ExpAt<double>& a, double s, double r0, double s0,
                                                              double t0, double dr, double ds, double* out) {
    const double sp = exp(a.lsp), rd = exp(a.lrd), eA = exp(a.A), eB = exp(a.B);
    const double dlsp = a.dA - a.drho, dlrd = a.dB + a.drho;  // A = ldt + rho + lsp, B = -ldt - rho + lrd
    const double dsp = sp > 0.0 ? sp * dlsp : 0.0, drd = rd > 0.0 ? rd * dlrd : 0.0;
    const double vp[3] = {dr * (a.rho * sp + s * (a.drho * sp + a.rho * dsp)), ds * (sp + s * dsp),
                          eA > 0.0 ? eA * (1.0 + s * a.dA) : 0.0};
    const double vd[3] = {(rd + s * drd) / dr, ((1.0 - a.rho) * rd + s * ((1.0 - a.rho) * drd - a.drho * rd)) / ds,
                          eB > 0.0 ? -eB * (1.0 + s * a.dB) : 0.0};
    const double v0[3] = {r0, s0, t0};
#pragma unroll
    for (int k = 0; k < 2; ++k) out[k] = fabs(vp[k]) <= fabs(vd[k]) ? vp[k] : v0[k] - vd[k];
    out[2] = t0 >= 0.0 ? t0 - vd[2] : vp[2];
}

// Projection of v0 onto D K_exp, D = diag(dr, ds, dt) (Theorem 3), all in FP64 with
// the safeguarded search.  L_cache (may be null): last log-offset of this cone, used
// as the Newton start and updated.
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
    exp_case4_setup(e, r0, s0, t0, dr, ds, log(dr), log(ds), log(dt), exp_ends(r0, s0, dr, ds));
    const double guess = L_cache ? *L_cache : NAN;
    double L;
    if (!exp_case4_solve(e, guess, L, evals)) { out[0] = 0.0; out[1] = 0.0; out[2] = 0.0; return; }
    if (L_cache) *L_cache = L;
    if (evals_out) *evals_out = evals;
    exp_case4_output(e, L, r0, s0, t0, dr, ds, out);
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

// ---------------------------------------------------------------------------
// Exponential cone, mixed precision: the same projection with the case tests
// screened in FP32 (FP64 only when the FP32 margin is too small), the root of h
// found in FP32 and polished by at most three FP64 Newton steps; anything the
// FP32 pass cannot settle (values outside the FP32 range, no convergence) falls
// back to exp_project.  FP64 transcendentals cost ~50x their FP32 forms on GB300.
// ---------------------------------------------------------------------------
// +1: surely in K_exp, -1: surely not, 0: undecided at FP32 precision
__host__ __device__ __forceinline__ int kexp_screen32(float r, float s, float t) {
    if (!(fabsf(r) < 1e30f && fabsf(s) < 1e30f && fabsf(t) < 1e30f)) return 0;
    if (s > 1e-30f) {
        if (t < 0.0f) return -1;
        if (!(t > 1e-30f)) return 0;
        const float lhs = logf(t) - logf(s), rhs = r / s;
        const float tol = 1e-4f * (1.0f + fabsf(lhs) + fabsf(rhs));
        return lhs - rhs > tol ? 1 : (lhs - rhs < -tol ? -1 : 0);
    }
    return s < -1e-30f ? -1 : 0;
}

// +1: surely in K_exp^*, -1: surely not, 0: undecided
__host__ __device__ __forceinline__ int kexpdual_screen32(float r, float s, float t) {
    if (!(fabsf(r) < 1e30f && fabsf(s) < 1e30f && fabsf(t) < 1e30f)) return 0;
    if (r < -1e-30f) {
        if (t < 0.0f) return -1;
        if (!(t > 1e-30f)) return 0;
        const float lhs = 1.0f + logf(t) - logf(-r), rhs = s / r;
        const float tol = 1e-4f * (1.0f + fabsf(lhs) + fabsf(rhs));
        return lhs - rhs > tol ? 1 : (lhs - rhs < -tol ? -1 : 0);
    }
    return r > 1e-30f ? -1 : 0;
}

// Points outside D K_exp (or its polar (D K_exp)° = D^-1 K_exp°) by less than the
// membership tests resolve: case 4's root then sits at the end of its interval, where the
// search converges slowly (dual iterates on the boundary of the dual cone at the solution
// make many such points).  By Moreau, returning v (or 0) errs by dist(v, D K_exp) (or
// dist(v, polar)); each function bounds it by the distance to a point of the set that
// differs from v only in t, with t moved past the computed boundary by a slack covering
// the rounding of the exponent and of exp.  INFINITY where that point does not exist.
template <typename R> struct ExpGapEps;
template <> struct ExpGapEps<double> { static constexpr double eps = 2.220446049250313e-16; };
template <> struct ExpGapEps<float> { static constexpr float eps = 1.1920929e-7f; };
template <typename R>
__host__ __device__ __forceinline__ R exp_gap_to_cone(R r0, R s0, R t0, R dr, R ds, R dt) {
    const R s = s0 / ds, q = (r0 / dr) / s;  // K_exp: s > 0, t >= s e^(r/s)
    if (!(s > R(0)) || !(fabs(q) < R(80))) return R(INFINITY);
    const R tb = dt * s * exp(q);
    const R tq = tb * (R(1) + (R(8) + R(2) * fabs(q)) * ExpGapEps<R>::eps);
    return t0 >= tq ? R(0) : tq - t0;
}
template <typename R>
__host__ __device__ __forceinline__ R exp_gap_to_polar(R r0, R s0, R t0, R dr, R ds, R dt) {
    const R a = dr * r0, q = ds * s0 / a - R(1);  // K_exp°: a > 0, c <= -a e^(b/a - 1)
    if (!(a > R(0)) || !(fabs(q) < R(80))) return R(INFINITY);
    const R tb = -a * exp(q) / dt;
    const R tq = tb * (R(1) + (R(8) + R(2) * fabs(q + R(1))) * ExpGapEps<R>::eps);
    return t0 <= tq ? R(0) : t0 - tq;
}

// ---------------------------------------------------------------------------
// Case-4 finish in the linear domain.  Away from the extremes (|rho| < 600, offset from the
// anchor above 1e-250) h of eq. h_rho and its derivative are formed directly from
// s~, r~ (eq. tilde_defs) and d~ at the offset delta of rho from the anchor:
//   h = d_t e^rho s_p - d_t^{-1} e^{-rho} r_d - t0,  s_p = s~ / (d_r d~),  r_d = d_s r~ / d~,
//   ds_p/drho = (r0 / d_r - s_p (2 rho - 1)) / d~,  dr_d/drho = (-d_s s0 - r_d (2 rho - 1)) / d~,
// (s~ = r0 (rho - a4) and r~ = s0 (a3 - rho) are affine in rho), one FP64 exp and three
// divisions per evaluation, where the log-domain evaluation needs five transcendentals.
// Newton's method in delta from the FP32 root; once a step is below 1e-8 min(1, delta) the
// result follows from the values at the last point to first order (error of order the
// step squared), per coordinate the smaller part as in exp_case4_output.
// ---------------------------------------------------------------------------
struct ExpLin {
    double rho, E, iE, sp, rd, sp_r, rd_r, h, dh;  // E = d_t e^rho, iE = 1 / E, *_r: d/drho
};

__host__ __device__ __forceinline__ bool exp_lin_eval(const ExpCase4& e, double idr, double delta, ExpLin& o) {
    const double dd = e.dir * delta;  // rho - anchor
    double rho, st, rt;
    if (e.anchor == 4) {
        rho = e.a4 + dd;
        st = e.r0 * dd;
        rt = (e.kind == 1) ? e.s0 * (e.w34 - dd) : e.tau * e.r0 - rho * e.s0;
    } else {
        rho = e.a3 + dd;
        rt = -e.s0 * dd;
        st = (e.kind == 1) ? e.r0 * (e.w34 + dd) : e.s0 * e.tau - e.r0 + e.r0 * rho;
    }
    const double dt_ = e.anchor == 4 ? e.dt4 + dd * ((2.0 * e.a4m1 + 1.0) + dd) : e.dt3 + dd * ((2.0 * e.a3 - 1.0) + dd);
    const double id = 1.0 / dt_;
    o.rho = rho;
    o.sp = st * id * idr;
    o.rd = e.ds * rt * id;
    o.E = exp(e.ldt + rho);
    o.iE = 1.0 / o.E;
    const double g = 2.0 * rho - 1.0;
    o.sp_r = (e.r0 * idr - o.sp * g) * id;
    o.rd_r = (-e.ds * e.s0 - o.rd * g) * id;
    o.h = o.E * o.sp - o.iE * o.rd - e.t0;
    o.dh = e.dir * (o.E * (o.sp + o.sp_r) + o.iE * (o.rd - o.rd_r));
    return o.sp > 0.0 && o.rd > 0.0 && o.E > 0.0 && o.E < INFINITY && isfinite(o.h) && isfinite(o.dh) && o.dh != 0.0;
}

// delta0: offset of the FP32 root; hi: upper end of the offsets (the half interval for
// r0, s0 > 0, else infinite).  Returns false when the point leaves (0, hi) or does not settle.
__host__ __device__ __forceinline__ bool exp_lin_polish(const ExpCase4& e, double delta0, double hi, double r0, double s0,
                                                        double t0, double dr, double ds, double* out, double* L_out,
                                                        int* ev) {
    const double idr = 1.0 / dr;
    double delta = delta0;
    for (int it = 0; it < 4; ++it) {
        ExpLin a;
        if (!exp_lin_eval(e, idr, delta, a)) return false;
        if (ev) ev[1] += 1;
        const double s = -a.h / a.dh;
        if (!isfinite(s)) return false;
        if (fabs(s) <= 1e-8 * fmin(1.0, delta)) {
            const double ds_ = e.dir * s;  // change of rho
            const double rho = a.rho + ds_;
            const double sp = a.sp + ds_ * a.sp_r, rd = a.rd + ds_ * a.rd_r;
            const double E = a.E * (1.0 + ds_), iE = a.iE * (1.0 - ds_);
            const double vp[3] = {dr * rho * sp, ds * sp, E * sp};
            const double vd[3] = {rd * idr, (1.0 - rho) * rd / ds, -iE * rd};
            const double v0[3] = {r0, s0, t0};
#pragma unroll
            for (int k = 0; k < 2; ++k) out[k] = fabs(vp[k]) <= fabs(vd[k]) ? vp[k] : v0[k] - vd[k];
            out[2] = t0 >= 0.0 ? t0 - vd[2] : vp[2];
            if (L_out) {  // the next search's starting point: FP32 precision is enough
                const double d1 = delta + s;
                *L_out = d1 > 1e-30 ? (double)logf((float)d1) : log(d1);
            }
            return true;
        }
        const double nd = delta + s;
        if (!(nd > 0.0 && nd < hi)) return false;
        delta = nd;
    }
    return false;
}

// Projection onto D K_exp with precomputed logs of the scales (lg[0..2] = log dr, ds, dt).
// L_cache (may be null): FP32 copy of the last log-offset of this cone.  mlp (may be
// null): device weights of the learned starting point, used when there is no cached
// root.  ev (may be null): ev[0] += FP32 and ev[1] += FP64 evaluations of h.
__host__ __device__ inline void exp_project_fast(double r0, double s0, double t0, double dr, double ds, double dt,
                                                 const double* lg, double* out, float* L_cache,
                                                 const float* mlp = nullptr, int* ev = nullptr) {
    // cases 1-3, screened in FP32; a point the FP64 test puts outside after an uncertain
    // screen is taken as inside when it is within 1e-14 |v| of the set (see exp_gap_to_cone)
    auto near = [&]() { return 1e-14 * sqrt(r0 * r0 + s0 * s0 + t0 * t0); };
    int c1 = kexp_screen32((float)r0 / (float)dr, (float)s0 / (float)ds, (float)t0 / (float)dt);
    if (c1 == 0) c1 = (in_kexp(r0 / dr, s0 / ds, t0 / dt) || exp_gap_to_cone(r0, s0, t0, dr, ds, dt) <= near()) ? 1 : -1;
    if (c1 > 0) { out[0] = r0; out[1] = s0; out[2] = t0; return; }
    int c2 = kexpdual_screen32(-(float)dr * (float)r0, -(float)ds * (float)s0, -(float)dt * (float)t0);
    if (c2 == 0)
        c2 = (in_kexp_dual(-dr * r0, -ds * s0, -dt * t0) || exp_gap_to_polar(r0, s0, t0, dr, ds, dt) <= near()) ? 1
                                                                                                              : -1;
    if (c2 > 0) { out[0] = 0.0; out[1] = 0.0; out[2] = 0.0; return; }
    if (r0 <= 0.0 && s0 <= 0.0) { out[0] = r0; out[1] = 0.0; out[2] = t0 > 0.0 ? t0 : 0.0; return; }
    // case 4: root in FP32
    const bool in_range = fabs(r0) < 1e30 && fabs(s0) < 1e30 && fabs(t0) < 1e30 && (r0 == 0.0 || fabs(r0) > 1e-30) &&
                          (s0 == 0.0 || fabs(s0) > 1e-30) && (t0 == 0.0 || fabs(t0) > 1e-30);
    ExpCase4T<float> ef;
    ExpEnds ends;
    float Lf = 0.0f;
    int evals = 0;
    bool ok = in_range;
    if (ok) {
        ends = exp_ends(r0, s0, dr, ds);
        exp_case4_setup(ef, r0, s0, t0, dr, ds, (float)lg[0], (float)lg[1], (float)lg[2], ends);
        // rho (rho - 1) + tau^2 must stay finite in FP32 over the search
        ok = fabsf(ef.a3) < 1e15f && fabsf(ef.a4) < 1e15f && fabsf(ef.tau) < 1e15f &&
             exp_case4_solve(ef, L_cache ? *L_cache : NAN, Lf, evals, mlp) &&
             !(Lf != Lf) && Lf < INFINITY;
    }
    if (ev) ev[0] += evals;
    if (ok && Lf == -INFINITY) {
        // FP32 puts the root at the anchor.  In FP64, F at a tiny offset delta_z = e^-200
        // is F at the anchor to all digits and dF = c delta_z, c = dF/ddelta there: the
        // anchor stands when F has the sign beyond the root or is zero to precision;
        // otherwise the root next to it is delta = -F / c, polished by Newton in delta.
        ExpCase4 e;
        exp_case4_setup(e, r0, s0, t0, dr, ds, lg[0], lg[1], lg[2], ends, ef.anchor);
        e.kind = ef.kind;
        e.anchor = ef.anchor;
        e.dir = (double)ef.dir;
        const double Lz = -200.0;
        double F, dF, rho, lsp, lrd, Fs;
        exp_F(e, Lz, F, dF, rho, lsp, lrd, Fs);
        if (ev) ev[1] += 1;
        const int sF = (F > 0.0) - (F < 0.0);
        if (F == F && Fs < INFINITY && (sF != ef.slo || fabs(F) <= 16.0 * RootTol<double>::collapse * Fs)) {
            if (L_cache) *L_cache = -INFINITY;
            exp_case4_output(e, -INFINITY, r0, s0, t0, dr, ds, out);
            if (ev) ev[1] += 1;
            return;
        }
        bool conv = false;
        double L = Lz;
        if (F == F && fabs(F) < INFINITY && fabs(dF) < 1e-60 && -F / dF > 0.0) {
            L = Lz + log(-F / dF);
            for (int it = 0; it < 4 && !conv; ++it) {
                exp_F(e, L, F, dF, rho, lsp, lrd, Fs);
                if (ev) ev[1] += 1;
                if (Fs < INFINITY && fabs(F) <= 4.0 * RootTol<double>::collapse * Fs) { conv = true; break; }
                const double st = -F / dF;
                if (!(st > -1.0) || !isfinite(st)) break;
                const double step = log1p(st);
                L += step;
                conv = fabs(step) <= RootTol<double>::newton * fmax(1.0, fabs(L));
            }
        }
        if (conv) {
            if (L_cache) *L_cache = (float)L;
            exp_case4_output(e, L, r0, s0, t0, dr, ds, out);
            if (ev) ev[1] += 1;
            return;
        }
        ok = false;
    }
    if (ok) {
        // FP64 polish from the FP32 root, same branch and anchor
        ExpCase4 e;
        exp_case4_setup(e, r0, s0, t0, dr, ds, lg[0], lg[1], lg[2], ends, ef.anchor, false);
        e.kind = ef.kind;
        e.anchor = ef.anchor;
        e.dir = (double)ef.dir;
        if (Lf > -575.0f) {  // linear domain when rho and the offset are moderate
            const double delta0 = Lf > -80.0f ? (double)expf(Lf) : exp((double)Lf);  // a starting point
            const double rho0 = (e.anchor == 4 ? e.a4 : e.a3) + e.dir * delta0;
            const double hi = e.kind == 1 ? 0.5 * fabs(e.w34) : INFINITY;
            double Lout;
            if (fabs(rho0) < 600.0 && exp_lin_polish(e, delta0, hi, r0, s0, t0, dr, ds, out, &Lout, ev)) {
                if (L_cache) *L_cache = (float)Lout;
                return;
            }
        }
        exp_case4_logs(e, r0, s0, t0, ef.anchor);
        // Newton steps s until one is small enough that the result at L + s follows from
        // the values at L to first order (error of order s^2)
        double L = (double)Lf;
        for (int it = 0; it < 3; ++it) {
            ExpAt<double> a;
            exp_eval(e, L, a);
            if (ev) ev[1] += 1;
            double st = 0.0;
            if (!(a.Fs < INFINITY && fabs(a.F) <= 4.0 * RootTol<double>::collapse * a.Fs)) {
                st = -a.F / a.dF;  // Newton in delta next to the anchor (see exp_newton), else in L
                st = ef.dm ? (st > -1.0 ? log1p(st) : NAN) : st;
                if (!isfinite(st)) break;
            }
            // the neglected second-order terms grow with (step x the log-derivatives of the
            // output terms A, B, log s_p, log r_d), which reach |rho| when rho is far from 0
            const double dmax = fmax(fmax(1.0, fmax(fabs(a.dA), fabs(a.dB))),
                                     fmax(fabs(a.dA - a.drho), fabs(a.dB + a.drho)));
            if (fabs(st) * dmax <= 1e-8) {  // (1e-7 left errors near 1e-12 on stressed inputs)
                if (L_cache) *L_cache = (float)(L + st);
                exp_case4_output_lin(a, st, r0, s0, t0, dr, ds, out);
                return;
            }
            L += st;
        }
    }
    double Lc = L_cache ? (double)*L_cache : NAN;
    int e64 = 0;
    exp_project(r0, s0, t0, dr, ds, dt, out, &Lc, &e64);
    if (ev) ev[1] += e64 + 1;
    if (L_cache) *L_cache = (float)Lc;
}

// Projection onto D^{-1} K_exp^* (Remark of App. A.2) with the mixed-precision search.
__host__ __device__ __forceinline__ void exp_dual_project_fast(double r, double s, double t, double dr, double ds,
                                                               double dt, const double* lg, double* out,
                                                               float* L_cache, const float* mlp = nullptr) {
    double p[3];
    exp_project_fast(-r, -s, -t, dr, ds, dt, lg, p, L_cache, mlp);
    out[0] = r + p[0];
    out[1] = s + p[1];
    out[2] = t + p[2];
}

}  // namespace pdcs

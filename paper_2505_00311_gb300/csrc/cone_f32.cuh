// cone_f32.cuh -- FP32 cone projections for the FP32-iterate mode.
//
// Same case analysis as cone_math.cuh (Theorem 1 for SOC / RSOC, Theorem 3 and the
// Remark of App. A.2 for exp and exp*), carried out in FP32 only: no FP64 polish.
// Used by the dual update while the iterates are FP32; the restart / termination
// checks always project in FP64 (cone_math.cuh).
#pragma once
#include "cone_math.cuh"

namespace pdcs {

// ---------------------------------------------------------------------------
// SOC, entries in registers (dim - 1 <= 32 R), weights w_i = dhat_i^{-2}
// ---------------------------------------------------------------------------
template <int R>
__device__ void soc_project_warp_f32(float* buf, const float* __restrict__ w, int dim, float* cache) {
    const int lane = threadIdx.x & 31;
    const int nx = dim - 1;
    const float t = buf[0];
    float xr[R], wr[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int i = lane + 32 * k;
        const bool in = i < nx;
        xr[k] = in ? buf[1 + i] : 0.0f;
        wr[k] = in ? w[i] : 1.0f;
    }
    float a = 0.0f, b = 0.0f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const float x2 = xr[k] * xr[k];
        a += x2 / wr[k];
        b += wr[k] * x2;
    }
    a = warp_sum_f(a);
    b = warp_sum_f(b);
    const float nDx = sqrtf(a), nDinvx = sqrtf(b);
    __syncwarp();
    if (t <= 0.0f && nDx <= -t) {  // case 1
#pragma unroll
        for (int k = 0; k < R; ++k) if (lane + 32 * k < nx) buf[1 + lane + 32 * k] = 0.0f;
        if (lane == 0) buf[0] = 0.0f;
        __syncwarp();
        return;
    }
    if (nDinvx <= t) return;  // case 2
    float mu = 1.0f;          // 2 lambda; case 3
    if (t != 0.0f) {          // case 4: search variable as in cone_math.cuh
        bool known, near = t > 0.0f && soc_cached_near(cache, known);
        if (t > 0.0f && !known) {  // sign of psi at mu = 1/2
            float S = 0.0f;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const float r = __frcp_rn(1.0f + 0.5f * wr[k]);
                S += wr[k] * xr[k] * xr[k] * r * r;
            }
            near = 0.5f * sqrtf(warp_sum_f(S)) < t;
        }
        const SocVar<float> V(t, near);
        auto ev = [&](float u, float& ph, float& dph, float& sc) {
            float S = 0.0f, S2 = 0.0f;
            const float m = V.mu(u);
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const float r = __frcp_rn(1.0f + m * wr[k]);
                const float term = wr[k] * xr[k] * xr[k] * r * r;
                S += term;
                S2 += wr[k] * term * r;
            }
            S = warp_sum_f(S);
            S2 = warp_sum_f(S2);
            V.psi(u, sqrtf(S), S2, ph, dph, sc);
        };
        const float u = soc_root<float>(ev, V.tpos, V.guess(t, nDinvx, cache), 2e-6f, 2e-7f, 100);
        if (cache && lane == 0) *cache = V.store(u);
        mu = V.mu(u);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const float y = xr[k] / (1.0f + mu * wr[k]);
        s += wr[k] * y * y;
        if (lane + 32 * k < nx) buf[1 + lane + 32 * k] = y;
    }
    s = warp_sum_f(s);
    __syncwarp();
    if (lane == 0) buf[0] = sqrtf(s);
    __syncwarp();
}

// SOC / RSOC of any size from an FP32 buffer: registers up to dim 129; larger blocks
// go through the FP64 scratch `tmp` (same rows) and the FP64 memory-loop projection
// onto Dr^{-1} K (kInv, scales dr).
__device__ __forceinline__ void soc_project_any_f32(float* buf, const float* __restrict__ w32, double* tmp,
                                                    const double* __restrict__ dr, int dim, bool rot,
                                                    float* cache) {
    const int lane = threadIdx.x & 31;
    const float r2 = 0.70710678118654752440f;
    const int nx = dim - 1;
    if (nx > 128) {
        for (int i = lane; i < dim; i += 32) tmp[i] = (double)buf[i];
        __syncwarp();
        if (rot) rsoc_project_warp<true>(tmp, dr, dim, nullptr);
        else soc_project_warp<true>(tmp, dr, dim, nullptr);
        for (int i = lane; i < dim; i += 32) buf[i] = (float)tmp[i];
        __syncwarp();
        return;
    }
    if (rot && lane == 0) {
        const float p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
    const int R = (nx + 31) / 32;
    if (R <= 1) soc_project_warp_f32<1>(buf, w32, dim, cache);
    else if (R == 2) soc_project_warp_f32<2>(buf, w32, dim, cache);
    else if (R == 3) soc_project_warp_f32<3>(buf, w32, dim, cache);
    else soc_project_warp_f32<4>(buf, w32, dim, cache);
    if (rot && lane == 0) {
        const float p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Exponential cone in FP32 (Theorem 3), log scales given
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool in_kexp_f(float r, float s, float t) {
    if (s > 0.0f) return t > 0.0f && (logf(t) - logf(s)) >= r / s;
    if (s == 0.0f) return t >= 0.0f && r <= 0.0f;
    return false;
}

__device__ __forceinline__ bool in_kexp_dual_f(float r, float s, float t) {
    if (r < 0.0f) return t > 0.0f && (1.0f + logf(t) - logf(-r)) >= s / r;
    if (r == 0.0f) return s >= 0.0f && t >= 0.0f;
    return false;
}

// Projection onto D K_exp in FP32; lg = log of the scales.  Falls back to the FP64
// search when the FP32 root search does not give a finite result.
__device__ inline void exp_project_f32(float r0, float s0, float t0, float dr, float ds, float dt, const float* lg,
                                       float* out, float* L_cache, const float* mlp = nullptr) {
    // a point within 1e-6 |v| of the cone (of its polar) is taken as inside (see exp_gap_to_cone)
    const float near = 1e-6f * sqrtf(r0 * r0 + s0 * s0 + t0 * t0);
    if (in_kexp_f(r0 / dr, s0 / ds, t0 / dt) || exp_gap_to_cone(r0, s0, t0, dr, ds, dt) <= near) {
        out[0] = r0; out[1] = s0; out[2] = t0;
        return;
    }
    if (in_kexp_dual_f(-dr * r0, -ds * s0, -dt * t0) || exp_gap_to_polar(r0, s0, t0, dr, ds, dt) <= near) {
        out[0] = 0.0f; out[1] = 0.0f; out[2] = 0.0f;
        return;
    }
    if (r0 <= 0.0f && s0 <= 0.0f) { out[0] = r0; out[1] = 0.0f; out[2] = t0 > 0.0f ? t0 : 0.0f; return; }
    ExpCase4T<float> e;
    e.r0 = r0; e.s0 = s0; e.t0 = t0; e.dr = dr; e.ds = ds;
    e.tau = ds / dr;
    e.ldr = lg[0]; e.lds = lg[1]; e.ldt = lg[2];
    const float ninf = -INFINITY;
    e.lr0 = r0 > 0.0f ? logf(r0) : ninf;
    e.ls0 = s0 > 0.0f ? logf(s0) : ninf;
    e.lt0 = t0 > 0.0f ? logf(t0) : (t0 < 0.0f ? logf(-t0) : ninf);
    e.a3 = s0 > 0.0f ? (r0 * ds) / (s0 * dr) : 0.0f;
    e.a4m1 = r0 > 0.0f ? -(s0 * ds) / (r0 * dr) : -1.0f;
    e.a4 = r0 > 0.0f ? 1.0f + e.a4m1 : 0.0f;
    e.w34 = e.a3 - e.a4;
    e.dt3 = s0 > 0.0f ? e.a3 * (e.a3 - 1.0f) + e.tau * e.tau : 0.0f;  // d~ at the interval ends
    e.dt4 = r0 > 0.0f ? e.a4 * e.a4m1 + e.tau * e.tau : 0.0f;
    int evals = 0;
    float L = 0.0f;
    bool ok = isfinite(e.a3) && isfinite(e.a4) && exp_case4_solve(e, L_cache ? *L_cache : NAN, L, evals, mlp) && !(L != L);
    float F, dF, rho, lsp, lrd, Fs;
    if (ok) {
        exp_F(e, L, F, dF, rho, lsp, lrd, Fs);
        ok = rho == rho;
    }
    if (!ok) {
        double o[3], Lc = NAN;
        exp_project((double)r0, (double)s0, (double)t0, (double)dr, (double)ds, (double)dt, o, &Lc, nullptr);
        out[0] = (float)o[0]; out[1] = (float)o[1]; out[2] = (float)o[2];
        return;
    }
    if (L_cache) *L_cache = L;
    const float sp = expf(lsp), rd = expf(lrd);
    const float vp[3] = {dr * rho * sp, ds * sp, expf(e.ldt + rho + lsp)};
    const float vd[3] = {rd / dr, (1.0f - rho) * rd / ds, -expf(-e.ldt - rho + lrd)};
    const float v0[3] = {r0, s0, t0};
#pragma unroll
    for (int k = 0; k < 2; ++k) out[k] = fabsf(vp[k]) <= fabsf(vd[k]) ? vp[k] : v0[k] - vd[k];
    out[2] = t0 >= 0.0f ? t0 - vd[2] : vp[2];
}

// Projection onto D^{-1} K_exp^* (Remark of App. A.2) in FP32.
__device__ __forceinline__ void exp_dual_project_f32(float r, float s, float t, float dr, float ds, float dt,
                                                     const float* lg, float* out, float* L_cache,
                                                     const float* mlp = nullptr) {
    float p[3];
    exp_project_f32(-r, -s, -t, dr, ds, dt, lg, p, L_cache, mlp);
    out[0] = r + p[0];
    out[1] = s + p[1];
    out[2] = t + p[2];
}

}  // namespace pdcs

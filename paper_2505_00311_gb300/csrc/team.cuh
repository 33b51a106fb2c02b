// team.cuh -- grid-wise projection of large second-order cones (Sec. 4, the grid-wise
// strategy: several blocks of one launch share one cone).
//
// A team is a contiguous range of G blocks of a cooperative launch (all blocks resident at
// once, so a block may wait for the others).  Block r of the team owns x entries
// [r ch, (r + 1) ch) of the cone (ch = ceil((dim - 1) / G)) and, for r = 0, the first row.
// Every sum over the cone is a team sum: a fixed-order block sum, one FP64 partial per
// block and quantity in a slot of its own, a team barrier, then every block adds the G
// partials in slot order.  All blocks of the team therefore hold bit-identical sums and
// take identical decisions; the root search (Theorem 1, the same mathematics and precision
// scheme as soc_project_warp_mp: FP32 safeguarded Newton on psi over FP32 copies, at most
// three FP64 Newton steps, FP64 search as fallback) runs in every block in lockstep.
// Partial slots are double-buffered by the parity of the team-sum count, so one barrier
// per sum suffices: a block can only rewrite a parity's slots after every block has passed
// the barrier that follows their reads of it.
//
// Waits are bounded: a block that spins for kTeamSpinLimit polls sets *abort, and a block
// that sees *abort set stops waiting; the callers turn that into a status (no trap, no
// fault).  A team of one block (G = 1) never waits.
#pragma once
#include "cone_math.cuh"
#include "dev.h"

namespace pdcs {

constexpr int kTeamSpinLimit = 1 << 21;  // polls of one barrier wait (each an L2 round trip or a sleep)
constexpr int kTeamUnroll = 8;           // loads in flight per thread in the D = I passes

__device__ __forceinline__ unsigned team_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void team_st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int team_ld_volatile(const int* p) { return *(volatile const int*)p; }

struct Team {
    int G, r;        // team size and this block's rank in it
    int slot;        // this block's partial slot (its block index in the launch)
    int slot0;       // the team's first slot
    int stride;      // slots per parity
    unsigned* bar;   // [count, generation] of the team's barrier
    double* part;    // 2 * stride * kTeamQ partials
    int* abort;      // set by a block whose wait timed out
    unsigned phase;  // team sums done so far (same in every block of the team)
    bool ok;         // false once a wait of this block gave up
};

// Sense-counting barrier over the team's blocks: the last block to arrive resets the
// count and bumps the generation the others poll.  Returns false (and sets *abort) when
// the wait gave up, or when another block already did.
__device__ __forceinline__ bool team_barrier(Team& tm) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = tm.ok ? 1 : 0;
        if (ok) {
            const unsigned g = team_ld_acquire(tm.bar + 1);
            __threadfence();
            const unsigned old = atomicAdd(tm.bar, 1u);
            if (old == (unsigned)tm.G - 1) {
                atomicExch(tm.bar, 0u);
                __threadfence();
                team_st_release(tm.bar + 1, g + 1u);
            } else {
                ok = 0;
                for (int it = 0; it < kTeamSpinLimit; ++it) {
                    if (team_ld_acquire(tm.bar + 1) != g) { ok = 1; break; }
                    if (team_ld_volatile(tm.abort) != 0) break;
                    if (it > 1024) __nanosleep(256);
                }
                if (!ok) atomicExch(tm.abort, 1);
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    tm.ok = s_ok != 0;
    return tm.ok;
}

// v[0..NQ): this block's per-thread values in, the team's totals out (in every thread).
template <int NQ>
__device__ __forceinline__ void team_sum(Team& tm, double (&v)[NQ]) {
    static_assert(NQ <= kTeamQ, "team_sum: too many quantities");
    __shared__ double sm[kTeamQ][kWarpsPerBlock];
    __shared__ double tot[kTeamQ];
    block_sum<NQ>(v, sm);
    if (tm.G == 1) {
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) tot[q] = v[q];
        }
    } else {
        double* P = tm.part + (size_t)(tm.phase & 1u) * tm.stride * kTeamQ;
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) P[(size_t)tm.slot * kTeamQ + q] = v[q];
        }
        team_barrier(tm);
        if (threadIdx.x < kWarp) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                double s = 0.0;
                for (int i = threadIdx.x; i < tm.G; i += kWarp) s += __ldcg(P + (size_t)(tm.slot0 + i) * kTeamQ + q);
                s = warp_sum(s);
                if (threadIdx.x == 0) tot[q] = s;
            }
        }
    }
    tm.phase += 1u;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = tot[q];
    __syncthreads();
}

// x entries [lo, hi) of block r of G over a cone of nx x entries
__device__ __forceinline__ void team_chunk(int nx, int G, int r, int& lo, int& hi) {
    const int ch = (nx + G - 1) / G;
    lo = min(nx, r * ch);
    hi = min(nx, lo + ch);
}

// Rows [row_lo, row_hi) of the cone (0 = its first row) that block r owns.
__device__ __forceinline__ void team_rows(int dim, int G, int r, int& row_lo, int& row_hi) {
    int lo, hi;
    team_chunk(dim - 1, G, r, lo, hi);
    row_lo = r == 0 ? 0 : 1 + lo;
    row_hi = 1 + hi;
}

// Projects the cone at buf[0..dim) (global memory) in place onto E K_soc, E as for
// soc_project_warp (weights wf(i) of the x entries; d: the block's scales for the FP64
// fallback, may be null), with every block of the team calling it with identical
// arguments after writing its own rows.  rot: rotated SOC through Q (rsoc_project_warp).
// cache: the cone's last root (may be null).  scr: 2 (dim - 1) floats of scratch for the
// FP32 copies.  Each block reads and writes only its own rows (plus reads of sums), so its
// rows are final when it returns.
template <bool kInv, typename WF>
__device__ void soc_team_project(double* buf, WF wf, const double* __restrict__ d, int dim, bool rot, float* cache,
                                 float* __restrict__ scr, Team& tm) {
    const double r2 = 0.70710678118654752440;
    const int nx = dim - 1;
    int lo, hi;
    team_chunk(nx, tm.G, tm.r, lo, hi);
    float* x32 = scr;
    float* w32 = scr + nx;
    const bool first = tm.r == 0;
    if (rot && first && threadIdx.x == 0) {
        const double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncthreads();
    if (wf.unit()) {  // Dhat = I: the textbook closed form; one FMA per entry, one product
        // kTeamUnroll independent loads per thread in flight (the sums stay in a fixed order)
        constexpr int U = kTeamUnroll;
        const int B = blockDim.x;
        double* x = buf + 1;
        double acc[U];
#pragma unroll
        for (int k = 0; k < U; ++k) acc[k] = 0.0;
        int i = lo + (int)threadIdx.x;
        for (; i + (U - 1) * B < hi; i += U * B) {
            double xv[U];
#pragma unroll
            for (int k = 0; k < U; ++k) xv[k] = x[i + k * B];
#pragma unroll
            for (int k = 0; k < U; ++k) acc[k] = fma(xv[k], xv[k], acc[k]);
        }
        for (; i < hi; i += B) acc[0] = fma(x[i], x[i], acc[0]);
        double nv[2] = {0.0, 0.0};
#pragma unroll
        for (int k = 0; k < U; ++k) nv[0] += acc[k];
        if (first && threadIdx.x == 0) nv[1] = buf[0];
        team_sum<2>(tm, nv);
        const double t = nv[1], nxn = sqrt(nv[0]);
        if (nxn > fabs(t)) {
            const double top = 0.5 * (t + nxn), sc = top / nxn;
            i = lo + (int)threadIdx.x;
            for (; i + (U - 1) * B < hi; i += U * B) {
                double xv[U];
#pragma unroll
                for (int k = 0; k < U; ++k) xv[k] = x[i + k * B];
#pragma unroll
                for (int k = 0; k < U; ++k) x[i + k * B] = xv[k] * sc;
            }
            for (; i < hi; i += B) x[i] *= sc;
            if (first && threadIdx.x == 0) buf[0] = top;
        } else if (t <= 0.0) {
            for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) buf[1 + i] = 0.0;
            if (first && threadIdx.x == 0) buf[0] = 0.0;
        }
        __syncthreads();
        if (rot && first && threadIdx.x == 0) {
            const double p = buf[0], q = buf[1];
            buf[0] = (p + q) * r2;
            buf[1] = (p - q) * r2;
        }
        __syncthreads();
        return;
    }
    // norms of the case tests, FP32 copies, range flags; t from the first block
    double nv[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
        const double x = buf[1 + i], w = wf(i);
        const double x2 = x * x;
        nv[0] += x2 / w;
        nv[1] += w * x2;
        x32[i] = (float)x;
        w32[i] = (float)w;
        if (!(w < 1e30 && w > 1e-30 && fabs(x) < 1e30)) nv[3] += 1.0;
    }
    if (first && threadIdx.x == 0) nv[2] = buf[0];
    team_sum<4>(tm, nv);
    const double t = nv[2];
    const double nDx = sqrt(nv[0]), nDinvx = sqrt(nv[1]);
    const bool rng = nv[3] == 0.0 && fabs(t) < 1e30 && fabs(t) > 1e-30 && nDinvx < 1e30;
    double mu = 1.0;  // case 3 (t == 0)
    bool zero = false, keep = false, fast = true;
    if (t <= 0.0 && nDx <= -t) zero = true;  // case 1
    else if (nDinvx <= t) keep = true;       // case 2
    else if (t != 0.0) {                     // case 4
        bool known = false, near = false;
        if (cache && t > 0.0) {
            const float cv = __ldcg(cache);
            const float m = cv < 0.0f ? -cv : 1.0f - cv;
            known = cv == cv && cv != 0.0f && m > 0.0f && m < 1.0f;
            near = known && m < 0.5f;
        }
        if (t > 0.0 && !known) {  // sign of psi at mu = 1/2
            double s[1] = {0.0};
            for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
                const double x = buf[1 + i], w = wf(i);
                const double r = 1.0 / (1.0 + 0.5 * w);
                s[0] += w * x * x * r * r;
            }
            team_sum<1>(tm, s);
            near = 0.5 * sqrt(s[0]) < t;
        }
        const SocVar<double> V(t, near);
        const SocVar<float> Vf(V);
        float* cache_in = nullptr;  // the cached start, read once above
        float cstart = cache ? __ldcg(cache) : 0.0f;
        if (cache) cache_in = &cstart;
        bool conv = false;
        double u = 0.0;
        if (rng) {
            auto ev32 = [&](float uu, float& ph, float& dph, float& sc) {
                const float m = Vf.mu(uu);
                float S = 0.0f, S2 = 0.0f;
                for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
                    const float w = w32[i], x = x32[i];
                    const float r = __frcp_rn(1.0f + m * w);
                    const float term = w * x * x * r * r;
                    S += term;
                    S2 += w * term * r;
                }
                double s[2] = {(double)S, (double)S2};
                team_sum<2>(tm, s);
                Vf.psi(uu, sqrtf((float)s[0]), (float)s[1], ph, dph, sc);
            };
            const float uf =
                soc_root<float>(ev32, V.tpos, (float)V.guess(t, nDinvx, cache_in), 2e-6f, 2e-7f, 100);
            u = (double)uf;
            if (uf > 0.0f && isfinite(uf)) {
                for (int it = 0; it < 3; ++it) {
                    const double m = V.mu(u);
                    double s[2] = {0.0, 0.0};
                    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
                        const double x = buf[1 + i], w = wf(i);
                        const double r = rcp_refined(1.0 + m * w);
                        const double term = w * x * x * r * r;
                        s[0] += term;
                        s[1] += w * term * r;
                    }
                    team_sum<2>(tm, s);
                    double ph, dph, sc;
                    V.psi(u, sqrt(s[0]), s[1], ph, dph, sc);
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
        if (!conv) {  // FP64 search with exact divisions
            fast = false;
            auto ev = [&](double uu, double& ph, double& dph, double& sc) {
                const double m = V.mu(uu);
                double s[2] = {0.0, 0.0};
                for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
                    const double x = buf[1 + i], w = wf(i);
                    const double r = 1.0 / (1.0 + m * w);
                    const double term = w * x * x * r * r;
                    s[0] += term;
                    s[1] += w * term * r;
                }
                team_sum<2>(tm, s);
                V.psi(uu, sqrt(s[0]), s[1], ph, dph, sc);
            };
            u = soc_root<double>(ev, V.tpos, V.guess(t, nDinvx, cache_in), RootTolSoc, 4e-16, 200);
        }
        if (cache && first && threadIdx.x == 0) *cache = V.store(u);
        mu = V.mu(u);
    }
    (void)d;
    if (zero) {
        for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) buf[1 + i] = 0.0;
        if (first && threadIdx.x == 0) buf[0] = 0.0;
    } else if (!keep) {
        double s[1] = {0.0};
        for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
            const double w = wf(i);
            const double y = fast ? buf[1 + i] * rcp_refined(1.0 + mu * w) : buf[1 + i] / (1.0 + mu * w);
            s[0] += w * y * y;
            buf[1 + i] = y;
        }
        team_sum<1>(tm, s);
        if (first && threadIdx.x == 0) buf[0] = sqrt(s[0]);
    }
    __syncthreads();
    if (rot && first && threadIdx.x == 0) {
        const double p = buf[0], q = buf[1];
        buf[0] = (p + q) * r2;
        buf[1] = (p - q) * r2;
    }
    __syncthreads();
}

}  // namespace pdcs

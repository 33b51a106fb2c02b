// setup_kernels.cuh -- one-off kernels of pdcs_create: diagonal rescaling,
// products for the power iteration, reductions.
#pragma once
#include "common.cuh"

namespace pdcs {

// Row norms of diag(dr) A diag(dc) for a CSR A (warp per row).  For the rows of
// K use (rs = dr, cs = dc); for the rows of K' use (rs = dc, cs = dr) with the
// product written as (dr_i * a) * dc_j in both cases, so both orientations see
// bitwise the same scaled entries.  kind 0: max |.|, kind 1: sum |.|.
__global__ void scaled_row_norms(int rows, const int* __restrict__ rp, const int* __restrict__ ci,
                                 const double* __restrict__ val, const double* __restrict__ own,
                                 const double* __restrict__ other, int own_is_dr, int kind, double* out) {
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = w; r < rows; r += nw) {
        const double so = own[r];
        double acc = 0.0;
        for (int p = rp[r] + lane; p < rp[r + 1]; p += 32) {
            const double sx = other[ci[p]];
            const double a = own_is_dr ? fabs((so * val[p]) * sx) : fabs((sx * val[p]) * so);
            acc = kind ? acc + a : fmax(acc, a);
        }
        acc = kind ? warp_sum(acc) : warp_max(acc);
        if (lane == 0) out[r] = acc;
    }
}

// Tie groups of rows to one norm (the max over the group): each group is
// [off, off + len).
__global__ void tie_groups(int ng, const int* __restrict__ off, const int* __restrict__ len, double* rn) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int o = off[g], L = len[g];
    double mx = 0.0;
    for (int i = 0; i < L; ++i) mx = fmax(mx, rn[o + i]);
    for (int i = 0; i < L; ++i) rn[o + i] = mx;
}

// d_i <- d_i / sqrt(norm_i) where norm_i > 0
__global__ void apply_norm(int k, const double* __restrict__ nrm, double* d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k && nrm[i] > 0.0) d[i] = d[i] / sqrt(nrm[i]);
}

// scaled values: out_p = (dr_row * val_p) * dc_col for K, and the same product for K'
__global__ void scale_values(int rows, const int* __restrict__ rp, const int* __restrict__ ci,
                             const double* __restrict__ val0, const double* __restrict__ own,
                             const double* __restrict__ other, int own_is_dr, double* out) {
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = w; r < rows; r += nw) {
        const double so = own[r];
        for (int p = rp[r] + lane; p < rp[r + 1]; p += 32) {
            const double sx = other[ci[p]];
            out[p] = own_is_dr ? (so * val0[p]) * sx : (sx * val0[p]) * so;
        }
    }
}

template <typename T>
__global__ void cast_vec(long long k, const double* __restrict__ in, T* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k; i += (long long)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}

// c~ = dc c, l~ = l / dc, u~ = u / dc ; h~ = dr h
__global__ void scale_cols(int n, const double* __restrict__ dc, const double* __restrict__ c,
                           const double* __restrict__ l, const double* __restrict__ u, double* cs, double* ls,
                           double* us) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    cs[j] = dc[j] * c[j];
    ls[j] = l[j] / dc[j];
    us[j] = u[j] / dc[j];
}

__global__ void scale_rows(int m, const double* __restrict__ dr, const double* __restrict__ h, double* hs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) hs[i] = dr[i] * h[i];
}

// Deterministic single-block reductions for setup: kind 0 sum of squares,
// 1 max |.|, 2 sum x*y.  Each thread's long strided sum carries Neumaier's compensation
// (a plain sum of the ~4,000 terms per thread of a 1M-vector loses ~1e-14).
__global__ void reduce_small(long long k, const double* __restrict__ a, const double* __restrict__ b, int kind,
                             double* out) {
    __shared__ double sm[2][kWarpsPerBlock];
    double v[2] = {0.0, 0.0};  // sum, compensation
    for (long long i = threadIdx.x; i < k; i += blockDim.x) {
        const double x = a[i];
        if (kind == 1) {
            v[0] = fmax(v[0], fabs(x));
            continue;
        }
        const double term = kind == 0 ? x * x : x * b[i];
        const double t = v[0] + term;
        v[1] += fabs(v[0]) >= fabs(term) ? (v[0] - t) + term : (term - t) + v[0];
        v[0] = t;
    }
    if (kind == 1) {
        double mx[1] = {v[0]};
        block_max<1>(mx, sm);
        if (threadIdx.x == 0) *out = mx[0];
        return;
    }
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) *out = v[0] + v[1];
}

// v <- u / s (s read from device)
__global__ void scale_by_inv(long long k, const double* __restrict__ u, const double* __restrict__ s, double* v) {
    const double inv = 1.0 / sqrt(*s);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k; i += (long long)gridDim.x * blockDim.x)
        v[i] = u[i] * inv;
}

// Per SOC row: weights of the dual projection onto Dr^{-1} K_soc, (dr_row / dr_first)^2,
// and of the primal projection onto Dr K_soc, (dr_first / dr_row)^2 (Theorem 1: w = dhat^-2).
__global__ void cone_constants(int n_soc, const int* __restrict__ off, const int* __restrict__ dim,
                               const double* __restrict__ dr, double* w, double* wp) {
    const int lane = threadIdx.x & 31;
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= n_soc) return;
    const int o = off[c], d = dim[c];
    const double d0 = dr[o];
    for (int i = lane; i < d; i += 32) {
        if (i == 0) { w[o] = 1.0; wp[o] = 1.0; continue; }
        const double q = dr[o + i] / d0, p = d0 / dr[o + i];
        w[o + i] = q * q;
        wp[o + i] = p * p;
    }
}

// Per exp cone: log dr of its three rows (scales of the rescaled cone, Theorem 3).
__global__ void exp_constants(int n_exp, int row0, const double* __restrict__ dr, double* lg) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_exp) return;
    for (int k = 0; k < 3; ++k) lg[3 * e + k] = log(dr[row0 + 3 * e + k]);
}

}  // namespace pdcs

// kernels.cuh -- per-iteration and per-check kernels of the PDCS solver.
//
// One PDHG evaluation (eq. PDHG on the rescaled program) is four launches:
//   primal_update  : applies the pending ReflectedHalpern update (Algorithm 1,
//                    step 6) and the eta-weighted average (step 7) to x and to the
//                    cached K'y, then xhat = Proj_[l,u](x - tau (c - K'y)) and
//                    per-block partials of ||xhat - x||^2;
//   spmv (K)       : K xhat into one of two buffers (the previous one is still
//                    needed by the pending Halpern update of K x);
//   dual_update    : the same pending update for y and the cached K x, then
//                    v = y + sigma (h - 2 K xhat + K x), yhat = Proj_{Dr^{-1} C*}(v)
//                    block by block (one thread per scalar row or exp cone, one
//                    warp per SOC / RSOC), partials of ||dy||^2 and dy'(K xhat - K x)
//                    (= dy' K dx, no extra product); its last block is the step
//                    controller (AdaptiveStepPDHG);
//   spmv (K')      : K' yhat, skipped when the step was rejected.
// The cached products follow from linearity: K z^{k+1} = ha K zhat + hb K z^k + hc K z^0.
#pragma once
#include "common.cuh"
#include "cone_f32.cuh"
#include "cone_math.cuh"
#include "team.cuh"
#include "dev.h"
#include "state.h"

namespace pdcs {

// ---------------------------------------------------------------------------
// SpMV: y = A x.  The rows are grouped in bins by length (host side, once per
// matrix); bin k runs lanes[k] lanes per row (a power of two, so that each lane
// takes a few entries), a warp covering 32 / lanes rows at a time, and the bins of
// the longest rows come first in the grid.  The matrix is stored bin by bin: binned
// row i has its entries at rp[i] .. rp[i+1] and is row list[i] of A, so the row
// bounds come from one contiguous array and the list only names the output.  Each
// lane issues U independent (column, value) loads before the gathers of x, for
// memory-level parallelism; its entries are summed in order, then the row's lanes by
// a shuffle tree, so a row's result depends only on its lane count.
// sel: 0 -> write y0;  1 -> write y0 / y1 by the parity of ctrl->attempts.
// skip: 0 never; 1 when not running; 2 when not running or the step was rejected.
// ---------------------------------------------------------------------------

// rows [0, count) of one bin: list, rp offset to the bin's first row
template <typename T, typename TO, int G, int U>
__device__ __forceinline__ void spmv_bin_rows(const int* __restrict__ list, int count, int wb, int nwb,
                                              const int* __restrict__ rp, const int* __restrict__ ci,
                                              const T* __restrict__ val, const T* __restrict__ x, TO* y) {
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31, g = lane / G, gl = lane % G;
    for (long long i0 = (long long)wb * RPW; i0 < count; i0 += (long long)nwb * RPW) {
        const long long i = i0 + g;
        T acc = T(0);
        int r = -1;
        if (i < count) {
            r = __ldg(list + i);
            const int e = __ldg(rp + i + 1);
            for (int p = __ldg(rp + i) + gl; p < e; p += G * U) {
                int c[U];
                T v[U], xv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int q = p + u * G;
                    c[u] = q < e ? __ldg(ci + q) : -1;
                    v[u] = q < e ? __ldg(val + q) : T(0);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : T(0);
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (c[u] >= 0) acc += v[u] * xv[u];
            }
        }
        acc = group_sum<G>(acc);
        if (r >= 0 && gl == 0) y[r] = (TO)acc;
    }
}

template <typename T, typename TO, int U>
__global__ void __launch_bounds__(kBlock) spmv_binned(SpmvBins B, const int* __restrict__ list,
                                                      const int* __restrict__ rp, const int* __restrict__ ci,
                                                      const T* __restrict__ val, const T* __restrict__ x, TO* y0,
                                                      TO* y1, const Ctrl* ctrl, int sel, int skip) {
    if (skip) {
        if (ctrl->status != kRunning) return;
        if (skip == 2 && !ctrl->pending) return;
    }
    TO* y = (sel == 1 && (ctrl->attempts & 1)) ? y1 : y0;
    int k = 0;
    while (k + 1 < B.nbins && (int)blockIdx.x >= B.blk[k + 1]) ++k;
    const int wb = ((int)blockIdx.x - B.blk[k]) * kWarpsPerBlock + (threadIdx.x >> 5);
    const int nwb = (B.blk[k + 1] - B.blk[k]) * kWarpsPerBlock;
    const int* l = list + B.row[k];
    const int* rb = rp + B.row[k];
    const int cnt = B.row[k + 1] - B.row[k];
    switch (B.lanes[k]) {
        case 1: spmv_bin_rows<T, TO, 1, U>(l, cnt, wb, nwb, rb, ci, val, x, y); break;
        case 2: spmv_bin_rows<T, TO, 2, U>(l, cnt, wb, nwb, rb, ci, val, x, y); break;
        case 4: spmv_bin_rows<T, TO, 4, U>(l, cnt, wb, nwb, rb, ci, val, x, y); break;
        case 8: spmv_bin_rows<T, TO, 8, U>(l, cnt, wb, nwb, rb, ci, val, x, y); break;
        case 16: spmv_bin_rows<T, TO, 16, U>(l, cnt, wb, nwb, rb, ci, val, x, y); break;
        default: spmv_bin_rows<T, TO, 32, U>(l, cnt, wb, nwb, rb, ci, val, x, y); break;
    }
}

// ---------------------------------------------------------------------------
// Sliced SpMV: y = A x with A stored in slices (SlicePlan).  One warp per slice: at each
// step every lane loads the next pair of entries of its row with one 8-byte (columns) and
// one 16-byte (FP64 values) load, the warp reading 256 + 512 contiguous bytes, then
// gathers x for both; a row's S lanes add their partial sums by a shuffle tree (S = 1:
// one accumulator in the row's order).  Rows longer than kSliceMaxLen come first in the
// grid, one warp each (lane-strided partial sums, then a shuffle tree).
// sel / skip as for spmv_binned.
// ---------------------------------------------------------------------------
template <typename T> struct Pair2;
template <> struct Pair2<double> { using type = double2; };
template <> struct Pair2<float> { using type = float2; };

template <typename T>
__device__ __forceinline__ T lane_group_sum(T v, int lg) {
    for (int o = (1 << lg) >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// xalt (may be null): the second x-hat buffer; with it x is the buffer Ctrl::xsel ^ xnext
// names (the iteration's K x-hat, see spmv_kt_primal)
template <typename T, typename TO>
__global__ void __launch_bounds__(kBlock) spmv_sliced(SlicePlan S, const int* __restrict__ ci,
                                                      const T* __restrict__ val, const T* __restrict__ x, TO* y0,
                                                      TO* y1, const Ctrl* ctrl, int sel, int skip,
                                                      const T* __restrict__ xalt) {
    if (skip) {
        if (ctrl->status != kRunning) return;
        if (skip == 2 && !ctrl->pending) return;
    }
    if (xalt && (ctrl->xsel ^ ctrl->xnext)) x = xalt;
    TO* y = (sel == 1 && (ctrl->attempts & 1)) ? y1 : y0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if ((int)blockIdx.x < S.nb_long) {
        const int r = (int)blockIdx.x * kWarpsPerBlock + w;
        if (r >= S.nlong) return;
        const int b = __ldg(S.long_rp + r), e = __ldg(S.long_rp + r + 1);
        T acc = T(0);
        for (int p = b + lane; p < e; p += 32) acc += __ldg(val + p) * __ldg(x + __ldg(ci + p));
        acc = group_sum<32>(acc);
        if (lane == 0) y[__ldg(S.long_row + r)] = (TO)acc;
        return;
    }
    using V2 = typename Pair2<T>::type;
    const int s = ((int)blockIdx.x - S.nb_long) * kWarpsPerBlock + w;
    if (s >= S.nslices) return;
    const int base = __ldg(S.slice_off + s);
    const int steps = (__ldg(S.slice_off + s + 1) - base) >> 6;
    const int lg = __ldg(S.slice_lg + s);
    const int2* cp = reinterpret_cast<const int2*>(ci + base) + lane;
    const V2* vp = reinterpret_cast<const V2*>(val + base) + lane;
    T acc = T(0);
    int q = 0;
    for (; q + 4 <= steps; q += 4) {  // four pairs in flight
        int2 c[4];
        V2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = __ldg(cp + 32 * (q + u));
            v[u] = __ldg(vp + 32 * (q + u));
        }
        T xv[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            xv[2 * u] = c[u].x >= 0 ? __ldg(x + c[u].x) : T(0);
            xv[2 * u + 1] = c[u].y >= 0 ? __ldg(x + c[u].y) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            acc += v[u].x * xv[2 * u];
            acc += v[u].y * xv[2 * u + 1];
        }
    }
    for (; q + 2 <= steps; q += 2) {  // two pairs in flight
        const int2 c0 = __ldg(cp + 32 * q), c1 = __ldg(cp + 32 * (q + 1));
        const V2 v0 = __ldg(vp + 32 * q), v1 = __ldg(vp + 32 * (q + 1));
        const T x0 = c0.x >= 0 ? __ldg(x + c0.x) : T(0);
        const T x1 = c0.y >= 0 ? __ldg(x + c0.y) : T(0);
        const T x2 = c1.x >= 0 ? __ldg(x + c1.x) : T(0);
        const T x3 = c1.y >= 0 ? __ldg(x + c1.y) : T(0);
        acc += v0.x * x0;
        acc += v0.y * x1;
        acc += v1.x * x2;
        acc += v1.y * x3;
    }
    if (q < steps) {
        const int2 c0 = __ldg(cp + 32 * q);
        const V2 v0 = __ldg(vp + 32 * q);
        const T x0 = c0.x >= 0 ? __ldg(x + c0.x) : T(0);
        const T x1 = c0.y >= 0 ? __ldg(x + c0.y) : T(0);
        acc += v0.x * x0;
        acc += v0.y * x1;
    }
    acc = lane_group_sum(acc, lg);
    if ((lane & ((1 << lg) - 1)) == 0) {
        const int r = __ldg(S.out_row + 32 * s + (lane >> lg));
        if (r >= 0) y[r] = (TO)acc;
    }
}

// K' y-hat fused with the next primal update (the epilogue of row j of K' is variable j):
// after an accepted step, the pending reflected-Halpern update of x_j and K'y_j (with this
// product as K' y-hat) and the average, then the next evaluation's
// x-hat_j = Proj_[l,u](x_j - tau (c_j - K'y_j)) with the controller's new tau, into the other
// x-hat buffer, and per-block partials of ||x-hat - x||^2 in the slots after primal_update's.
// The same arithmetic as primal_update_body, element by element.  Skipped (like the plain
// K' product) when the step was rejected; block 0 sets Ctrl::xnext.
template <typename T>
__global__ void __launch_bounds__(kBlock) spmv_kt_primal(SlicePlan S, const int* __restrict__ ci,
                                                         const T* __restrict__ val, Dev<T> D) {
    Ctrl* C = D.ctrl;
    if (C->status != kRunning || !C->pending) return;
    __shared__ double sm[1][kWarpsPerBlock];
    const T ha = (T)C->ha, hb = (T)C->hb, hc = (T)C->hc, hw = (T)C->hw, tau = (T)C->tau;
    const T* xcur = C->xsel ? D.xh1 : D.xh;
    T* xnew = C->xsel ? D.xh : D.xh1;
    const T* __restrict__ yh = D.yh;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T dx2 = T(0);
    auto epilogue = [&](int j, T ktyh) {
        T x = D.x[j], kty = D.kty[j];
        x = ha * xcur[j] + hb * x + hc * D.x0[j];
        kty = ha * ktyh + hb * kty + hc * D.kty0[j];
        D.x[j] = x;
        D.kty[j] = kty;
        if (hw != T(0)) D.xsum[j] += hw * x;
        const T xh = fmin(fmax(x - tau * (D.c[j] - kty), D.l[j]), D.u[j]);
        xnew[j] = xh;
        const T dx = xh - x;
        dx2 += dx * dx;
    };
    if ((int)blockIdx.x < S.nb_long) {
        const int r = (int)blockIdx.x * kWarpsPerBlock + w;
        if (r < S.nlong) {
            const int b = __ldg(S.long_rp + r), e = __ldg(S.long_rp + r + 1);
            T acc = T(0);
            for (int p = b + lane; p < e; p += 32) acc += __ldg(val + p) * __ldg(yh + __ldg(ci + p));
            acc = group_sum<32>(acc);
            if (lane == 0) epilogue(__ldg(S.long_row + r), acc);
        }
    } else {
        using V2 = typename Pair2<T>::type;
        const int s = ((int)blockIdx.x - S.nb_long) * kWarpsPerBlock + w;
        if (s < S.nslices) {
            const int base = __ldg(S.slice_off + s);
            const int steps = (__ldg(S.slice_off + s + 1) - base) >> 6;
            const int lg = __ldg(S.slice_lg + s);
            const int2* cp = reinterpret_cast<const int2*>(ci + base) + lane;
            const V2* vp = reinterpret_cast<const V2*>(val + base) + lane;
            T acc = T(0);
            int q = 0;
            for (; q + 4 <= steps; q += 4) {
                int2 c[4];
                V2 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    c[u] = __ldg(cp + 32 * (q + u));
                    v[u] = __ldg(vp + 32 * (q + u));
                }
                T xv[8];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    xv[2 * u] = c[u].x >= 0 ? __ldg(yh + c[u].x) : T(0);
                    xv[2 * u + 1] = c[u].y >= 0 ? __ldg(yh + c[u].y) : T(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    acc += v[u].x * xv[2 * u];
                    acc += v[u].y * xv[2 * u + 1];
                }
            }
            for (; q + 2 <= steps; q += 2) {
                const int2 c0 = __ldg(cp + 32 * q), c1 = __ldg(cp + 32 * (q + 1));
                const V2 v0 = __ldg(vp + 32 * q), v1 = __ldg(vp + 32 * (q + 1));
                const T x0 = c0.x >= 0 ? __ldg(yh + c0.x) : T(0);
                const T x1 = c0.y >= 0 ? __ldg(yh + c0.y) : T(0);
                const T x2 = c1.x >= 0 ? __ldg(yh + c1.x) : T(0);
                const T x3 = c1.y >= 0 ? __ldg(yh + c1.y) : T(0);
                acc += v0.x * x0;
                acc += v0.y * x1;
                acc += v1.x * x2;
                acc += v1.y * x3;
            }
            if (q < steps) {
                const int2 c0 = __ldg(cp + 32 * q);
                const V2 v0 = __ldg(vp + 32 * q);
                const T x0 = c0.x >= 0 ? __ldg(yh + c0.x) : T(0);
                const T x1 = c0.y >= 0 ? __ldg(yh + c0.y) : T(0);
                acc += v0.x * x0;
                acc += v0.y * x1;
            }
            acc = lane_group_sum(acc, lg);
            if ((lane & ((1 << lg) - 1)) == 0) {
                const int r = __ldg(S.out_row + 32 * s + (lane >> lg));
                if (r >= 0) epilogue(r, acc);
            }
        }
    }
    double a[1] = {(double)dx2};
    block_sum<1>(a, sm);
    if (threadIdx.x == 0) {
        D.part[D.pl.off_px + D.px_f0 + blockIdx.x] = a[0];
        if (blockIdx.x == 0) C->xnext = 1;
    }
}

// Fills the sliced storage of a CSR matrix (rows in order: rp, ci, val) for plan S: one
// thread per slot (lane of a slice, or long row); values converted to TD; cis or vals may
// be null.
template <typename TD>
__global__ void __launch_bounds__(kBlock) sliced_copy(SlicePlan S, const int* __restrict__ rp,
                                                      const int* __restrict__ ci, const double* __restrict__ val,
                                                      int* __restrict__ cis, TD* __restrict__ vals) {
    const long long slots = 32LL * S.nslices + S.nlong;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < slots;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < 32LL * S.nslices) {
            const int s = (int)(t >> 5), lane = (int)(t & 31);
            const int lg = S.slice_lg[s], g = lane & ((1 << lg) - 1), j = lane >> lg;
            const int base = S.slice_off[s], steps = (S.slice_off[s + 1] - base) >> 6;
            const int r = S.out_row[32 * s + j];
            const int b = r >= 0 ? rp[r] : 0, len = r >= 0 ? rp[r + 1] - b : 0;
            for (int q = 0; q < steps; ++q) {
                const int p = (q << lg) + g;  // pair of the row held at this step
                for (int h = 0; h < 2; ++h) {
                    const int k = 2 * p + h;
                    const long long dst = base + 64LL * q + 2 * lane + h;
                    if (cis) cis[dst] = k < len ? ci[b + k] : -1;
                    if (vals) vals[dst] = k < len ? (TD)val[b + k] : TD(0);
                }
            }
        } else {
            const int jj = (int)(t - 32LL * S.nslices);
            const int r = S.long_row[jj], b = rp[r], len = rp[r + 1] - b, dst = S.long_rp[jj];
            for (int k = 0; k < len; ++k) {
                if (cis) cis[dst + k] = ci[b + k];
                if (vals) vals[dst + k] = (TD)val[b + k];
            }
        }
    }
}

// Stores a CSR matrix (rows in order, row pointer rp) bin by bin: binned row i is row
// list[i]; rpb (the binned row pointer) is given.  One warp per binned row; the
// entries keep their order within the row.  Values are converted to TD.
template <typename TS, typename TD>
__global__ void __launch_bounds__(kBlock) bin_rows_copy(int rows, const int* __restrict__ list,
                                                        const int* __restrict__ rp, const int* __restrict__ ci,
                                                        const TS* __restrict__ val, const int* __restrict__ rpb,
                                                        int* __restrict__ cib, TD* __restrict__ valb) {
    const int lane = threadIdx.x & 31;
    for (long long i = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); i < rows;
         i += (long long)gridDim.x * kWarpsPerBlock) {
        const int r = list[i];
        const int src = rp[r], len = rp[r + 1] - src, dst = rpb[i];
        for (int p = lane; p < len; p += 32) {
            if (cib) cib[dst + p] = ci[src + p];
            valb[dst + p] = (TD)val[src + p];
        }
    }
}

// ---------------------------------------------------------------------------
// last-block helper: returns true in every thread of the block that finished last
// ---------------------------------------------------------------------------
// (total: the blocks taking part, possibly spread over several concurrent kernels)
__device__ __forceinline__ bool last_block(Ctrl* C, unsigned int total) {
    __shared__ unsigned int s_ticket;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = atomicAdd(&C->ticket, 1u);
    __syncthreads();
    const bool last = s_ticket == total - 1;
    if (last) __threadfence();
    return last;
}
__device__ __forceinline__ bool last_block(Ctrl* C) { return last_block(C, gridDim.x); }

// Deterministic sum of part[0..cnt) by one block (fixed per-thread strides + fixed tree).
__device__ __forceinline__ double block_reduce_parts(const double* part, int cnt, double (*sm)[kWarpsPerBlock]) {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) v[0] += __ldcg(part + i);
    block_sum<1>(v, sm);
    return v[0];  // valid in thread 0
}

__device__ __forceinline__ double block_max_parts(const double* part, int cnt, double (*sm)[kWarpsPerBlock]) {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) v[0] = fmax(v[0], __ldcg(part + i));
    block_max<1>(v, sm);
    return v[0];
}

// ---------------------------------------------------------------------------
// primal update
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void primal_update_body(const Dev<T>& D, int qidx) {
    (void)qidx;
    Ctrl* C = D.ctrl;
    if (C->status != kRunning) return;
    if (C->xnext) {  // formed by the previous evaluation's K' product (spmv_kt_primal)
        if (threadIdx.x == 0) D.part[D.pl.off_px + blockIdx.x] = 0.0;
        return;
    }
    __shared__ double sm[1][kWarpsPerBlock];
    const bool pend = C->pending != 0;
    const T ha = (T)C->ha, hb = (T)C->hb, hc = (T)C->hc, hw = (T)C->hw, tau = (T)C->tau;
    T* xhat = C->xsel ? D.xh1 : D.xh;
    if (threadIdx.x == 0)  // the fused product's slots hold an earlier evaluation's partials
        for (int b = D.px_f0 + (int)blockIdx.x; b < D.pl.primal_blocks; b += gridDim.x) D.part[D.pl.off_px + b] = 0.0;
    T acc_t = T(0);  // per-thread partial in the iterate precision, then FP64 across threads
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D.n; j += stride) {
        T x = D.x[j], kty = D.kty[j];
        if (pend) {
            x = ha * xhat[j] + hb * x + hc * D.x0[j];
            kty = ha * D.ktyh[j] + hb * kty + hc * D.kty0[j];
            D.x[j] = x;
            D.kty[j] = kty;
            if (hw != T(0)) D.xsum[j] += hw * x;
        }
        T xh = fmin(fmax(x - tau * (D.c[j] - kty), D.l[j]), D.u[j]);
        xhat[j] = xh;
        const T dx = xh - x;
        if ((unsigned)(j - D.pc_lo) >= (unsigned)D.pc_len) acc_t += dx * dx;  // cone blocks: pc_apply
    }
    double acc[1] = {(double)acc_t};
    block_sum<1>(acc, sm);
    if (threadIdx.x == 0) D.part[D.pl.off_px + blockIdx.x] = acc[0];
}

// Halpern update of one dual row (returns the updated y; writes y, kx, ysum).
template <typename T>
__device__ __forceinline__ void dual_row_halpern(const Dev<T>& D, int i, bool pend, T ha, T hb, T hc, T hw,
                                                 const T* kxh_prev, T& y, T& kx) {
    y = D.y[i];
    kx = D.kx[i];
    if (pend) {
        y = ha * D.yh[i] + hb * y + hc * D.y0[i];
        kx = ha * kxh_prev[i] + hb * kx + hc * D.kx0[i];
        D.y[i] = y;
        D.kx[i] = kx;
        if (hw != T(0)) D.ysum[i] += hw * y;
    }
}

// AdaptiveStepPDHG decision and Algorithm 1 bookkeeping (run by the last block).
template <typename T>
__device__ void step_controller(const Dev<T>& D, double (*sm)[kWarpsPerBlock]) {
    Ctrl* C = D.ctrl;
    const double nx2 = block_reduce_parts(D.part + D.pl.off_px, D.pl.primal_blocks, sm);
    const double ny2 = block_reduce_parts(D.part + D.pl.off_dy, D.pl.dual_blocks, sm);
    const double itr = block_reduce_parts(D.part + D.pl.off_dy + D.pl.dual_blocks, D.pl.dual_blocks, sm);
    if (threadIdx.x != 0) return;
    C->ticket = 0;
    C->attempts += 1;
    if (C->xnext) {  // this evaluation's x-hat was the precomputed one: it is now the current
        C->xsel ^= 1;
        C->xnext = 0;
    }
    if (!isfinite(nx2) || !isfinite(ny2) || !isfinite(itr)) {
        C->status = kNumericError;
        C->pending = 0;
        return;
    }
    const double eta = C->eta, om = C->omega;
    bool accept = true;
    if (C->step_mode == 0) {
        const double inter = fabs(itr);
        const double move = om * nx2 + ny2 / om;
        const double eta_max = inter > 0.0 ? move / (2.0 * inter) : INFINITY;
        const double j1 = (double)C->attempts + 1.0;
        const double t1 = (1.0 - pow(j1, -0.3)) * eta_max;
        const double t2 = (1.0 + pow(j1, -0.6)) * eta;
        accept = eta <= eta_max;
        C->eta = fmin(t1, t2);
    }
    if (accept) {
        C->pending = 1;
        if (C->step_mode == 2) {  // plain PDHG: z <- zhat
            C->ha = 1.0; C->hb = 0.0; C->hc = 0.0; C->hw = 0.0;
        } else {
            const double kk = (double)C->k;
            const double a = (kk + 1.0) / (kk + 2.0), be = C->beta;
            C->ha = a * (1.0 + be);
            C->hb = -a * be;
            C->hc = 1.0 / (kk + 2.0);
            C->hw = eta;
            C->wsum += eta;
        }
        C->k += 1;
        C->accepted += 1;
    } else {
        C->pending = 0;
    }
    C->tau = C->eta / C->omega;
    C->sigma = C->eta * C->omega;
}

// ---------------------------------------------------------------------------
// dual update + projection + step controller
//
// Three cone roles over disjoint row ranges: scalar rows (one thread each), SOC / RSOC
// blocks (one warp each) and exp cones (one thread each).  Each role is a device function
// of its own; the single-program path launches each as its own kernel (concurrent
// branches of the evaluation graph, each with the registers it needs), a batch runs them
// as block ranges of one kernel.  Either way every block writes its partials of
// ||dy||^2 and dy'(K xhat - K x) to the slot of its global role-block index
// (exp blocks first, then SOC, then scalar), and the last block to finish, over all roles,
// runs the step controller: the sums are the same whatever the launch form.
// ---------------------------------------------------------------------------
template <typename T>
struct DualCoef {
    const T* p;      // K xhat of this evaluation
    const T* pprev;  // K xhat of the previous one (pending Halpern update of K x)
    bool pend;
    T ha, hb, hc, hw, sigma;
};

template <typename T>
__device__ __forceinline__ DualCoef<T> dual_coef(const Dev<T>& D) {
    const Ctrl* C = D.ctrl;
    const long long att = C->attempts;
    DualCoef<T> k;
    k.p = (att & 1) ? D.kxh1 : D.kxh0;
    k.pprev = (att & 1) ? D.kxh0 : D.kxh1;
    k.pend = C->pending != 0;
    k.ha = (T)C->ha; k.hb = (T)C->hb; k.hc = (T)C->hc; k.hw = (T)C->hw; k.sigma = (T)C->sigma;
    return k;
}

// scalar rows [0, m_scalar): block sb of nb_scal
template <typename T>
__device__ __forceinline__ void dual_scalar_rows(const Dev<T>& D, const DualCoef<T>& k, int sb, T (&acc)[2]) {
    const int stride = D.nb_scal * blockDim.x;
    for (int i = sb * blockDim.x + threadIdx.x; sb < D.nb_scal && i < D.m_scalar; i += stride) {
        T y, kx;
        dual_row_halpern(D, i, k.pend, k.ha, k.hb, k.hc, k.hw, k.pprev, y, kx);
        const T pi = k.p[i];
        const T v = y + k.sigma * (D.h[i] - T(2) * pi + kx);
        const T yh = (i < D.m_zero) ? v : fmax(v, T(0));
        D.yh[i] = yh;
        const T dy = yh - y;
        acc[0] += dy * dy;
        acc[1] += dy * (pi - kx);
    }
}

// One SOC / RSOC cone by a whole warp on global memory
template <typename T>
__device__ __forceinline__ void dual_soc_cone(const Dev<T>& D, const DualCoef<T>& k, int cidx, T (&acc)[2]) {
    const int lane = threadIdx.x & 31;
    {
        const int o = D.soc_off[cidx], dim = D.soc_dim[cidx];
        for (int i = lane; i < dim; i += 32) {
            T y, kx;
            dual_row_halpern(D, o + i, k.pend, k.ha, k.hb, k.hc, k.hw, k.pprev, y, kx);
            D.yh[o + i] = y + k.sigma * (D.h[o + i] - T(2) * k.p[o + i] + kx);
        }
        __syncwarp();
        if constexpr (sizeof(T) == 8)
            soc_project_any<true>(D.yh + o, D.soc_w + o + 1, D.dr + o, dim, D.soc_rot[cidx] != 0, D.soc_lam + cidx,
                                  reinterpret_cast<float*>(D.scr + o),  // scratch unused during the update
                                  D.soc_wp + o + 1);
        else
            soc_project_any_f32(D.yh + o, D.soc_w32 + o + 1, D.scr + o, D.dr + o, dim, D.soc_rot[cidx] != 0,
                                D.soc_lam + cidx);
        for (int i = lane; i < dim; i += 32) {
            const T dy = D.yh[o + i] - D.y[o + i];
            acc[0] += dy * dy;
            acc[1] += dy * (k.p[o + i] - D.kx[o + i]);
        }
        __syncwarp();
    }
}

// SOC / RSOC blocks: block sb of nb_soc, one warp per cone (batches, FP32 iterates)
template <typename T>
__device__ __forceinline__ void dual_soc_blocks(const Dev<T>& D, const DualCoef<T>& k, int sb, T (&acc)[2]) {
    const int wid = threadIdx.x >> 5;
    const int stride = D.nb_soc * (blockDim.x >> 5);
    for (int cidx = sb * (blockDim.x >> 5) + wid; cidx < D.n_soc; cidx += stride) dual_soc_cone(D, k, cidx, acc);
}

// One tile of cones (tile t, one warp): the pending Halpern update and v of its rows into
// shared memory (coalesced over the tile's rows), the projections by lane groups of S
// lanes (soc_seg_project), then yhat and the partials from shared memory.
template <int S>
__device__ __forceinline__ void soc_tile_project(const Dev<double>& D, int t, double* sv, const double* sw,
                                                 const double* swi, float* sxf, float* swf, int lane) {
    const int c0 = D.tile_cone0[t], nc = D.tile_cone0[t + 1] - c0;
    const int grp = lane / S, g = lane % S;
    if (grp >= nc) return;
    const int so = D.soc_so[c0 + grp];  // staged offset of the group's cone
    const int cone = D.soc_order[c0 + grp];
    const int o = D.soc_off[cone], dim = D.soc_dim[cone];
    const unsigned gmask = S == 32 ? 0xffffffffu : (((1u << S) - 1u) << (grp * S));
    (void)o;
    soc_seg_project<S>(sv + so, sw + so + 1, swi + so + 1, sxf + so, swf + so, dim, D.soc_rot[cone] != 0,
                       D.soc_lam + cone, gmask, g);
}

__device__ __forceinline__ void dual_soc_tile(const Dev<double>& D, const DualCoef<double>& k, int t,
                                              double (&acc)[2]) {
    extern __shared__ double soc_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // per warp: value, weight, inverse weight (doubles), then FP32 copies of value and weight
    double* sv = soc_smem + (size_t)wid * (kSocTileRows * 4);
    double* sw = sv + kSocTileRows;
    double* swi = sw + kSocTileRows;
    float* sxf = reinterpret_cast<float*>(swi + kSocTileRows);
    float* swf = sxf + kSocTileRows;
    const int r0 = D.tile_row0[t], nr = D.tile_row0[t + 1] - r0;
    for (int q = lane; q < nr; q += 32) {
        const int i = D.soc_trow[r0 + q];
        double y, kx;
        dual_row_halpern(D, i, k.pend, k.ha, k.hb, k.hc, k.hw, k.pprev, y, kx);
        sv[q] = y + k.sigma * (D.h[i] - 2.0 * k.p[i] + kx);
        sw[q] = D.soc_w[i];   // weight of the dual projection (1 on a cone's first row, unused)
        swi[q] = D.soc_wp[i];
    }
    __syncwarp();
    switch (D.tile_lg[t]) {
        case 0: soc_tile_project<1>(D, t, sv, sw, swi, sxf, swf, lane); break;
        case 1: soc_tile_project<2>(D, t, sv, sw, swi, sxf, swf, lane); break;
        case 2: soc_tile_project<4>(D, t, sv, sw, swi, sxf, swf, lane); break;
        case 3: soc_tile_project<8>(D, t, sv, sw, swi, sxf, swf, lane); break;
        case 4: soc_tile_project<16>(D, t, sv, sw, swi, sxf, swf, lane); break;
        default: soc_tile_project<32>(D, t, sv, sw, swi, sxf, swf, lane); break;
    }
    __syncwarp();
    for (int q = lane; q < nr; q += 32) {
        const int i = D.soc_trow[r0 + q];
        const double yh = sv[q];
        D.yh[i] = yh;
        const double dy = yh - D.y[i];
        acc[0] += dy * dy;
        acc[1] += dy * (k.p[i] - D.kx[i]);
    }
    __syncwarp();  // the staged rows are read before the next tile overwrites them
}

// the tiles, dealt round-robin over the tile blocks (block b takes tiles b, b + nb, ...;
// largest cones first), so every block gets the same share of the work to within a tile
__device__ __forceinline__ void dual_soc_tiles(const Dev<double>& D, const DualCoef<double>& k, double (&acc)[2]) {
    const int nb = D.nb_tiles;
    for (int t = (int)blockIdx.x + (int)(threadIdx.x >> 5) * nb; t < D.n_tiles; t += kWarpsPerBlock * nb)
        dual_soc_tile(D, k, t, acc);
}

// the large cones (after the tiles in soc_order), a warp each: block lb of the SOC blocks
// beyond the tiles
__device__ __forceinline__ void dual_soc_large(const Dev<double>& D, const DualCoef<double>& k, int lb,
                                               double (&acc)[2]) {
    const int wid = threadIdx.x >> 5;
    const int nbl = D.nb_soc - D.nb_tiles;
    const int base = D.tile_cone0[D.n_tiles];
    for (int j = lb * kWarpsPerBlock + wid; j < D.n_large; j += nbl * kWarpsPerBlock)
        dual_soc_cone(D, k, D.soc_order[base + j], acc);
}

// Exponential-family blocks of the exp region: kind 0 is K_exp, kind 1 (EXP_DUAL) is K_exp^*.
// For scales D (row scales d, logs lg) and v, the projections onto D C_e (primal side) and
// onto (D C_e)^* (dual side):
//   K_exp  : D K_exp directly, D^{-1} K_exp^* by the Remark (v + Proj_{D K_exp}(-v));
//   K_exp^*: D K_exp^* = (D^{-1})^{-1} K_exp^* by the Remark with the inverse scales, and
//            (D K_exp^*)^* = D^{-1} K_exp directly with the inverse scales.
// (the K_exp^* blocks in a call of their own, so that the K_exp path compiles as before)
static __device__ __noinline__ void exp_block_project_inv(bool dual_side, double r, double s, double t, double d0,
                                                          double d1, double d2, const double* lg, double* out,
                                                          float* cache, const float* mlp) {
    const double li[3] = {-lg[0], -lg[1], -lg[2]};
    if (dual_side) exp_project_fast(r, s, t, 1.0 / d0, 1.0 / d1, 1.0 / d2, li, out, cache, mlp);
    else exp_dual_project_fast(r, s, t, 1.0 / d0, 1.0 / d1, 1.0 / d2, li, out, cache, mlp);
}
__device__ __forceinline__ void exp_block_project(bool kdual, bool dual_side, double r, double s, double t,
                                                  double d0, double d1, double d2, const double* lg, double* out,
                                                  float* cache, const float* mlp) {
    if (kdual) {
        exp_block_project_inv(dual_side, r, s, t, d0, d1, d2, lg, out, cache, mlp);
        return;
    }
    if (dual_side) exp_dual_project_fast(r, s, t, d0, d1, d2, lg, out, cache, mlp);
    else exp_project_fast(r, s, t, d0, d1, d2, lg, out, cache, mlp);
}
static __device__ __noinline__ void exp_block_project_inv_f32(float r, float s, float t, float d0, float d1, float d2,
                                                              const float* lg, float* out, float* cache,
                                                              const float* mlp) {
    const float li[3] = {-lg[0], -lg[1], -lg[2]};
    exp_project_f32(r, s, t, 1.0f / d0, 1.0f / d1, 1.0f / d2, li, out, cache, mlp);
}
__device__ __forceinline__ void exp_block_project_f32(bool kdual, float r, float s, float t, float d0, float d1,
                                                      float d2, const float* lg, float* out, float* cache,
                                                      const float* mlp) {  // dual side
    if (kdual) {
        exp_block_project_inv_f32(r, s, t, d0, d1, d2, lg, out, cache, mlp);
        return;
    }
    exp_dual_project_f32(r, s, t, d0, d1, d2, lg, out, cache, mlp);
}
template <typename T>
__device__ __forceinline__ bool exp_kind_dual(const Dev<T>& D, int e) {
    return D.exp_kind != nullptr && D.exp_kind[e] != 0;
}

// exp cones: block b of nb_exp, one thread per cone (exp_pb per block)
template <typename T>
__device__ __forceinline__ void dual_exp_cones(const Dev<T>& D, const DualCoef<T>& k, int b, T (&acc)[2]) {
    const int stride = D.nb_exp * D.exp_pb;
    for (int e = b * D.exp_pb + threadIdx.x; threadIdx.x < D.exp_pb && e < D.n_exp; e += stride) {
        const int r = D.exp_row0 + 3 * e;
        T y[3], kx[3], v[3], out[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            dual_row_halpern(D, r + q, k.pend, k.ha, k.hb, k.hc, k.hw, k.pprev, y[q], kx[q]);
            v[q] = y[q] + k.sigma * (D.h[r + q] - T(2) * k.p[r + q] + kx[q]);
        }
        const bool kd = exp_kind_dual(D, e);
        if constexpr (sizeof(T) == 8)
            exp_block_project(kd, true, v[0], v[1], v[2], D.dr[r], D.dr[r + 1], D.dr[r + 2], D.exp_lg + 3 * e, out,
                              D.exp_L + e, D.exp_mlp);
        else
            exp_block_project_f32(kd, v[0], v[1], v[2], (float)D.dr[r], (float)D.dr[r + 1], (float)D.dr[r + 2],
                                  D.exp_lg32 + 3 * e, out, D.exp_L + e, D.exp_mlp);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const T yh = (T)out[q];
            D.yh[r + q] = yh;
            const T dy = yh - y[q];
            acc[0] += dy * dy;
            acc[1] += dy * (k.p[r + q] - kx[q]);
        }
    }
}

// partials of role-block gb (global index), then the controller in the last block of all
template <typename T>
__device__ __forceinline__ void dual_finish(const Dev<T>& D, int gb, const T (&acc_t)[2]) {
    __shared__ double sm[2][kWarpsPerBlock];
    double acc[2] = {(double)acc_t[0], (double)acc_t[1]};
    block_sum<2>(acc, sm);
    if (threadIdx.x == 0) {
        D.part[D.pl.off_dy + gb] = acc[0];
        D.part[D.pl.off_dy + D.pl.dual_blocks + gb] = acc[1];
    }
    if (last_block(D.ctrl, (unsigned)D.pl.dual_blocks)) step_controller(D, sm);
}

// all roles as block ranges of one launch (batches): exp blocks, then SOC, then scalar
template <typename T>
__device__ __forceinline__ void dual_update_body(const Dev<T>& D, int qidx) {
    (void)qidx;
    if (D.ctrl->status != kRunning) return;
    const DualCoef<T> k = dual_coef(D);
    T acc[2] = {T(0), T(0)};  // per-thread partials in the iterate precision, then FP64
    const int b = blockIdx.x;
    if (b >= D.nb_exp + D.nb_soc) dual_scalar_rows(D, k, b - D.nb_exp - D.nb_soc, acc);
    else if (b >= D.nb_exp) dual_soc_blocks(D, k, b - D.nb_exp, acc);
    else dual_exp_cones(D, k, b, acc);
    dual_finish(D, b, acc);
}

// one role per kernel (single programs; the three run concurrently)
template <typename T>
__global__ void __launch_bounds__(kBlock) dual_scalar(Dev<T> D) {
    if (D.ctrl->status != kRunning) return;
    const DualCoef<T> k = dual_coef(D);
    T acc[2] = {T(0), T(0)};
    dual_scalar_rows(D, k, blockIdx.x, acc);
    dual_finish(D, D.nb_exp + D.nb_soc + (int)blockIdx.x, acc);
}
template <typename T>
__global__ void __launch_bounds__(kBlock, 3) dual_soc(Dev<T> D) {
    if (D.ctrl->status != kRunning) return;
    const DualCoef<T> k = dual_coef(D);
    T acc[2] = {T(0), T(0)};
    if constexpr (sizeof(T) == 8) {  // FP64: tiles by lane groups, then the large cones
        if ((int)blockIdx.x < D.nb_tiles) dual_soc_tiles(D, k, acc);
        else dual_soc_large(D, k, (int)blockIdx.x - D.nb_tiles, acc);
    } else {
        dual_soc_blocks(D, k, blockIdx.x, acc);
    }
    dual_finish(D, D.nb_exp + (int)blockIdx.x, acc);
}
template <typename T>
__global__ void __launch_bounds__(kBlock, 2) dual_exp(Dev<T> D) {
    if (D.ctrl->status != kRunning) return;
    const DualCoef<T> k = dual_coef(D);
    T acc[2] = {T(0), T(0)};
    dual_exp_cones(D, k, blockIdx.x, acc);
    dual_finish(D, (int)blockIdx.x, acc);
}

// ---------------------------------------------------------------------------
// flush: apply a pending Halpern update without a PDHG step (before a check)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void flush_primal_body(const Dev<T>& D, int qidx) {
    (void)qidx;
    Ctrl* C = D.ctrl;
    if (C->status != kRunning || !C->pending || C->xnext) return;  // xnext: applied already
    const T ha = (T)C->ha, hb = (T)C->hb, hc = (T)C->hc, hw = (T)C->hw;
    const T* xhat = C->xsel ? D.xh1 : D.xh;
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D.n; j += stride) {
        const T x = ha * xhat[j] + hb * D.x[j] + hc * D.x0[j];
        D.x[j] = x;
        D.kty[j] = ha * D.ktyh[j] + hb * D.kty[j] + hc * D.kty0[j];
        if (hw != T(0)) D.xsum[j] += hw * x;
    }
}

template <typename T>
__device__ __forceinline__ void flush_dual_body(const Dev<T>& D, int qidx) {
    (void)qidx;
    Ctrl* C = D.ctrl;
    if (C->status != kRunning || !C->pending) return;
    // the pending evaluation is attempts - 1; its K xhat sits in buffer (attempts - 1) & 1
    const T* pprev = ((C->attempts - 1) & 1) ? D.kxh1 : D.kxh0;
    const T ha = (T)C->ha, hb = (T)C->hb, hc = (T)C->hc, hw = (T)C->hw;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D.m; i += stride) {
        T y, kx;
        dual_row_halpern(D, i, true, ha, hb, hc, hw, pprev, y, kx);
    }
}

// ---------------------------------------------------------------------------
// check: candidates (Algorithm 1 step 8), their KKT, restart controller
// ---------------------------------------------------------------------------
__device__ __forceinline__ int n_candidates(const Ctrl* C) {
    return (C->check_mode == 1 || C->step_mode == 2 || !(C->wsum > 0.0)) ? 1 : 2;
}

// xc[q] = Proj_[l,u](source_q): q = 0 current z, q = 1 the average zsum / wsum
template <typename T>
__device__ __forceinline__ void cand_primal_body(const Dev<T>& D, int qidx) {
    const Ctrl* C = D.ctrl;
    if (C->status != kRunning) return;
    const int q = qidx;
    if (q >= n_candidates(C)) return;
    const double iw = q ? 1.0 / C->wsum : 0.0;
    double* out = D.xc + (size_t)q * D.n;
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D.n; j += stride) {
        const double s = q ? (double)D.xsum[j] * iw : (double)D.x[j];
        out[j] = fmin(fmax(s, D.l64[j]), D.u64[j]);
    }
}

// yc[q] = Proj_{Dr^{-1} C*}(source_q), same block split as dual_update
template <typename T>
__device__ __forceinline__ void cand_dual_body(const Dev<T>& D, int qidx) {
    const Ctrl* C = D.ctrl;
    if (C->status != kRunning) return;
    const int q = qidx;
    if (q >= n_candidates(C)) return;
    const double iw = q ? 1.0 / C->wsum : 0.0;
    double* out = D.yc + (size_t)q * D.m;
    const T* src = q ? D.ysum : D.y;
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    auto val = [&](int i) { return q ? (double)src[i] * iw : (double)src[i]; };
    if (b >= D.nb_exp + D.nb_soc) {  // scalar rows (blocks dispatched last)
        const int sb = b - D.nb_exp - D.nb_soc;  // idle beyond this program's split (batches)
        const int stride = D.nb_scal * blockDim.x;
        for (int i = sb * blockDim.x + threadIdx.x; sb < D.nb_scal && i < D.m_scalar; i += stride) {
            const double v = val(i);
            out[i] = (i < D.m_zero) ? v : fmax(v, 0.0);
        }
    } else if (b >= D.nb_exp) {  // SOC / RSOC blocks
        const int stride = D.nb_soc * kWarpsPerBlock;
        for (int cidx = (b - D.nb_exp) * kWarpsPerBlock + wid; cidx < D.n_soc; cidx += stride) {
            if (D.soc_huge && D.soc_huge[cidx]) continue;  // grid-wise (soc_team)
            const int o = D.soc_off[cidx], dim = D.soc_dim[cidx];
            for (int i = lane; i < dim; i += 32) out[o + i] = val(o + i);
            __syncwarp();
            soc_project_any<true>(out + o, D.soc_w + o + 1, D.dr + o, dim, D.soc_rot[cidx] != 0, nullptr,
                                  reinterpret_cast<float*>(D.scr + (size_t)q * D.m + o), D.soc_wp + o + 1);
        }
    } else {
        const int stride = D.nb_exp * D.exp_pb;
        for (int e = b * D.exp_pb + threadIdx.x; threadIdx.x < D.exp_pb && e < D.n_exp; e += stride) {
            const int r = D.exp_row0 + 3 * e;
            double o3[3];
            exp_block_project(exp_kind_dual(D, e), true, val(r), val(r + 1), val(r + 2), D.dr[r], D.dr[r + 1],
                              D.dr[r + 2], D.exp_lg + 3 * e, o3, nullptr, D.exp_mlp);
            out[r] = o3[0];
            out[r + 1] = o3[1];
            out[r + 2] = o3[2];
        }
    }
}

// Primal-side KKT partials of candidate q = blockIdx.y (rows of K):
//   kpRp2  : ||v - Proj_{Dr C}(v)||^2, v = K~ xc - h~       (restart metric, scaled)
//   kpHy   : h~' yc                                          (dual objective part)
//   kpDy2  : ||yc - y0||^2                                   (primal weight update)
//   kpRmax : ||w - Proj_C(w)||_inf, w = K x - h = v / dr      (err_p numerator)
//   kpKxmax: ||K x||_inf, kpPmax: ||Proj_C(K x - h)||_inf     (err_p denominator)
template <typename T>
__device__ __forceinline__ void kkt_primal_body(const Dev<T>& D, int qidx) {
    const Ctrl* C = D.ctrl;
    if (C->status != kRunning) return;
    const int q = qidx;
    if (q >= n_candidates(C)) return;
    __shared__ double sm[3][kWarpsPerBlock];
    const double* kx = D.kxc + (size_t)q * D.m;
    const double* yc = D.yc + (size_t)q * D.m;
    double* s1 = D.scr + (size_t)q * D.m;  // scratch: scaled residual point
    double sums[3] = {0.0, 0.0, 0.0};      // rp2, hy, dy2
    double mx[3] = {0.0, 0.0, 0.0};        // rmax, kxmax, pmax
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    auto common = [&](int i) {
        sums[1] += D.h64[i] * yc[i];
        const double dy = yc[i] - (double)D.y0[i];
        sums[2] += dy * dy;
        mx[1] = fmax(mx[1], fabs(kx[i] / D.dr[i]));
    };
    if (b >= D.nb_exp + D.nb_soc) {  // scalar rows (blocks dispatched last)
        const int sb = b - D.nb_exp - D.nb_soc;  // idle beyond this program's split (batches)
        const int stride = D.nb_scal * blockDim.x;
        for (int i = sb * blockDim.x + threadIdx.x; sb < D.nb_scal && i < D.m_scalar; i += stride) {
            const double v = kx[i] - D.h64[i];
            const double w = v / D.dr[i];
            double rs, ru, pu;
            if (i < D.m_zero) { rs = v; ru = w; pu = 0.0; }
            else { rs = fmin(v, 0.0); ru = fmin(w, 0.0); pu = fmax(w, 0.0); }
            sums[0] += rs * rs;
            mx[0] = fmax(mx[0], fabs(ru));
            mx[2] = fmax(mx[2], fabs(pu));
            common(i);
        }
    } else if (b >= D.nb_exp) {  // SOC / RSOC blocks
        const int stride = D.nb_soc * kWarpsPerBlock;
        for (int cidx = (b - D.nb_exp) * kWarpsPerBlock + wid; cidx < D.n_soc; cidx += stride) {
            if (D.soc_huge && D.soc_huge[cidx]) continue;  // grid-wise (soc_team)
            const int o = D.soc_off[cidx], dim = D.soc_dim[cidx];
            const bool rot = D.soc_rot[cidx] != 0;
            // scaled residual: project v onto Dr K
            for (int i = lane; i < dim; i += 32) s1[o + i] = kx[o + i] - D.h64[o + i];
            __syncwarp();
            soc_project_any<false>(s1 + o, D.soc_wp + o + 1, D.dr + o, dim, rot, nullptr, nullptr, D.soc_w + o + 1);
            for (int i = lane; i < dim; i += 32) {
                const double v = kx[o + i] - D.h64[o + i];
                const double r = v - s1[o + i];
                sums[0] += r * r;
            }
            __syncwarp();
            // unscaled residual: project w = v / dr onto K (D = I)
            for (int i = lane; i < dim; i += 32) s1[o + i] = (kx[o + i] - D.h64[o + i]) / D.dr[o + i];
            __syncwarp();
            soc_project_any<false>(s1 + o, nullptr, nullptr, dim, rot, nullptr);
            for (int i = lane; i < dim; i += 32) {
                const double w = (kx[o + i] - D.h64[o + i]) / D.dr[o + i];
                mx[0] = fmax(mx[0], fabs(w - s1[o + i]));
                mx[2] = fmax(mx[2], fabs(s1[o + i]));
                common(o + i);
            }
            __syncwarp();
        }
    } else {
        const int stride = D.nb_exp * D.exp_pb;
        for (int e = b * D.exp_pb + threadIdx.x; threadIdx.x < D.exp_pb && e < D.n_exp; e += stride) {
            const int r = D.exp_row0 + 3 * e;
            double v[3], w[3], ps[3], pu[3];
            for (int k = 0; k < 3; ++k) {
                v[k] = kx[r + k] - D.h64[r + k];
                w[k] = v[k] / D.dr[r + k];
            }
            const double lg0[3] = {0.0, 0.0, 0.0};
            const bool kd = exp_kind_dual(D, e);
            exp_block_project(kd, false, v[0], v[1], v[2], D.dr[r], D.dr[r + 1], D.dr[r + 2], D.exp_lg + 3 * e, ps,
                              nullptr, D.exp_mlp);
            exp_block_project(kd, false, w[0], w[1], w[2], 1.0, 1.0, 1.0, lg0, pu, nullptr, D.exp_mlp);
            for (int k = 0; k < 3; ++k) {
                const double rs = v[k] - ps[k];
                sums[0] += rs * rs;
                mx[0] = fmax(mx[0], fabs(w[k] - pu[k]));
                mx[2] = fmax(mx[2], fabs(pu[k]));
                common(r + k);
            }
        }
    }
    block_sum<3>(sums, sm);
    block_max<3>(mx, sm);
    if (threadIdx.x == 0) {
        const int nb = D.pl.kktp_blocks;
        double* P = D.part + D.pl.off_kp + (size_t)q * kKktPN * nb;
        P[kpRp2 * nb + b] = sums[0];
        P[kpHy * nb + b] = sums[1];
        P[kpDy2 * nb + b] = sums[2];
        P[kpRmax * nb + b] = mx[0];
        P[kpKxmax * nb + b] = mx[1];
        P[kpPmax * nb + b] = mx[2];
    }
}

// Proj onto Lambda_j (eq. defn_Lambda1) from the bound pattern of column j
__device__ __forceinline__ double proj_lambda(double lam, double l, double u) {
    const bool lf = isfinite(l), uf = isfinite(u);
    if (!lf && !uf) return 0.0;
    if (!lf) return fmin(lam, 0.0);
    if (!uf) return fmax(lam, 0.0);
    return lam;
}

// restart / termination controller, run by the last block of kkt_dual
template <typename T>
__device__ void check_controller(const Dev<T>& D, double (*sm)[kWarpsPerBlock]) {
    Ctrl* C = D.ctrl;
    const int nc = n_candidates(C);
    double kp[2][kKktPN], kd[2][kKktDN];
    for (int q = 0; q < nc; ++q) {
        const int nbp = D.pl.kktp_blocks, nbd = D.pl.kktd_blocks;
        const double* P = D.part + D.pl.off_kp + (size_t)q * kKktPN * nbp;
        const double* Q = D.part + D.pl.off_kd + (size_t)q * kKktDN * nbd;
        kp[q][kpRp2] = block_reduce_parts(P + kpRp2 * nbp, nbp, sm);
        kp[q][kpHy] = block_reduce_parts(P + kpHy * nbp, nbp, sm);
        kp[q][kpDy2] = block_reduce_parts(P + kpDy2 * nbp, nbp, sm);
        kp[q][kpRmax] = block_max_parts(P + kpRmax * nbp, nbp, sm);
        kp[q][kpKxmax] = block_max_parts(P + kpKxmax * nbp, nbp, sm);
        kp[q][kpPmax] = block_max_parts(P + kpPmax * nbp, nbp, sm);
        kd[q][kdRd2] = block_reduce_parts(Q + kdRd2 * nbd, nbd, sm);
        kd[q][kdPobj] = block_reduce_parts(Q + kdPobj * nbd, nbd, sm);
        kd[q][kdBterm] = block_reduce_parts(Q + kdBterm * nbd, nbd, sm);
        kd[q][kdDx2] = block_reduce_parts(Q + kdDx2 * nbd, nbd, sm);
        kd[q][kdDmax] = block_max_parts(Q + kdDmax * nbd, nbd, sm);
        kd[q][kdKtymax] = block_max_parts(Q + kdKtymax * nbd, nbd, sm);
    }
    if (threadIdx.x != 0) return;
    C->ticket = 0;
    double err[2][3], comp[2][3], emax[2];
    bool finite = true;
    for (int q = 0; q < nc; ++q) {
        const double pobj = kd[q][kdPobj];
        const double dobj = kp[q][kpHy] + kd[q][kdBterm];
        const double gap = fabs(pobj - dobj);
        err[q][0] = kp[q][kpRmax] / (1.0 + fmax(C->hmax, fmax(kp[q][kpKxmax], kp[q][kpPmax])));
        err[q][1] = kd[q][kdDmax] / (1.0 + fmax(C->cmax, kd[q][kdKtymax]));
        err[q][2] = gap / (1.0 + fmax(fabs(pobj), fabs(dobj)));
        comp[q][0] = kp[q][kpRp2];
        comp[q][1] = kd[q][kdRd2];
        comp[q][2] = gap;
        emax[q] = fmax(err[q][0], fmax(err[q][1], err[q][2]));
        finite = finite && isfinite(emax[q]) && isfinite(comp[q][0]) && isfinite(comp[q][1]);
    }
    C->restart_now = 0;
    C->pending = 0;
    C->xnext = 0;  // a restart may move x: the next primal update forms x-hat again
    C->n_cand = nc;
    if (!finite) { C->status = kNumericError; return; }
    // solution = the better candidate of this check (current first)
    int sol = 0;
    if (nc == 2 && emax[1] < emax[0]) sol = 1;
    C->sol_cand = sol;
    for (int k = 0; k < 3; ++k) C->err[k] = err[sol][k];
    C->pobj = kd[sol][kdPobj];
    C->dobj = kp[sol][kpHy] + kd[sol][kdBterm];
    const double om = C->omega;
    auto phi_of = [&](const double* cc, double w) { return sqrt(w * cc[0] + cc[1] / w + cc[2] * cc[2]); };
    if (C->check_mode == 1) {  // initial evaluation of the anchor
        for (int k = 0; k < 3; ++k) C->comp0[k] = comp[0][k];
        C->phi0 = phi_of(comp[0], om);
        C->phi_prev = INFINITY;
        C->check_mode = 0;
        return;
    }
    if (C->tol > 0.0) {
        for (int q = 0; q < nc; ++q) {
            if (err[q][0] <= C->tol && err[q][1] <= C->tol && err[q][2] <= C->tol) {
                C->sol_cand = q;
                for (int k = 0; k < 3; ++k) C->err[k] = err[q][k];
                C->pobj = kd[q][kdPobj];
                C->dobj = kp[q][kpHy] + kd[q][kdBterm];
                C->status = kConverged;
                return;
            }
        }
    }
    if (C->step_mode == 2) return;  // plain PDHG: no restarts
    double phi[2];
    for (int q = 0; q < nc; ++q) phi[q] = phi_of(comp[q], om);
    const int best = (nc == 2 && phi[1] < phi[0]) ? 1 : 0;
    const double pc = phi[best];
    const bool restart = (pc <= 0.2 * C->phi0) || (pc <= 0.8 * C->phi0 && pc > C->phi_prev) ||
                         ((double)C->k >= 0.36 * (double)C->accepted);
    C->phi_prev = pc;
    if (!restart) return;
    const double dx = sqrt(kd[best][kdDx2]), dy = sqrt(kp[best][kpDy2]);
    double w = om;
    if (dx > 1e-10 && dy > 1e-10) w = exp(0.5 * log(dy / dx) + 0.5 * log(om));
    C->omega = w;
    C->tau = C->eta / w;
    C->sigma = C->eta * w;
    C->best = best;
    C->restart_now = 1;
    C->wsum = 0.0;
    C->k = 0;
    C->restarts += 1;
    for (int k = 0; k < 3; ++k) C->comp0[k] = comp[best][k];
    C->phi0 = phi_of(comp[best], w);
    C->phi_prev = INFINITY;
}

// Dual-side KKT partials of candidate q (columns of K), then the controller.
//   kdRd2  : ||lambda~ - Proj_Lambda(lambda~)||^2, lambda~ = c~ - K~' yc
//   kdPobj : c~' xc;  kdBterm : sum l~ mu^+ - u~ mu^-, mu = Proj_Lambda(lambda~)
//   kdDx2  : ||xc - x0||^2
//   kdDmax : ||lambda - Proj_Lambda(lambda)||_inf (original scale), kdKtymax : ||K'y||_inf
template <typename T>
__device__ __forceinline__ void kkt_dual_body(const Dev<T>& D, int qidx) {
    (void)qidx;
    Ctrl* C = D.ctrl;
    if (C->status != kRunning) return;
    const int nc = n_candidates(C);
    __shared__ double sm[4][kWarpsPerBlock];
    for (int q = 0; q < nc; ++q) {
        const double* xc = D.xc + (size_t)q * D.n;
        const double* kty = D.ktyc + (size_t)q * D.n;
        double sums[4] = {0.0, 0.0, 0.0, 0.0};
        double mx[2] = {0.0, 0.0};
        const int stride = gridDim.x * blockDim.x;
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D.n; j += stride) {
            const double ls = D.l64[j], us = D.u64[j];
            const double lam = D.c64[j] - kty[j];
            // a primal cone block's reduced costs were projected onto K_p^* by pc_apply; its
            // variables add no bound term (the infimum of mu'x over K_p is 0)
            const bool in_pc = (unsigned)(j - D.pc_lo) < (unsigned)D.pc_len;
            const double mu = in_pc ? D.pc_mu[(size_t)q * D.pc_len + (j - D.pc_lo)] : proj_lambda(lam, ls, us);
            sums[0] += (lam - mu) * (lam - mu);
            sums[1] += D.c64[j] * xc[j];
            if (!in_pc && mu > 0.0) sums[2] += ls * mu;
            if (!in_pc && mu < 0.0) sums[2] += us * mu;
            const double dx = xc[j] - (double)D.x0[j];
            sums[3] += dx * dx;
            const double lu = lam / D.dc[j];
            mx[0] = fmax(mx[0], fabs(lu - (in_pc ? mu / D.dc[j] : proj_lambda(lu, D.l_orig[j], D.u_orig[j]))));
            mx[1] = fmax(mx[1], fabs(kty[j] / D.dc[j]));
        }
        block_sum<4>(sums, sm);
        block_max<2>(mx, sm);
        if (threadIdx.x == 0) {
            const int nb = D.pl.kktd_blocks;
            double* Q = D.part + D.pl.off_kd + (size_t)q * kKktDN * nb;
            Q[kdRd2 * nb + blockIdx.x] = sums[0];
            Q[kdPobj * nb + blockIdx.x] = sums[1];
            Q[kdBterm * nb + blockIdx.x] = sums[2];
            Q[kdDx2 * nb + blockIdx.x] = sums[3];
            Q[kdDmax * nb + blockIdx.x] = mx[0];
            Q[kdKtymax * nb + blockIdx.x] = mx[1];
        }
    }
    if (last_block(C)) check_controller(D, sm);
}

// restart: z^{t+1,0} <- candidate `best` (and its cached products), averages reset
template <typename T>
__device__ __forceinline__ void restart_primal_body(const Dev<T>& D, int qidx) {
    (void)qidx;
    const Ctrl* C = D.ctrl;
    if (!C->restart_now) return;
    const int q = C->best;
    const double* xc = D.xc + (size_t)q * D.n;
    const double* kt = D.ktyc + (size_t)q * D.n;
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D.n; j += stride) {
        D.x[j] = D.x0[j] = (T)xc[j];
        D.kty[j] = D.kty0[j] = (T)kt[j];
        D.xsum[j] = T(0);
    }
}

template <typename T>
__device__ __forceinline__ void restart_dual_body(const Dev<T>& D, int qidx) {
    (void)qidx;
    const Ctrl* C = D.ctrl;
    if (!C->restart_now) return;
    const int q = C->best;
    const double* yc = D.yc + (size_t)q * D.m;
    const double* kx = D.kxc + (size_t)q * D.m;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D.m; i += stride) {
        D.y[i] = D.y0[i] = (T)yc[i];
        D.kx[i] = D.kx0[i] = (T)kx[i];
        D.ysum[i] = T(0);
    }
}


// ---------------------------------------------------------------------------
// Grid-wise projection of the large SOC / RSOC cones (team.cuh), one cooperative launch
// of team_nb blocks per use:
//   kTeamDual : the dual update's rows of those cones (FP64 iterates): pending Halpern
//               update, v, yhat = Proj(v), partials of ||dy||^2 and dy'(K xhat - K x) in the
//               dual-update slots after the role blocks; takes part in the step
//               controller's ticket like the role kernels;
//   kTeamCand : the dual candidates' projections (cand_dual skips these cones);
//   kTeamKkt  : the primal-side KKT partials of these cones' rows (kkt_primal skips them),
//               in the slots after kkt_primal's blocks.
// A block in no team entry writes zero partials.
// ---------------------------------------------------------------------------
enum TeamMode { kTeamDual = 0, kTeamCand = 1, kTeamKkt = 2 };

template <typename T>
__device__ __forceinline__ Team make_team(const Dev<T>& D, int e) {
    Team tm;
    tm.G = D.team_g[e];
    tm.slot0 = D.team_b0[e];
    tm.r = (int)blockIdx.x - tm.slot0;
    tm.slot = blockIdx.x;
    tm.stride = D.team_nb;
    tm.bar = D.team_bar + 2 * e;
    tm.part = D.team_part;
    tm.abort = &D.ctrl->team_abort;
    tm.phase = 0u;
    tm.ok = true;
    return tm;
}

template <typename T>
__device__ __forceinline__ bool in_team(const Dev<T>& D, int e) {
    const int b0 = D.team_b0[e];
    return (int)blockIdx.x >= b0 && (int)blockIdx.x < b0 + D.team_g[e];
}

// Records a wait that gave up (status kTimeout; the host reports PDCS_ERR_DEVICE_TIMEOUT).
__device__ __forceinline__ void team_report(Ctrl* C, bool ok) {
    if (!ok && threadIdx.x == 0) atomicExch(&C->status, (int)kTimeout);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) soc_team(Dev<T> D, int mode) {
    Ctrl* C = D.ctrl;
    if (C->status != kRunning) return;
    bool ok = true;
    if (mode == kTeamDual) {
        if constexpr (sizeof(T) == 8) {
            const DualCoef<T> k = dual_coef(D);
            T acc[2] = {T(0), T(0)};
            for (int e = 0; e < D.n_team; ++e) {
                if (!in_team(D, e)) continue;
                Team tm = make_team(D, e);
                const int c = D.team_cone[e], o = D.soc_off[c], dim = D.soc_dim[c];
                int rl, rh;
                team_rows(dim, tm.G, tm.r, rl, rh);
                for (int i = rl + (int)threadIdx.x; i < rh; i += blockDim.x) {
                    T y, kx;
                    dual_row_halpern(D, o + i, k.pend, k.ha, k.hb, k.hc, k.hw, k.pprev, y, kx);
                    D.yh[o + i] = y + k.sigma * (D.h[o + i] - T(2) * k.p[o + i] + kx);
                }
                __syncthreads();
                soc_team_project<true>(D.yh + o, SocWeightsArray{D.soc_w + o + 1, D.soc_wp + o + 1}, D.dr + o, dim,
                                       D.soc_rot[c] != 0, D.soc_lam + c, reinterpret_cast<float*>(D.scr + o), tm);
                for (int i = rl + (int)threadIdx.x; i < rh; i += blockDim.x) {
                    const T dy = D.yh[o + i] - D.y[o + i];
                    acc[0] += dy * dy;
                    acc[1] += dy * (k.p[o + i] - D.kx[o + i]);
                }
                ok = ok && tm.ok;
            }
            team_report(C, ok);
            dual_finish(D, D.team_gb0 + (int)blockIdx.x, acc);
        }
        return;
    }
    const int nc = n_candidates(C);
    for (int q = 0; q < nc; ++q) {
        if (mode == kTeamCand) {
            const double iw = q ? 1.0 / C->wsum : 0.0;
            double* out = D.yc + (size_t)q * D.m;
            const T* src = q ? D.ysum : D.y;
            for (int e = 0; e < D.n_team; ++e) {
                if (!in_team(D, e)) continue;
                Team tm = make_team(D, e);
                const int c = D.team_cone[e], o = D.soc_off[c], dim = D.soc_dim[c];
                int rl, rh;
                team_rows(dim, tm.G, tm.r, rl, rh);
                for (int i = rl + (int)threadIdx.x; i < rh; i += blockDim.x)
                    out[o + i] = q ? (double)src[o + i] * iw : (double)src[o + i];
                __syncthreads();
                soc_team_project<true>(out + o, SocWeightsArray{D.soc_w + o + 1, D.soc_wp + o + 1}, D.dr + o, dim,
                                       D.soc_rot[c] != 0, nullptr,
                                       reinterpret_cast<float*>(D.scr + (size_t)q * D.m + o), tm);
                ok = ok && tm.ok;
            }
        } else {
            __shared__ double sm[3][kWarpsPerBlock];
            const double* kx = D.kxc + (size_t)q * D.m;
            const double* yc = D.yc + (size_t)q * D.m;
            double* s1 = D.scr + (size_t)q * D.m;
            double sums[3] = {0.0, 0.0, 0.0};  // rp2, hy, dy2
            double mx[3] = {0.0, 0.0, 0.0};    // rmax, kxmax, pmax
            for (int e = 0; e < D.n_team; ++e) {
                if (!in_team(D, e)) continue;
                Team tm = make_team(D, e);
                const int c = D.team_cone[e], o = D.soc_off[c], dim = D.soc_dim[c];
                const bool rot = D.soc_rot[c] != 0;
                // FP32 copies in the other candidate's scratch rows of this cone (free here)
                float* f32 = reinterpret_cast<float*>(D.scr + (size_t)(1 - q) * D.m + o);
                int rl, rh;
                team_rows(dim, tm.G, tm.r, rl, rh);
                // scaled residual: project v = K~ xc - h~ onto Dr K
                for (int i = rl + (int)threadIdx.x; i < rh; i += blockDim.x) s1[o + i] = kx[o + i] - D.h64[o + i];
                __syncthreads();
                soc_team_project<false>(s1 + o, SocWeightsArray{D.soc_wp + o + 1, D.soc_w + o + 1}, D.dr + o, dim,
                                        rot, nullptr, f32, tm);
                for (int i = rl + (int)threadIdx.x; i < rh; i += blockDim.x) {
                    const double r = (kx[o + i] - D.h64[o + i]) - s1[o + i];
                    sums[0] += r * r;
                }
                __syncthreads();
                // unscaled residual: project w = v / dr onto K (D = I)
                for (int i = rl + (int)threadIdx.x; i < rh; i += blockDim.x)
                    s1[o + i] = (kx[o + i] - D.h64[o + i]) / D.dr[o + i];
                __syncthreads();
                soc_team_project<false>(s1 + o, SocWeightsArray{nullptr, nullptr}, nullptr, dim, rot, nullptr, f32,
                                        tm);
                for (int i = rl + (int)threadIdx.x; i < rh; i += blockDim.x) {
                    const double w = (kx[o + i] - D.h64[o + i]) / D.dr[o + i];
                    mx[0] = fmax(mx[0], fabs(w - s1[o + i]));
                    mx[2] = fmax(mx[2], fabs(s1[o + i]));
                    sums[1] += D.h64[o + i] * yc[o + i];
                    const double dy = yc[o + i] - (double)D.y0[o + i];
                    sums[2] += dy * dy;
                    mx[1] = fmax(mx[1], fabs(kx[o + i] / D.dr[o + i]));
                }
                __syncthreads();
                ok = ok && tm.ok;
            }
            block_sum<3>(sums, sm);
            block_max<3>(mx, sm);
            if (threadIdx.x == 0) {
                const int nb = D.pl.kktp_blocks, b = D.team_kb0 + (int)blockIdx.x;
                double* P = D.part + D.pl.off_kp + (size_t)q * kKktPN * nb;
                P[kpRp2 * nb + b] = sums[0];
                P[kpHy * nb + b] = sums[1];
                P[kpDy2 * nb + b] = sums[2];
                P[kpRmax * nb + b] = mx[0];
                P[kpKxmax * nb + b] = mx[1];
                P[kpPmax * nb + b] = mx[2];
            }
        }
    }
    team_report(C, ok);
}

// ---------------------------------------------------------------------------
// Batched SpMV (FP64 programs): program blockIdx.z.  mode 0: K xhat into the buffer of
// the evaluation's parity; 1: K' yhat (skipped after a rejected step); 2: K xc[q];
// 3: K' yc[q] (q = blockIdx.y).  Blocks beyond a program's plan are idle.
// ---------------------------------------------------------------------------
template <int U>
__global__ void __launch_bounds__(kBlock) spmv_batch(const Dev<double>* __restrict__ Ds, int mode) {
    const Dev<double>& D = Ds[blockIdx.z];
    const Ctrl* C = D.ctrl;
    if (C->status != kRunning) return;
    if (mode == 1 && !C->pending) return;
    const bool kt = mode == 1 || mode == 3;
    const SpmvBins& B = kt ? D.binsKT : D.binsK;
    if ((int)blockIdx.x >= B.blk[B.nbins]) return;
    int k = 0;
    while (k + 1 < B.nbins && (int)blockIdx.x >= B.blk[k + 1]) ++k;
    const int wb = ((int)blockIdx.x - B.blk[k]) * kWarpsPerBlock + (threadIdx.x >> 5);
    const int nwb = (B.blk[k + 1] - B.blk[k]) * kWarpsPerBlock;
    const int* l = (kt ? D.listKT : D.listK) + B.row[k];
    const int cnt = B.row[k + 1] - B.row[k];
    const int* rp = (kt ? D.rpT : D.rp) + B.row[k];
    const int q = blockIdx.y;
    const double* x;
    double* y;
    if (mode == 0) { x = D.xh; y = (C->attempts & 1) ? D.kxh1 : D.kxh0; }
    else if (mode == 1) { x = D.yh; y = D.ktyh; }
    else if (mode == 2) { x = D.xc + (size_t)q * D.n; y = D.kxc + (size_t)q * D.m; }
    else { x = D.yc + (size_t)q * D.m; y = D.ktyc + (size_t)q * D.n; }
    const int* ci = kt ? D.ciT : D.ci;
    const double* val = kt ? D.valT : D.val;
    switch (B.lanes[k]) {
        case 1: spmv_bin_rows<double, double, 1, U>(l, cnt, wb, nwb, rp, ci, val, x, y); break;
        case 2: spmv_bin_rows<double, double, 2, U>(l, cnt, wb, nwb, rp, ci, val, x, y); break;
        case 4: spmv_bin_rows<double, double, 4, U>(l, cnt, wb, nwb, rp, ci, val, x, y); break;
        case 8: spmv_bin_rows<double, double, 8, U>(l, cnt, wb, nwb, rp, ci, val, x, y); break;
        case 16: spmv_bin_rows<double, double, 16, U>(l, cnt, wb, nwb, rp, ci, val, x, y); break;
        default: spmv_bin_rows<double, double, 32, U>(l, cnt, wb, nwb, rp, ci, val, x, y); break;
    }
}

// ---------------------------------------------------------------------------
// Primal cone blocks x2 in K_p (Sec. 2, eq. prob_cp with n2 > 0): SOC / RSOC cones over
// variables.  Their column scales are tied per block, so D^{-1} K_p = K_p and the projection
// is the textbook one: (t, x) -> itself if ||x|| <= t, 0 if ||x|| <= -t, else
// a (1, x / ||x||) with a = (t + ||x||) / 2; an RSOC block is rotated by
// Q = [[1, 1], [1, -1]] / sqrt2 (+) I first and back after.  Two launches over the grid
// (cone k = blockIdx.x, chunk b = blockIdx.y, source q = blockIdx.z): pc_reduce writes each
// chunk's sum of squares of the (rotated) x part and, from chunk 0, the (rotated) first entry;
// pc_apply sums a cone's chunk partials in a fixed order (the same in every block of the cone)
// and projects its chunk.  Sources: kPcHat the x-hat of this evaluation, projected in place,
// with the cone variables' ||x-hat - x||^2 partials (primal_update leaves them out) in the
// primal slots after primal_update's; kPcCand the candidates, in place; kPcLam the candidates'
// reduced costs lambda = c - K'y, projected onto K_p^* (= K_p) into pc_mu for kkt_dual.
// ---------------------------------------------------------------------------
constexpr double kSqrtHalf = 0.70710678118654752440;

template <typename T>
__device__ __forceinline__ bool pc_active(const Dev<T>& D, int mode, int q) {
    const Ctrl* C = D.ctrl;
    if (C->status != kRunning) return false;
    if (mode == kPcHat) return C->xnext == 0;
    return q < n_candidates(C);
}

// entry j (a variable of a cone block) of source q
template <typename T>
__device__ __forceinline__ double pc_src(const Dev<T>& D, int mode, int q, int j) {
    if (mode == kPcHat) return (double)(D.ctrl->xsel ? D.xh1 : D.xh)[j];
    if (mode == kPcCand) return D.xc[(size_t)q * D.n + j];
    return D.c64[j] - D.ktyc[(size_t)q * D.n + j];
}

template <typename T>
__global__ void __launch_bounds__(kBlock) pc_reduce(Dev<T> D, int mode) {
    const int k = blockIdx.x, b = blockIdx.y, q = blockIdx.z;
    if (!pc_active(D, mode, q)) return;
    __shared__ double sm[1][kWarpsPerBlock];
    const int o = D.pc_off[k], d = D.pc_dim[k];
    const bool rot = D.pc_rot[k] != 0;
    const int i0 = b * kPcChunk, i1 = min(d, i0 + kPcChunk);
    double acc[1] = {0.0};
    for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x) {
        if (i == 0) continue;  // t
        const double v = pc_src(D, mode, q, o + i);
        const double w = (rot && i == 1) ? (pc_src(D, mode, q, o) - v) * kSqrtHalf : v;
        acc[0] += w * w;
    }
    block_sum<1>(acc, sm);
    if (threadIdx.x == 0) {
        D.pc_ss[((size_t)q * D.n_pc + k) * D.pc_nch + b] = acc[0];
        if (b == 0) {
            const double v0 = pc_src(D, mode, q, o);
            D.pc_t[(size_t)q * D.n_pc + k] = rot ? (v0 + pc_src(D, mode, q, o + 1)) * kSqrtHalf : v0;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) pc_apply(Dev<T> D, int mode) {
    const int k = blockIdx.x, b = blockIdx.y, q = blockIdx.z;
    if (!pc_active(D, mode, q)) return;
    __shared__ double sm[1][kWarpsPerBlock];
    __shared__ double s_t, s_sc;
    const int o = D.pc_off[k], d = D.pc_dim[k];
    const bool rot = D.pc_rot[k] != 0;
    const int i0 = b * kPcChunk, i1 = min(d, i0 + kPcChunk);
    double* slot = D.part + D.pl.off_px + D.pc_slot0 + (size_t)k * D.pc_nch + b;
    if (i0 >= i1) {
        if (mode == kPcHat && threadIdx.x == 0) *slot = 0.0;
        return;
    }
    const double ss = block_reduce_parts(D.pc_ss + ((size_t)q * D.n_pc + k) * D.pc_nch, D.pc_nch, sm);
    if (threadIdx.x == 0) {
        const double t = D.pc_t[(size_t)q * D.n_pc + k], nx = sqrt(ss);
        if (nx <= t) { s_t = t; s_sc = 1.0; }
        else if (nx <= -t) { s_t = 0.0; s_sc = 0.0; }
        else { const double a = 0.5 * (t + nx); s_t = a; s_sc = a / nx; }
    }
    __syncthreads();
    const double tn = s_t, sc = s_sc;
    T* xhat = D.ctrl->xsel ? D.xh1 : D.xh;
    double acc[1] = {0.0};
    auto put = [&](int j, double val) {
        if (mode == kPcHat) {
            xhat[j] = (T)val;
            const double dx = (double)(T)val - (double)D.x[j];
            acc[0] += dx * dx;
        } else if (mode == kPcCand) {
            D.xc[(size_t)q * D.n + j] = val;
        } else {
            D.pc_mu[(size_t)q * D.pc_len + (j - D.pc_lo)] = val;
        }
    };
    for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x) {
        if (rot && i == 1) continue;  // written with entry 0
        if (i == 0) {
            if (rot) {
                const double p1 = sc * ((pc_src(D, mode, q, o) - pc_src(D, mode, q, o + 1)) * kSqrtHalf);
                const double e0 = (tn + p1) * kSqrtHalf, e1 = (tn - p1) * kSqrtHalf;
                put(o, e0);
                put(o + 1, e1);
            } else {
                put(o, tn);
            }
        } else {
            put(o + i, sc * pc_src(D, mode, q, o + i));
        }
    }
    if (mode == kPcHat) {
        block_sum<1>(acc, sm);
        if (threadIdx.x == 0) *slot = acc[0];
    }
}

// ---------------------------------------------------------------------------
// Launch wrappers: one program (the view by value), or a batch of programs in one
// launch (views in device memory; the program is blockIdx.z, the candidate blockIdx.y).
// A batch shares one grid: every program is set up with the same block counts.
// ---------------------------------------------------------------------------
#define PDCS_KERNEL_PAIR(name)                                                               \
    template <typename T>                                                                    \
    __global__ void __launch_bounds__(kBlock) name(Dev<T> D) {                               \
        name##_body(D, blockIdx.y);                                                          \
    }                                                                                        \
    template <typename T>                                                                    \
    __global__ void __launch_bounds__(kBlock) name##_batch(const Dev<T>* __restrict__ Ds) {  \
        name##_body(Ds[blockIdx.z], blockIdx.y);                                             \
    }
PDCS_KERNEL_PAIR(primal_update)
PDCS_KERNEL_PAIR(dual_update)
PDCS_KERNEL_PAIR(flush_primal)
PDCS_KERNEL_PAIR(flush_dual)
PDCS_KERNEL_PAIR(cand_primal)
PDCS_KERNEL_PAIR(cand_dual)
PDCS_KERNEL_PAIR(kkt_primal)
PDCS_KERNEL_PAIR(kkt_dual)
PDCS_KERNEL_PAIR(restart_primal)
PDCS_KERNEL_PAIR(restart_dual)
#undef PDCS_KERNEL_PAIR

}  // namespace pdcs

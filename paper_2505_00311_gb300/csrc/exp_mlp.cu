// exp_mlp.cu -- the learned starting point of the exponential-cone root search:
// training pairs from the plain projector, forward / backward / Adam kernels, and
// projection statistics with and without the network.  Offline entry points: host
// arrays in, host arrays out, device memory allocated per call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/pdcs.h"
#include "common.cuh"
#include "cone_math.cuh"

using namespace pdcs;

static_assert(kExpMlpParams == PDCS_EXP_MLP_PARAMS, "parameter count");
static_assert(kExpMlpIn == PDCS_EXP_MLP_IN && kExpMlpHidden == PDCS_EXP_MLP_HIDDEN, "shape");

namespace {

constexpr int H = kExpMlpHidden, NI = kExpMlpIn;
// offsets of the parameter blocks
constexpr int oW1 = 0, oB1 = oW1 + H * NI, oW2 = oB1 + H, oB2 = oW2 + H * H, oW3 = oB2 + H, oB3 = oW3 + H;
// per-sample record of the forward / backward pass: x, h1, h2, delta1, delta2, delta3
constexpr int rX = 0, rH1 = rX + NI, rH2 = rH1 + H, rD1 = rH2 + H, rD2 = rD1 + H, rD3 = rD2 + H, kRec = rD3 + 1;

// ---- training pairs: case 4 of Theorem 3, plain FP64 search from no starting point
__global__ void dataset_kernel(long long n, const double* __restrict__ v, const double* __restrict__ d, float* feat,
                               float* target, int* flag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        flag[i] = 0;
        const double r0 = v[3 * i], s0 = v[3 * i + 1], t0 = v[3 * i + 2];
        const double dr = d[3 * i], ds = d[3 * i + 1], dt = d[3 * i + 2];
        if (!(dr > 0.0 && ds > 0.0 && dt > 0.0)) continue;
        if (in_kexp(r0 / dr, s0 / ds, t0 / dt) || in_kexp_dual(-dr * r0, -ds * s0, -dt * t0) ||
            (r0 <= 0.0 && s0 <= 0.0))
            continue;
        ExpCase4 e;
        exp_case4_setup(e, r0, s0, t0, dr, ds, log(dr), log(ds), log(dt), exp_ends(r0, s0, dr, ds));
        double L = 0.0;
        int evals = 0;
        // roots farther than e^-50 from the endpoint (about 2 % of N(0, 1) inputs, with a
        // tail to e^-36000) are left out: the search reaches them from its bracket, and as
        // regression targets they would swamp the typical range
        if (!exp_case4_solve(e, (double)NAN, L, evals) || !(fabs(L) <= 50.0)) continue;
        exp_mlp_features(e, feat + NI * i);
        target[i] = (float)L;
        flag[i] = 1;
    }
}

// ---- forward and backward pass of one sample per thread (loss = mean of (y - target)^2)
__global__ void fwd_bwd_kernel(int B, const float* __restrict__ feat, const float* __restrict__ target,
                               const long long* __restrict__ idx, const float* __restrict__ W, float* rec,
                               float* sq) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const long long k = idx ? idx[b] : b;
    float x[NI], z1[H], h1[H], z2[H], h2[H];
    for (int j = 0; j < NI; ++j) x[j] = feat[NI * k + j];
    for (int i = 0; i < H; ++i) {
        float a = W[oB1 + i];
        for (int j = 0; j < NI; ++j) a = fmaf(W[oW1 + i * NI + j], x[j], a);
        z1[i] = a;
        h1[i] = fmaxf(a, 0.0f);
    }
    float y = W[oB3];
    for (int i = 0; i < H; ++i) {
        float a = W[oB2 + i];
        for (int j = 0; j < H; ++j) a = fmaf(W[oW2 + i * H + j], h1[j], a);
        z2[i] = a;
        h2[i] = fmaxf(a, 0.0f);
        y = fmaf(W[oW3 + i], h2[i], y);
    }
    const float err = y - target[k];
    sq[b] = err * err;
    const float d3 = 2.0f * err / (float)B;  // dLoss/dy
    float d2[H];
    for (int i = 0; i < H; ++i) d2[i] = z2[i] > 0.0f ? W[oW3 + i] * d3 : 0.0f;
    float* r = rec + (size_t)kRec * b;
    for (int j = 0; j < H; ++j) {
        float a = 0.0f;
        for (int i = 0; i < H; ++i) a = fmaf(W[oW2 + i * H + j], d2[i], a);
        r[rD1 + j] = z1[j] > 0.0f ? a : 0.0f;
    }
    for (int j = 0; j < NI; ++j) r[rX + j] = x[j];
    for (int i = 0; i < H; ++i) {
        r[rH1 + i] = h1[i];
        r[rH2 + i] = h2[i];
        r[rD2 + i] = d2[i];
    }
    r[rD3] = d3;
}

// ---- gradient of one parameter per thread (sum over the batch in sample order), then
// the loss (thread 0 of block 0) and, when adam is set, the Adam update of the parameter
__device__ __forceinline__ float param_grad(int p, int B, const float* __restrict__ rec) {
    int a = -1, c = -1;  // factors: rec[a] * rec[c] (c < 0: the factor is 1)
    if (p < oB1) { a = rD1 + p / NI; c = rX + p % NI; }
    else if (p < oW2) { a = rD1 + (p - oB1); }
    else if (p < oB2) { a = rD2 + (p - oW2) / H; c = rH1 + (p - oW2) % H; }
    else if (p < oW3) { a = rD2 + (p - oB2); }
    else if (p < oB3) { a = rD3; c = rH2 + (p - oW3); }
    else { a = rD3; }
    float g = 0.0f;
    for (int b = 0; b < B; ++b) {
        const float* r = rec + (size_t)kRec * b;
        g = fmaf(r[a], c >= 0 ? r[c] : 1.0f, g);
    }
    return g;
}

__global__ void grad_kernel(int B, const float* __restrict__ rec, const float* __restrict__ sq, float* grad,
                            float* loss, float* W, float* m1, float* m2, int adam, float lr, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) {
        double s = 0.0;
        for (int b = 0; b < B; ++b) s += sq[b];
        *loss = (float)(s / B);
    }
    if (p >= kExpMlpParams) return;
    const float g = param_grad(p, B, rec);
    if (grad) grad[p] = g;
    if (adam) {
        const float mm = 0.9f * m1[p] + 0.1f * g;
        const float vv = 0.999f * m2[p] + 0.001f * g * g;
        m1[p] = mm;
        m2[p] = vv;
        W[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
    }
}

// SplitMix64 (Steele, Lea and Flood, 2014): minibatch indices drawn with replacement
__global__ void draw_kernel(int B, long long n, unsigned long long seed, long long step, long long* idx) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(step * B + b + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    idx[b] = (long long)(z % (unsigned long long)n);
}

// ---- cold-start projections with and without the network, with evaluation counts
__global__ void stats_kernel(long long n, const double* __restrict__ v, const double* __restrict__ d,
                             const float* mlp, double* out, int* evals) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double dr = d[3 * i], ds = d[3 * i + 1], dt = d[3 * i + 2];
        const double lg[3] = {log(dr), log(ds), log(dt)};
        int ev[2] = {0, 0};
        exp_project_fast(v[3 * i], v[3 * i + 1], v[3 * i + 2], dr, ds, dt, lg, out + 3 * i, nullptr, mlp, ev);
        evals[2 * i] = ev[0];
        evals[2 * i + 1] = ev[1];
    }
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    template <typename T>
    cudaError_t alloc(size_t count) { return cudaMalloc(&p, sizeof(T) * (count ? count : 1)); }
    template <typename T>
    T* as() { return static_cast<T*>(p); }
};

#define CKE(call)                                        \
    do {                                                 \
        if ((call) != cudaSuccess) return PDCS_ERR_CUDA; \
    } while (0)

int grid_for(long long k) { return (int)std::max(1LL, std::min((k + 255) / 256, 4096LL)); }

}  // namespace

extern "C" {

pdcs_status pdcs_exp_mlp_dataset(int64_t n, const double* v, const double* d, float* features, float* target,
                                 int64_t* kept) {
    if (n < 0 || (n > 0 && (!v || !d || !features || !target)) || !kept) return PDCS_ERR_INVALID;
    *kept = 0;
    if (n == 0) return PDCS_OK;
    DevBuf dv, dd, df, dt, dfl;
    CKE(dv.alloc<double>(3 * n)); CKE(dd.alloc<double>(3 * n)); CKE(df.alloc<float>(NI * n));
    CKE(dt.alloc<float>(n)); CKE(dfl.alloc<int>(n));
    CKE(cudaMemcpy(dv.p, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
    CKE(cudaMemcpy(dd.p, d, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
    dataset_kernel<<<grid_for(n), 256>>>(n, dv.as<double>(), dd.as<double>(), df.as<float>(), dt.as<float>(),
                                         dfl.as<int>());
    CKE(cudaGetLastError());
    std::vector<float> f((size_t)NI * n), t(n);
    std::vector<int> fl(n);
    CKE(cudaMemcpy(f.data(), df.p, sizeof(float) * NI * n, cudaMemcpyDeviceToHost));
    CKE(cudaMemcpy(t.data(), dt.p, sizeof(float) * n, cudaMemcpyDeviceToHost));
    CKE(cudaMemcpy(fl.data(), dfl.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!fl[i]) continue;
        for (int j = 0; j < NI; ++j) features[NI * k + j] = f[NI * i + j];
        target[k] = t[i];
        ++k;
    }
    *kept = k;
    return PDCS_OK;
}

pdcs_status pdcs_exp_mlp_loss_grad(int64_t n, const float* features, const float* target, const float* weights,
                                   float* grad, float* loss) {
    if (n < 1 || n > (1LL << 30) || !features || !target || !weights || !grad || !loss) return PDCS_ERR_INVALID;
    const int B = (int)n;
    DevBuf df, dt, dw, drec, dsq, dg, dl;
    CKE(df.alloc<float>(NI * n)); CKE(dt.alloc<float>(n)); CKE(dw.alloc<float>(kExpMlpParams));
    CKE(drec.alloc<float>((size_t)kRec * n)); CKE(dsq.alloc<float>(n)); CKE(dg.alloc<float>(kExpMlpParams));
    CKE(dl.alloc<float>(1));
    CKE(cudaMemcpy(df.p, features, sizeof(float) * NI * n, cudaMemcpyHostToDevice));
    CKE(cudaMemcpy(dt.p, target, sizeof(float) * n, cudaMemcpyHostToDevice));
    CKE(cudaMemcpy(dw.p, weights, sizeof(float) * kExpMlpParams, cudaMemcpyHostToDevice));
    fwd_bwd_kernel<<<(B + 127) / 128, 128>>>(B, df.as<float>(), dt.as<float>(), nullptr, dw.as<float>(),
                                             drec.as<float>(), dsq.as<float>());
    grad_kernel<<<(kExpMlpParams + 127) / 128, 128>>>(B, drec.as<float>(), dsq.as<float>(), dg.as<float>(),
                                                      dl.as<float>(), dw.as<float>(), nullptr, nullptr, 0, 0.f, 1.f,
                                                      1.f);
    CKE(cudaGetLastError());
    CKE(cudaMemcpy(grad, dg.p, sizeof(float) * kExpMlpParams, cudaMemcpyDeviceToHost));
    CKE(cudaMemcpy(loss, dl.p, sizeof(float), cudaMemcpyDeviceToHost));
    return PDCS_OK;
}

pdcs_status pdcs_exp_mlp_train(int64_t n, const float* features, const float* target, int32_t steps, int32_t batch,
                               float lr, uint64_t seed, float* weights, float* loss_trace) {
    if (n < 1 || steps < 0 || batch < 1 || batch > (1 << 22) || !(lr > 0.0f) || !features || !target || !weights)
        return PDCS_ERR_INVALID;
    const int B = batch;
    DevBuf df, dt, dw, drec, dsq, dl, dm1, dm2, didx, dtrace;
    CKE(df.alloc<float>(NI * n)); CKE(dt.alloc<float>(n)); CKE(dw.alloc<float>(kExpMlpParams));
    CKE(drec.alloc<float>((size_t)kRec * B)); CKE(dsq.alloc<float>(B)); CKE(dl.alloc<float>(1));
    CKE(dm1.alloc<float>(kExpMlpParams)); CKE(dm2.alloc<float>(kExpMlpParams)); CKE(didx.alloc<long long>(B));
    CKE(dtrace.alloc<float>(steps));
    CKE(cudaMemcpy(df.p, features, sizeof(float) * NI * n, cudaMemcpyHostToDevice));
    CKE(cudaMemcpy(dt.p, target, sizeof(float) * n, cudaMemcpyHostToDevice));
    CKE(cudaMemcpy(dw.p, weights, sizeof(float) * kExpMlpParams, cudaMemcpyHostToDevice));
    CKE(cudaMemset(dm1.p, 0, sizeof(float) * kExpMlpParams));
    CKE(cudaMemset(dm2.p, 0, sizeof(float) * kExpMlpParams));
    double b1t = 1.0, b2t = 1.0;
    for (int s = 0; s < steps; ++s) {
        b1t *= 0.9;
        b2t *= 0.999;
        draw_kernel<<<(B + 255) / 256, 256>>>(B, n, seed, s, didx.as<long long>());
        fwd_bwd_kernel<<<(B + 127) / 128, 128>>>(B, df.as<float>(), dt.as<float>(), didx.as<long long>(),
                                                 dw.as<float>(), drec.as<float>(), dsq.as<float>());
        grad_kernel<<<(kExpMlpParams + 127) / 128, 128>>>(B, drec.as<float>(), dsq.as<float>(), nullptr,
                                                          dtrace.as<float>() + s, dw.as<float>(), dm1.as<float>(),
                                                          dm2.as<float>(), 1, lr, (float)(1.0 - b1t),
                                                          (float)(1.0 - b2t));
    }
    CKE(cudaGetLastError());
    CKE(cudaMemcpy(weights, dw.p, sizeof(float) * kExpMlpParams, cudaMemcpyDeviceToHost));
    if (loss_trace && steps > 0) CKE(cudaMemcpy(loss_trace, dtrace.p, sizeof(float) * steps, cudaMemcpyDeviceToHost));
    return PDCS_OK;
}

pdcs_status pdcs_exp_proj_stats(int64_t n, const double* v, const double* d, const float* weights, double* out,
                                int32_t* evals) {
    if (n < 0 || (n > 0 && (!v || !d || !out || !evals))) return PDCS_ERR_INVALID;
    if (n == 0) return PDCS_OK;
    DevBuf dv, dd, dout, dev, dw;
    CKE(dv.alloc<double>(3 * n)); CKE(dd.alloc<double>(3 * n)); CKE(dout.alloc<double>(3 * n));
    CKE(dev.alloc<int>(2 * n));
    CKE(cudaMemcpy(dv.p, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
    CKE(cudaMemcpy(dd.p, d, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
    if (weights) {
        CKE(dw.alloc<float>(kExpMlpParams));
        CKE(cudaMemcpy(dw.p, weights, sizeof(float) * kExpMlpParams, cudaMemcpyHostToDevice));
    }
    stats_kernel<<<grid_for(n), 256>>>(n, dv.as<double>(), dd.as<double>(), weights ? dw.as<float>() : nullptr,
                                       dout.as<double>(), dev.as<int>());
    CKE(cudaGetLastError());
    CKE(cudaMemcpy(out, dout.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    CKE(cudaMemcpy(evals, dev.p, sizeof(int) * 2 * n, cudaMemcpyDeviceToHost));
    return PDCS_OK;
}

}  // extern "C"

// mlp.cu -- a small fully connected network (ReLU hidden layers, linear output, mean
// squared error) with its forward, backward and Adam kernels: the warm-start predictor
// of parametric program families (initial dual iterate and primal weight from a summary
// of the instance data).  Offline entry points: host arrays in and out, device memory
// allocated per call.  FP32 throughout with sums in a fixed order (deterministic).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "../../include/pdcs.h"

namespace {

struct Net {
    int L = 0;                   // weight layers
    std::vector<int> sz;         // L + 1 widths
    std::vector<size_t> wo, bo;  // offsets of W_l (out x in) and b_l in the parameter vector
    size_t params = 0;
    int widest = 0;
    bool init(int n_layers, const int32_t* sizes) {
        if (n_layers < 1 || n_layers > PDCS_MLP_MAX_LAYERS || !sizes) return false;
        L = n_layers;
        sz.assign(sizes, sizes + L + 1);
        for (int w : sz)
            if (w < 1 || w > PDCS_MLP_MAX_WIDTH) return false;
        widest = *std::max_element(sz.begin(), sz.end());
        params = 0;
        for (int l = 0; l < L; ++l) {
            wo.push_back(params);
            params += (size_t)sz[l + 1] * sz[l];
            bo.push_back(params);
            params += sz[l + 1];
        }
        return true;
    }
};

// Z = X W' + b (B x dout); Y = relu(Z) for hidden layers, Y = Z for the output layer
__global__ void dense_fwd(int B, int din, int dout, const float* __restrict__ X, const float* __restrict__ W,
                          const float* __restrict__ b, float* Z, float* Y, int relu) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * dout) return;
    const int s = (int)(t / dout), o = (int)(t % dout);
    const float* x = X + (size_t)s * din;
    const float* w = W + (size_t)o * din;
    float a = b[o];
    for (int i = 0; i < din; ++i) a = fmaf(w[i], x[i], a);
    Z[t] = a;
    Y[t] = relu ? fmaxf(a, 0.0f) : a;
}

// The same layer on the tensor cores: X and W rounded to BF16 as they are loaded, products
// accumulated in FP32 by mma.sync m16n8k16 tiles (one warp per 16 x 8 tile of Z, K in steps of
// 16, zero padding past din), bias and ReLU in FP32.  Fragment layout of the PTX ISA for
// m16n8k16 with 16-bit operands: lane = 4 g + t; A rows g and g + 8, columns 2t, 2t + 1 and
// 8 + 2t, 9 + 2t; B (k x n, "col") columns n = g, rows 2t, 2t + 1 and 8 + 2t, 9 + 2t;
// C rows g and g + 8, columns 2t, 2t + 1.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

__global__ void dense_fwd_bf16(int B, int din, int dout, const float* __restrict__ X, const float* __restrict__ W,
                               const float* __restrict__ b, float* Z, float* Y, int relu) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int tn = (dout + 7) / 8;
    if (warp >= (long long)((B + 15) / 16) * tn) return;  // whole warps
    const int m0 = (int)(warp / tn) * 16, n0 = (int)(warp % tn) * 8;
    const int g = lane >> 2, t = lane & 3;
    auto xa = [&](int r, int k) { return (r < B && k < din) ? X[(size_t)r * din + k] : 0.0f; };
    auto wb = [&](int n, int k) { return (n < dout && k < din) ? W[(size_t)n * din + k] : 0.0f; };
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int k0 = 0; k0 < din; k0 += 16) {
        const int ka = k0 + 2 * t, kb = k0 + 8 + 2 * t;
        const uint32_t a0 = pack_bf16(xa(m0 + g, ka), xa(m0 + g, ka + 1));
        const uint32_t a1 = pack_bf16(xa(m0 + g + 8, ka), xa(m0 + g + 8, ka + 1));
        const uint32_t a2 = pack_bf16(xa(m0 + g, kb), xa(m0 + g, kb + 1));
        const uint32_t a3 = pack_bf16(xa(m0 + g + 8, kb), xa(m0 + g + 8, kb + 1));
        const uint32_t b0 = pack_bf16(wb(n0 + g, ka), wb(n0 + g, ka + 1));
        const uint32_t b1 = pack_bf16(wb(n0 + g, kb), wb(n0 + g, kb + 1));
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = m0 + g + (q >= 2 ? 8 : 0), n = n0 + 2 * t + (q & 1);
        if (r < B && n < dout) {
            const float z = c[q] + b[n];
            Z[(size_t)r * dout + n] = z;
            Y[(size_t)r * dout + n] = relu ? fmaxf(z, 0.0f) : z;
        }
    }
}

// output error: dZ = 2 (Y - T) / (B dout), squared errors for the loss
__global__ void out_err(int B, int dout, const float* __restrict__ Y, const float* __restrict__ T,
                        const long long* __restrict__ idx, float* dZ, float* sq) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * dout) return;
    const int s = (int)(t / dout), o = (int)(t % dout);
    const long long k = idx ? idx[s] : s;
    const float e = Y[t] - T[(size_t)k * dout + o];
    sq[t] = e * e;
    dZ[t] = 2.0f * e / ((float)B * (float)dout);
}

// gradients of layer l: gW[o][i] = sum_s dZ[s][o] X[s][i], gb[o] = sum_s dZ[s][o]
__global__ void dense_grad(int B, int din, int dout, const float* __restrict__ X, const float* __restrict__ dZ,
                           float* gW, float* gb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= dout * (din + 1)) return;
    const int o = t / (din + 1), i = t % (din + 1);
    float a = 0.0f;
    for (int s = 0; s < B; ++s) a = fmaf(dZ[(size_t)s * dout + o], i < din ? X[(size_t)s * din + i] : 1.0f, a);
    if (i < din) gW[(size_t)o * din + i] = a;
    else gb[o] = a;
}

// back-propagated error into the previous hidden layer: dZp = (dZ W) masked by Zp > 0
__global__ void dense_back(int B, int din, int dout, const float* __restrict__ dZ, const float* __restrict__ W,
                           const float* __restrict__ Zp, float* dZp) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * din) return;
    const int s = (int)(t / din), i = (int)(t % din);
    float a = 0.0f;
    for (int o = 0; o < dout; ++o) a = fmaf(dZ[(size_t)s * dout + o], W[(size_t)o * din + i], a);
    dZp[t] = Zp[t] > 0.0f ? a : 0.0f;
}

__global__ void gather_rows(int B, int d, const float* __restrict__ X, const long long* __restrict__ idx, float* out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * d) return;
    const int s = (int)(t / d), j = (int)(t % d);
    out[t] = X[(size_t)idx[s] * d + j];
}

__global__ void sum_loss(long long k, const float* __restrict__ sq, float* loss) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double a = 0.0;
        for (long long i = 0; i < k; ++i) a += sq[i];
        *loss = (float)(a / (double)k);
    }
}

__global__ void adam_step(long long P, const float* __restrict__ g, float* W, float* m1, float* m2, float lr, float c1,
                          float c2) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const float mm = 0.9f * m1[p] + 0.1f * g[p];
    const float vv = 0.999f * m2[p] + 0.001f * g[p] * g[p];
    m1[p] = mm;
    m2[p] = vv;
    W[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
}

// SplitMix64 (Steele, Lea and Flood, 2014): minibatch rows drawn with replacement
__global__ void draw_rows(int B, long long n, unsigned long long seed, long long step, long long* idx) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(step * B + b + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    idx[b] = (long long)(z % (unsigned long long)n);
}

inline int blocks(long long k) { return (int)std::max(1LL, (k + 255) / 256); }

struct DevMem {
    std::vector<void*> ptrs;
    ~DevMem() { for (void* p : ptrs) cudaFree(p); }
    template <typename T>
    T* get(size_t count, cudaError_t& e) {
        void* p = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(&p, sizeof(T) * std::max<size_t>(count, 1));
        if (p) ptrs.push_back(p);
        return static_cast<T*>(p);
    }
};

// Work buffers of a batch of B rows: pre-activations and outputs of every layer, errors.
struct Work {
    std::vector<float*> Z, Y, dZ;
    float *sq = nullptr, *grad = nullptr, *loss = nullptr;
    cudaError_t alloc(DevMem& M, const Net& N, int B) {
        cudaError_t e = cudaSuccess;
        Z.resize(N.L + 1);
        Y.resize(N.L + 1);
        dZ.resize(N.L + 1);
        for (int l = 1; l <= N.L; ++l) {
            Z[l] = M.get<float>((size_t)B * N.sz[l], e);
            Y[l] = M.get<float>((size_t)B * N.sz[l], e);
            dZ[l] = M.get<float>((size_t)B * N.sz[l], e);
        }
        sq = M.get<float>((size_t)B * N.sz[N.L], e);
        grad = M.get<float>(N.params, e);
        loss = M.get<float>(1, e);
        return e;
    }
};

// forward pass of B rows X (already on the device); output in w.Y[L]
void forward(const Net& N, int B, const float* X, const float* W, Work& w) {
    const float* in = X;
    for (int l = 0; l < N.L; ++l) {
        const long long k = (long long)B * N.sz[l + 1];
        dense_fwd<<<blocks(k), 256>>>(B, N.sz[l], N.sz[l + 1], in, W + N.wo[l], W + N.bo[l], w.Z[l + 1], w.Y[l + 1],
                                      l + 1 < N.L);
        in = w.Y[l + 1];
    }
}

// the forward pass with every layer on the tensor cores (dense_fwd_bf16)
void forward_bf16(const Net& N, int B, const float* X, const float* W, Work& w) {
    const float* in = X;
    for (int l = 0; l < N.L; ++l) {
        const long long tiles = (long long)((B + 15) / 16) * ((N.sz[l + 1] + 7) / 8);
        dense_fwd_bf16<<<blocks(tiles * 32), 256>>>(B, N.sz[l], N.sz[l + 1], in, W + N.wo[l], W + N.bo[l],
                                                    w.Z[l + 1], w.Y[l + 1], l + 1 < N.L);
        in = w.Y[l + 1];
    }
}

// loss and gradient of B rows (targets T indexed by idx, or in order when idx is null)
void loss_grad(const Net& N, int B, const float* X, const float* T, const long long* idx, const float* W, Work& w) {
    forward(N, B, X, W, w);
    const int L = N.L;
    const long long ko = (long long)B * N.sz[L];
    out_err<<<blocks(ko), 256>>>(B, N.sz[L], w.Y[L], T, idx, w.dZ[L], w.sq);
    sum_loss<<<1, 32>>>(ko, w.sq, w.loss);
    for (int l = L - 1; l >= 0; --l) {
        const float* in = l == 0 ? X : w.Y[l];
        const int din = N.sz[l], dout = N.sz[l + 1];
        dense_grad<<<blocks((long long)dout * (din + 1)), 256>>>(B, din, dout, in, w.dZ[l + 1], w.grad + N.wo[l],
                                                                  w.grad + N.bo[l]);
        if (l > 0)
            dense_back<<<blocks((long long)B * din), 256>>>(B, din, dout, w.dZ[l + 1], W + N.wo[l], w.Z[l], w.dZ[l]);
    }
}

}  // namespace

#define CKM(e)                                                            \
    do {                                                                  \
        if ((e) != cudaSuccess) return (e) == cudaErrorMemoryAllocation   \
                                           ? PDCS_ERR_OOM                 \
                                           : PDCS_ERR_CUDA;               \
    } while (0)

extern "C" {

int64_t pdcs_mlp_params(int32_t n_layers, const int32_t* sizes) {
    Net N;
    return N.init(n_layers, sizes) ? (int64_t)N.params : -1;
}

pdcs_status pdcs_mlp_forward(int32_t n_layers, const int32_t* sizes, int64_t n, const float* X, const float* W,
                             float* Y) {
    Net N;
    if (!N.init(n_layers, sizes) || n < 1 || n > (1 << 24) || !X || !W || !Y) return PDCS_ERR_INVALID;
    const int B = (int)n;
    DevMem M;
    Work w;
    cudaError_t e = w.alloc(M, N, B);
    float* dX = M.get<float>((size_t)B * N.sz[0], e);
    float* dW = M.get<float>(N.params, e);
    CKM(e);
    CKM(cudaMemcpy(dX, X, sizeof(float) * B * N.sz[0], cudaMemcpyHostToDevice));
    CKM(cudaMemcpy(dW, W, sizeof(float) * N.params, cudaMemcpyHostToDevice));
    forward(N, B, dX, dW, w);
    CKM(cudaGetLastError());
    CKM(cudaMemcpy(Y, w.Y[N.L], sizeof(float) * B * N.sz[N.L], cudaMemcpyDeviceToHost));
    return PDCS_OK;
}

pdcs_status pdcs_mlp_forward_bf16(int32_t n_layers, const int32_t* sizes, int64_t n, const float* X, const float* W,
                                  float* Y) {
    Net N;
    if (!N.init(n_layers, sizes) || n < 1 || n > (1 << 24) || !X || !W || !Y) return PDCS_ERR_INVALID;
    const int B = (int)n;
    DevMem M;
    Work w;
    cudaError_t e = w.alloc(M, N, B);
    float* dX = M.get<float>((size_t)B * N.sz[0], e);
    float* dW = M.get<float>(N.params, e);
    CKM(e);
    CKM(cudaMemcpy(dX, X, sizeof(float) * B * N.sz[0], cudaMemcpyHostToDevice));
    CKM(cudaMemcpy(dW, W, sizeof(float) * N.params, cudaMemcpyHostToDevice));
    forward_bf16(N, B, dX, dW, w);
    CKM(cudaGetLastError());
    CKM(cudaMemcpy(Y, w.Y[N.L], sizeof(float) * B * N.sz[N.L], cudaMemcpyDeviceToHost));
    return PDCS_OK;
}

pdcs_status pdcs_mlp_loss_grad(int32_t n_layers, const int32_t* sizes, int64_t n, const float* X, const float* T,
                               const float* W, float* grad, float* loss) {
    Net N;
    if (!N.init(n_layers, sizes) || n < 1 || n > (1 << 24) || !X || !T || !W || !grad || !loss)
        return PDCS_ERR_INVALID;
    const int B = (int)n;
    DevMem M;
    Work w;
    cudaError_t e = w.alloc(M, N, B);
    float* dX = M.get<float>((size_t)B * N.sz[0], e);
    float* dT = M.get<float>((size_t)B * N.sz[N.L], e);
    float* dW = M.get<float>(N.params, e);
    CKM(e);
    CKM(cudaMemcpy(dX, X, sizeof(float) * B * N.sz[0], cudaMemcpyHostToDevice));
    CKM(cudaMemcpy(dT, T, sizeof(float) * B * N.sz[N.L], cudaMemcpyHostToDevice));
    CKM(cudaMemcpy(dW, W, sizeof(float) * N.params, cudaMemcpyHostToDevice));
    loss_grad(N, B, dX, dT, nullptr, dW, w);
    CKM(cudaGetLastError());
    CKM(cudaMemcpy(grad, w.grad, sizeof(float) * N.params, cudaMemcpyDeviceToHost));
    CKM(cudaMemcpy(loss, w.loss, sizeof(float), cudaMemcpyDeviceToHost));
    return PDCS_OK;
}

pdcs_status pdcs_mlp_train(int32_t n_layers, const int32_t* sizes, int64_t n, const float* X, const float* T,
                           int32_t steps, int32_t batch, float lr, uint64_t seed, float* W, float* loss_trace) {
    Net N;
    if (!N.init(n_layers, sizes) || n < 1 || steps < 0 || batch < 1 || batch > (1 << 20) || !(lr > 0.0f) || !X ||
        !T || !W)
        return PDCS_ERR_INVALID;
    const int B = batch;
    DevMem M;
    Work w;
    cudaError_t e = w.alloc(M, N, B);
    float* dX = M.get<float>((size_t)n * N.sz[0], e);
    float* dT = M.get<float>((size_t)n * N.sz[N.L], e);
    float* dW = M.get<float>(N.params, e);
    float* m1 = M.get<float>(N.params, e);
    float* m2 = M.get<float>(N.params, e);
    float* xb = M.get<float>((size_t)B * N.sz[0], e);
    long long* idx = M.get<long long>(B, e);
    float* trace = M.get<float>(std::max(steps, 1), e);
    CKM(e);
    CKM(cudaMemcpy(dX, X, sizeof(float) * n * N.sz[0], cudaMemcpyHostToDevice));
    CKM(cudaMemcpy(dT, T, sizeof(float) * n * N.sz[N.L], cudaMemcpyHostToDevice));
    CKM(cudaMemcpy(dW, W, sizeof(float) * N.params, cudaMemcpyHostToDevice));
    CKM(cudaMemset(m1, 0, sizeof(float) * N.params));
    CKM(cudaMemset(m2, 0, sizeof(float) * N.params));
    double b1t = 1.0, b2t = 1.0;
    for (int s = 0; s < steps; ++s) {
        b1t *= 0.9;
        b2t *= 0.999;
        draw_rows<<<blocks(B), 256>>>(B, n, seed, s, idx);
        gather_rows<<<blocks((long long)B * N.sz[0]), 256>>>(B, N.sz[0], dX, idx, xb);
        loss_grad(N, B, xb, dT, idx, dW, w);
        CKM(cudaMemcpyAsync(trace + s, w.loss, sizeof(float), cudaMemcpyDeviceToDevice));
        adam_step<<<blocks((long long)N.params), 256>>>((long long)N.params, w.grad, dW, m1, m2, lr,
                                                         (float)(1.0 - b1t), (float)(1.0 - b2t));
    }
    CKM(cudaGetLastError());
    CKM(cudaMemcpy(W, dW, sizeof(float) * N.params, cudaMemcpyDeviceToHost));
    if (loss_trace && steps > 0) CKM(cudaMemcpy(loss_trace, trace, sizeof(float) * steps, cudaMemcpyDeviceToHost));
    return PDCS_OK;
}

}  // extern "C"

// proj.cu -- pdcs_proj_cones_device: blockwise projection of a device vector
// onto D C or D^{-1} C* (eq. multi_cone_proj), the projection step of the
// solver exposed on its own for parity tests and projection benchmarks.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/pdcs.h"
#include "common.cuh"
#include "cone_math.cuh"

using namespace pdcs;

namespace {

// scalar blocks: one warp per block of rows; soc: one warp per cone; exp: one thread per cone
__global__ void proj_scalar(int nb, const int* __restrict__ off, const int* __restrict__ dim,
                            const unsigned char* __restrict__ type, const double* v, int dual, double* out) {
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = w; k < nb; k += nw) {
        const int o = off[k], d = dim[k];
        const bool zero = type[k] == kZero;
        for (int i = lane; i < d; i += 32) {
            const double x = v[o + i];
            out[o + i] = zero ? (dual ? x : 0.0) : fmax(x, 0.0);
        }
    }
}

__global__ void proj_soc(int nc, const int* __restrict__ off, const int* __restrict__ dim,
                         const unsigned char* __restrict__ rot, const double* v, const double* d, int dual,
                         double* out, float* scr) {
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = w; k < nc; k += nw) {
        const int o = off[k], dm = dim[k];
        if (out != v)
            for (int i = lane; i < dm; i += 32) out[o + i] = v[o + i];
        __syncwarp();
        const double* dd = d ? d + o : nullptr;
        // the solver's mixed-precision search (FP32 root, FP64 polish), weights from the
        // scales; blocks beyond the registers keep an FP32 copy in scr (2 floats per row)
        float* sc = scr ? scr + 2LL * o : nullptr;
        if (dual) soc_project_scaled<true>(out + o, dd, dm, rot[k] != 0, sc);
        else soc_project_scaled<false>(out + o, dd, dm, rot[k] != 0, sc);
    }
}

__global__ void proj_exp(int ne, const int* __restrict__ off, const double* v, const double* d, int dual, double* out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ne; k += stride) {
        const int o = off[k];
        const double r = v[o], s = v[o + 1], t = v[o + 2];
        const double dr = d ? d[o] : 1.0, ds = d ? d[o + 1] : 1.0, dt = d ? d[o + 2] : 1.0;
        const double lg[3] = {d ? log(dr) : 0.0, d ? log(ds) : 0.0, d ? log(dt) : 0.0};
        double p[3];
        // the solver's mixed-precision search (FP32 screening and root, FP64 result)
        if (dual) exp_dual_project_fast(r, s, t, dr, ds, dt, lg, p, nullptr);
        else exp_project_fast(r, s, t, dr, ds, dt, lg, p, nullptr);
        out[o] = p[0];
        out[o + 1] = p[1];
        out[o + 2] = p[2];
    }
}

}  // namespace

extern "C" pdcs_status pdcs_proj_cones_device(const double* v, const double* d, int64_t m, const pdcs_cone* cones,
                                              int64_t n_cones, int32_t dual, double* out, void* cuda_stream) {
    if (!v || !out || !cones || n_cones < 1 || m < 1 || m > 0x7fffffff) return PDCS_ERR_INVALID;
    std::vector<int> s_off, s_dim, soc_off, soc_dim, exp_off;
    std::vector<unsigned char> s_type, soc_rot;
    long long o = 0;
    for (int64_t k = 0; k < n_cones; ++k) {
        const int t = cones[k].type;
        const long long dm = cones[k].dim;
        if (t < PDCS_CONE_ZERO || t > PDCS_CONE_EXP || dm < 1 || (t == PDCS_CONE_EXP && dm != 3) ||
            (t == PDCS_CONE_RSOC && dm < 2))
            return PDCS_ERR_INVALID;
        if (t == PDCS_CONE_ZERO || t == PDCS_CONE_NONNEG) {
            s_off.push_back((int)o); s_dim.push_back((int)dm); s_type.push_back((unsigned char)t);
        } else if (t == PDCS_CONE_EXP) {
            exp_off.push_back((int)o);
        } else {
            soc_off.push_back((int)o); soc_dim.push_back((int)dm); soc_rot.push_back(t == PDCS_CONE_RSOC);
        }
        o += dm;
    }
    if (o != m) return PDCS_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t ns = s_off.size(), nc = soc_off.size(), ne = exp_off.size();
    const size_t bytes = sizeof(int) * (2 * ns + 2 * nc + ne) + ns + nc + 64;
    char* buf = nullptr;
    if (cudaMallocAsync(&buf, bytes, s) != cudaSuccess) return PDCS_ERR_CUDA;
    std::vector<char> host(bytes, 0);
    size_t p = 0;
    auto put = [&](const void* src, size_t sz) { std::copy((const char*)src, (const char*)src + sz, host.data() + p); size_t q = p; p += sz; return q; };
    const size_t o_soff = put(s_off.data(), sizeof(int) * ns), o_sdim = put(s_dim.data(), sizeof(int) * ns);
    const size_t o_coff = put(soc_off.data(), sizeof(int) * nc), o_cdim = put(soc_dim.data(), sizeof(int) * nc);
    const size_t o_eoff = put(exp_off.data(), sizeof(int) * ne);
    const size_t o_styp = put(s_type.data(), ns), o_crot = put(soc_rot.data(), nc);
    cudaError_t e = cudaMemcpyAsync(buf, host.data(), bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host staging buffer is pageable and local
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && ns) {
        const int g = (int)std::min<long long>((ns + 7) / 8, (long long)sms * 16);
        proj_scalar<<<g, kBlock, 0, s>>>((int)ns, (int*)(buf + o_soff), (int*)(buf + o_sdim),
                                         (unsigned char*)(buf + o_styp), v, dual, out);
    }
    float* scr = nullptr;  // FP32 copies of the blocks beyond the registers
    bool big = false;
    for (int dm : soc_dim) big = big || dm - 1 > 128;
    if (e == cudaSuccess && big && cudaMallocAsync(&scr, sizeof(float) * 2 * (size_t)m, s) != cudaSuccess) scr = nullptr;
    if (e == cudaSuccess && nc) {
        const int g = (int)std::min<long long>((nc + 7) / 8, (long long)sms * 16);
        proj_soc<<<g, kBlock, 0, s>>>((int)nc, (int*)(buf + o_coff), (int*)(buf + o_cdim),
                                      (unsigned char*)(buf + o_crot), v, d, dual, out, scr);
    }
    if (scr) cudaFreeAsync(scr, s);
    if (e == cudaSuccess && ne) {
        const int g = (int)std::min<long long>((ne + kBlock - 1) / kBlock, (long long)sms * 16);
        proj_exp<<<g, kBlock, 0, s>>>((int)ne, (int*)(buf + o_eoff), v, d, dual, out);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFreeAsync(buf, s);
    return e == cudaSuccess ? PDCS_OK : PDCS_ERR_CUDA;
}

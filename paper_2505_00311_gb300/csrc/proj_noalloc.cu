// proj_noalloc.cu -- pdcs_proj_cones_device_noalloc: the blockwise cone projection
// for callers that must not allocate device memory.  Its only scratch (the copied
// cone list and the row offset of every cone) lives in one file-scope device array
// of fixed size, so a call performs no cudaMalloc / cudaFree and no allocating
// library routine.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pdcs.h"
#include "common.cuh"
#include "cone_math.cuh"

using namespace pdcs;

namespace {

// Scratch: PDCS_NOALLOC_MAX_CONES cone records followed by as many 64-bit row offsets
// (6 MiB for 262,144 cones).  Every GPU that loads the library holds it until exit.
constexpr size_t kConeBytes = sizeof(pdcs_cone) * (size_t)PDCS_NOALLOC_MAX_CONES;
constexpr size_t kScratchBytes = kConeBytes + sizeof(long long) * (size_t)PDCS_NOALLOC_MAX_CONES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device.  In host code the
// symbol name is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

cudaError_t scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Exclusive prefix sum of the cone dimensions into the offsets (one block).
__global__ void noalloc_offsets(long long nc, const pdcs_cone* __restrict__ cones, long long* off) {
    __shared__ long long part[1024];
    const int t = threadIdx.x;
    const long long chunk = (nc + blockDim.x - 1) / blockDim.x;
    const long long b = t * chunk, e = (b + chunk < nc) ? b + chunk : nc;
    long long s = 0;
    for (long long k = b; k < e; ++k) s += cones[k].dim;
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        long long acc = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const long long v = part[i];
            part[i] = acc;
            acc += v;
        }
    }
    __syncthreads();
    long long acc = part[t];
    for (long long k = b; k < e; ++k) {
        off[k] = acc;
        acc += cones[k].dim;
    }
}

// One warp per cone: scalar cones loop over their rows, SOC / RSOC by the warp
// projection (Theorem 1), exp cones by lane 0 (Theorem 3 / the Remark).
__global__ void noalloc_project(long long nc, const pdcs_cone* __restrict__ cones, const long long* __restrict__ off,
                                const double* v, const double* d, int dual, double* out) {
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = w; k < nc; k += nw) {
        const int type = cones[k].type;
        const long long o = off[k];
        const int dm = (int)cones[k].dim;
        if (type == kZero || type == kNonneg) {
            for (int i = lane; i < dm; i += 32) {
                const double x = v[o + i];
                out[o + i] = type == kZero ? (dual ? x : 0.0) : fmax(x, 0.0);
            }
        } else if (type == kSoc || type == kRsoc) {
            if (out != v)
                for (int i = lane; i < dm; i += 32) out[o + i] = v[o + i];
            __syncwarp();
            const double* dd = d ? d + o : nullptr;
            if (type == kRsoc) {
                if (dual) rsoc_project_warp<true>(out + o, dd, dm, nullptr);
                else rsoc_project_warp<false>(out + o, dd, dm, nullptr);
            } else {
                if (dual) soc_project_warp<true>(out + o, dd, dm, nullptr);
                else soc_project_warp<false>(out + o, dd, dm, nullptr);
            }
        } else if (lane == 0) {
            const double r = v[o], s = v[o + 1], t = v[o + 2];
            const double dr = d ? d[o] : 1.0, ds = d ? d[o + 1] : 1.0, dt = d ? d[o + 2] : 1.0;
            double p[3];
            if (dual) exp_dual_project(r, s, t, dr, ds, dt, p, nullptr, nullptr);
            else exp_project(r, s, t, dr, ds, dt, p, nullptr, nullptr);
            out[o] = p[0];
            out[o + 1] = p[1];
            out[o + 2] = p[2];
        }
        __syncwarp();
    }
}

}  // namespace

extern "C" pdcs_status pdcs_proj_cones_device_noalloc(const double* v, const double* d, int64_t m,
                                                      const pdcs_cone* cones, int64_t n_cones, int32_t dual,
                                                      double* out, void* cuda_stream) {
    if (!v || !out || !cones || n_cones < 1 || m < 1 || m > 0x7fffffff) return PDCS_ERR_INVALID;
    if (n_cones > PDCS_NOALLOC_MAX_CONES) return PDCS_ERR_INVALID;
    long long tot = 0;
    for (int64_t k = 0; k < n_cones; ++k) {
        const int t = cones[k].type;
        const long long dm = cones[k].dim;
        if (t < PDCS_CONE_ZERO || t > PDCS_CONE_EXP || dm < 1 || dm > 0x7fffffff || (t == PDCS_CONE_EXP && dm != 3) ||
            (t == PDCS_CONE_RSOC && dm < 2))
            return PDCS_ERR_INVALID;
        tot += dm;
    }
    if (tot != m) return PDCS_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PDCS_ERR_CUDA;
    void* base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) return PDCS_ERR_CUDA;
    pdcs_cone* dcones = reinterpret_cast<pdcs_cone*>(base);
    long long* doff = reinterpret_cast<long long*>(static_cast<unsigned char*>(base) + kConeBytes);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemcpyAsync(dcones, cones, sizeof(pdcs_cone) * (size_t)n_cones, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return PDCS_ERR_CUDA;
    noalloc_offsets<<<1, 1024, 0, s>>>(n_cones, dcones, doff);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long grid = (n_cones + kWarpsPerBlock - 1) / kWarpsPerBlock;
    noalloc_project<<<(int)(grid < (long long)sms * 16 ? grid : (long long)sms * 16), kBlock, 0, s>>>(
        n_cones, dcones, doff, v, d, dual, out);
    return cudaGetLastError() == cudaSuccess ? PDCS_OK : PDCS_ERR_CUDA;
}

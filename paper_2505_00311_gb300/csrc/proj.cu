// proj.cu -- pdcs_proj_cones_device: blockwise projection of a device vector
// onto D C or D^{-1} C* (eq. multi_cone_proj), the projection step of the
// solver exposed on its own for parity tests and projection benchmarks; and the
// projection plan (pdcs_proj_plan_*), which builds the cone layout once and then only
// enqueues kernels, picking the strategy of each SOC cone by its dimension (Sec. 4:
// warp-wise up to kTeamMinDim rows, then teams of blocks of a cooperative launch).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pdcs.h"
#include "common.cuh"
#include "cone_math.cuh"
#include "team.cuh"

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

// kind (may be null): 1 for a K_exp^* (EXP_DUAL) block, projected with the inverse scales
// (D K_exp^* by the Remark, its dual D^{-1} K_exp directly)
__global__ void proj_exp(int ne, const int* __restrict__ off, const unsigned char* __restrict__ kind, const double* v,
                         const double* d, int dual, double* out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ne; k += stride) {
        const int o = off[k];
        const double r = v[o], s = v[o + 1], t = v[o + 2];
        const double dr = d ? d[o] : 1.0, ds = d ? d[o + 1] : 1.0, dt = d ? d[o + 2] : 1.0;
        const double lg[3] = {d ? log(dr) : 0.0, d ? log(ds) : 0.0, d ? log(dt) : 0.0};
        double p[3];
        // the solver's mixed-precision search (FP32 screening and root, FP64 result)
        if (kind && kind[k]) {
            const double li[3] = {-lg[0], -lg[1], -lg[2]};
            if (dual) exp_project_fast(r, s, t, 1.0 / dr, 1.0 / ds, 1.0 / dt, li, p, nullptr);
            else exp_dual_project_fast(r, s, t, 1.0 / dr, 1.0 / ds, 1.0 / dt, li, p, nullptr);
        } else if (dual) {
            exp_dual_project_fast(r, s, t, dr, ds, dt, lg, p, nullptr);
        } else {
            exp_project_fast(r, s, t, dr, ds, dt, lg, p, nullptr);
        }
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
    std::vector<unsigned char> s_type, soc_rot, exp_kind;
    long long o = 0;
    for (int64_t k = 0; k < n_cones; ++k) {
        const int t = cones[k].type;
        const long long dm = cones[k].dim;
        const bool ex = t == PDCS_CONE_EXP || t == PDCS_CONE_EXP_DUAL;
        if (t < PDCS_CONE_ZERO || t > PDCS_CONE_EXP_DUAL || dm < 1 || (ex && dm != 3) || (t == PDCS_CONE_RSOC && dm < 2))
            return PDCS_ERR_INVALID;
        if (t == PDCS_CONE_ZERO || t == PDCS_CONE_NONNEG) {
            s_off.push_back((int)o); s_dim.push_back((int)dm); s_type.push_back((unsigned char)t);
        } else if (ex) {
            exp_off.push_back((int)o);
            exp_kind.push_back(t == PDCS_CONE_EXP_DUAL);
        } else {
            soc_off.push_back((int)o); soc_dim.push_back((int)dm); soc_rot.push_back(t == PDCS_CONE_RSOC);
        }
        o += dm;
    }
    if (o != m) return PDCS_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t ns = s_off.size(), nc = soc_off.size(), ne = exp_off.size();
    const size_t bytes = sizeof(int) * (2 * ns + 2 * nc + ne) + ns + nc + ne + 64;
    char* buf = nullptr;
    if (cudaMallocAsync(&buf, bytes, s) != cudaSuccess) return PDCS_ERR_CUDA;
    std::vector<char> host(bytes, 0);
    size_t p = 0;
    auto put = [&](const void* src, size_t sz) { std::copy((const char*)src, (const char*)src + sz, host.data() + p); size_t q = p; p += sz; return q; };
    const size_t o_soff = put(s_off.data(), sizeof(int) * ns), o_sdim = put(s_dim.data(), sizeof(int) * ns);
    const size_t o_coff = put(soc_off.data(), sizeof(int) * nc), o_cdim = put(soc_dim.data(), sizeof(int) * nc);
    const size_t o_eoff = put(exp_off.data(), sizeof(int) * ne);
    const size_t o_styp = put(s_type.data(), ns), o_crot = put(soc_rot.data(), nc);
    const size_t o_ekind = put(exp_kind.data(), ne);
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
        proj_exp<<<g, kBlock, 0, s>>>((int)ne, (int*)(buf + o_eoff), (unsigned char*)(buf + o_ekind), v, d, dual,
                                      out);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFreeAsync(buf, s);
    return e == cudaSuccess ? PDCS_OK : PDCS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Projection plan
// ---------------------------------------------------------------------------
namespace {

constexpr int kPlanRowsPerBlock = 32768;  // x entries per block of a team (large SOC cones)
constexpr int kPlanEntriesPerLane = 32;   // D = I, small cones: lanes per cone S = 2^lg, dim <= 32 S

// D = I, SOC / RSOC cones of at most 4096 rows by lane groups: slice k holds 32 / S cones
// of one group size S = 2^lg[k] (cones c0[k] .. c0[k + 1] - 1 of the sorted list), one group
// per cone; lane g of a group takes rows 1 + g, 1 + g + S, ...  The textbook closed form
// (t + ||x||) / 2 (1, x / ||x||) when ||x|| > |t| (Q-transformed rows 1-2 for RSOC), 0 in
// the polar cone, v itself in the cone.  The per-cone scalar work (square root, division)
// is shared by the 32 / S cones of a warp instruction.
__global__ void __launch_bounds__(kBlock) proj_soc_unit(int nslices, const int* __restrict__ c0,
                                                        const unsigned char* __restrict__ lgs,
                                                        const int* __restrict__ off, const int* __restrict__ dim,
                                                        const unsigned char* __restrict__ rot,
                                                        const double* __restrict__ v, double* __restrict__ out) {
    const double r2 = 0.70710678118654752440;
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = w; k < nslices; k += nw) {
        const int lg = lgs[k], S = 1 << lg, g = lane & (S - 1);
        const int c = c0[k] + (lane >> lg);
        const bool ok = c < c0[k + 1];
        const int o = ok ? off[c] : 0, d = ok ? dim[c] : 0;
        const bool rq = ok && rot[c] != 0;
        double t = 0.0, x1 = 0.0, a = 0.0;
        if (ok) {
            t = v[o];
            if (d > 1) x1 = v[o + 1];
            if (rq) {
                const double p = t, q = x1;
                t = (p + q) * r2;
                x1 = (p - q) * r2;
            }
            if (g == 0 && d > 1) a = x1 * x1;
            for (int i = 1 + g + (g == 0 ? S : 0); i < d; i += S) a = fma(v[o + i], v[o + i], a);
        }
        for (int q = S >> 1; q > 0; q >>= 1) a += __shfl_xor_sync(0xffffffffu, a, q);
        if (!ok) continue;
        const double nx = sqrt(a);
        if (nx > fabs(t)) {
            const double top = 0.5 * (t + nx), sc = top / nx;
            for (int i = 1 + g + (g == 0 ? S : 0); i < d; i += S) out[o + i] = v[o + i] * sc;
            if (g == 0) {
                const double y1 = x1 * sc;
                if (rq) {
                    out[o] = (top + y1) * r2;
                    out[o + 1] = (top - y1) * r2;
                } else {
                    out[o] = top;
                    if (d > 1) out[o + 1] = y1;
                }
            }
        } else if (t <= 0.0) {
            for (int i = g; i < d; i += S) out[o + i] = 0.0;
        } else if (out != v) {
            for (int i = g; i < d; i += S) out[o + i] = v[o + i];
        }
    }
}

struct PlanTeams {
    int n_team, nb;
    const int* off;
    const int* dim;
    const unsigned char* rot;
    const int* b0;
    const int* g;
    unsigned* bar;
    double* part;
    int* abort;
};

// Large SOC / RSOC cones: entry e by blocks [b0[e], b0[e] + g[e]) (team.cuh), in table
// order; each block copies its own rows of v to out, then the team projects in place.
template <bool kInv>
__global__ void __launch_bounds__(kBlock) proj_team(PlanTeams T, const double* v, const double* d, double* out,
                                                    float* scr) {
    for (int e = 0; e < T.n_team; ++e) {
        const int b0 = T.b0[e], G = T.g[e];
        if ((int)blockIdx.x < b0 || (int)blockIdx.x >= b0 + G) continue;
        Team tm;
        tm.G = G; tm.slot0 = b0; tm.r = (int)blockIdx.x - b0; tm.slot = blockIdx.x; tm.stride = T.nb;
        tm.bar = T.bar + 2 * e; tm.part = T.part; tm.abort = T.abort; tm.phase = 0u; tm.ok = true;
        const int o = T.off[e], dim = T.dim[e];
        int rl, rh;
        team_rows(dim, G, tm.r, rl, rh);
        if (out != v)
            for (int i = rl + (int)threadIdx.x; i < rh; i += blockDim.x) out[o + i] = v[o + i];
        __syncthreads();
        const double* dd = d ? d + o : nullptr;
        soc_team_project<kInv>(out + o, SocWeightsScales<kInv>{dd, dd ? dd[0] : 1.0}, dd, dim, T.rot[e] != 0,
                               nullptr, scr + 2LL * o, tm);
        if (!tm.ok) return;
    }
}

}  // namespace

struct pdcs_proj_plan {
    int64_t m = 0;
    int sms = 152;
    int ns = 0, nc = 0, ne = 0;
    int *s_off = nullptr, *s_dim = nullptr, *c_off = nullptr, *c_dim = nullptr, *e_off = nullptr;
    unsigned char *s_type = nullptr, *c_rot = nullptr, *e_kind = nullptr;
    bool big_warp = false;  // a warp cone beyond the registers (FP32 copies in scr)
    int nsl = 0;            // lane-group slices of the warp cones (D = I runs)
    int* sl_c0 = nullptr;
    unsigned char* sl_lg = nullptr;
    PlanTeams T{};
    float* scr = nullptr;
    void* base = nullptr;
};

extern "C" pdcs_status pdcs_proj_plan_create(int64_t m, const pdcs_cone* cones, int64_t n_cones, void* cuda_stream,
                                             pdcs_proj_plan** out) {
    if (!out) return PDCS_ERR_INVALID;
    *out = nullptr;
    if (!cones || n_cones < 1 || m < 1 || m > 0x7fffffff) return PDCS_ERR_INVALID;
    std::vector<int> s_off, s_dim, c_off, c_dim, e_off, big;
    std::vector<unsigned char> s_type, c_rot, e_kind;
    std::vector<long long> offs(n_cones);
    long long o = 0, soc_rows = 0;
    for (int64_t k = 0; k < n_cones; ++k) {
        const int t = cones[k].type;
        const long long dm = cones[k].dim;
        const bool ex = t == PDCS_CONE_EXP || t == PDCS_CONE_EXP_DUAL;
        if (t < PDCS_CONE_ZERO || t > PDCS_CONE_EXP_DUAL || dm < 1 || (ex && dm != 3) ||
            (t == PDCS_CONE_RSOC && dm < 2) || o + dm > m)
            return PDCS_ERR_INVALID;
        offs[k] = o;
        if (t == PDCS_CONE_ZERO || t == PDCS_CONE_NONNEG) {
            s_off.push_back((int)o); s_dim.push_back((int)dm); s_type.push_back((unsigned char)t);
        } else if (ex) {
            e_off.push_back((int)o);
            e_kind.push_back(t == PDCS_CONE_EXP_DUAL);
        } else if (dm > kTeamMinDim) {
            big.push_back((int)k);
            soc_rows += dm;
        } else {
            c_off.push_back((int)o); c_dim.push_back((int)dm); c_rot.push_back(t == PDCS_CONE_RSOC);
        }
        o += dm;
    }
    if (o != m) return PDCS_ERR_INVALID;
    pdcs_proj_plan* P = new (std::nothrow) pdcs_proj_plan;
    if (!P) return PDCS_ERR_OOM;
    P->m = m;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int dm : c_dim) P->big_warp = P->big_warp || dm - 1 > 128;
    // teams of the large cones, largest first, packed into waves of at most one block per SM
    std::stable_sort(big.begin(), big.end(), [&](int a, int b) { return cones[a].dim > cones[b].dim; });
    int occ = 0;
    if (!big.empty() && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, proj_team<false>, kBlock, 0) != cudaSuccess)
        occ = 0;
    // up to four blocks per SM: the D = I passes are bound by the loads in flight per SM
    const int NB = P->sms * std::max(1, std::min(occ, 4));
    std::vector<int> t_off, t_dim, t_b0, t_g;
    std::vector<unsigned char> t_rot;
    if (!big.empty() && occ >= 1) {
        int free_b = NB;
        for (int k : big) {
            const long long nx = cones[k].dim - 1;
            const int g = (int)std::min<long long>(NB, std::max<long long>(1, (nx + kPlanRowsPerBlock - 1) / kPlanRowsPerBlock));
            if (g > free_b) free_b = NB;
            t_off.push_back((int)offs[k]); t_dim.push_back((int)cones[k].dim);
            t_rot.push_back(cones[k].type == PDCS_CONE_RSOC);
            t_b0.push_back(NB - free_b); t_g.push_back(g);
            free_b -= g;
        }
    } else {  // no cooperative launch possible: the large cones go warp by warp
        for (int k : big) {
            c_off.push_back((int)offs[k]); c_dim.push_back((int)cones[k].dim);
            c_rot.push_back(cones[k].type == PDCS_CONE_RSOC);
            P->big_warp = true;
        }
    }
    const int nt = (int)t_off.size();
    // warp cones sorted by the lane-group size of the D = I kernel (S = 2^lg, the smallest with
    // dim <= kPlanEntriesPerLane S, at most 32), cut into slices of 32 / S cones
    std::vector<int> sl_c0;
    std::vector<unsigned char> sl_lg;
    {
        const size_t nc0 = c_off.size();
        std::vector<unsigned char> lg(nc0);
        for (size_t k = 0; k < nc0; ++k) {
            int l = 0;
            while (l < 5 && c_dim[k] > kPlanEntriesPerLane * (1 << l)) ++l;
            lg[k] = (unsigned char)l;
        }
        std::vector<size_t> ord(nc0);
        for (size_t k = 0; k < nc0; ++k) ord[k] = k;
        std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return lg[a] < lg[b]; });
        std::vector<int> o2(nc0), d2(nc0);
        std::vector<unsigned char> r2(nc0);
        for (size_t k = 0; k < nc0; ++k) { o2[k] = c_off[ord[k]]; d2[k] = c_dim[ord[k]]; r2[k] = c_rot[ord[k]]; }
        c_off.swap(o2); c_dim.swap(d2); c_rot.swap(r2);
        for (size_t k = 0; k < nc0;) {
            const int l = lg[ord[k]], per = 32 >> l;
            sl_c0.push_back((int)k);
            sl_lg.push_back((unsigned char)l);
            size_t e = k;
            while (e < nc0 && e < k + per && lg[ord[e]] == l) ++e;
            k = e;
        }
        sl_c0.push_back((int)nc0);
    }
    P->nsl = (int)sl_lg.size();
    P->ns = (int)s_off.size(); P->nc = (int)c_off.size(); P->ne = (int)e_off.size();
    // one device allocation: the lists, the team barriers and partials, the abort flag, and
    // the FP32 scratch (2 floats per row) of the large cones' scaled projections
    const bool need_scr = P->big_warp || nt > 0;
    size_t bytes = 0;
    auto take = [&](size_t sz) { size_t q = bytes; bytes += (sz + 255) / 256 * 256; return q; };
    const size_t o_soff = take(sizeof(int) * P->ns), o_sdim = take(sizeof(int) * P->ns), o_styp = take(P->ns);
    const size_t o_coff = take(sizeof(int) * P->nc), o_cdim = take(sizeof(int) * P->nc), o_crot = take(P->nc);
    const size_t o_eoff = take(sizeof(int) * P->ne), o_ekind = take(P->ne);
    const size_t o_slc0 = take(sizeof(int) * (P->nsl + 1)), o_sllg = take(P->nsl);
    const size_t o_toff = take(sizeof(int) * nt), o_tdim = take(sizeof(int) * nt), o_trot = take(nt);
    const size_t o_tb0 = take(sizeof(int) * nt), o_tg = take(sizeof(int) * nt);
    const size_t o_bar = take(sizeof(unsigned) * (2 * nt + 2)), o_part = take(sizeof(double) * 2 * NB * kTeamQ);
    const size_t o_abort = take(sizeof(int));
    const size_t o_scr = take(need_scr ? sizeof(float) * 2 * (size_t)m : 0);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (cudaMalloc(&P->base, bytes) != cudaSuccess) {
        delete P;
        return PDCS_ERR_OOM;
    }
    char* b = (char*)P->base;
    std::vector<char> host(o_scr, 0);
    auto put = [&](size_t at, const void* src, size_t sz) { if (sz) std::memcpy(host.data() + at, src, sz); };
    put(o_soff, s_off.data(), sizeof(int) * P->ns); put(o_sdim, s_dim.data(), sizeof(int) * P->ns);
    put(o_styp, s_type.data(), P->ns);
    put(o_coff, c_off.data(), sizeof(int) * P->nc); put(o_cdim, c_dim.data(), sizeof(int) * P->nc);
    put(o_crot, c_rot.data(), P->nc);
    put(o_eoff, e_off.data(), sizeof(int) * P->ne); put(o_ekind, e_kind.data(), P->ne);
    put(o_slc0, sl_c0.data(), sizeof(int) * (P->nsl + 1)); put(o_sllg, sl_lg.data(), P->nsl);
    put(o_toff, t_off.data(), sizeof(int) * nt); put(o_tdim, t_dim.data(), sizeof(int) * nt);
    put(o_trot, t_rot.data(), nt); put(o_tb0, t_b0.data(), sizeof(int) * nt); put(o_tg, t_g.data(), sizeof(int) * nt);
    cudaError_t e = cudaMemcpyAsync(b, host.data(), o_scr, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the staging buffer is pageable and local
    if (e != cudaSuccess) {
        cudaFree(P->base);
        delete P;
        return PDCS_ERR_CUDA;
    }
    P->s_off = (int*)(b + o_soff); P->s_dim = (int*)(b + o_sdim); P->s_type = (unsigned char*)(b + o_styp);
    P->c_off = (int*)(b + o_coff); P->c_dim = (int*)(b + o_cdim); P->c_rot = (unsigned char*)(b + o_crot);
    P->e_off = (int*)(b + o_eoff); P->e_kind = (unsigned char*)(b + o_ekind);
    P->sl_c0 = (int*)(b + o_slc0); P->sl_lg = (unsigned char*)(b + o_sllg);
    P->T.n_team = nt; P->T.nb = NB;
    P->T.off = (int*)(b + o_toff); P->T.dim = (int*)(b + o_tdim); P->T.rot = (unsigned char*)(b + o_trot);
    P->T.b0 = (int*)(b + o_tb0); P->T.g = (int*)(b + o_tg);
    P->T.bar = (unsigned*)(b + o_bar); P->T.part = (double*)(b + o_part); P->T.abort = (int*)(b + o_abort);
    P->scr = need_scr ? (float*)(b + o_scr) : nullptr;
    *out = P;
    return PDCS_OK;
}

extern "C" pdcs_status pdcs_proj_plan_run(pdcs_proj_plan* P, const double* v, const double* d, int32_t dual,
                                          double* out, void* cuda_stream) {
    if (!P || !v || !out) return PDCS_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int sms = P->sms;
    if (P->ns) {
        const int g = (int)std::min<long long>((P->ns + 7) / 8, (long long)sms * 16);
        proj_scalar<<<g, kBlock, 0, s>>>(P->ns, P->s_off, P->s_dim, P->s_type, v, dual, out);
    }
    if (P->nc && d == nullptr) {  // D = I: closed form by lane groups (primal and dual: K_soc is self-dual)
        const int g = (int)std::min<long long>((P->nsl + 7) / 8, (long long)sms * 16);
        proj_soc_unit<<<g, kBlock, 0, s>>>(P->nsl, P->sl_c0, P->sl_lg, P->c_off, P->c_dim, P->c_rot, v, out);
    } else if (P->nc) {
        const int g = (int)std::min<long long>((P->nc + 7) / 8, (long long)sms * 16);
        proj_soc<<<g, kBlock, 0, s>>>(P->nc, P->c_off, P->c_dim, P->c_rot, v, d, dual, out,
                                      P->big_warp ? P->scr : nullptr);
    }
    cudaError_t e = cudaSuccess;
    if (P->T.n_team) {
        PlanTeams T = P->T;
        float* scr = P->scr;
        void* args[] = {(void*)&T, (void*)&v, (void*)&d, (void*)&out, (void*)&scr};
        const void* fn = dual ? (const void*)proj_team<true> : (const void*)proj_team<false>;
        e = cudaLaunchCooperativeKernel(fn, dim3(T.nb), dim3(kBlock), args, 0, s);
    }
    if (P->ne) {
        const int g = (int)std::min<long long>((P->ne + kBlock - 1) / kBlock, (long long)sms * 16);
        proj_exp<<<g, kBlock, 0, s>>>(P->ne, P->e_off, P->e_kind, v, d, dual, out);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? PDCS_OK : PDCS_ERR_CUDA;
}

extern "C" pdcs_status pdcs_proj_plan_check(pdcs_proj_plan* P, void* cuda_stream) {
    if (!P) return PDCS_ERR_INVALID;
    if (!P->T.n_team) return cudaStreamSynchronize((cudaStream_t)cuda_stream) == cudaSuccess ? PDCS_OK : PDCS_ERR_CUDA;
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, P->T.abort, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return PDCS_ERR_CUDA;
    return flag ? PDCS_ERR_DEVICE_TIMEOUT : PDCS_OK;
}

extern "C" void pdcs_proj_plan_destroy(pdcs_proj_plan* P) {
    if (!P) return;
    cudaDeviceSynchronize();
    cudaFree(P->base);
    delete P;
}

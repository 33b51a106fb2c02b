// kern_impl.cuh -- definitions of the launchers declared in launch.h for one value type
// (PDCS_DEFINE_LAUNCHERS(T) in each kernel translation unit).
#pragma once
#include "kernels.cuh"
#include "launch.h"

// dynamic shared memory of dual_soc: the SOC tiles of the FP64 path (one per warp)
template <typename T>
constexpr int dual_soc_smem() {
    return sizeof(T) == 8 ? pdcs::kWarpsPerBlock * pdcs::kSocTileRows * 32 : 0;
}

#define PDCS_DEFINE_LAUNCHERS(T)                                                                                   \
    namespace pdcs {                                                                                               \
    void k_primal_update(const Dev<T>& D, dim3 g, cudaStream_t s) { primal_update<T><<<g, kBlock, 0, s>>>(D); }   \
    void k_dual_update(const Dev<T>& D, dim3 g, cudaStream_t s) { dual_update<T><<<g, kBlock, 0, s>>>(D); }       \
    void k_dual_scalar(const Dev<T>& D, cudaStream_t s) {                                                          \
        if (D.nb_scal > 0) dual_scalar<T><<<D.nb_scal, kBlock, 0, s>>>(D);                                         \
    }                                                                                                              \
    void k_dual_soc(const Dev<T>& D, cudaStream_t s) {                                                             \
        if (D.nb_soc > 0) dual_soc<T><<<D.nb_soc, kBlock, dual_soc_smem<T>(), s>>>(D);                             \
    }                                                                                                              \
    cudaError_t k_prepare(const Dev<T>*) {                                                                         \
        return cudaFuncSetAttribute(dual_soc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, dual_soc_smem<T>()); \
    }                                                                                                              \
    void k_dual_exp(const Dev<T>& D, cudaStream_t s) {                                                             \
        if (D.nb_exp > 0) dual_exp<T><<<D.nb_exp, kBlock, 0, s>>>(D);                                              \
    }                                                                                                              \
    void k_flush_primal(const Dev<T>& D, dim3 g, cudaStream_t s) { flush_primal<T><<<g, kBlock, 0, s>>>(D); }     \
    void k_flush_dual(const Dev<T>& D, dim3 g, cudaStream_t s) { flush_dual<T><<<g, kBlock, 0, s>>>(D); }         \
    void k_cand_primal(const Dev<T>& D, dim3 g, cudaStream_t s) { cand_primal<T><<<g, kBlock, 0, s>>>(D); }       \
    void k_cand_dual(const Dev<T>& D, dim3 g, cudaStream_t s) { cand_dual<T><<<g, kBlock, 0, s>>>(D); }           \
    void k_kkt_primal(const Dev<T>& D, dim3 g, cudaStream_t s) { kkt_primal<T><<<g, kBlock, 0, s>>>(D); }         \
    void k_kkt_dual(const Dev<T>& D, dim3 g, cudaStream_t s) { kkt_dual<T><<<g, kBlock, 0, s>>>(D); }             \
    void k_restart_primal(const Dev<T>& D, dim3 g, cudaStream_t s) { restart_primal<T><<<g, kBlock, 0, s>>>(D); } \
    void k_restart_dual(const Dev<T>& D, dim3 g, cudaStream_t s) { restart_dual<T><<<g, kBlock, 0, s>>>(D); }     \
    cudaError_t k_soc_team(const Dev<T>& D, int mode, cudaStream_t s) {                                            \
        if (D.team_nb <= 0) return cudaSuccess;                                                                    \
        Dev<T> Dv = D;                                                                                             \
        int md = mode;                                                                                             \
        void* args[] = {(void*)&Dv, (void*)&md};                                                                   \
        return cudaLaunchCooperativeKernel((const void*)soc_team<T>, dim3(D.team_nb), dim3(kBlock), args, 0, s);   \
    }                                                                                                              \
    void k_pc(const Dev<T>& D, int mode, int nq, cudaStream_t s) {                                                 \
        if (D.n_pc <= 0) return;                                                                                   \
        const dim3 g(D.n_pc, D.pc_nch, nq);                                                                        \
        pc_reduce<T><<<g, kBlock, 0, s>>>(D, mode);                                                                \
        pc_apply<T><<<g, kBlock, 0, s>>>(D, mode);                                                                 \
    }                                                                                                              \
    int k_team_occupancy(const Dev<T>*) {                                                                          \
        int occ = 0;                                                                                               \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, soc_team<T>, kBlock, 0) == cudaSuccess ? occ : 0; \
    }                                                                                                              \
    void k_spmv(const SpmvBins& B, int unroll, cudaStream_t s, const int* list, const int* rp, const int* ci,     \
                const T* val, const T* x, T* y0, T* y1, const Ctrl* ctrl, int sel, int skip) {                     \
        const int grid = B.blk[B.nbins];                                                                           \
        if (grid <= 0) return;                                                                                     \
        switch (unroll) {                                                                                          \
            case 1: spmv_binned<T, T, 1><<<grid, kBlock, 0, s>>>(B, list, rp, ci, val, x, y0, y1, ctrl, sel, skip); break; \
            case 4: spmv_binned<T, T, 4><<<grid, kBlock, 0, s>>>(B, list, rp, ci, val, x, y0, y1, ctrl, sel, skip); break; \
            default: spmv_binned<T, T, 2><<<grid, kBlock, 0, s>>>(B, list, rp, ci, val, x, y0, y1, ctrl, sel, skip); break; \
        }                                                                                                          \
    }                                                                                                              \
    void k_spmv_sliced(const SlicePlan& S, cudaStream_t s, const int* ci, const T* val, const T* x, T* y0, T* y1, \
                       const Ctrl* ctrl, int sel, int skip, const T* xalt) {                                       \
        if (S.grid > 0) spmv_sliced<T, T><<<S.grid, kBlock, 0, s>>>(S, ci, val, x, y0, y1, ctrl, sel, skip, xalt); \
    }                                                                                                              \
    void k_spmv_kt_primal(const SlicePlan& S, cudaStream_t s, const int* ci, const T* val, const Dev<T>& D) {     \
        if (S.grid > 0) spmv_kt_primal<T><<<S.grid, kBlock, 0, s>>>(S, ci, val, D);                               \
    }                                                                                                              \
    void k_sliced_copy(const SlicePlan& S, int grid, cudaStream_t s, const int* rp, const int* ci,                \
                       const double* val, int* cis, T* vals) {                                                     \
        sliced_copy<T><<<grid, kBlock, 0, s>>>(S, rp, ci, val, cis, vals);                                        \
    }                                                                                                              \
    void k_bin_rows_copy(int grid, cudaStream_t s, int rows, const int* list, const int* rp, const int* ci,       \
                         const double* val, const int* rpb, int* cib, T* valb) {                                   \
        bin_rows_copy<double, T><<<grid, kBlock, 0, s>>>(rows, list, rp, ci, val, rpb, cib, valb);                 \
    }                                                                                                              \
    }

// launch.h -- host functions that launch the solver's kernels.  They are defined in the
// kernel translation units (kern_f64.cu, kern_f32.cu, kern_batch.cu), which compile in
// parallel; the host code (solver.cu) sees only these declarations.
#pragma once
#include <cuda_runtime.h>

#include "dev.h"

namespace pdcs {

#define PDCS_DECLARE_LAUNCHERS(T)                                                                                  \
    void k_primal_update(const Dev<T>& D, dim3 g, cudaStream_t s);                                                \
    void k_dual_update(const Dev<T>& D, dim3 g, cudaStream_t s);                                                  \
    void k_dual_scalar(const Dev<T>& D, cudaStream_t s);                                                          \
    void k_dual_soc(const Dev<T>& D, cudaStream_t s);                                                             \
    void k_dual_exp(const Dev<T>& D, cudaStream_t s);                                                             \
    /* once per process and device, before the first launch: kernel attributes (shared memory) */                 \
    cudaError_t k_prepare(const Dev<T>*);                                                                          \
    void k_flush_primal(const Dev<T>& D, dim3 g, cudaStream_t s);                                                 \
    void k_flush_dual(const Dev<T>& D, dim3 g, cudaStream_t s);                                                   \
    void k_cand_primal(const Dev<T>& D, dim3 g, cudaStream_t s);                                                  \
    void k_cand_dual(const Dev<T>& D, dim3 g, cudaStream_t s);                                                    \
    void k_kkt_primal(const Dev<T>& D, dim3 g, cudaStream_t s);                                                   \
    void k_kkt_dual(const Dev<T>& D, dim3 g, cudaStream_t s);                                                     \
    void k_restart_primal(const Dev<T>& D, dim3 g, cudaStream_t s);                                               \
    void k_restart_dual(const Dev<T>& D, dim3 g, cudaStream_t s);                                                 \
    /* grid-wise SOC cones (soc_team, mode 0 dual update, 1 candidates, 2 KKT): a cooperative  */                  \
    /* launch of D.team_nb blocks; nothing when D.team_nb == 0 */                                                  \
    cudaError_t k_soc_team(const Dev<T>& D, int mode, cudaStream_t s);                                            \
    /* primal cone blocks (pc_reduce then pc_apply; mode kPcHat, kPcCand or kPcLam over nq sources); */            \
    /* nothing when D.n_pc == 0 */                                                                                 \
    void k_pc(const Dev<T>& D, int mode, int nq, cudaStream_t s);                                                 \
    /* resident blocks per SM of soc_team (0 on error) */                                                          \
    int k_team_occupancy(const Dev<T>*);                                                                           \
    /* y = A x over the binned rows of B (see spmv_binned); unroll 1, 2 or 4 */                                    \
    void k_spmv(const SpmvBins& B, int unroll, cudaStream_t s, const int* list, const int* rp, const int* ci,     \
                const T* val, const T* x, T* y0, T* y1, const Ctrl* ctrl, int sel, int skip);                      \
    /* y = A x in the sliced storage of plan S (see spmv_sliced) */                                                 \
    void k_spmv_sliced(const SlicePlan& S, cudaStream_t s, const int* ci, const T* val, const T* x, T* y0, T* y1, \
                       const Ctrl* ctrl, int sel, int skip, const T* xalt);                                        \
    /* K' y-hat in the sliced storage of S with the next primal update in its epilogue (spmv_kt_primal) */        \
    void k_spmv_kt_primal(const SlicePlan& S, cudaStream_t s, const int* ci, const T* val, const Dev<T>& D);      \
    /* a CSR matrix (rows in order, FP64 values) in the sliced storage of S, values as T (vals may be null) */     \
    void k_sliced_copy(const SlicePlan& S, int grid, cudaStream_t s, const int* rp, const int* ci,                \
                       const double* val, int* cis, T* vals);                                                      \
    /* a CSR matrix (FP64 values) stored bin by bin with values of type T */                                       \
    void k_bin_rows_copy(int grid, cudaStream_t s, int rows, const int* list, const int* rp, const int* ci,       \
                         const double* val, const int* rpb, int* cib, T* valb);

PDCS_DECLARE_LAUNCHERS(double)
PDCS_DECLARE_LAUNCHERS(float)
#undef PDCS_DECLARE_LAUNCHERS

// Batches of FP64 programs (views in device memory; program = blockIdx.z).
enum BatchKernel {
    kbPrimalUpdate, kbDualUpdate, kbFlushPrimal, kbFlushDual, kbCandPrimal, kbCandDual, kbKktPrimal, kbKktDual,
    kbRestartPrimal, kbRestartDual
};
void k_batch(BatchKernel which, const Dev<double>* views, dim3 g, cudaStream_t s);
void k_spmv_batch(const Dev<double>* views, dim3 g, int mode, cudaStream_t s);

}  // namespace pdcs

// kern_batch.cu -- the solver's kernels for batches of FP64 programs.
#include "kernels.cuh"
#include "launch.h"

namespace pdcs {

void k_batch(BatchKernel which, const Dev<double>* views, dim3 g, cudaStream_t s) {
    switch (which) {
        case kbPrimalUpdate: primal_update_batch<double><<<g, kBlock, 0, s>>>(views); break;
        case kbDualUpdate: dual_update_batch<double><<<g, kBlock, 0, s>>>(views); break;
        case kbFlushPrimal: flush_primal_batch<double><<<g, kBlock, 0, s>>>(views); break;
        case kbFlushDual: flush_dual_batch<double><<<g, kBlock, 0, s>>>(views); break;
        case kbCandPrimal: cand_primal_batch<double><<<g, kBlock, 0, s>>>(views); break;
        case kbCandDual: cand_dual_batch<double><<<g, kBlock, 0, s>>>(views); break;
        case kbKktPrimal: kkt_primal_batch<double><<<g, kBlock, 0, s>>>(views); break;
        case kbKktDual: kkt_dual_batch<double><<<g, kBlock, 0, s>>>(views); break;
        case kbRestartPrimal: restart_primal_batch<double><<<g, kBlock, 0, s>>>(views); break;
        case kbRestartDual: restart_dual_batch<double><<<g, kBlock, 0, s>>>(views); break;
    }
}

void k_spmv_batch(const Dev<double>* views, dim3 g, int mode, cudaStream_t s) {
    spmv_batch<4><<<g, kBlock, 0, s>>>(views, mode);
}

}  // namespace pdcs

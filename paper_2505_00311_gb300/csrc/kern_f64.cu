// kern_f64.cu -- the solver's kernels for FP64 iterates (and the FP64 checks).
#include "kern_impl.cuh"
PDCS_DEFINE_LAUNCHERS(double)

// kern_f32.cu -- the solver's kernels for FP32 iterates (FP32-iterate mode).
#include "kern_impl.cuh"
PDCS_DEFINE_LAUNCHERS(float)

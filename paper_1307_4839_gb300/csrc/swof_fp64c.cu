// swof_fp64c.cu -- the FP64 stencil kernels again, with multiply-add
// contraction (built without -fmad=false): within 1e-12 of the oracle under
// its dt sequence, not bit for bit.  Selected per context by
// swof_set_fp64_contraction.
#define SWOF_FP64_CONTRACT 1
#include "swof_fp64.cu"

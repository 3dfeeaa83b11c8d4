// swof_fp64_reg.cu -- FP64 register-prefetch forms of the stage kernels.
// Built with -fmad=false and IEEE division / square root, like the FP64
// ring forms, so both give the oracle's values bit for bit.
#include "swof_reg.cuh"

SWOF_KERNELS_BEGIN

template int launch_stage_reg<double, 1, false>(int, const Params &, const Fields<double> &, cudaStream_t);
template int launch_stage_reg<double, 2, false>(int, const Params &, const Fields<double> &, cudaStream_t);
template int launch_stage_reg<double, 1, true>(int, const Params &, const Fields<double> &, cudaStream_t);

SWOF_KERNELS_END

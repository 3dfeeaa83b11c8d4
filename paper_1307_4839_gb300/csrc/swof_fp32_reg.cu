// swof_fp32_reg.cu -- FP32 register-prefetch forms of the stage kernels.
#include "swof_reg.cuh"

namespace swof {

template int launch_stage_reg<float, 1, false>(int, const Params &, const Fields<float> &, cudaStream_t);
template int launch_stage_reg<float, 2, false>(int, const Params &, const Fields<float> &, cudaStream_t);
template int launch_stage_reg<float, 1, true>(int, const Params &, const Fields<float> &, cudaStream_t);

}  // namespace swof

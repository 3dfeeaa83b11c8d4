// swof_fp64c_reg.cu -- register-prefetch forms of the contracted FP64
// stage kernels (see swof_fp64c.cu).
#define SWOF_FP64_CONTRACT 1
#include "swof_fp64_reg.cu"

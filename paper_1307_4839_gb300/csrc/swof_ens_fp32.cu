// swof_ens_fp32.cu -- FP32 instantiation of the
// ensemble kernel (built with -Xptxas -dlcm=cg, see swof_ensemble.cuh).
#include "swof_ensemble.cuh"

namespace swof {

int launch_ensemble_fp32(const void *desc, int ntx, int grid, void *stream)
{
    return launch_ensemble_t<float>(*static_cast<const EnsDesc<float> *>(desc), ntx, grid, (cudaStream_t)stream);
}

int ensemble_max_grid_fp32(int ntx, int *grid) { return ensemble_max_grid_t<float>(ntx, grid); }

}  // namespace swof

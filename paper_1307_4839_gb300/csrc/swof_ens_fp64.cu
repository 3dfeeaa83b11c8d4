// swof_ens_fp64.cu -- FP64 (-fmad=false, bit-identical to the single-grid FP64 path) instantiation of the
// ensemble kernel (built with -Xptxas -dlcm=cg, see swof_ensemble.cuh).
#include "swof_ensemble.cuh"

namespace swof {

int launch_ensemble_fp64(const void *desc, int ntx, int grid, void *stream)
{
    return launch_ensemble_t<double>(*static_cast<const EnsDesc<double> *>(desc), ntx, grid, (cudaStream_t)stream);
}

int ensemble_max_grid_fp64(int ntx, int *grid) { return ensemble_max_grid_t<double>(ntx, grid); }

}  // namespace swof

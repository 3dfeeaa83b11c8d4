// swof_fp64.cu -- FP64 instantiation of the stencil kernels.  Built with
// -fmad=false (no contraction of a*b+c) and IEEE division / square root so
// that every value matches the FP64 oracle's operation order bit for bit.
// swof_fp64c.cu compiles this file again with contraction allowed
// (SWOF_FP64_CONTRACT=1): launch_fp64c(), kernels in swof::fp64c.
#include "swof_kernels.cuh"
#include "swof_skip.cuh"

namespace swof {

#if SWOF_FP64_CONTRACT
const Launch &launch_fp64c()
#else
const Launch &launch_fp64()
#endif
{
    static const Launch L = {configure_t<double>, launch_ghosts_t<double>, launch_lambda_t<double>, launch_ring_t<double>,
                             launch_stage_t<double, 1>, launch_stage_t<double, 2>,
                             launch_stage1_o1_t<double>, launch_commit_o1_t<double>, launch_gauges_t<double>, launch_hmax_t<double>,
                             launch_pack1_t<double>,
                             launch_reduce_t<double>, stage_slots, launch_unpack_t<double>,
                             launch_pack_t<double>, launch_probe_t<double>};
    return L;
}

}  // namespace swof

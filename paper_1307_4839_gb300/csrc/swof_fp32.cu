// swof_fp32.cu -- FP32 bulk instantiation of the stencil kernels (difference
// form of z, FMA contraction allowed).  dt, time and budgets stay FP64.
#include "swof_kernels.cuh"
#include "swof_skip.cuh"

namespace swof {

const Launch &launch_fp32()
{
    static const Launch L = {configure_t<float>, launch_ghosts_t<float>, launch_lambda_t<float>, launch_ring_t<float>,
                             launch_stage_t<float, 1>, launch_stage_t<float, 2>,
                             launch_stage1_o1_t<float>, launch_commit_o1_t<float>, launch_gauges_t<float>, launch_hmax_t<float>,
                             launch_pack1_t<float>,
                             launch_reduce_t<float>, stage_slots, launch_unpack_t<float>,
                             launch_pack_t<float>, launch_probe_t<float>};
    return L;
}

}  // namespace swof

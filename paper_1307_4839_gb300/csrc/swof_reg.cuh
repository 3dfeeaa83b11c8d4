// swof_reg.cuh -- dispatch of the register-prefetch forms of the stage
// kernels (tile shapes N_RING_SHAPES..N_TILE_SHAPES - 1), instantiated in
// swof_fp32_reg.cu and swof_fp64_reg.cu so that both forms compile in
// parallel.
#pragma once
#include "swof_kernels.cuh"

SWOF_KERNELS_BEGIN

template <typename T, int STAGE, bool ORD1>
int launch_stage_reg(int cfg, const Params &P, const Fields<T> &F, cudaStream_t s)
{
    switch (cfg - N_RING_SHAPES) {
    case 1: return launch_sweep_reg<T, STAGE, 128, 64, ORD1>(P, F, s);
    case 2: return launch_sweep_reg<T, STAGE, 256, 32, ORD1>(P, F, s);
    case 3: return launch_sweep_reg<T, STAGE, 64, 64, ORD1>(P, F, s);
    case 4: return launch_sweep_reg<T, STAGE, 64, 16, ORD1>(P, F, s);
    default: return launch_sweep_reg<T, STAGE, 128, 32, ORD1>(P, F, s);
    }
}

SWOF_KERNELS_END

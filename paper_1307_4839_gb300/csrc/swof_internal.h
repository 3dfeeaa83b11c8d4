// swof_internal.h -- device-side data layout and launcher declarations of
// libswof (not part of the public ABI; see include/swof.h).
//
// Layout in HBM (padded SoA, one array per field):
//   (ny + 4) rows of `pitch` elements; row r holds grid row j = r - 2
//   (2 ghost rows below and above, Sec. 6.1: two layers at second order).
//   Within a row, element lpad + i is cell i, i in [-2, nx + 1]; lpad is 2
//   in both precisions, so the first ghost cell (i = -2) and the first
//   column of every stage tile (tile widths NTX - 4 are multiples of 4) sit
//   on a 16-byte boundary, as the stage kernels' tensor copies need.  pitch
//   is a multiple of 128 bytes; the columns past nx + 1 stay zero.
//   Corner ghosts are never read and stay zero.
#pragma once
#include <cuda.h>

#include <cstddef>
#include <cstdint>

#include "../../include/swof.h"

// Debug build: device-side index checks (libswof_debug.so; see swof.h).
#ifndef SWOF_BOUNDS_CHECK
#define SWOF_BOUNDS_CHECK 0
#endif

// The FP64 stencil is built twice: bit for bit with the oracle (-fmad=false)
// and with multiply-add contraction (swof_fp64c*.cu, SWOF_FP64_CONTRACT=1).
// The kernel headers open their namespace with SWOF_KERNELS_BEGIN, which in
// the contracted build adds an inline namespace, so the two builds' kernels
// and launchers have distinct symbols in one library.
#ifndef SWOF_FP64_CONTRACT
#define SWOF_FP64_CONTRACT 0
#endif
#if SWOF_FP64_CONTRACT
#define SWOF_KERNELS_BEGIN namespace swof { inline namespace fp64c {
#define SWOF_KERNELS_END } }
#else
#define SWOF_KERNELS_BEGIN namespace swof {
#define SWOF_KERNELS_END }
#endif

namespace swof {

// Per-context control block in device memory: the CFL reduction words, the
// dt of the step being taken, simulated time and latched status.
struct DevCtl {
    unsigned long long lam_bits[2];   // max wave speed x, y (bits of a double >= 0)
    unsigned long long lam2_bits[2];  // same at U* (CFL check)
    unsigned int done;                // blocks finished in the wave-speed kernel
    unsigned int done2;               // blocks finished in the U* check
    int status;                       // latched SWOF_E* (0 = ok)
    int rain_active;                  // rain falls during the current step
    double t;                         // simulated time (start of next step)
    double dt, dtdx, dtdy, rdt;       // current step: dt, dt/dx, dt/dy, dt*R
    double last_dt;
    long long steps;
    long long cfl_viol;
    double rain_in;                   // FP64 budget: rain volume
    int dt_seq_pos, dt_seq_n;
    float fdt, fdtdx, fdtdy, frdt;    // the same four in FP32 for the FP32 kernels
    long long gauge_n;                // gauge records written
    long long live_tiles, tiles;      // dry-tile skipping: tiles processed / offered
};

// Scalar parameters (by value into every kernel).
struct Params {
    int nx, ny, pitch, lpad;
    double dx, dy;
    double g, cfl, h_dry, dt_max, dt_min, t_end;
    int cfl_mode, friction, infiltration, check_cfl;
    int bc[4];                 // SWOF_BC_* per edge W, E, S, N
    int order;                 // 1: first order (one Euler stage); else 2
    double bc_h[4], bc_q[4];   // imposed edge depth / discharge
    double cf;                 // friction factor C_f (scalar, Sec. 2.1)
    double rain_rate, rain_t_on, rain_t_off;
    double ks, psi, dtheta;
    double dt_fixed;
    double area;               // unused by the arithmetic; dx*dy
    // FP32 copies of the scalars the FP32 kernels use (no FP64 on their path)
    float fg, fh_dry, fcf, fpsi, fdtheta, fks;
    float fdx, fdy;            // cell sizes for the FP32 budget terms
    float fbc_h[4], fbc_q[4];
    int tile_cfg;              // stage-1 kernel shape, index into the sweep shapes
    int tile_cfg2;             // stage-2 kernel shape
    int no_budget;             // 1: stage kernels leave the budget slots alone (timing runs)
    int fuse_lambda;           // 1: stage 2 adds the wave speeds of U^{n+1} of its tile interiors
    int lam_partial;           // 1: the wave-speed kernel only reduces (no dt control)
    int *status;               // the context's latched status word (debug build: failed index checks)
};

// Stage-kernel shapes: threads per CTA along x, rows per CTA, and how the
// input rows arrive (ring = 1: the TMA ring with the dry fast path; 0: the
// one-row register prefetch).  Shapes 5..9 are the register forms of 0..4.
struct TileShape {
    int ntx, h, ring;
};
constexpr int N_TILE_SHAPES = 10;
constexpr int N_RING_SHAPES = 5;
constexpr TileShape TILE_SHAPES[N_TILE_SHAPES] = {{128, 32, 1}, {128, 64, 1}, {256, 32, 1}, {64, 64, 1},
                                                  {64, 16, 1},  {128, 32, 0}, {128, 64, 0}, {256, 32, 0},
                                                  {64, 64, 0},  {64, 16, 0}};
constexpr int SHALLOW_SHAPE = 4;      // dry-tile skipping: short column walks
inline int max_stage_blocks(int nx, int ny)
{
    int m = 0;
    for (int k = 0; k < N_TILE_SHAPES; ++k) {
        int w = TILE_SHAPES[k].ntx - 4, h = TILE_SHAPES[k].h;
        int b = ((nx + w - 1) / w) * ((ny + h - 1) / h);
        m = b > m ? b : m;
    }
    return m;
}

// TMA tensor maps of a context's padded fields for one stage-tile width
// (box NTX columns x RING_ROWS rows): h, qx, qy, h1, qx1, qy1, then z (FP64)
// or dz_x, dz_y (FP32).  Passed to the stage kernels by value.
struct SweepMaps {
    CUtensorMap m[8];
};
constexpr int N_MAP_WIDTHS = 3;                 // tile widths NTX = 64, 128, 256
constexpr int RING_ROWS = 4;                    // rows per tensor copy of the stage ring
inline int map_width_index(int ntx) { return ntx == 64 ? 0 : (ntx == 128 ? 1 : 2); }

// cuTensorMapEncodeTiled, looked up from the driver at run time
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled();

// Device pointers of one context.  T = double (FP64) or float (FP32).
template <typename T>
struct Fields {
    T *h, *qx, *qy;            // U^n (updated in place by stage 2)
    T *h1, *qx1, *qy1;         // U* (stage-1 output)
    T *z;                      // FP64 path: topography (padded)
    T *dzx, *dzy;              // FP32 path: z(i+1)-z(i), z(j+1)-z(j) per face (padded)
    T *cfmap;                  // per-cell friction factor C_f (padded) or nullptr
    T *ksmap;                  // per-cell K_s (padded) or nullptr
    T *vinf;                   // infiltrated depth (padded)
    double *outflow_slots;     // per-block FP64 budget accumulators
    double *infil_slots;
    const int *ring_cols;      // columns / rows whose wave speeds stage 2 leaves out
    const int *ring_rows;      //   (tile-edge columns/rows for the current tile shape)
    int n_ring_cols, n_ring_rows;
    int ring_tw, ring_th, ring_tgx;   // that shape's tile width, height, tiles per row
    const double *dt_seq;      // replayed dt values or nullptr
    double *dt_hist;           // dt of every step
    long long dt_hist_cap;
    DevCtl *ctl;
    T *hmax;                   // running maximum depth (padded) or nullptr
    const long long *gauge_off;  // padded offsets of the gauge cells
    int n_gauges;
    long long gauge_cap;
    double *gauge_rec;         // [gauge_cap][1 + 3 n_gauges]
    unsigned char *tile_act;   // dry-tile skipping: tile holds water after the step
    unsigned char *tile_live;  //   tile processed in the current step (nullptr: off)
    const SweepMaps *tmaps;    // host memory: the stage kernels' tensor maps per tile width
};

// Launchers, one set per precision (swof_fp64.cu, swof_fp32.cu).  All
// enqueue on `stream` and return cudaError_t as int.
struct Launch {
    int (*configure)();              // per-device kernel attributes
    int (*ghosts)(const Params &, void *fields, void *stream);
    int (*lambda)(const Params &, void *fields, void *stream);
    int (*lambda_ring)(const Params &, void *fields, void *stream);
    int (*stage1)(const Params &, void *fields, void *stream);
    int (*stage2)(const Params &, void *fields, void *stream);
    int (*stage1_o1)(const Params &, void *fields, void *stream);   // first-order stage
    int (*commit_o1)(const Params &, void *fields, void *stream);   // first-order step end
    int (*gauges)(const Params &, void *fields, void *stream);
    int (*hmax)(const Params &, void *fields, void *stream);
    int (*pack1)(const Params &, const void *src, double *dst, void *stream);
    int (*reduce)(const Params &, void *fields, double *out, int nslots, void *stream);
    int (*slots)(const Params &);    // number of per-block slots the stage kernels use
    // dense [ny][nx] device arrays (dtype SWOF_FP64/FP32) <-> padded state
    int (*unpack)(const Params &, void *fields, const void *h, const void *qx, const void *qy,
                  int dtype, void *stream);
    int (*pack)(const Params &, void *fields, void *h, void *qx, void *qy, int dtype, void *stream);
    // debug build: form the padded index of cell (i, j) through the checked path
    int (*probe)(const Params &, void *fields, int i, int j, void *stream);
};

const Launch &launch_fp64();
const Launch &launch_fp64c();   // FP64 with multiply-add contraction
const Launch &launch_fp32();

}  // namespace swof

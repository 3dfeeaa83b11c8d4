// swof_d8.cu -- D8 flow directions of a DEM (sm_103a), the eight-neighbour
// example of arXiv 1307.4839 Sec. 5.2: for every cell, the neighbour of
// smallest elevation among those strictly below it (code 1..8 = E, NE, N,
// NW, W, SW, S, SE; 0 when none is lower; ties to the first code;
// neighbours outside the grid, or at z <= nodata when a no-data value is
// given, are no candidates).
//
// 4 bytes read and 1 written per cell.  A warp owns a strip of 256
// columns (8 per lane, two 16-byte loads per lane and row) and walks an
// equal share of its rows with a three-row register window; the columns beside the
// strip come from the neighbouring lanes by shuffle, and from two scalar
// loads at the strip's ends.  The next row is loaded one iteration ahead.
// Without a no-data value the selection is three instructions per
// neighbour; it is what bounds the kernel (issue), not the bytes.
// Values outside the grid are NaN, which no comparison selects.  The grid
// is one wave of resident blocks, each looping over work items.
// Rows whose width is not a multiple of 4 (or unaligned arrays) take the
// same walk with one column per lane.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/swof.h"

namespace {

constexpr int D8_ROWS = 64;       // rows per work item (general widths)
constexpr int D8_WARPS = 8;       // warps per block

__device__ __forceinline__ float nanf_() { return __int_as_float(0x7fc00000); }

// code of one cell from its value and its 8 neighbours in code order
template <bool NODATA>
__device__ __forceinline__ unsigned d8_code(float c, float e, float ne, float n, float nw, float w, float sw, float s,
                                            float se, float nodata)
{
    float best = c;
    unsigned code = 0;
    const float v[8] = {e, ne, n, nw, w, sw, s, se};
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if ((!NODATA || v[k] > nodata) && v[k] < best) {
            best = v[k];
            code = k + 1;
        }
    return code;
}

// One row of a 256-column strip: lane values x[1..8] (two 16-byte loads),
// x[0] / x[9] the columns left of / right of the lane's eight.
struct Row8 {
    float x[10];
};

__device__ __forceinline__ Row8 load_row8(const float *__restrict__ z, int nx, int ny, int row, int c0, int lane)
{
    Row8 r;
    float4 a = make_float4(nanf_(), nanf_(), nanf_(), nanf_()), b = a;
    const int col = c0 + 8 * lane;
    const bool rin = row >= 0 && row < ny;
    const float *p = z + (size_t)row * nx + col;
    if (rin && col < nx) a = __ldg(reinterpret_cast<const float4 *>(p));
    if (rin && col + 4 < nx) b = __ldg(reinterpret_cast<const float4 *>(p + 4));
    float l = __shfl_up_sync(0xffffffffu, b.w, 1);
    float rr = __shfl_down_sync(0xffffffffu, a.x, 1);
    if (lane == 0) l = (rin && c0 > 0) ? __ldg(z + (size_t)row * nx + c0 - 1) : nanf_();
    if (lane == 31) rr = (rin && c0 + 256 < nx) ? __ldg(z + (size_t)row * nx + c0 + 256) : nanf_();
    r.x[0] = l;
    r.x[1] = a.x; r.x[2] = a.y; r.x[3] = a.z; r.x[4] = a.w;
    r.x[5] = b.x; r.x[6] = b.y; r.x[7] = b.z; r.x[8] = b.w;
    r.x[9] = rr;
    return r;
}

template <bool NODATA>
__global__ void __launch_bounds__(32 * D8_WARPS) k_d8_vec(const float *__restrict__ z, int nx, int ny, float nodata,
                                                         unsigned char *__restrict__ dir)
{
    const int lane = threadIdx.x & 31;
    // every warp of the (one-wave) grid gets one equal run of rows of a strip
    const int strips = (nx + 255) / 256;
    const long long warps = (long long)gridDim.x * D8_WARPS;
    const int chunks = (int)(warps / strips > 0 ? warps / strips : 1);
    const int rows = (ny + chunks - 1) / chunks;
    const long long items = (long long)strips * chunks;
    for (long long it = (long long)blockIdx.x * D8_WARPS + (threadIdx.x >> 5); it < items; it += warps) {
        const int c0 = (int)(it % strips) * 256, r0 = (int)(it / strips) * rows;
        const int r1 = r0 + rows < ny ? r0 + rows : ny;
        const int col = c0 + 8 * lane;
        if (r0 >= r1) continue;
        Row8 s = load_row8(z, nx, ny, r0 - 1, c0, lane);
        Row8 c = load_row8(z, nx, ny, r0, c0, lane);
        Row8 n = load_row8(z, nx, ny, r0 + 1, c0, lane);
        for (int j = r0; j < r1; ++j) {
            Row8 p = load_row8(z, nx, ny, j + 2, c0, lane);      // one row ahead
            unsigned out[2] = {0u, 0u};
#pragma unroll
            for (int e = 1; e <= 8; ++e) {
                unsigned k = d8_code<NODATA>(c.x[e], c.x[e + 1], n.x[e + 1], n.x[e], n.x[e - 1], c.x[e - 1],
                                             s.x[e - 1], s.x[e], s.x[e + 1], nodata);
                out[(e - 1) >> 2] |= k << (8 * ((e - 1) & 3));
            }
            unsigned char *d = dir + (size_t)j * nx + col;
            if (col < nx) *reinterpret_cast<unsigned *>(d) = out[0];
            if (col + 4 < nx) *reinterpret_cast<unsigned *>(d + 4) = out[1];
            s = c;
            c = n;
            n = p;
        }
    }
}

// general widths: one column per lane, 32-column strips
__device__ __forceinline__ void load_row1(const float *__restrict__ z, int nx, int ny, int row, int c0, int lane,
                                          float &l, float &m, float &r)
{
    const int col = c0 + lane;
    const bool rin = row >= 0 && row < ny;
    m = (rin && col < nx) ? __ldg(z + (size_t)row * nx + col) : nanf_();
    l = __shfl_up_sync(0xffffffffu, m, 1);
    r = __shfl_down_sync(0xffffffffu, m, 1);
    if (lane == 0) l = (rin && c0 > 0) ? __ldg(z + (size_t)row * nx + c0 - 1) : nanf_();
    if (lane == 31) r = (rin && c0 + 32 < nx) ? __ldg(z + (size_t)row * nx + c0 + 32) : nanf_();
}

template <bool NODATA>
__global__ void __launch_bounds__(32 * D8_WARPS) k_d8_any(const float *__restrict__ z, int nx, int ny, float nodata,
                                                         unsigned char *__restrict__ dir)
{
    const int lane = threadIdx.x & 31;
    const int strips = (nx + 31) / 32, bands = (ny + D8_ROWS - 1) / D8_ROWS;
    const long long items = (long long)strips * bands;
    for (long long it = (long long)blockIdx.x * D8_WARPS + (threadIdx.x >> 5); it < items;
         it += (long long)gridDim.x * D8_WARPS) {
        const int c0 = (int)(it % strips) * 32, r0 = (int)(it / strips) * D8_ROWS;
        const int col = c0 + lane;
        float sl, sm, sr, cl, cm, cr, nl, nm, nr;
        load_row1(z, nx, ny, r0 - 1, c0, lane, sl, sm, sr);
        load_row1(z, nx, ny, r0, c0, lane, cl, cm, cr);
        load_row1(z, nx, ny, r0 + 1, c0, lane, nl, nm, nr);
        for (int j = r0; j < r0 + D8_ROWS && j < ny; ++j) {
            float al, am, ar;
            load_row1(z, nx, ny, j + 2, c0, lane, al, am, ar);
            unsigned k = d8_code<NODATA>(cm, cr, nr, nm, nl, cl, sl, sm, sr, nodata);
            if (col < nx) dir[(size_t)j * nx + col] = (unsigned char)k;
            sl = cl; sm = cm; sr = cr;
            cl = nl; cm = nm; cr = nr;
            nl = al; nm = am; nr = ar;
        }
    }
}

}  // namespace

template <bool NODATA>
int d8_launch(const float *z, int nx, int ny, float nodata, unsigned char *dir, cudaStream_t s)
{
    const bool vec = nx % 4 == 0 && ((uintptr_t)z & 15) == 0 && ((uintptr_t)dir & 3) == 0;
    const long long items = vec ? (long long)((nx + 255) / 256) * ny       // up to one row per warp
                                : (long long)((nx + 31) / 32) * ((ny + D8_ROWS - 1) / D8_ROWS);
    long long blocks = (items + D8_WARPS - 1) / D8_WARPS;
    static int per_sm[2] = {0, 0}, sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_d8_vec<NODATA>, 32 * D8_WARPS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_d8_any<NODATA>, 32 * D8_WARPS, 0);
        if (sms < 1) sms = 152;
    }
    const long long cap = (long long)sms * (per_sm[vec ? 0 : 1] > 0 ? per_sm[vec ? 0 : 1] : 4);
    if (blocks > cap) blocks = cap;
    if (vec)
        k_d8_vec<NODATA><<<(int)blocks, 32 * D8_WARPS, 0, s>>>(z, nx, ny, nodata, dir);
    else
        k_d8_any<NODATA><<<(int)blocks, 32 * D8_WARPS, 0, s>>>(z, nx, ny, nodata, dir);
    return cudaGetLastError() == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

extern "C" int swof_flow_directions(const float *z, int nx, int ny, const float *nodata, unsigned char *dir,
                                    void *stream)
{
    if (!z || !dir || nx < 1 || ny < 1) return SWOF_EINVAL;
    if ((long long)nx * ny > (1LL << 40)) return SWOF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return nodata ? d8_launch<true>(z, nx, ny, *nodata, dir, s) : d8_launch<false>(z, nx, ny, 0.0f, dir, s);
}

// swof_noalloc.cu -- swof_volume_noalloc: water volume and minimum depth of a
// caller-owned depth field, with no device allocation at all.
//
// Who needs this: code that may not call cudaMalloc -- a host that hands
// every byte of device memory to its own pool allocator (a cudaMalloc behind
// its back could fail or fragment the pool), or a real-time loop where an
// allocation is not allowed because it can synchronise the device.  Such a
// caller passes its own input and output pointers; the only scratch is the
// file-scope array below, fixed at load time.
//
// The reduction is the same deterministic two-pass scheme as the diagnostics
// reduction of a context, but over dense rows: pass 1 writes one partial sum
// and one minimum per grid row into the static array, pass 2 combines the
// rows in a fixed order.  Every call overwrites every row slot it reads, so
// nothing has to be cleared between calls; the array keeps the last call's
// contents.  Two calls that overlap on the GPU (different streams, or host
// threads) share the array and race: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/swof.h"

namespace {

constexpr int ROW_THREADS = 256;
constexpr int ROW_BLOCKS = 1216;  // 8 per SM on a 152-SM GB300

// Scratch: [2 * SWOF_NOALLOC_MAX_ROWS] doubles = (sum, min) per row (1 MiB).
static __device__ __align__(256) double g_rows[2 * SWOF_NOALLOC_MAX_ROWS];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double *g_rows_ptr[MAX_DEVICES] = {};

template <typename S>
__global__ void k_row_partials(const S *h, int nx, int ny, double *rows);
__global__ void k_rows_final(const double *rows, int ny, double area, double *out);

// Device address of g_rows on the current device, looked up once per device
// (host code cannot use the symbol itself as a device pointer).  The same
// one-time set-up also loads this file's three kernels on the device
// (cudaFuncGetAttributes), so no later call has a module load left to do.
int rows_ptr(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return SWOF_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_rows_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rows);
        if (e != cudaSuccess || !p) return SWOF_ECUDA;
        cudaFuncAttributes a;
        if (cudaFuncGetAttributes(&a, k_row_partials<double>) != cudaSuccess ||
            cudaFuncGetAttributes(&a, k_row_partials<float>) != cudaSuccess ||
            cudaFuncGetAttributes(&a, k_rows_final) != cudaSuccess)
            return SWOF_ECUDA;
        g_rows_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_rows_ptr[dev];
    return SWOF_OK;
}

// min that keeps a NaN (fmin would drop it): a field holding NaN reports
// NaN as its minimum depth, so a positivity check on out[1] sees it
__device__ __forceinline__ double min_nan(double m, double v) { return (v != v || m != m) ? NAN : fmin(m, v); }

__device__ __forceinline__ void block_sum_min(double &s, double &m, double *rs, double *rm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m = min_nan(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        rs[threadIdx.x >> 5] = s;
        rm[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s = 0.0;
        m = INFINITY;
        for (int w = 0; w < ROW_THREADS / 32; ++w) {
            s += rs[w];
            m = min_nan(m, rm[w]);
        }
    }
    __syncthreads();
}

template <typename S>
__global__ void __launch_bounds__(ROW_THREADS) k_row_partials(const S *h, int nx, int ny, double *rows)
{
    __shared__ double rs[ROW_THREADS / 32], rm[ROW_THREADS / 32];
    for (int j = blockIdx.x; j < ny; j += gridDim.x) {
        double s = 0.0, m = INFINITY;
        const S *row = h + (size_t)j * (size_t)nx;
        for (int i = threadIdx.x; i < nx; i += ROW_THREADS) {
            double v = (double)row[i];
            s += v;
            m = min_nan(m, v);
        }
        block_sum_min(s, m, rs, rm);
        if (threadIdx.x == 0) {
            rows[2 * j] = s;
            rows[2 * j + 1] = m;
        }
    }
}

__global__ void __launch_bounds__(ROW_THREADS) k_rows_final(const double *rows, int ny, double area, double *out)
{
    __shared__ double rs[ROW_THREADS / 32], rm[ROW_THREADS / 32];
    double s = 0.0, m = INFINITY;
    for (int j = threadIdx.x; j < ny; j += ROW_THREADS) {
        s += rows[2 * j];
        m = min_nan(m, rows[2 * j + 1]);
    }
    block_sum_min(s, m, rs, rm);
    if (threadIdx.x == 0) {
        out[0] = s * area;
        out[1] = m;
    }
}

}  // namespace

extern "C" int swof_volume_noalloc(const void *h, int nx, int ny, int dtype, double dx, double dy,
                                   double *out, void *stream)
{
    if (!h || !out || nx < 1 || ny < 1 || !(dx > 0) || !(dy > 0)) return SWOF_EINVAL;
    if (dtype != SWOF_FP64 && dtype != SWOF_FP32) return SWOF_EINVAL;
    if (ny > SWOF_NOALLOC_MAX_ROWS) return SWOF_EINVAL;   // beyond the fixed scratch
    // a CUDA error already pending on this thread belongs to the caller's own
    // earlier work: leave it to the caller, launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return SWOF_ECUDA;
    double *rows = nullptr;
    int st = rows_ptr(&rows);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int blocks = ny < ROW_BLOCKS ? ny : ROW_BLOCKS;
    if (dtype == SWOF_FP64)
        k_row_partials<double><<<blocks, ROW_THREADS, 0, s>>>(static_cast<const double *>(h), nx, ny, rows);
    else
        k_row_partials<float><<<blocks, ROW_THREADS, 0, s>>>(static_cast<const float *>(h), nx, ny, rows);
    k_rows_final<<<1, ROW_THREADS, 0, s>>>(rows, ny, dx * dy, out);
    return cudaGetLastError() == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

// swof_unet.cu -- the learned surrogate: a 4-level convolutional U-Net on
// coarsened shallow-water fields, trained and run with the tcgen05 kernels of
// swof_conv.cuh (BF16 weights and activations, FP32 accumulation, FP32
// master weights, gradients and AdamW moments).
//
// Topology (base width C, levels l = 0..3 at resolution H >> l, width C << l):
//   encoder  l: conv3x3 -> GELU -> conv3x3 -> GELU   (the second writes the
//               first half of the level's concatenation buffer), then 2x2
//               average pooling to the next level;
//   bottom  (l = 3): the same two convolutions, no pooling;
//   decoder  l = 2, 1, 0: 2x2 stride-2 transposed conv of the level below
//               into the second half of the concatenation buffer, then
//               conv3x3 -> GELU -> conv3x3 -> GELU;
//   output: 1x1 conv to 16 channels (the first `out_ch` are used), FP32.
// Inputs are NHWC bf16 with 16 channels (the first `in_ch` used, normalised
// by the caller-given mean / scale); the network predicts the normalised
// increment of the state over the surrogate's time span.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/swof.h"
#include "swof_conv.cuh"

namespace swof {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// Small kernels
__device__ __forceinline__ float gelu_grad(float z)
{
    const float phi = 0.39894228040143268f * __expf(-0.5f * z * z);
    const float Phi = 0.5f * (1.0f + erf_as(z * 0.70710678118654752f));
    return Phi + z * phi;
}

// dz[p][n] = dy[p][dyc0 + n] * (act ? gelu'(z[p][n]) : 1), bf16 compact output
__global__ void k_act_bwd(const float *dy, int dyc, int dyc0, const bf16 *z, int act, bf16 *dz, long long P, int N)
{
    long long total = P * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long p = i / N;
        int n = (int)(i - p * N);
        float g = dy[p * dyc + dyc0 + n];
        if (act) g *= gelu_grad(__bfloat162float(z[i]));
        dz[i] = __float2bfloat16_rn(g);
    }
}

// column sums of a bf16 [P][N] matrix into db[n % nb] (atomics)
// Column sums of dz in two fixed-order passes (the result does not depend
// on the order blocks run in): k_colsum writes each block's sums part[b][n]
// (each thread owns one column n and a strided set of rows; the block's row
// lanes are added in lane order), k_colsum_fin adds, per bias b, the columns
// n = b (mod nb) and the blocks in index order to db[b].
__global__ void k_colsum(const bf16 *dz, long long P, int N, float *part)
{
    extern __shared__ float lanes[];           // [rlanes][N]
    int n = threadIdx.x % N;
    int rlane = threadIdx.x / N, rlanes = blockDim.x / N;
    float s = 0.0f;
    for (long long p = blockIdx.x * (long long)rlanes + rlane; p < P; p += (long long)gridDim.x * rlanes)
        s += __bfloat162float(dz[p * N + n]);
    if (rlane < rlanes) lanes[rlane * N + n] = s;
    __syncthreads();
    if (rlane == 0) {
        float t = 0.0f;
        for (int r = 0; r < rlanes; ++r) t += lanes[r * N + n];
        part[(long long)blockIdx.x * N + n] = t;
    }
}
__global__ void k_colsum_fin(const float *part, int blocks, int N, int nb, float *db)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        float t = 0.0f;
        for (int k = 0; k < blocks; ++k)
            for (int n = b; n < N; n += nb) t += part[(long long)k * N + n];
        db[b] += t;
    }
}

// 2x2 average pooling: x (channels [xc0, xc0+C) of stride cx) at H x W ->
// y compact [B][H/2][W/2][C].  One thread per output pixel and 8-channel
// group (C, cx and xc0 multiples of 8): four 16-byte loads, one store.
template <typename I>
__global__ void k_pool_fwd(const bf16 *x, int cx, int xc0, int B, int H, int W, int C, bf16 *y)
{
    const I G = (I)(C >> 3), Wo = (I)(W / 2), Ho = (I)(H / 2);
    const I total = (I)B * Ho * Wo * G;
    for (I i = (I)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (I)gridDim.x * blockDim.x) {
        const I q = i / G, g = i - q * G;
        const I r = q / Wo, xo = q - r * Wo;
        const I b = r / Ho, yo = r - b * Ho;
        const long long base = ((long long)b * H + 2 * (long long)yo) * W + 2 * (long long)xo;
        const int c0 = xc0 + 8 * (int)g;
        uint4 a = *reinterpret_cast<const uint4 *>(x + base * cx + c0);
        uint4 bq = *reinterpret_cast<const uint4 *>(x + (base + 1) * cx + c0);
        uint4 cq = *reinterpret_cast<const uint4 *>(x + (base + W) * cx + c0);
        uint4 dq = *reinterpret_cast<const uint4 *>(x + (base + W + 1) * cx + c0);
        const bf16 *pa = reinterpret_cast<const bf16 *>(&a), *pb = reinterpret_cast<const bf16 *>(&bq);
        const bf16 *pc = reinterpret_cast<const bf16 *>(&cq), *pd = reinterpret_cast<const bf16 *>(&dq);
        __align__(16) bf16 t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float s = __bfloat162float(pa[k]) + __bfloat162float(pb[k]) + __bfloat162float(pc[k]) +
                      __bfloat162float(pd[k]);
            t[k] = __float2bfloat16_rn(0.25f * s);
        }
        *reinterpret_cast<uint4 *>(y + (long long)q * C + 8 * (long long)g) = *reinterpret_cast<const uint4 *>(t);
    }
}

// dx[..][xc0 + c] += dy / 4 for the four fine pixels of each coarse pixel
__global__ void k_pool_bwd_add(const float *dy, int B, int H, int W, int C, float *dx, int cx, int xc0)
{
    long long total = (long long)B * (H / 2) * (W / 2) * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        int c = (int)(i % C);
        long long q = i / C;
        int xo = (int)(q % (W / 2));
        long long r = q / (W / 2);
        int yo = (int)(r % (H / 2));
        int b = (int)(r / (H / 2));
        long long base = ((long long)b * H + 2 * yo) * W + 2 * xo;
        float g = 0.25f * dy[i];
        dx[base * cx + xc0 + c] += g;
        dx[(base + 1) * cx + xc0 + c] += g;
        dx[(base + W) * cx + xc0 + c] += g;
        dx[(base + W + 1) * cx + xc0 + c] += g;
    }
}

// Mean squared error over the first nch of 16 output channels; writes the
// gradient d(pred) = 2 (pred - tgt) / (P * nch) (0 on unused channels) and
// writes each block's loss sum (FP64) to part[block] (k_sum_blocks adds them).
__global__ void k_mse(const float *pred, const float *tgt, long long P, int nch, float *dpred, double *part)
{
    __shared__ double red[32];
    double s = 0.0;
    const float scale = 2.0f / (float)(P * nch);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * 16; i += (long long)gridDim.x * blockDim.x) {
        long long p = i >> 4;
        int c = (int)(i & 15);
        float g = 0.0f;
        if (c < nch) {
            float d = pred[i] - tgt[p * nch + c];
            s += (double)d * d;
            g = scale * d;
        }
        dpred[i] = g;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}
// the loss: the blocks' sums in index order
__global__ void k_sum_blocks(const double *part, int n, double *loss)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < n; ++k) t += part[k];
        *loss += t;
    }
}

__global__ void k_adamw(float *w, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                        float eps, float wd, float bc1, float bc2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.0f - b1) * gi;
        float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float upd = (mi / bc1) / (sqrtf(vi / bc2) + eps);
        w[i] = w[i] - lr * (upd + wd * w[i]);
    }
}

__global__ void k_to_bf16(const float *src, bf16 *dst, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

// Data-gradient weights: wd[ci][tap' * cout + co] = w[co][(taps-1-tap') * cin_p + ci]
// (taps = 9 for 3x3, 1 for 1x1); and the transposed conv's wd[ci][n] = w[n][ci].
__global__ void k_make_wd(const float *w, int cout, int Kp, int cin_p, int taps, int flip, bf16 *wd, int rows, int Kpd)
{
    long long total = (long long)rows * Kpd;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        int ci = (int)(i / Kpd), k = (int)(i % Kpd);
        float val = 0.0f;
        int tapd = k / cout, co = k % cout;
        if (tapd < taps) {
            int tap = flip ? taps - 1 - tapd : tapd;
            val = w[(long long)co * Kp + tap * cin_p + ci];
        }
        wd[i] = __float2bfloat16_rn(val);
    }
}

__global__ void k_replicate_bias(const float *b, int n, int reps, float *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n * reps) out[i] = b[i % n];
}

// state [B][4][H][W] fp32 (h, hu, hv, z) -> x [B*H*W][16] bf16 normalised
template <typename I>
__global__ void k_pack_input(const float *state, int nin, int B, int H, int W, const float *mean, const float *inv,
                             bf16 *x)
{
    // one thread per pixel: the nin channel planes read coalesced across
    // threads, the pixel's 16 channels written as two 16-byte stores; index
    // arithmetic in I (32-bit when the batch fits)
    const I HW = (I)H * W, P = (I)B * HW;
    for (I p = (I)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (I)gridDim.x * blockDim.x) {
        const I b = p / HW, r = p - b * HW;
        __align__(16) bf16 t[16];
#pragma unroll
        for (int c = 0; c < 16; ++c)
            t[c] = __float2bfloat16_rn(c < nin ? (state[((long long)b * nin + c) * HW + r] - mean[c]) * inv[c] : 0.0f);
        uint4 *d = reinterpret_cast<uint4 *>(x + (long long)p * 16);
        d[0] = reinterpret_cast<const uint4 *>(t)[0];
        d[1] = reinterpret_cast<const uint4 *>(t)[1];
    }
}

// The prediction's 1x1 output convolution and residual update in one pass:
// out[b][c] = in[b][c] + scale[c] * (bias[c] + sum_k x[p][k] w[c][k]) for
// c < nout, NCHW fp32.  x: bf16 [P][C] (C a multiple of 8), w: bf16 rows of
// Kp.  One thread per pixel; the products of bf16 values are exact in FP32
// and accumulate in FP32, as on the tensor cores (nout <= 16 outputs are
// too few columns for an MMA tile).
template <typename I>
__global__ void k_head_residual(const bf16 *x, int C, const bf16 *w, int Kp, const float *bias, const float *in,
                                int nin, int nout, int B, int H, int W, const float *scale, float *out)
{
    extern __shared__ float swt[];            // [nout][C]
    for (int i = threadIdx.x; i < nout * C; i += blockDim.x) swt[i] = __bfloat162float(w[(i / C) * Kp + i % C]);
    __syncthreads();
    const I HW = (I)H * W, P = (I)B * HW;
    for (I p = (I)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (I)gridDim.x * blockDim.x) {
        float acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0.0f;
        for (int k0 = 0; k0 < C; k0 += 8) {
            uint4 v = *reinterpret_cast<const uint4 *>(x + (long long)p * C + k0);
            const bf16 *pv = reinterpret_cast<const bf16 *>(&v);
            float xf[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) xf[j] = __bfloat162float(pv[j]);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (c < nout) {
                    const float4 w0 = *reinterpret_cast<const float4 *>(swt + c * C + k0);
                    const float4 w1 = *reinterpret_cast<const float4 *>(swt + c * C + k0 + 4);
                    acc[c] = fmaf(xf[0], w0.x, acc[c]);
                    acc[c] = fmaf(xf[1], w0.y, acc[c]);
                    acc[c] = fmaf(xf[2], w0.z, acc[c]);
                    acc[c] = fmaf(xf[3], w0.w, acc[c]);
                    acc[c] = fmaf(xf[4], w1.x, acc[c]);
                    acc[c] = fmaf(xf[5], w1.y, acc[c]);
                    acc[c] = fmaf(xf[6], w1.z, acc[c]);
                    acc[c] = fmaf(xf[7], w1.w, acc[c]);
                }
        }
        const I b = p / HW, r = p - b * HW;
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c < nout)
                out[((long long)b * nout + c) * HW + r] =
                    in[((long long)b * nin + c) * HW + r] + (acc[c] + bias[c]) * scale[c];
    }
}

// target tgt[p][c] = (next[b][c] - in[b][c]) / scale[c]
__global__ void k_target(const float *in, int nin, const float *next, int nout, int B, int H, int W,
                         const float *scale, float *tgt)
{
    long long HW = (long long)H * W, P = (long long)B * HW;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * nout; i += (long long)gridDim.x * blockDim.x) {
        long long p = i / nout;
        int c = (int)(i - p * nout);
        long long b = p / HW, q = p - b * HW;
        tgt[i] = (next[(b * nout + c) * HW + q] - in[(b * nin + c) * HW + q]) / scale[c];
    }
}

inline int grid_for(long long n) { long long g = (n + 255) / 256; return (int)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16); }

// ---------------------------------------------------------------------------
// Launchers of the tensor-core kernels.  Each keeps, per device, the
// dynamic shared memory it has opted its kernel into and the resident CTAs
// of the whole GPU (persistent grids); the first launch on a device sets
// them, under one lock so that host threads may share the library.
constexpr int MAX_DEVICES = 64;
std::mutex g_launch_attr_lock;

inline int current_device()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= MAX_DEVICES) d = 0;
    return d;
}

// resident CTAs of kernel f on device dev at `threads` threads and `smem`
// bytes of dynamic shared memory (at least one per SM)
template <typename Kern>
int resident_ctas(Kern f, int threads, size_t smem, int dev)
{
    int n = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess || n < 1) n = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return n * (sms > 0 ? sms : 152);
}

template <int NT>
int conv_launch(const ConvArgs &A, cudaStream_t s)
{
    size_t smem = ConvCfg<NT>::SMEM;
    static int per_dev[MAX_DEVICES] = {};   // resident CTAs of the GPU (persistent grid)
    const int dev = current_device();
    int per_sm;
    {
        std::lock_guard<std::mutex> g(g_launch_attr_lock);
        if (!per_dev[dev]) {
            if (cudaFuncSetAttribute(k_conv<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return SWOF_ECUDA;
            per_dev[dev] = resident_ctas(k_conv<NT>, ConvCfg<NT>::THREADS, smem, dev);
        }
        per_sm = per_dev[dev];
    }
    long long M = (long long)A.B * A.H * A.W;
    long long tiles = (M + 127) / 128;
    long long gy = A.ntot / NT;
    long long gx = (4LL * per_sm + gy - 1) / gy;
    if (gx > tiles) gx = tiles;
    if (gx < 1) gx = 1;
    dim3 grid((unsigned)gx, (unsigned)gy);
    k_conv<NT><<<grid, ConvCfg<NT>::THREADS, smem, s>>>(A);
    return cudaGetLastError() == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

// ---- TMA tensor maps (the encoder comes from the driver at run time) ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    // looked up once per process (a function-local static is initialised
    // once even with several host threads)
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiledFn>(p);
        return nullptr;
    }();
    return fn;
}

// Output tensor map of the TMA-store epilogue, for a bf16 output y alone
// (no pre-activation or FP32 output): NHWC -- the [pixels][cy] array, box
// {pw, 32}; SCATTER_UP2 -- the 2H x 2W output as [output rows][x][sub-x][cy]
// (x the input column), box {pw, 1, 32, 1}, when each warp's 32 pixels lie
// in one input row (W a multiple of 32).  pw = 64, 32 or 16 columns
// (128-, 64- or 32-byte swizzle).  Sets A.ystage = pw, or 0 (plain stores)
// where the layout does not allow it.
int epi_tma_map(ConvArgs &A, int nt, CUtensorMap *m)
{
    A.ystage = 0;
    std::memset(m, 0, sizeof(*m));
    if (!A.y || A.ypre || A.yf || nt < 32 || (A.cy * 2) % 16 || (A.yc0 * 2) % 16 ||
        (reinterpret_cast<uintptr_t>(A.y) & 15))
        return SWOF_OK;
    int pw;                       // each epilogue warp takes nt / 2 columns
    if (A.store == STORE_NHWC) {
        pw = nt / 2 < 64 ? nt / 2 : 64;
    } else {
        if (A.W % 32 || A.cout_up % 32) return SWOF_OK;
        pw = A.cout_up < 64 ? A.cout_up : 64;
    }
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return SWOF_ECUDA;
    const CUtensorMapSwizzle sz = pw == 64   ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : pw == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                             : CU_TENSOR_MAP_SWIZZLE_32B;
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r;
    if (A.store == STORE_NHWC) {
        cuuint64_t d[2] = {(cuuint64_t)A.cy, (cuuint64_t)A.B * A.H * A.W};
        cuuint64_t st[1] = {(cuuint64_t)A.cy * 2};
        cuuint32_t bx[2] = {(cuuint32_t)pw, 32};
        r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)A.y, d, st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sz,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        cuuint64_t d[4] = {(cuuint64_t)A.cy, 2, (cuuint64_t)A.W, (cuuint64_t)A.B * 2 * A.H};
        cuuint64_t st[3] = {(cuuint64_t)A.cy * 2, (cuuint64_t)A.cy * 4, (cuuint64_t)A.W * A.cy * 4};
        cuuint32_t bx[4] = {(cuuint32_t)pw, 1, 32, 1};
        r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)A.y, d, st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sz,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return SWOF_ECUDA;
    A.ystage = pw;
    return SWOF_OK;
}

template <int NT, int CB>
int conv_halo_launch(const ConvArgs &A0, cudaStream_t s)
{
    using Cfg = HaloCfg<NT, CB>;
    ConvArgs A = A0;
    CUtensorMap ymap;
    if (int e = epi_tma_map(A, NT, &ymap)) return e;
    int stage_out = A.ystage ? epi_stage_bytes(A.ystage) : 0;
    if (stage_out && Cfg::stages(A.Kp, stage_out) < 2) {    // no room: plain stores
        A.ystage = 0;
        stage_out = 0;
    }
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return SWOF_ECUDA;
    CUtensorMap tmap;
    cuuint64_t dims[4] = {(cuuint64_t)A.cin, (cuuint64_t)A.W, (cuuint64_t)A.H, (cuuint64_t)A.B};
    cuuint64_t strides[3] = {(cuuint64_t)A.cx * 2, (cuuint64_t)A.W * A.cx * 2, (cuuint64_t)A.H * A.W * A.cx * 2};
    cuuint32_t box[4] = {(cuuint32_t)CB, (cuuint32_t)HALO_PX, (cuuint32_t)HALO_ROWS, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    const CUtensorMapSwizzle sz = CB == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : CB == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                             : CU_TENSOR_MAP_SWIZZLE_32B;
    if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)(A.x + A.xc0), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return SWOF_ECUDA;
    const int stages = Cfg::stages(A.Kp, stage_out);
    if (stages < 2) return SWOF_EINVAL;
    const size_t smem = Cfg::smem(A.Kp, stages, stage_out);
    // the opt-in grows to the largest stage count asked for so far; the
    // resident CTAs are those of the size set last
    static int per_dev[MAX_DEVICES] = {};
    static size_t smem_set[MAX_DEVICES] = {};
    const int dev = current_device();
    int per_sm;
    {
        std::lock_guard<std::mutex> g(g_launch_attr_lock);
        if (smem > smem_set[dev]) {
            if (cudaFuncSetAttribute(k_conv_halo<NT, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return SWOF_ECUDA;
            smem_set[dev] = smem;
            per_dev[dev] = 0;
        }
        if (!per_dev[dev]) per_dev[dev] = resident_ctas(k_conv_halo<NT, CB>, Cfg::THREADS, smem, dev);
        per_sm = per_dev[dev];
    }
    const long long tiles = (long long)A.B * A.H * A.W / 128;
    const long long gy = A.ntot / NT;
    long long gx = (per_sm + gy - 1) / gy;
    if (gx > tiles) gx = tiles;
    if (gx < 1) gx = 1;
    k_conv_halo<NT, CB><<<dim3((unsigned)gx, (unsigned)gy), Cfg::THREADS, smem, s>>>(A, tmap, ymap, stages);
    return cudaGetLastError() == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

// TMA maps of a same-resolution layer: the input slice (NHWC, channel
// stride cx, offset xc0) with a 128-pixel tile box of 8 channels, and the
// weight rows [ntot][Kp] with a box of 8 columns x NT rows; SW: boxes of 64
// channels / 64 columns, written with the 128-byte swizzle.
template <int NT, bool SW>
int conv_tma_launch(const ConvArgs &A0, cudaStream_t s)
{
    using Cfg = TmaCfg<NT>;
    ConvArgs A = A0;
    CUtensorMap ymap;
    if (int e = epi_tma_map(A, NT, &ymap)) return e;
    const size_t smem = Cfg::SMEM + (A.ystage ? (size_t)epi_stage_bytes(A.ystage) : 0);
    constexpr size_t smem_max = Cfg::SMEM + EPI_STAGE_BYTES_MAX;
    static_assert(smem_max <= 227 * 1024, "TMA-operand conv: shared memory over the limit");
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return SWOF_ECUDA;
    CUtensorMap xmap, wmap;
    const int bw = A.W >= 128 ? 128 : A.W, bh = A.W >= 128 ? 1 : 128 / A.W;
    const CUtensorMapSwizzle sz = SW ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE;
    const cuuint32_t kbox = SW ? 64 : 8;
    cuuint64_t xd[4] = {(cuuint64_t)A.cin, (cuuint64_t)A.W, (cuuint64_t)A.H, (cuuint64_t)A.B};
    cuuint64_t xs[3] = {(cuuint64_t)A.cx * 2, (cuuint64_t)A.W * A.cx * 2, (cuuint64_t)A.H * A.W * A.cx * 2};
    cuuint32_t xb[4] = {kbox, (cuuint32_t)bw, (cuuint32_t)bh, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)(A.x + A.xc0), xd, xs, xb, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return SWOF_ECUDA;
    cuuint64_t wd[2] = {(cuuint64_t)A.Kp, (cuuint64_t)A.ntot};
    cuuint64_t ws[1] = {(cuuint64_t)A.Kp * 2};
    cuuint32_t wb[2] = {kbox, (cuuint32_t)NT};
    if (enc(&wmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)A.w, wd, ws, wb, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            sz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return SWOF_ECUDA;
    static int per_dev[MAX_DEVICES] = {};
    const int dev = current_device();
    int per_sm;
    {
        std::lock_guard<std::mutex> g(g_launch_attr_lock);
        if (!per_dev[dev]) {
            if (cudaFuncSetAttribute(k_conv_tma<NT, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_max) != cudaSuccess)
                return SWOF_ECUDA;
            per_dev[dev] = resident_ctas(k_conv_tma<NT, SW>, Cfg::THREADS, smem_max, dev);
        }
        per_sm = per_dev[dev];
    }
    const long long tiles = (long long)A.B * A.H * A.W / 128;
    const long long gy = A.ntot / NT;
    long long gx = (per_sm + gy - 1) / gy;
    if (gx > tiles) gx = tiles;
    if (gx < 1) gx = 1;
    k_conv_tma<NT, SW><<<dim3((unsigned)gx, (unsigned)gy), Cfg::THREADS, smem, s>>>(A, xmap, wmap, ymap);
    return cudaGetLastError() == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

// Same-resolution layers whose 128-pixel tiles are boxes of the image (a
// segment of one row, or whole rows) take the TMA-operand kernel.
bool tma_ok(const ConvArgs &A)
{
    const bool box = (A.W % 128 == 0) || (128 % A.W == 0 && A.H % (128 / A.W) == 0);
    return A.gather == GATHER_SAME && (A.ks == 1 || A.ks == 3) && box && ((A.xc0 * 2) % 16 == 0) &&
           ((A.cx * 2) % 16 == 0) && A.H <= 65535 && A.Kp % 64 == 0;
}

// Channel block of the halo kernel: the widest of 64, 32, 16 (dividing cin)
// whose halo stages fit in shared memory beside the resident weight tile;
// 0 if none does.
template <int NT>
int halo_cb(const ConvArgs &A)
{
    if (A.cin % 64 == 0 && HaloCfg<NT, 64>::stages(A.Kp) >= 2) return 64;
    if (A.cin % 32 == 0 && HaloCfg<NT, 32>::stages(A.Kp) >= 3) return 32;
    if (A.cin % 16 == 0 && HaloCfg<NT, 16>::stages(A.Kp) >= 3) return 16;
    return 0;
}

template <int NT>
int conv_halo(const ConvArgs &A, cudaStream_t s)
{
    switch (halo_cb<NT>(A)) {
    case 16: return conv_halo_launch<NT, 16>(A, s);
    case 32: return conv_halo_launch<NT, 32>(A, s);
    case 64: return conv_halo_launch<NT, 64>(A, s);
    default: return SWOF_EINVAL;
    }
}

// 3x3 layers over rows of >= 128 pixels whose weight tile fits in shared
// memory (beside the halo stages) take the TMA halo kernel; the rest the
// gather kernel.
bool halo_ok(const ConvArgs &A, int nt)
{
    if (!(A.gather == GATHER_SAME && A.ks == 3 && A.store == STORE_NHWC && A.W % 128 == 0 && A.cin >= 16 &&
          ((A.xc0 * 2) % 16 == 0) && ((A.cx * 2) % 16 == 0) && A.H <= 65535 &&
          (size_t)nt * A.Kp * 2 <= (size_t)HaloCfg<32, 64>::WMAX))
        return false;
    switch (nt) {
    case 16: return halo_cb<16>(A) != 0;
    case 32: return halo_cb<32>(A) != 0;
    case 64: return halo_cb<64>(A) != 0;
    case 128: return halo_cb<128>(A) != 0;
    default: return false;
    }
}

int conv(ConvArgs A, cudaStream_t s)
{
    int nt = A.ntot >= 256 ? 256 : A.ntot;
    if (A.ntot % nt) return SWOF_EINVAL;
    if (A.cin < 8 || (A.cin & (A.cin - 1)) || (long long)A.B * A.H * A.W >= (1LL << 31) / 4)
        return SWOF_EINVAL;
    A.cin_shift = 0;
    while ((1 << A.cin_shift) < A.cin) ++A.cin_shift;
    if (halo_ok(A, nt)) {
        switch (nt) {
        case 16: return conv_halo<16>(A, s);
        case 32: return conv_halo<32>(A, s);
        case 64: return conv_halo<64>(A, s);
        case 128: return conv_halo<128>(A, s);
        default: break;
        }
    }
    // (16-column layers -- the 1x1 output convolution -- stay on the gather
    // kernel: measured 35 us there against 54 us with TMA boxes at 256^2 x 8)
    if (tma_ok(A)) {
        // one swizzled 64-channel box per K chunk when every chunk lies in one tap
        const bool sw = A.cin % 64 == 0 && A.Kp == A.ks * A.ks * A.cin;
        switch (nt) {
        case 32: return sw ? conv_tma_launch<32, true>(A, s) : conv_tma_launch<32, false>(A, s);
        case 64: return sw ? conv_tma_launch<64, true>(A, s) : conv_tma_launch<64, false>(A, s);
        case 128: return sw ? conv_tma_launch<128, true>(A, s) : conv_tma_launch<128, false>(A, s);
        case 256: return sw ? conv_tma_launch<256, true>(A, s) : conv_tma_launch<256, false>(A, s);
        default: break;
        }
    }
    switch (nt) {
    case 16: return conv_launch<16>(A, s);
    case 32: return conv_launch<32>(A, s);
    case 64: return conv_launch<64>(A, s);
    case 128: return conv_launch<128>(A, s);
    case 256: return conv_launch<256>(A, s);
    default: return SWOF_EINVAL;
    }
}

// Column tile of the weight-gradient kernel for a row length ncols, and the
// grid of one launch: gx x gy output tiles, the P pixels split over gz CTAs
// (about two CTAs per SM in all) of chunks_per_cta 64-pixel chunks each.
int wgrad_nt(int ncols) { return ncols % 256 == 0 ? 256 : (ncols % 128 == 0 ? 128 : 64); }
void wgrad_grid(int nrows, int ncols, long long P, unsigned *gx, unsigned *gy, unsigned *gz, int *chunks_per_cta)
{
    const int NT = wgrad_nt(ncols);
    const long long chunks = (P + 63) / 64;
    *gx = (unsigned)((nrows + 127) / 128);
    *gy = (unsigned)((ncols + NT - 1) / NT);
    long long splits = (2 * 152) / ((long long)*gx * *gy);
    if (splits < 1) splits = 1;
    if (splits > chunks) splits = chunks;
    *chunks_per_cta = (int)((chunks + splits - 1) / splits);
    *gz = (unsigned)((chunks + *chunks_per_cta - 1) / *chunks_per_cta);
}

template <int NT>
int wgrad_launch(WgradArgs A, int ncols, cudaStream_t s)
{
    size_t smem = sizeof(ConvSmem) + 1024;
    if (cudaFuncSetAttribute(k_wgrad<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SWOF_ECUDA;
    unsigned gx, gy, gz;
    wgrad_grid(A.nrows, ncols, (long long)A.B * A.H * A.W, &gx, &gy, &gz, &A.chunks_per_cta);
    k_wgrad<NT><<<dim3(gx, gy, gz), 128, smem, s>>>(A);
    if (cudaGetLastError() != cudaSuccess) return SWOF_ECUDA;
    const long long n = (long long)A.nrows * A.Kp;
    long long blocks = (n + 255) / 256;
    if (blocks > 4 * 152) blocks = 4 * 152;
    k_wgrad_sum<<<(unsigned)blocks, 256, 0, s>>>(A.part, (int)gz, n, A.dw);
    return cudaGetLastError() == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

int wgrad(WgradArgs A, int ncols, cudaStream_t s)
{
    if (A.cin < 8 || (A.cin & (A.cin - 1)) || (long long)A.B * A.H * A.W >= (1LL << 31) / 4 || !A.part)
        return SWOF_EINVAL;
    A.cin_shift = 0;
    while ((1 << A.cin_shift) < A.cin) ++A.cin_shift;
    switch (wgrad_nt(ncols)) {
    case 256: return wgrad_launch<256>(A, ncols, s);
    case 128: return wgrad_launch<128>(A, ncols, s);
    default: return wgrad_launch<64>(A, ncols, s);
    }
}

}  // namespace swof

// ---------------------------------------------------------------------------
// The network
using swof::bf16;

namespace {

enum LayerKind { K_CONV3 = 0, K_CONV1 = 1, K_CONVT = 2 };

struct Layer {
    int kind, cin, cin_p, cout, act;
    int ncols;          // GEMM columns of the forward (cout, or 4*cout for the transposed conv)
    int Kp;             // forward K padded (row length of w)
    int Kpd;            // data-gradient K padded
    size_t woff, boff;  // offsets in the flat parameter arrays
    size_t nw, nb;
};

struct Act {            // an NHWC bf16 activation slot
    bf16 *p;
    int c, c0;          // channel stride / offset
};

}  // namespace

struct swof_unet {
    int C, in_ch, out_ch, H, W, maxB;
    std::vector<Layer> layers;    // 0,1: enc0; 2,3: enc1; 4,5: enc2; 6,7: bottom; 8: up2, 9,10: dec2;
                                  // 11: up1, 12,13: dec1; 14: up0, 15,16: dec0; 17: out
    size_t nparam = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // flat FP32 (weights then biases)
    bf16 *wbf = nullptr;          // bf16 forward weights (same layout as w's weight part)
    bf16 *wd = nullptr;           // data-gradient weights
    size_t nwd = 0;
    float *bias_rep = nullptr;    // replicated transposed-conv biases
    std::vector<size_t> wd_off;
    std::vector<std::vector<char>> dummy;
    // activations (per level l)
    std::vector<bf16 *> ea, ea_pre, eb_pre, cat, pool, da, da_pre, db, db_pre;
    bf16 *x0 = nullptr, *bott = nullptr, *bott_pre = nullptr, *dz = nullptr;
    float *out = nullptr, *tgt = nullptr, *gpred = nullptr;
    // gradients (FP32)
    std::vector<float *> g_ea, g_cat, g_pool, g_da, g_db;
    float *g_bott = nullptr;
    double *loss = nullptr;
    int *err = nullptr;
    float *norm = nullptr;        // mean[16], inv[16], scale[16] (device)
    float *wg_part = nullptr;     // partial sums: weight-gradient pixel splits, bias-gradient and loss blocks
    size_t wg_part_n = 0;
    long long step = 0;
    std::vector<void *> allocs;
};

namespace {

template <typename T>
T *dmalloc(swof_unet *u, size_t n, int *st)
{
    if (*st) return nullptr;
    void *p = nullptr;
    if (cudaMalloc(&p, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
        *st = SWOF_ENOMEM;
        return nullptr;
    }
    cudaMemset(p, 0, (n ? n : 1) * sizeof(T));
    u->allocs.push_back(p);
    return static_cast<T *>(p);
}

int pad64(int k) { return (k + 63) / 64 * 64; }

Layer make_layer(int kind, int cin, int cout, int act)
{
    Layer L{};
    L.kind = kind;
    L.cin = cin;
    L.cin_p = cin < 16 ? 16 : cin;
    L.cout = cout;
    L.act = act;
    L.ncols = kind == K_CONVT ? 4 * cout : cout;
    int taps = kind == K_CONV3 ? 9 : 1;
    L.Kp = pad64(taps * L.cin_p);
    L.Kpd = kind == K_CONVT ? pad64(4 * cout) : pad64(taps * cout);
    L.nw = (size_t)L.ncols * L.Kp;
    L.nb = (size_t)cout;
    return L;
}

// SplitMix64 + Box-Muller: reproducible initial weights
struct Rng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uni() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return std::sqrt(-2.0 * std::log(uni())) * std::cos(6.283185307179586 * uni()); }
};

cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

float *W(swof_unet *u, int l) { return u->w + u->layers[l].woff; }
float *Bv(swof_unet *u, int l) { return u->w + u->layers[l].boff; }
float *GW(swof_unet *u, int l) { return u->g + u->layers[l].woff; }
float *GB(swof_unet *u, int l) { return u->g + u->layers[l].boff; }
bf16 *WB(swof_unet *u, int l) { return u->wbf + u->layers[l].woff; }

// refresh bf16 weights, data-gradient weights and replicated biases from the FP32 master
int refresh_weights(swof_unet *u, cudaStream_t s)
{
    size_t nw = u->layers.back().woff + u->layers.back().nw;
    swof::k_to_bf16<<<swof::grid_for((long long)nw), 256, 0, s>>>(u->w, u->wbf, (long long)nw);
    for (size_t l = 0; l < u->layers.size(); ++l) {
        const Layer &L = u->layers[l];
        int rows = L.cin_p, taps = L.kind == K_CONV3 ? 9 : (L.kind == K_CONV1 ? 1 : 4);
        if (L.kind == K_CONVT) {
            // wd[ci][n] = w[n][ci]: a 1-tap "flip" over n = (sub, co) columns
            swof::k_make_wd<<<swof::grid_for((long long)rows * L.Kpd), 256, 0, s>>>(
                W(u, (int)l), L.ncols, L.Kp, L.cin_p, 1, 0, u->wd + u->wd_off[l], rows, L.Kpd);
        } else {
            swof::k_make_wd<<<swof::grid_for((long long)rows * L.Kpd), 256, 0, s>>>(
                W(u, (int)l), L.cout, L.Kp, L.cin_p, taps, 1, u->wd + u->wd_off[l], rows, L.Kpd);
        }
    }
    // transposed-conv biases replicated over the 4 sub-positions
    int off = 0;
    for (size_t l = 0; l < u->layers.size(); ++l) {
        const Layer &L = u->layers[l];
        if (L.kind != K_CONVT) continue;
        swof::k_replicate_bias<<<(4 * L.cout + 255) / 256, 256, 0, s>>>(Bv(u, (int)l), L.cout, 4, u->bias_rep + off);
        off += 4 * L.cout;
    }
    return cudaGetLastError() == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

float *rep_bias(swof_unet *u, int l)
{
    int off = 0;
    for (int k = 0; k < l; ++k)
        if (u->layers[k].kind == K_CONVT) off += 4 * u->layers[k].cout;
    return u->bias_rep + off;
}

// forward of one layer on B samples at resolution h x w (output grid)
int fwd_layer(swof_unet *u, int l, int B, int h, int w, Act in, Act out, bf16 *pre, float *outf, int outf_c,
              cudaStream_t s)
{
    const Layer &L = u->layers[l];
    swof::ConvArgs A{};
    A.x = in.p;
    A.B = B;
    A.H = h;
    A.W = w;
    A.cx = in.c;
    A.xc0 = in.c0;
    A.cin = L.cin_p;
    A.ks = L.kind == K_CONV3 ? 3 : 1;
    A.gather = swof::GATHER_SAME;
    A.w = WB(u, l);
    A.Kp = L.Kp;
    A.bias = L.kind == K_CONVT ? rep_bias(u, l) : Bv(u, l);
    A.ntot = L.ncols;
    A.y = out.p;
    A.ypre = pre;
    A.yf = outf;
    A.cy = outf ? outf_c : out.c;
    A.yc0 = outf ? 0 : out.c0;
    A.act = L.act;
    A.pre_round = 1;
    A.store = L.kind == K_CONVT ? swof::SCATTER_UP2 : swof::STORE_NHWC;
    A.cout_up = L.cout;
    A.err = u->err;
    return swof::conv(A, s);
}

// backward of one layer: dy (FP32, channels [dyc0, dyc0 + cout) of stride
// dyc, at the layer's output grid oh x ow) -> weight/bias gradients and,
// when dx is given, the input gradient (FP32, channels [dxc0, ...) of dxc).
int bwd_layer(swof_unet *u, int l, int B, int ih, int iw, Act in, const float *dy, int dyc, int dyc0,
              const bf16 *pre, float *dx, int dxc, int dxc0, cudaStream_t s)
{
    const Layer &L = u->layers[l];
    const bool up = L.kind == K_CONVT;
    const int oh = up ? 2 * ih : ih, ow = up ? 2 * iw : iw;
    const long long Po = (long long)B * oh * ow, Pi = (long long)B * ih * iw;
    // dz = dy * act'(pre), compact bf16 [Po][cout]
    swof::k_act_bwd<<<swof::grid_for(Po * L.cout), 256, 0, s>>>(dy, dyc, dyc0, pre, L.act, u->dz, Po, L.cout);
    // bias gradient
    {
        int per = 256 / L.cout > 0 ? 256 / L.cout : 1;
        int threads = per * L.cout;
        if (threads > 1024) threads = L.cout;
        long long blocks = (Po + per - 1) / per;
        if (blocks > 1024) blocks = 1024;
        swof::k_colsum<<<(unsigned)blocks, threads, threads * sizeof(float), s>>>(u->dz, Po, L.cout, u->wg_part);
        swof::k_colsum_fin<<<1, 256, 0, s>>>(u->wg_part, (int)blocks, L.cout, L.cout, GB(u, l));
    }
    // weight gradient
    swof::WgradArgs G{};
    G.g = u->dz;
    G.gc = L.cout;
    G.gmode = up ? swof::GATHER_UP2 : swof::GATHER_SAME;
    G.cout_up = L.cout;
    G.x = in.p;
    G.cx = in.c;
    G.xc0 = in.c0;
    G.cin = L.cin_p;
    G.ks = L.kind == K_CONV3 ? 3 : 1;
    G.B = B;
    G.H = ih;
    G.W = iw;
    G.nrows = L.ncols;
    G.Kp = L.Kp;
    G.dw = GW(u, l);
    G.part = u->wg_part;
    G.err = u->err;
    {
        unsigned gx, gy, gz;
        int cpc;
        swof::wgrad_grid(G.nrows, L.Kp, (long long)B * ih * iw, &gx, &gy, &gz, &cpc);
        if ((size_t)gz * (size_t)G.nrows * (size_t)G.Kp > u->wg_part_n) return SWOF_EINVAL;   // (sized at creation)
    }
    int st = swof::wgrad(G, L.Kp, s);
    if (st || !dx) return st;
    // data gradient
    swof::ConvArgs A{};
    A.x = u->dz;
    A.B = B;
    A.H = ih;
    A.W = iw;
    A.cx = L.cout;
    A.xc0 = 0;
    A.cin = L.cout;
    A.ks = L.kind == K_CONV3 ? 3 : 1;
    A.gather = up ? swof::GATHER_UP2 : swof::GATHER_SAME;
    A.w = u->wd + u->wd_off[l];
    A.Kp = L.Kpd;
    A.bias = nullptr;
    A.ntot = L.cin_p;
    A.yf = dx;
    A.cy = dxc;
    A.yc0 = dxc0;
    A.act = swof::ACT_NONE;
    A.store = swof::STORE_NHWC;
    A.err = u->err;
    (void)Pi;
    return swof::conv(A, s);
}

// keep_pre = false (inference): the pre-activations are not stored (the
// activations still use their bf16-rounded values, as in training).
int forward(swof_unet *u, int B, cudaStream_t s, bool keep_pre = true, bool head = true)
{
    int st = SWOF_OK;
    auto pre = [&](bf16 *p) { return keep_pre ? p : nullptr; };
    const int C = u->C;
    Act in{u->x0, 16, 0};
    for (int l = 0; l < 4 && !st; ++l) {
        int h = u->H >> l, w = u->W >> l, c = C << l;
        if (l > 0) {
            int hp = u->H >> (l - 1), wp = u->W >> (l - 1), cp = C << (l - 1);
            long long n = (long long)B * h * w * cp;
            if (n < (1LL << 31))
                swof::k_pool_fwd<unsigned><<<swof::grid_for(n / 8), 256, 0, s>>>(u->cat[l - 1], 2 * cp, 0, B, hp, wp, cp,
                                                                            u->pool[l]);
            else
                swof::k_pool_fwd<long long><<<swof::grid_for(n / 8), 256, 0, s>>>(u->cat[l - 1], 2 * cp, 0, B, hp, wp,
                                                                             cp, u->pool[l]);
            in = Act{u->pool[l], cp, 0};
        }
        st = fwd_layer(u, 2 * l, B, h, w, in, Act{u->ea[l], c, 0}, pre(u->ea_pre[l]), nullptr, 0, s);
        Act o = l < 3 ? Act{u->cat[l], 2 * c, 0} : Act{u->bott, c, 0};
        if (!st)
            st = fwd_layer(u, 2 * l + 1, B, h, w, Act{u->ea[l], c, 0}, o, pre(l < 3 ? u->eb_pre[l] : u->bott_pre),
                           nullptr, 0, s);
    }
    Act below{u->bott, C << 3, 0};
    for (int l = 2; l >= 0 && !st; --l) {
        int h = u->H >> l, w = u->W >> l, c = C << l;
        int base = 8 + 3 * (2 - l);
        // transposed conv from the level below (its grid) into the second half of cat[l]
        st = fwd_layer(u, base, B, h / 2, w / 2, below, Act{u->cat[l], 2 * c, c}, nullptr, nullptr, 0, s);
        if (!st) st = fwd_layer(u, base + 1, B, h, w, Act{u->cat[l], 2 * c, 0}, Act{u->da[l], c, 0},
                                pre(u->da_pre[l]), nullptr, 0, s);
        if (!st) st = fwd_layer(u, base + 2, B, h, w, Act{u->da[l], c, 0}, Act{u->db[l], c, 0},
                                pre(u->db_pre[l]), nullptr, 0, s);
        below = Act{u->db[l], c, 0};
    }
    if (!st && head) st = fwd_layer(u, 17, B, u->H, u->W, below, Act{nullptr, 16, 0}, nullptr, u->out, 16, s);
    return st;
}

int backward(swof_unet *u, int B, cudaStream_t s)
{
    const int C = u->C;
    int st = SWOF_OK;
    // output layer: dy = d(loss)/d(pred) in gpred
    st = bwd_layer(u, 17, B, u->H, u->W, Act{u->db[0], C, 0}, u->gpred, 16, 0, nullptr, u->g_db[0], C, 0, s);
    for (int l = 0; l <= 2 && !st; ++l) {
        // process levels top-down in the decoder order: level 0 first (closest to the output)
        int h = u->H >> l, w = u->W >> l, c = C << l;
        int base = 8 + 3 * (2 - l);
        st = bwd_layer(u, base + 2, B, h, w, Act{u->da[l], c, 0}, u->g_db[l], c, 0, u->db_pre[l], u->g_da[l], c, 0, s);
        if (!st) st = bwd_layer(u, base + 1, B, h, w, Act{u->cat[l], 2 * c, 0}, u->g_da[l], c, 0, u->da_pre[l],
                                u->g_cat[l], 2 * c, 0, s);
        // transposed conv: its output gradient is the second half of g_cat[l]
        Act below = l < 2 ? Act{u->db[l + 1], 2 * c, 0} : Act{u->bott, 8 * C, 0};
        float *gbelow = l < 2 ? u->g_db[l + 1] : u->g_bott;
        if (!st) st = bwd_layer(u, base, B, h / 2, w / 2, below, u->g_cat[l], 2 * c, c, nullptr, gbelow, 2 * c, 0, s);
    }
    // bottom and encoder, deepest first
    for (int l = 3; l >= 0 && !st; --l) {
        int h = u->H >> l, w = u->W >> l, c = C << l;
        Act in_b{u->ea[l], c, 0};
        const float *dyb = l < 3 ? u->g_cat[l] : u->g_bott;
        int dybc = l < 3 ? 2 * c : c;
        st = bwd_layer(u, 2 * l + 1, B, h, w, in_b, dyb, dybc, 0, l < 3 ? u->eb_pre[l] : u->bott_pre, u->g_ea[l], c, 0, s);
        Act in_a = l == 0 ? Act{u->x0, 16, 0} : Act{u->pool[l], C << (l - 1), 0};
        float *gin = l == 0 ? nullptr : u->g_pool[l];
        if (!st) st = bwd_layer(u, 2 * l, B, h, w, in_a, u->g_ea[l], c, 0, u->ea_pre[l], gin, C << (l > 0 ? l - 1 : 0), 0, s);
        if (!st && l > 0) {
            int hp = u->H >> (l - 1), wp = u->W >> (l - 1), cp = C << (l - 1);
            long long n = (long long)B * h * w * cp;
            swof::k_pool_bwd_add<<<swof::grid_for(n), 256, 0, s>>>(u->g_pool[l], B, hp, wp, cp, u->g_cat[l - 1], 2 * cp, 0);
        }
    }
    return st ? st : (cudaGetLastError() == cudaSuccess ? SWOF_OK : SWOF_ECUDA);
}

}  // namespace

// Loss and gradients for the packed input in x0 and the target in tgt
// ([P][out_ch] FP32); gradients replace the previous ones.
int loss_and_grads(swof_unet *u, int B, cudaStream_t s)
{
    long long P = (long long)B * u->H * u->W;
    cudaMemsetAsync(u->g, 0, u->nparam * sizeof(float), s);
    cudaMemsetAsync(u->loss, 0, sizeof(double), s);
    int st = forward(u, B, s);
    if (st) return st;
    const int mb = swof::grid_for(P * 16);
    swof::k_mse<<<mb, 256, 0, s>>>(u->out, u->tgt, P, u->out_ch, u->gpred, reinterpret_cast<double *>(u->wg_part));
    swof::k_sum_blocks<<<1, 32, 0, s>>>(reinterpret_cast<const double *>(u->wg_part), mb, u->loss);
    return backward(u, B, s);
}

int adamw(swof_unet *u, float lr, float b1, float b2, float eps, float wd, cudaStream_t s)
{
    u->step++;
    float bc1 = 1.0f - std::pow(b1, (float)u->step), bc2 = 1.0f - std::pow(b2, (float)u->step);
    swof::k_adamw<<<swof::grid_for((long long)u->nparam), 256, 0, s>>>(u->w, u->g, u->m, u->v, (long long)u->nparam,
                                                                         lr, b1, b2, eps, wd, bc1, bc2);
    return refresh_weights(u, s);
}

int read_status(swof_unet *u, cudaStream_t s, double *loss_host)
{
    int err = 0;
    double l = 0.0;
    if (cudaMemcpyAsync(&err, u->err, sizeof err, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SWOF_ECUDA;
    if (cudaMemcpyAsync(&l, u->loss, sizeof l, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SWOF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SWOF_ECUDA;
    if (loss_host) *loss_host = l;
    return err ? SWOF_ETIMEOUT : SWOF_OK;
}

void swof_unet_dims(const swof_unet *u, int *d)
{
    d[0] = u->in_ch, d[1] = u->out_ch, d[2] = u->H, d[3] = u->W, d[4] = u->maxB;
}

extern "C" {

int swof_unet_create(int base, int in_ch, int out_ch, int H, int W, int max_batch, unsigned long long seed,
                     swof_unet **out)
{
    if (!out) return SWOF_EINVAL;
    *out = nullptr;
    if (base < 16 || base % 16 || base > 64 || in_ch < 1 || in_ch > 16 || out_ch < 1 || out_ch > 16 ||
        H < 16 || W < 16 || H % 8 || W % 8 || max_batch < 1)
        return SWOF_EINVAL;
    swof_unet *u = new (std::nothrow) swof_unet();
    if (!u) return SWOF_ENOMEM;
    u->C = base;
    u->in_ch = in_ch;
    u->out_ch = out_ch;
    u->H = H;
    u->W = W;
    u->maxB = max_batch;
    const int C = base;
    auto add = [&](int kind, int cin, int cout, int act) { u->layers.push_back(make_layer(kind, cin, cout, act)); };
    add(K_CONV3, in_ch, C, 1);
    add(K_CONV3, C, C, 1);
    for (int l = 1; l < 4; ++l) {
        add(K_CONV3, C << (l - 1), C << l, 1);
        add(K_CONV3, C << l, C << l, 1);
    }
    for (int l = 2; l >= 0; --l) {
        add(K_CONVT, C << (l + 1), C << l, 0);
        add(K_CONV3, 2 * (C << l), C << l, 1);
        add(K_CONV3, C << l, C << l, 1);
    }
    add(K_CONV1, C, 16, 0);
    size_t off = 0;
    for (Layer &L : u->layers) {
        L.woff = off;
        off += L.nw;
    }
    for (Layer &L : u->layers) {
        L.boff = off;
        off += L.nb;
    }
    u->nparam = off;
    size_t nwd = 0;
    for (Layer &L : u->layers) {
        u->wd_off.push_back(nwd);
        nwd += (size_t)L.cin_p * L.Kpd;
    }
    u->nwd = nwd;
    int st = SWOF_OK;
    u->w = dmalloc<float>(u, off, &st);
    u->g = dmalloc<float>(u, off, &st);
    u->m = dmalloc<float>(u, off, &st);
    u->v = dmalloc<float>(u, off, &st);
    u->wbf = dmalloc<bf16>(u, off, &st);
    u->wd = dmalloc<bf16>(u, nwd, &st);
    int nrep = 0;
    for (Layer &L : u->layers)
        if (L.kind == K_CONVT) nrep += 4 * L.cout;
    u->bias_rep = dmalloc<float>(u, (size_t)nrep, &st);
    u->err = dmalloc<int>(u, 1, &st);
    u->loss = dmalloc<double>(u, 1, &st);
    u->norm = dmalloc<float>(u, 48, &st);
    const long long B = max_batch;
    long long P0 = B * H * W;
    u->x0 = dmalloc<bf16>(u, (size_t)(P0 * 16), &st);
    u->out = dmalloc<float>(u, (size_t)(P0 * 16), &st);
    u->tgt = dmalloc<float>(u, (size_t)(P0 * 16), &st);
    u->gpred = dmalloc<float>(u, (size_t)(P0 * 16), &st);
    size_t maxdz = 0;
    for (int l = 0; l < 4; ++l) {
        long long P = B * (H >> l) * (W >> l);
        int c = C << l;
        u->ea.push_back(dmalloc<bf16>(u, (size_t)(P * c), &st));
        u->ea_pre.push_back(dmalloc<bf16>(u, (size_t)(P * c), &st));
        u->g_ea.push_back(dmalloc<float>(u, (size_t)(P * c), &st));
        u->eb_pre.push_back(l < 3 ? dmalloc<bf16>(u, (size_t)(P * c), &st) : nullptr);
        u->cat.push_back(l < 3 ? dmalloc<bf16>(u, (size_t)(P * 2 * c), &st) : nullptr);
        u->g_cat.push_back(l < 3 ? dmalloc<float>(u, (size_t)(P * 2 * c), &st) : nullptr);
        u->pool.push_back(l > 0 ? dmalloc<bf16>(u, (size_t)(P * (c / 2)), &st) : nullptr);
        u->g_pool.push_back(l > 0 ? dmalloc<float>(u, (size_t)(P * (c / 2)), &st) : nullptr);
        u->da.push_back(l < 3 ? dmalloc<bf16>(u, (size_t)(P * c), &st) : nullptr);
        u->da_pre.push_back(l < 3 ? dmalloc<bf16>(u, (size_t)(P * c), &st) : nullptr);
        u->db.push_back(l < 3 ? dmalloc<bf16>(u, (size_t)(P * c), &st) : nullptr);
        u->db_pre.push_back(l < 3 ? dmalloc<bf16>(u, (size_t)(P * c), &st) : nullptr);
        u->g_da.push_back(l < 3 ? dmalloc<float>(u, (size_t)(P * c), &st) : nullptr);
        u->g_db.push_back(l < 3 ? dmalloc<float>(u, (size_t)(P * c), &st) : nullptr);
        maxdz = maxdz > (size_t)(P * 2 * c) ? maxdz : (size_t)(P * 2 * c);
    }
    {
        long long P3 = B * (H >> 3) * (W >> 3);
        u->bott = dmalloc<bf16>(u, (size_t)(P3 * (C << 3)), &st);
        u->bott_pre = dmalloc<bf16>(u, (size_t)(P3 * (C << 3)), &st);
        u->g_bott = dmalloc<float>(u, (size_t)(P3 * (C << 3)), &st);
    }
    maxdz = maxdz > (size_t)(P0 * 16) ? maxdz : (size_t)(P0 * 16);
    u->dz = dmalloc<bf16>(u, maxdz, &st);
    {
        // partial sums of the weight gradients: the largest splits x rows x
        // columns over the layers (a layer's pixel count is at most P0, and
        // fewer pixels give no more splits)
        size_t need = 0;
        for (const Layer &L : u->layers) {
            unsigned gx, gy, gz;
            int cpc;
            swof::wgrad_grid(L.ncols, L.Kp, P0, &gx, &gy, &gz, &cpc);
            size_t n = (size_t)gz * (size_t)L.ncols * (size_t)L.Kp;
            need = need > n ? need : n;
        }
        // (also the bias-gradient and loss partial sums: <= 1024 blocks x 256
        // columns of floats, 152 x 16 doubles)
        need = need > (size_t)1024 * 256 ? need : (size_t)1024 * 256;
        u->wg_part = dmalloc<float>(u, need, &st);
        u->wg_part_n = need;
    }
    if (!st) {
        // Kaiming-normal weights (std sqrt(2 / fan_in)), zero biases, in the
        // logical entries of each padded row
        std::vector<float> hw(off, 0.0f);
        Rng rng{seed * 0x9E3779B97F4A7C15ull + 12345u};
        for (const Layer &L : u->layers) {
            int taps = L.kind == K_CONV3 ? 9 : 1;
            int fan = (L.kind == K_CONVT ? 1 : taps) * L.cin;
            double sd = std::sqrt(2.0 / fan);
            if (L.kind == K_CONV1) sd *= 0.1;   // small initial increments
            for (int n = 0; n < L.ncols; ++n)
                for (int t = 0; t < taps; ++t)
                    for (int c = 0; c < L.cin; ++c) hw[L.woff + (size_t)n * L.Kp + t * L.cin_p + c] = (float)(sd * rng.normal());
        }
        st = cudaMemcpy(u->w, hw.data(), off * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
        std::vector<float> nrm(48, 0.0f);
        for (int c = 0; c < 16; ++c) {
            nrm[16 + c] = 1.0f;
            nrm[32 + c] = 1.0f;
        }
        if (!st) st = cudaMemcpy(u->norm, nrm.data(), 48 * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
        if (!st) st = refresh_weights(u, nullptr);
        if (!st) st = cudaDeviceSynchronize() == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
    }
    if (st) {
        swof_unet_destroy(u);
        return st;
    }
    *out = u;
    return SWOF_OK;
}

void swof_unet_destroy(swof_unet *u)
{
    if (!u) return;
    cudaDeviceSynchronize();
    for (void *p : u->allocs) cudaFree(p);
    delete u;
}

long long swof_unet_param_count(const swof_unet *u) { return u ? (long long)u->nparam : 0; }

int swof_unet_layout(const swof_unet *u, int layer, int *info)
{
    if (!u || !info || layer < 0 || layer >= (int)u->layers.size()) return SWOF_EINVAL;
    const Layer &L = u->layers[(size_t)layer];
    info[0] = L.kind;
    info[1] = L.cin;
    info[2] = L.cin_p;
    info[3] = L.cout;
    info[4] = L.ncols;
    info[5] = L.Kp;
    info[6] = (int)L.woff;
    info[7] = (int)L.boff;
    info[8] = L.act;
    return (int)u->layers.size();
}

int swof_unet_get_params(swof_unet *u, float *host)
{
    if (!u || !host) return SWOF_EINVAL;
    return cudaMemcpy(host, u->w, u->nparam * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

int swof_unet_set_params(swof_unet *u, const float *host)
{
    if (!u || !host) return SWOF_EINVAL;
    if (cudaMemcpy(u->w, host, u->nparam * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return SWOF_ECUDA;
    int st = refresh_weights(u, nullptr);
    return st ? st : (cudaDeviceSynchronize() == cudaSuccess ? SWOF_OK : SWOF_ECUDA);
}

int swof_unet_get_grads(swof_unet *u, float *host)
{
    if (!u || !host) return SWOF_EINVAL;
    return cudaMemcpy(host, u->g, u->nparam * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

int swof_unet_set_norm(swof_unet *u, const float *mean, const float *scale_in, const float *scale_out)
{
    if (!u || !mean || !scale_in || !scale_out) return SWOF_EINVAL;
    std::vector<float> nrm(48, 0.0f);
    for (int c = 0; c < 16; ++c) {
        nrm[16 + c] = 1.0f;
        nrm[32 + c] = 1.0f;
    }
    for (int c = 0; c < u->in_ch; ++c) {
        if (!(scale_in[c] > 0.0f)) return SWOF_EINVAL;
        nrm[c] = mean[c];
        nrm[16 + c] = 1.0f / scale_in[c];
    }
    for (int c = 0; c < u->out_ch; ++c) {
        if (!(scale_out[c] > 0.0f)) return SWOF_EINVAL;
        nrm[32 + c] = scale_out[c];
    }
    return cudaMemcpy(u->norm, nrm.data(), 48 * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

// Forward on raw network inputs: x bf16 [B*H*W][16] (device) -> out fp32 [B*H*W][16] (device).
int swof_unet_forward_raw(swof_unet *u, const void *x, int B, float *y, void *stream)
{
    if (!u || !x || !y || B < 1 || B > u->maxB) return SWOF_EINVAL;
    cudaStream_t s = S(stream);
    long long P = (long long)B * u->H * u->W;
    if (cudaMemcpyAsync(u->x0, x, (size_t)P * 16 * sizeof(bf16), cudaMemcpyDeviceToDevice, s) != cudaSuccess) return SWOF_ECUDA;
    int st = forward(u, B, s);
    if (st) return st;
    return cudaMemcpyAsync(y, u->out, (size_t)P * 16 * sizeof(float), cudaMemcpyDeviceToDevice, s) == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

// Loss and gradients (no update) on raw inputs and targets: x bf16
// [P][16] and tgt fp32 [P][out_ch] (device).  Synchronises; *loss_host
// gets the sum of squared errors (nullable).
int swof_unet_grads_raw(swof_unet *u, const void *x, const float *tgt, int B, double *loss_host, void *stream)
{
    if (!u || !x || !tgt || B < 1 || B > u->maxB) return SWOF_EINVAL;
    cudaStream_t s = S(stream);
    long long P = (long long)B * u->H * u->W;
    cudaMemsetAsync(u->err, 0, sizeof(int), s);
    if (cudaMemcpyAsync(u->x0, x, (size_t)P * 16 * sizeof(bf16), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(u->tgt, tgt, (size_t)P * u->out_ch * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return SWOF_ECUDA;
    int st = loss_and_grads(u, B, s);
    return st ? st : read_status(u, s, loss_host);
}

// Diagnostics: copy an internal activation of the last forward (bf16 or
// fp32) to host as fp32.  which: 0 input x0, 1 ea, 2 ea_pre, 3 cat, 4 pool,
// 5 da, 6 db, 7 bottom, 8 output; level l; n values.
int swof_unet_activation(swof_unet *u, int which, int l, float *host, long long n)
{
    if (!u || !host || n < 0 || l < 0 || l > 3) return SWOF_EINVAL;
    const void *src = nullptr;
    bool isbf = true;
    switch (which) {
    case 0: src = u->x0; break;
    case 1: src = u->ea[l]; break;
    case 2: src = u->ea_pre[l]; break;
    case 3: src = u->cat[l]; break;
    case 4: src = u->pool[l]; break;
    case 5: src = u->da[l]; break;
    case 6: src = u->db[l]; break;
    case 7: src = u->bott; break;
    case 8: src = u->out; isbf = false; break;
    default: return SWOF_EINVAL;
    }
    if (!src) return SWOF_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return SWOF_ECUDA;
    if (!isbf) return cudaMemcpy(host, src, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
    std::vector<uint16_t> tmp((size_t)n);
    if (cudaMemcpy(tmp.data(), src, (size_t)n * 2, cudaMemcpyDeviceToHost) != cudaSuccess) return SWOF_ECUDA;
    for (long long i = 0; i < n; ++i) {
        uint32_t b = (uint32_t)tmp[(size_t)i] << 16;
        std::memcpy(&host[i], &b, 4);
    }
    return SWOF_OK;
}

// the input packing, with 32-bit index arithmetic when the batch fits
void pack_input(const float *in, swof_unet *u, int B, long long P, cudaStream_t s)
{
    if (P * 16 < (1LL << 31))
        swof::k_pack_input<unsigned><<<swof::grid_for(P), 256, 0, s>>>(in, u->in_ch, B, u->H, u->W, u->norm,
                                                                     u->norm + 16, u->x0);
    else
        swof::k_pack_input<long long><<<swof::grid_for(P), 256, 0, s>>>(in, u->in_ch, B, u->H, u->W, u->norm,
                                                                       u->norm + 16, u->x0);
}

// One AdamW update of the FP32 master weights from the current gradients.
int swof_unet_adamw(swof_unet *u, float lr, float beta1, float beta2, float eps, float weight_decay, void *stream)
{
    if (!u || !(lr >= 0.0f)) return SWOF_EINVAL;
    return adamw(u, lr, beta1, beta2, eps, weight_decay, S(stream));
}

// Training step on states: in [B][in_ch][H][W] (h, hu, hv, z), next
// [B][out_ch][H][W] (h, hu, hv a span later), FP32 device.  The network
// learns (next - in) / scale_out from (in - mean) / scale_in.
int swof_surrogate_train_step(swof_unet *u, const float *in, const float *next, int B, float lr, float weight_decay,
                              double *loss_host, void *stream)
{
    if (!u || !in || !next || B < 1 || B > u->maxB) return SWOF_EINVAL;
    cudaStream_t s = S(stream);
    long long P = (long long)B * u->H * u->W;
    cudaMemsetAsync(u->err, 0, sizeof(int), s);
    pack_input(in, u, B, P, s);
    swof::k_target<<<swof::grid_for(P * u->out_ch), 256, 0, s>>>(in, u->in_ch, next, u->out_ch, B, u->H, u->W,
                                                                   u->norm + 32, u->tgt);
    int st = loss_and_grads(u, B, s);
    if (!st) st = adamw(u, lr, 0.9f, 0.999f, 1e-8f, weight_decay, s);
    return st ? st : read_status(u, s, loss_host);
}

// Prediction: out[b] = in[b][0:out_ch] + scale_out * net((in - mean) / scale_in), FP32 device.
int swof_surrogate_predict(swof_unet *u, const float *in, int B, float *out, void *stream)
{
    if (!u || !in || !out || B < 1 || B > u->maxB) return SWOF_EINVAL;
    cudaStream_t s = S(stream);
    long long P = (long long)B * u->H * u->W;
    pack_input(in, u, B, P, s);
    int st = forward(u, B, s, false, false);
    if (st) return st;
    const Layer &L = u->layers[17];
    const size_t hs = (size_t)u->out_ch * u->C * sizeof(float);
    if (P * 16 < (1LL << 31))
        swof::k_head_residual<unsigned><<<swof::grid_for(P), 256, hs, s>>>(
            u->db[0], u->C, WB(u, 17), L.Kp, Bv(u, 17), in, u->in_ch, u->out_ch, B, u->H, u->W, u->norm + 32, out);
    else
        swof::k_head_residual<long long><<<swof::grid_for(P), 256, hs, s>>>(
            u->db[0], u->C, WB(u, 17), L.Kp, Bv(u, 17), in, u->in_ch, u->out_ch, B, u->H, u->W, u->norm + 32, out);
    return cudaGetLastError() == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

}  // extern "C"

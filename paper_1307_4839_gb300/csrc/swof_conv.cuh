// swof_conv.cuh -- implicit-GEMM convolutions of the learned surrogate on
// the tcgen05 tensor cores (BF16 operands, FP32 accumulation in TMEM).
//
// Activations are NHWC bf16 (channel stride cx, channel offset xc0, so a
// layer can read or write a slice of a concatenation buffer).  A layer is
// one GEMM  out[p, n] = sum_k A[p, k] W[n, k]  over output pixels p:
//   GATHER_SAME : k = tap * cin + c, A[p, k] = x[p + offset(tap), c] for a
//                 ks x ks stencil (ks = 3 or 1) at the same resolution, zero
//                 outside the image (conv forward, and data gradients with
//                 flipped / transposed weights);
//   GATHER_UP2  : k = (a*2 + b) * cin + c, A[p, k] = x[(2y+a, 2x+b), c] of a
//                 tensor at twice the resolution (data gradient of the 2x2
//                 stride-2 transposed convolution).
// Epilogue: + bias, optional GELU (pre-activation kept for the backward),
// bf16 and/or fp32 stores; SCATTER_UP2 writes column n = (a*2+b)*cout + o
// to pixel (2y+a, 2x+b), channel o (transposed-conv forward).
// The K loop is double-buffered: the CTA stages chunk k+1 while the tensor
// core works on chunk k; every wait is bounded.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tc05.cuh"

namespace swof {

enum { GATHER_SAME = 0, GATHER_UP2 = 1 };
enum { STORE_NHWC = 0, SCATTER_UP2 = 1 };
enum { ACT_NONE = 0, ACT_GELU = 1 };

struct ConvArgs {
    const __nv_bfloat16 *x;    // input activations (NHWC)
    int B, H, W;               // output-pixel grid (input grid for GATHER_UP2 is 2H x 2W)
    int cx, xc0, cin;          // input channel stride, offset, count (cin multiple of 8)
    int ks;                    // 3 or 1 (GATHER_SAME)
    int gather;
    const __nv_bfloat16 *w;    // [ntot][Kp] weights, K-major, zero-padded
    int Kp;                    // padded K (multiple of 64)
    const float *bias;         // [ntot] or null
    int ntot;                  // total GEMM columns
    __nv_bfloat16 *y;          // output (post-activation), may be null
    __nv_bfloat16 *ypre;       // pre-activation output, compact [pixels][ntot], may be null
    float *yf;                 // fp32 output, may be null
    int cy, yc0;               // output channel stride / offset (bf16 and fp32 outputs)
    int act;
    int store;                 // STORE_NHWC or SCATTER_UP2
    int cout_up;               // SCATTER_UP2: output channels
    int *err;
};

constexpr long long CONV_WAIT_LIMIT = 1LL << 22;

__device__ __forceinline__ float gelu_f(float v) { return 0.5f * v * (1.0f + erff(v * 0.70710678118654752f)); }

struct __align__(1024) ConvSmem {
    uint8_t a[2][128 * 64 * 2];
    uint8_t b[2][256 * 64 * 2];
    unsigned long long bar[2];
    uint32_t tmem;
};

// Stage the 128 x 64 chunk of the implicit A matrix (pixels m0.., columns k0..).
__device__ __forceinline__ void stage_a(uint8_t *dst, const ConvArgs &A, long long m0, int k0, long long M)
{
    const int taps = (A.gather == GATHER_SAME) ? A.ks * A.ks : 4;
    const int half = A.ks >> 1;
    const int hw = A.H * A.W;
    for (int v = threadIdx.x; v < 128 * 8; v += blockDim.x) {
        int r = v >> 3, j = v & 7;
        uint4 val = make_uint4(0, 0, 0, 0);
        long long p = m0 + r;
        int k = k0 + 8 * j;
        int tap = k / A.cin, c = k - tap * A.cin;
        if (p < M && tap < taps) {
            int b = (int)(p / hw), rem = (int)(p - (long long)b * hw);
            int yy = rem / A.W, xx = rem - yy * A.W;
            long long src = -1;
            if (A.gather == GATHER_SAME) {
                int sy = yy + tap / A.ks - half, sx = xx + tap % A.ks - half;
                if (sy >= 0 && sy < A.H && sx >= 0 && sx < A.W) src = ((long long)b * A.H + sy) * A.W + sx;
            } else {
                int sy = 2 * yy + (tap >> 1), sx = 2 * xx + (tap & 1);
                src = ((long long)b * 2 * A.H + sy) * (2 * A.W) + sx;
            }
            if (src >= 0) val = *reinterpret_cast<const uint4 *>(A.x + src * A.cx + A.xc0 + c);
        }
        *reinterpret_cast<uint4 *>(dst + tc05::canon_off(r, 8 * j)) = val;
    }
}

// Stage rows n0..n0+nrows-1 of W, columns k0..k0+63.
__device__ __forceinline__ void stage_b(uint8_t *dst, const __nv_bfloat16 *w, int n0, int nrows, int Kp, int k0)
{
    for (int v = threadIdx.x; v < nrows * 8; v += blockDim.x) {
        int r = v >> 3, j = v & 7;
        uint4 val = *reinterpret_cast<const uint4 *>(w + (long long)(n0 + r) * Kp + k0 + 8 * j);
        *reinterpret_cast<uint4 *>(dst + tc05::canon_off(r, 8 * j)) = val;
    }
}

// One CTA: 128 output pixels x NT columns (column tile blockIdx.y).
template <int NT>
__global__ void __launch_bounds__(128) k_conv(ConvArgs A)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    ConvSmem &S = *reinterpret_cast<ConvSmem *>(smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(smem_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = (long long)A.B * A.H * A.W;
    const long long m0 = (long long)blockIdx.x * 128;
    const int n0 = blockIdx.y * NT;
    if (warp == 0) {
        tc05::tmem_alloc(tc05::smem_u32(&S.tmem), 256);
        tc05::tmem_relinquish();
    }
    if (tid == 0) {
        tc05::mbar_init(tc05::smem_u32(&S.bar[0]), 1);
        tc05::mbar_init(tc05::smem_u32(&S.bar[1]), 1);
    }
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t idesc = tc05::idesc_bf16(128, NT);
    const int nk = A.Kp / 64;
    int bad = 0;
    uint32_t phase[2] = {0u, 0u};
    for (int kc = 0; kc < nk; ++kc) {
        const int s = kc & 1;
        if (kc >= 2) {
            if (!tc05::mbar_wait(tc05::smem_u32(&S.bar[s]), phase[s], CONV_WAIT_LIMIT)) bad = 1;
            phase[s] ^= 1u;
        }
        if (__syncthreads_or(bad)) break;
        stage_a(S.a[s], A, m0, kc * 64, M);
        stage_b(S.b[s], A.w, n0, NT, A.Kp, kc * 64);
        tc05::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc05::fence_after();
            const uint32_t a0 = tc05::smem_u32(S.a[s]), b0 = tc05::smem_u32(S.b[s]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                tc05::mma_bf16(tmem, tc05::sdesc(a0 + q * 256, tc05::CANON_LBO, tc05::CANON_SBO),
                               tc05::sdesc(b0 + q * 256, tc05::CANON_LBO, tc05::CANON_SBO), idesc,
                               (kc > 0 || q > 0) ? 1u : 0u);
            tc05::mma_commit(tc05::smem_u32(&S.bar[s]));
        }
    }
    if (!bad) {
        for (int kc = (nk >= 2 ? nk - 2 : 0); kc < nk; ++kc) {
            const int s = kc & 1;
            if (!tc05::mbar_wait(tc05::smem_u32(&S.bar[s]), phase[s], CONV_WAIT_LIMIT)) bad = 1;
            phase[s] ^= 1u;
        }
    }
    tc05::fence_after();
    if (!__syncthreads_or(bad)) {
        const long long p = m0 + warp * 32 + lane;
        const int hw = A.H * A.W;
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += 16) {
            float v[16];
            tc05::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (p >= M) continue;
            const int col0 = n0 + c0;
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (A.bias) v[i] += A.bias[col0 + i];
            long long dst;           // pixel index in the output tensor
            int ch;                  // first channel written
            if (A.store == STORE_NHWC) {
                dst = p;
                ch = A.yc0 + col0;
            } else {                 // 16 columns share one sub-position (cout_up multiple of 16)
                int sub = col0 / A.cout_up, o = col0 - sub * A.cout_up;
                int b = (int)(p / hw), rem = (int)(p - (long long)b * hw);
                int yy = rem / A.W, xx = rem - yy * A.W;
                dst = ((long long)b * 2 * A.H + 2 * yy + (sub >> 1)) * (2 * A.W) + 2 * xx + (sub & 1);
                ch = A.yc0 + o;
            }
            if (A.yf) {
#pragma unroll
                for (int i = 0; i < 16; ++i) A.yf[dst * A.cy + ch + i] = v[i];
            }
            if (A.ypre) {   // compact, indexed by the GEMM row and column
                __align__(16) __nv_bfloat16 t[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) t[i] = __float2bfloat16_rn(v[i]);
                uint4 *d = reinterpret_cast<uint4 *>(A.ypre + p * A.ntot + col0);
                d[0] = reinterpret_cast<uint4 *>(t)[0];
                d[1] = reinterpret_cast<uint4 *>(t)[1];
            }
            if (A.y) {
                __align__(16) __nv_bfloat16 t[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    // the activation acts on the bf16-rounded pre-activation
                    float z = A.ypre ? __bfloat162float(__float2bfloat16_rn(v[i])) : v[i];
                    t[i] = __float2bfloat16_rn(A.act == ACT_GELU ? gelu_f(z) : z);
                }
                uint4 *d = reinterpret_cast<uint4 *>(A.y + dst * A.cy + ch);
                d[0] = reinterpret_cast<uint4 *>(t)[0];
                d[1] = reinterpret_cast<uint4 *>(t)[1];
            }
        }
    } else if (tid == 0 && A.err) {
        atomicExch(A.err, 1);
    }
    tc05::fence_before();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, 256);
}

}  // namespace swof

namespace swof {

// ---------------------------------------------------------------------------
// Weight gradient:  dW[n][k] += sum_p G[p, n] * X[p, k]  (FP32 atomics),
// a GEMM with M' = n (output columns of the layer), N' = k, reduced over
// pixels p.  G is the layer's output gradient (bf16, [P][gc]) -- for the
// transposed conv gathered from the 2x-resolution tensor (row n = sub *
// cout + o); X is the layer's input, gathered like the forward A operand
// (3x3 taps or 1x1).  Both are staged transposed (pixels along K) with an
// 8 x 8 register transpose of bf16 blocks.
struct WgradArgs {
    const __nv_bfloat16 *g;    // output gradient
    int gc, gmode, cout_up;    // its channel stride; GATHER_SAME or GATHER_UP2 (transposed conv)
    const __nv_bfloat16 *x;    // layer input
    int cx, xc0, cin, ks;      // input channel stride / offset / count, stencil (3 or 1)
    int B, H, W;               // pixel grid of the reduction
    int nrows;                 // M' (number of valid rows n)
    int Kp;                    // row length of dW (padded K)
    float *dw;                 // [nrows][Kp] FP32, accumulated atomically
    int chunks_per_cta;        // pixel chunks (64 pixels) per CTA
    int *err;
};

// 8 x 8 transpose of bf16: in[i] holds row i (8 values); out[j] gets column j.
__device__ __forceinline__ void transpose8(const uint4 (&in)[8], uint4 (&out)[8])
{
    const unsigned short *s = reinterpret_cast<const unsigned short *>(in);
    unsigned short *d = reinterpret_cast<unsigned short *>(out);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) d[j * 8 + i] = s[i * 8 + j];
}

__device__ __forceinline__ uint4 load_g(const WgradArgs &A, long long p, int n, long long P)
{
    if (p >= P || n >= A.nrows) return make_uint4(0, 0, 0, 0);
    if (A.gmode == GATHER_SAME) return *reinterpret_cast<const uint4 *>(A.g + p * A.gc + n);
    const int hw = A.H * A.W;
    int sub = n / A.cout_up, o = n - sub * A.cout_up;
    int b = (int)(p / hw), rem = (int)(p - (long long)b * hw);
    int yy = rem / A.W, xx = rem - yy * A.W;
    long long q = ((long long)b * 2 * A.H + 2 * yy + (sub >> 1)) * (2 * A.W) + 2 * xx + (sub & 1);
    return *reinterpret_cast<const uint4 *>(A.g + q * A.gc + o);
}

__device__ __forceinline__ uint4 load_x(const WgradArgs &A, long long p, int k, long long P)
{
    const int taps = A.ks * A.ks;
    int tap = k / A.cin, c = k - tap * A.cin;
    if (p >= P || tap >= taps) return make_uint4(0, 0, 0, 0);
    const int hw = A.H * A.W, half = A.ks >> 1;
    int b = (int)(p / hw), rem = (int)(p - (long long)b * hw);
    int yy = rem / A.W, xx = rem - yy * A.W;
    int sy = yy + tap / A.ks - half, sx = xx + tap % A.ks - half;
    if (sy < 0 || sy >= A.H || sx < 0 || sx >= A.W) return make_uint4(0, 0, 0, 0);
    return *reinterpret_cast<const uint4 *>(A.x + (((long long)b * A.H + sy) * A.W + sx) * A.cx + A.xc0 + c);
}

template <int NT>
__global__ void __launch_bounds__(128) k_wgrad(WgradArgs A)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    ConvSmem &S = *reinterpret_cast<ConvSmem *>(smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(smem_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long P = (long long)A.B * A.H * A.W;
    const int nb0 = blockIdx.x * 128;       // rows n
    const int kb0 = blockIdx.y * NT;        // columns k
    const long long total_chunks = (P + 63) / 64;
    const long long c_begin = (long long)blockIdx.z * A.chunks_per_cta;
    long long c_end = c_begin + A.chunks_per_cta;
    if (c_end > total_chunks) c_end = total_chunks;
    if (c_begin >= c_end) return;           // uniform: nothing allocated yet
    if (warp == 0) {
        tc05::tmem_alloc(tc05::smem_u32(&S.tmem), 256);
        tc05::tmem_relinquish();
    }
    if (tid == 0) {
        tc05::mbar_init(tc05::smem_u32(&S.bar[0]), 1);
        tc05::mbar_init(tc05::smem_u32(&S.bar[1]), 1);
    }
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t idesc = tc05::idesc_bf16(128, NT);
    const int nk = (int)(c_end - c_begin);
    int bad = 0;
    uint32_t phase[2] = {0u, 0u};
    for (int kc = 0; kc < nk; ++kc) {
        const int s = kc & 1;
        if (kc >= 2) {
            if (!tc05::mbar_wait(tc05::smem_u32(&S.bar[s]), phase[s], CONV_WAIT_LIMIT)) bad = 1;
            phase[s] ^= 1u;
        }
        if (__syncthreads_or(bad)) break;
        const long long p0 = (c_begin + kc) * 64;
        // A' = G^T: 16 row blocks (n) x 8 pixel blocks, one per thread
        {
            int nb = tid & 15, pb = tid >> 4;
            uint4 in[8], out[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) in[i] = load_g(A, p0 + pb * 8 + i, nb0 + nb * 8, P);
            transpose8(in, out);
#pragma unroll
            for (int r = 0; r < 8; ++r)
                *reinterpret_cast<uint4 *>(S.a[s] + tc05::canon_off(nb * 8 + r, pb * 8)) = out[r];
        }
        // B' = X^T: NT/8 row blocks (k) x 8 pixel blocks
        for (int blk = tid; blk < (NT / 8) * 8; blk += 128) {
            int kbk = blk % (NT / 8), pb = blk / (NT / 8);
            uint4 in[8], out[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) in[i] = load_x(A, p0 + pb * 8 + i, kb0 + kbk * 8, P);
            transpose8(in, out);
#pragma unroll
            for (int r = 0; r < 8; ++r)
                *reinterpret_cast<uint4 *>(S.b[s] + tc05::canon_off(kbk * 8 + r, pb * 8)) = out[r];
        }
        tc05::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc05::fence_after();
            const uint32_t a0 = tc05::smem_u32(S.a[s]), b0 = tc05::smem_u32(S.b[s]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                tc05::mma_bf16(tmem, tc05::sdesc(a0 + q * 256, tc05::CANON_LBO, tc05::CANON_SBO),
                               tc05::sdesc(b0 + q * 256, tc05::CANON_LBO, tc05::CANON_SBO), idesc,
                               (kc > 0 || q > 0) ? 1u : 0u);
            tc05::mma_commit(tc05::smem_u32(&S.bar[s]));
        }
    }
    if (!bad) {
        for (int kc = (nk >= 2 ? nk - 2 : 0); kc < nk; ++kc) {
            const int s = kc & 1;
            if (!tc05::mbar_wait(tc05::smem_u32(&S.bar[s]), phase[s], CONV_WAIT_LIMIT)) bad = 1;
            phase[s] ^= 1u;
        }
    }
    tc05::fence_after();
    if (!__syncthreads_or(bad)) {
        const int n = nb0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += 16) {
            float v[16];
            tc05::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (n < A.nrows) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (kb0 + c0 + i < A.Kp) atomicAdd(&A.dw[(long long)n * A.Kp + kb0 + c0 + i], v[i]);
            }
        }
    } else if (tid == 0 && A.err) {
        atomicExch(A.err, 1);
    }
    tc05::fence_before();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, 256);
}

}  // namespace swof

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
// The forward K loop is a multi-stage cp.async pipeline (the weight-gradient
// kernel double-buffers); every wait is bounded.
#pragma once
#include <cuda.h>
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
    int cx, xc0, cin;          // input channel stride, offset, count (cin a power of two >= 8)
    int cin_shift;             // log2(cin)
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
    int pre_round;             // 1: the activation acts on the bf16-rounded pre-activation
    int store;                 // STORE_NHWC or SCATTER_UP2
    int cout_up;               // SCATTER_UP2: output channels
    int ystage;                // 32 or 64: bf16 output y staged in shared memory per piece of that many
                               // columns and written by TMA stores (k_conv_halo, k_conv_tma); 0: plain stores
    int *err;
};

constexpr long long CONV_WAIT_LIMIT = 1LL << 22;

// erf(x) by Abramowitz & Stegun, Handbook of Mathematical Functions, formula
// 7.1.28: 1 - (1 + a1 x + ... + a6 x^6)^-16 for x >= 0 (|error| <= 3e-7),
// odd extension; one reciprocal, no exponential.  The surrogate rounds its
// activations to bf16 (relative 4e-3), far above this error.
__device__ __forceinline__ float erf_as(float x)
{
    const float a = fabsf(x);
    float p = 0.0000430638f;
    p = fmaf(p, a, 0.0002765672f);
    p = fmaf(p, a, 0.0001520143f);
    p = fmaf(p, a, 0.0092705272f);
    p = fmaf(p, a, 0.0422820123f);
    p = fmaf(p, a, 0.0705230784f);
    p = fmaf(p, a, 1.0f);
    p = p * p;
    p = p * p;
    p = p * p;
    p = p * p;                         // (...)^16; +inf for large x -> erf = 1
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p));
    return copysignf(1.0f - r, x);
}
// GELU(v) = v Phi(v) = 0.5 v (1 + erf(v / sqrt 2)).  With r = (1 + a1 x + ...
// + a6 x^6)^-16 at x = |v| / sqrt 2 (the tail term of 7.1.28 above),
// 1 + erf = 2 - r for v >= 0 and r for v < 0, so GELU = v - v r / 2 or v r / 2:
// no 1 - r, sign transfer or 1 + erf, and the negative tail keeps r's
// relative accuracy.
__device__ __forceinline__ float gelu_f(float v)
{
    const float a = fabsf(v) * 0.70710678118654752f;
    float p = 0.0000430638f;
    p = fmaf(p, a, 0.0002765672f);
    p = fmaf(p, a, 0.0001520143f);
    p = fmaf(p, a, 0.0092705272f);
    p = fmaf(p, a, 0.0422820123f);
    p = fmaf(p, a, 0.0705230784f);
    p = fmaf(p, a, 1.0f);
    p = p * p;
    p = p * p;
    p = p * p;
    p = p * p;
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p));
    const float h = (0.5f * v) * r;
    return v >= 0.0f ? v - h : h;
}

struct __align__(1024) ConvSmem {
    uint8_t a[2][128 * 64 * 2];
    uint8_t b[2][256 * 64 * 2];
    unsigned long long bar[2];
    uint32_t tmem;
};

// ---- cp.async (16-byte copies global -> shared through L1, which keeps
// the 3x3 taps' re-reads of a pixel on chip; zero-filled when the
// source size is 0) ----
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Pipeline depth and shared-memory footprint of k_conv<NT>.
template <int NT>
struct ConvCfg {
    static constexpr int STAGES = NT >= 256 ? 3 : (NT >= 128 ? 4 : 6);
    static constexpr int A_BYTES = 128 * 64 * 2;
    static constexpr int B_BYTES = NT * 64 * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int TC = NT < 32 ? 32 : NT;           // columns of one accumulator
    static constexpr int TMEM_COLS = 2 * TC;               // two accumulators
#ifndef CONV_PRODUCER_WARPS
#define CONV_PRODUCER_WARPS 4
#endif
    static constexpr int PRODUCER_WARPS = CONV_PRODUCER_WARPS;
    static constexpr int THREADS = 32 * (PRODUCER_WARPS + 5);   // producers, 1 MMA, 4 epilogue warps
    static constexpr int BIAS_BYTES = 256 * 4;
    static constexpr int BAR_BYTES = (2 * STAGES + 4) * 8 + 16;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + BIAS_BYTES + BAR_BYTES + 1024;
};

// Bounded mbarrier wait that also gives up when another role has aborted;
// a wait that runs out raises the abort flag.
__device__ __forceinline__ bool conv_wait(uint32_t bar, uint32_t parity, volatile int *abort)
{
    for (long long i = 0; i < CONV_WAIT_LIMIT; ++i) {
        if (tc05::mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 63 && *abort) return false;
    }
    *abort = 1;
    return false;
}

// Epilogue of one 128-pixel tile for the 32 pixel rows of TMEM lane quarter
// `quarter` (this warp): accumulator columns at TMEM address tb + c, bias
// from shared memory, optional pre-activation, activation, stores.
template <int NT>
__device__ __forceinline__ void conv_tile_epilogue(const ConvArgs &A, uint32_t tmem, int acc_col, int quarter,
                                                   long long m0, int n0, long long M, const float *sbias, int cb = 0,
                                                   int ce = NT)
{
    const int lane = threadIdx.x & 31;
    const int hw = A.H * A.W;
    const long long p = m0 + quarter * 32 + lane;
    const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)acc_col;
#pragma unroll 1
    for (int c0 = cb; c0 < ce; c0 += 16) {
        float v[16];
        tc05::tmem_ld16(tb + (uint32_t)c0, v);
        if (p >= M) continue;
        const int col0 = n0 + c0;
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] += sbias[c0 + i];
        long long dst;           // pixel index in the output tensor
        int ch;                  // first channel written
        if (A.store == STORE_NHWC) {
            dst = p;
            ch = A.yc0 + col0;
        } else {                 // 16 columns share one sub-position (cout_up multiple of 16)
            const int sub = col0 / A.cout_up, o = col0 - sub * A.cout_up;
            const int b = (int)(p / hw), rem = (int)(p - (long long)b * hw);
            const int yy = rem / A.W, xx = rem - yy * A.W;
            dst = ((long long)b * 2 * A.H + 2 * yy + (sub >> 1)) * (2 * A.W) + 2 * xx + (sub & 1);
            ch = A.yc0 + o;
        }
        if (A.yf) {
            float4 *dp = reinterpret_cast<float4 *>(A.yf + dst * A.cy + ch);
#pragma unroll
            for (int i = 0; i < 4; ++i) dp[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
        if (A.ypre) {   // compact, indexed by the GEMM row and column
            __align__(16) __nv_bfloat16 t[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) t[i] = __float2bfloat16_rn(v[i]);
            uint4 *dp = reinterpret_cast<uint4 *>(A.ypre + p * A.ntot + col0);
            dp[0] = reinterpret_cast<uint4 *>(t)[0];
            dp[1] = reinterpret_cast<uint4 *>(t)[1];
        }
        if (A.y) {
            __align__(16) __nv_bfloat16 t[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                // the activation acts on the bf16-rounded pre-activation
                const float z = A.pre_round ? __bfloat162float(__float2bfloat16_rn(v[i])) : v[i];
                t[i] = __float2bfloat16_rn(A.act == ACT_GELU ? gelu_f(z) : z);
            }
            uint4 *dp = reinterpret_cast<uint4 *>(A.y + dst * A.cy + ch);
            dp[0] = reinterpret_cast<uint4 *>(t)[0];
            dp[1] = reinterpret_cast<uint4 *>(t)[1];
        }
    }
}

// Shared-memory staging of the TMA-store epilogue: per epilogue warp one
// (pw = 64) or two buffers of 32 rows (its pixels) x pw bf16 columns
// (pw = A.ystage), in the swizzled layout of the output tensor map (128-,
// 64- or 32-byte swizzle for rows of 64, 32 or 16 columns), so the 32
// lanes' 16-byte writes of one chunk hit distinct bank groups.
constexpr int EPI_WARPS = 8;                                 // two per TMEM lane quarter
__host__ __device__ constexpr int epi_bufs(int pw) { return pw == 64 ? 1 : 2; }
__host__ __device__ constexpr int epi_stage_bytes(int pw) { return EPI_WARPS * epi_bufs(pw) * 32 * pw * 2; }
constexpr int EPI_STAGE_BYTES_MAX = 32 * 1024;               // epi_stage_bytes(16 / 32 / 64) <= 32 KB
__device__ __forceinline__ uint32_t epi_swz(int r, int j, int pw)
{
    return pw == 64   ? (uint32_t)(r * 128 + ((j ^ (r & 7)) << 4))                 // 128-byte swizzle
           : pw == 32 ? (uint32_t)(r * 64 + ((j ^ ((r >> 1) & 3)) << 4))           // 64-byte swizzle
                      : (uint32_t)(r * 32 + ((j ^ ((r >> 2) & 1)) << 4));          // 32-byte swizzle
}

// The same epilogue for a bf16 output y only, through shared memory and TMA
// stores: per piece of pw columns each lane writes its pixel's row into the
// warp's staging buffer, lane 0 stores the 32 x pw block with one tensor
// copy (NHWC: box {pw, 32} at (channel, pixel); SCATTER_UP2: the warp's 32
// pixels are consecutive x of one input row, box {pw, 1, 32, 1} at
// (channel, sub-x, x, output row)).  Two buffers alternate; a buffer is
// rewritten only after the store that read it has finished reading.
template <int NT>
__device__ __forceinline__ void conv_tile_epilogue_tma(const ConvArgs &A, uint32_t tmem, int acc_col, int quarter,
                                                       long long m0, int n0, const float *sbias,
                                                       const CUtensorMap *ymap, uint8_t *stg, uint32_t &nbuf,
                                                       int cb, int ce)
{
    const int lane = threadIdx.x & 31;
    const int pw = A.ystage;
    const long long p0 = m0 + quarter * 32;
    const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)acc_col;
    int b = 0, yy = 0, xx0 = 0;
    if (A.store != STORE_NHWC) {
        const int hw = A.H * A.W;
        b = (int)(p0 / hw);
        const int rem = (int)(p0 - (long long)b * hw);
        yy = rem / A.W;
        xx0 = rem - yy * A.W;
    }
#pragma unroll 1
    for (int pc = cb; pc < ce; pc += pw) {
        uint8_t *buf = stg + (epi_bufs(pw) == 2 ? (nbuf & 1) : 0) * (32 * pw * 2);
        if (lane == 0) {
            if (epi_bufs(pw) == 2)
                tc05::bulk_wait_read<1>();
            else
                tc05::bulk_wait_read<0>();
        }
        __syncwarp();
#pragma unroll 1
        for (int c0 = 0; c0 < pw; c0 += 16) {
            float v[16];
            tc05::tmem_ld16(tb + (uint32_t)(pc + c0), v);
            __align__(16) __nv_bfloat16 t[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float x = v[i] + sbias[pc + c0 + i];
                // the activation acts on the bf16-rounded pre-activation
                const float z = A.pre_round ? __bfloat162float(__float2bfloat16_rn(x)) : x;
                t[i] = __float2bfloat16_rn(A.act == ACT_GELU ? gelu_f(z) : z);
            }
            *reinterpret_cast<uint4 *>(buf + epi_swz(lane, c0 >> 3, pw)) = reinterpret_cast<uint4 *>(t)[0];
            *reinterpret_cast<uint4 *>(buf + epi_swz(lane, (c0 >> 3) + 1, pw)) = reinterpret_cast<uint4 *>(t)[1];
        }
        tc05::fence_async_smem();
        __syncwarp();
        if (lane == 0) {
            const int col = n0 + pc;
            if (A.store == STORE_NHWC) {
                tc05::tma_store_2d(ymap, tc05::smem_u32(buf), A.yc0 + col, (int)p0);
            } else {
                const int sub = col / A.cout_up, o = col - sub * A.cout_up;
                tc05::tma_store_4d(ymap, tc05::smem_u32(buf), A.yc0 + o, sub & 1, xx0, b * 2 * A.H + 2 * yy + (sub >> 1));
            }
            tc05::bulk_commit();
        }
        ++nbuf;
    }
}

// One persistent CTA handles the 128-pixel tiles m = blockIdx.x,
// blockIdx.x + gridDim.x, ... of column tile blockIdx.y (NT columns), with
// warp roles:
//   warps 0-3  producers: gather the implicit A rows (8 pixel rows and one
//              16-byte column per thread, coordinates decoded once per tile)
//              and the weight rows with cp.async into a STAGES-deep ring;
//              after a chunk's copies land, fence them to the async proxy
//              and arrive on its `full` barrier;
//   warp 4     one thread issues the tcgen05 MMAs of each chunk into one of
//              two TMEM accumulators and commits to the chunk's `empty`
//              barrier (slot reusable) and, per tile, to `acc_full`;
//   warps 5-8  epilogue: drain the finished accumulator (each warp its
//              32 TMEM lanes), bias, activation, stores; arrive on
//              `acc_empty`, so the next-but-one tile may reuse it.
// Loads, MMAs and epilogues of different chunks and tiles overlap; no
// CTA-wide barrier inside the loop.  Every wait is bounded.
template <int NT>
__global__ void __launch_bounds__(ConvCfg<NT>::THREADS) k_conv(ConvArgs A)
{
    using Cfg = ConvCfg<NT>;
    constexpr int S = Cfg::STAGES;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(smem_raw) & 1023)) & 1023);
    float *sbias = reinterpret_cast<float *>(base + S * Cfg::STAGE_BYTES);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(base + S * Cfg::STAGE_BYTES + Cfg::BIAS_BYTES);
    unsigned long long *empty = full + S;
    unsigned long long *accf = empty + S;
    unsigned long long *acce = accf + 2;
    uint32_t *tmem_word = reinterpret_cast<uint32_t *>(acce + 2);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_word + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = (long long)A.B * A.H * A.W;
    const int tiles = (int)((M + 127) / 128);
    const int n0 = blockIdx.y * NT;
    const int nk = A.Kp / 64;
    const int my_tiles = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int G = my_tiles * nk;
    if (G == 0) return;             // uniform: nothing allocated yet
    constexpr int PW = Cfg::PRODUCER_WARPS, PT = 32 * PW;   // producer warps / threads
    constexpr int RPT = 1024 / PT;                          // A rows per producer thread
    constexpr int RSTEP = PT / 8;                           // row step between them
    if (warp == PW) {
        tc05::tmem_alloc(tc05::smem_u32(tmem_word), Cfg::TMEM_COLS);
        tc05::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc05::mbar_init(tc05::smem_u32(&full[q]), PT);
            tc05::mbar_init(tc05::smem_u32(&empty[q]), 1);
        }
        for (int q = 0; q < 2; ++q) {
            tc05::mbar_init(tc05::smem_u32(&accf[q]), 1);
            tc05::mbar_init(tc05::smem_u32(&acce[q]), 128);
        }
        *abort = 0;
    }
    for (int i = tid; i < NT; i += Cfg::THREADS) sbias[i] = A.bias ? A.bias[n0 + i] : 0.0f;
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    const uint32_t tmem = *tmem_word;
    const uint32_t sbase = tc05::smem_u32(base);
    const int hw = A.H * A.W;

    if (warp < PW) {
        // ---------------- producers ----------------
        const int j = tid & 7;
        const int taps = (A.gather == GATHER_SAME) ? A.ks * A.ks : 4;
        const int half = A.ks >> 1;
        int ry[RPT], rx[RPT], rbase[RPT];
        int dec_tile = -1;
        auto decode = [&](int ti) {           // rows r_i = r0 + RSTEP i, RSTEP pixels apart
            const int m0 = ((int)blockIdx.x + ti * (int)gridDim.x) * 128;
            int p = m0 + (tid >> 3);
            int b = p / hw, rem = p - b * hw;
            int y = rem / A.W, x = rem - y * A.W;
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                if (p < (int)M) {
                    ry[i] = y;
                    rx[i] = x;
                    rbase[i] = (A.gather == GATHER_SAME) ? p : (b * 2 * A.H + 2 * y) * (2 * A.W) + 2 * x;
                } else {
                    ry[i] = rx[i] = 0;
                    rbase[i] = -1;
                }
                p += RSTEP;
                x += RSTEP;
                while (x >= A.W) {
                    x -= A.W;
                    if (++y == A.H) {
                        y = 0;
                        ++b;
                    }
                }
            }
            dec_tile = ti;
        };
        int g = 0;
#pragma unroll 1
        for (; g < G; ++g) {
            const int slot = g % S;
            if (!conv_wait(tc05::smem_u32(&empty[slot]), (uint32_t)(((g / S) & 1) ^ 1), abort)) break;
            const int ti = g / nk, kc = g - ti * nk;
            if (ti != dec_tile) decode(ti);
            const uint32_t sa = sbase + slot * Cfg::STAGE_BYTES, sb = sa + Cfg::A_BYTES;
            const int k = kc * 64 + 8 * j;
            const int tap = k >> A.cin_shift, c = k & (A.cin - 1);
            int dy = 0, dx = 0, toff;
            if (A.gather == GATHER_SAME) {
                const int ty = A.ks == 3 ? (tap * 11) >> 5 : 0;      // tap / 3 for tap < 9
                dy = ty - half;
                dx = tap - ty * A.ks - half;
                toff = dy * A.W + dx;
            } else {
                toff = (tap >> 1) * (2 * A.W) + (tap & 1);
            }
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int r = (tid >> 3) + RSTEP * i;
                bool ok = rbase[i] >= 0 && tap < taps;
                if (A.gather == GATHER_SAME) {
                    const int sy = ry[i] + dy, sx = rx[i] + dx;
                    ok = ok && sy >= 0 && sy < A.H && sx >= 0 && sx < A.W;
                }
                const __nv_bfloat16 *src = ok ? A.x + (long long)(rbase[i] + toff) * A.cx + A.xc0 + c : A.x;
                cp_async16(sa + tc05::canon_off(r, 8 * j), src, ok ? 16u : 0u);
            }
            for (int v = tid; v < NT * 8; v += PT) {
                const int r = v >> 3, jj = v & 7;
                cp_async16(sb + tc05::canon_off(r, 8 * jj), A.w + (long long)(n0 + r) * A.Kp + kc * 64 + 8 * jj, 16u);
            }
            cp_async_commit();
            if (g >= S - 2) {                 // chunk g - (S - 2) has landed
                cp_async_wait<S - 2>();
                tc05::fence_async_smem();
                mbar_arrive(tc05::smem_u32(&full[(g - (S - 2)) % S]));
            }
        }
        cp_async_wait<0>();
        tc05::fence_async_smem();
        if (g == G)
            for (int q = (G > S - 2 ? G - (S - 2) : 0); q < G; ++q) mbar_arrive(tc05::smem_u32(&full[q % S]));
    } else if (warp == PW) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            const uint32_t idesc = tc05::idesc_bf16(128, NT);
            bool ok = true;
#pragma unroll 1
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                const int acc = lt & 1;
                if (!conv_wait(tc05::smem_u32(&acce[acc]), (uint32_t)(((lt >> 1) & 1) ^ 1), abort)) break;
                tc05::fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * Cfg::TC);
#pragma unroll 1
                for (int kc = 0; kc < nk; ++kc) {
                    const int g = lt * nk + kc, slot = g % S;
                    if (!conv_wait(tc05::smem_u32(&full[slot]), (uint32_t)((g / S) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    tc05::fence_after();
                    const uint32_t a0 = sbase + slot * Cfg::STAGE_BYTES, b0 = a0 + Cfg::A_BYTES;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        tc05::mma_bf16(d, tc05::sdesc(a0 + q * 256, tc05::CANON_LBO, tc05::CANON_SBO),
                                       tc05::sdesc(b0 + q * 256, tc05::CANON_LBO, tc05::CANON_SBO), idesc,
                                       (kc > 0 || q > 0) ? 1u : 0u);
                    tc05::mma_commit(tc05::smem_u32(&empty[slot]));
                }
                if (ok) tc05::mma_commit(tc05::smem_u32(&accf[acc]));
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3;       // TMEM lanes 32 * quarter ..
#pragma unroll 1
        for (int lt = 0; lt < my_tiles; ++lt) {
            const int acc = lt & 1;
            if (!conv_wait(tc05::smem_u32(&accf[acc]), (uint32_t)((lt >> 1) & 1), abort)) break;
            tc05::fence_after();
            const long long m0 = ((long long)blockIdx.x + (long long)lt * gridDim.x) * 128;
            conv_tile_epilogue<NT>(A, tmem, acc * Cfg::TC, quarter, m0, n0, M, sbias);
            tc05::fence_before();
            mbar_arrive(tc05::smem_u32(&acce[acc]));
        }
    }
    tc05::fence_before();
    __syncthreads();
    if (*abort && tid == 0 && A.err) atomicExch(A.err, 1);
    if (warp == PW) tc05::tmem_dealloc(tmem, Cfg::TMEM_COLS);
}


// ---------------------------------------------------------------------------
// 3x3 convolution over image rows of W >= 128 pixels (W a multiple of 128)
// without a gather.  A tile is 128 consecutive pixels (h, w0 .. w0+127) of
// one image row.  For each block of CB input channels (16, 32 or 64) the
// producer loads the tile's halo -- rows h-1 .. h+1, pixels w0-1 .. w0+128 --
// with ONE TMA box of CB channels x 130 pixels x 3 rows, zero-filled outside
// the image: 390 rows of CB * 2 bytes, one per halo pixel, written with the
// swizzle of that row width.  In that layout the A operand of tap (dy, dx)
// is the 128 rows starting at halo pixel (1 + dy) * 130 + 1 + dx: a K-major
// swizzled descriptor started at that row (the swizzle follows the address).
// (Boxes one 8-channel plane wide, 16-byte rows, kept the TMA unit busy for
// ~1.2 cycles per row and set the pace of these layers.)  The whole weight
// tile [NT][Kp] stays in shared memory.
// Warp roles: 0 TMA producer, 1 MMA issue, 2-9 epilogue (two warps per
// TMEM lane quarter, each draining half of the columns).  Four TMEM
// accumulators (two at 256 columns): with 32 or 64 output channels a tile's
// MMAs are short, and the MMAs of tile t + NACC wait for tile t's epilogue
// to have drained its accumulator, so more accumulators hide more of the
// epilogue's latency.  The halo ring has S stages, as many as fit beside the
// weights (2 .. 6).
constexpr int HALO_PX = 130, HALO_ROWS = 3;

template <int NT, int CB>
struct HaloCfg {
    static constexpr int MAX_STAGES = 6;
    static constexpr int ROW_BYTES = CB * 2;                              // one halo pixel's CB channels
    static constexpr int BOX_BYTES = HALO_PX * HALO_ROWS * ROW_BYTES;
    static constexpr int STAGE_BYTES = (BOX_BYTES + 1023) / 1024 * 1024;  // stages on swizzle-group boundaries
    static constexpr int WMAX = 160 * 1024;                // resident weight tile limit
    static constexpr int SMEM_MAX = 227 * 1024;
    static constexpr int TC = NT < 32 ? 32 : NT;
    static constexpr int NACC = TC <= 128 ? 4 : 2;        // TMEM accumulators (4 x TC <= 512 columns)
    static constexpr int TMEM_COLS = NACC * TC;
    static constexpr int THREADS = 32 * (2 + EPI_WARPS);   // producer, MMA issuer, epilogue warps
    static size_t smem(int Kp, int stages, int stage_out = 0)
    {
        return (size_t)stages * STAGE_BYTES + (size_t)NT * Kp * 2 + 256 * 4 + (2 * MAX_STAGES + 2 * NACC) * 8 + 16 + 1024 +
               (size_t)stage_out;
    }
    // the deepest ring (2 .. MAX_STAGES) that fits beside the weights (and
    // stage_out bytes of output staging); 0 if none
    static int stages(int Kp, int stage_out = 0)
    {
        for (int sgs = MAX_STAGES; sgs >= 2; --sgs)
            if (smem(Kp, sgs, stage_out) <= (size_t)SMEM_MAX) return sgs;
        return 0;
    }
};

template <int NT, int CB>
__global__ void __launch_bounds__(HaloCfg<NT, CB>::THREADS)
    k_conv_halo(ConvArgs A, const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap ymap, int S)
{
    using Cfg = HaloCfg<NT, CB>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *stg = smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(smem_raw) & 1023)) & 1023);
    uint8_t *base = stg + (A.ystage ? epi_stage_bytes(A.ystage) : 0);   // TMA-store staging first (1024-aligned)
    uint8_t *wsm = base + S * Cfg::STAGE_BYTES;                        // weights, canonical per 64-chunk
    float *sbias = reinterpret_cast<float *>(wsm + (size_t)NT * A.Kp * 2);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(sbias + 256);
    unsigned long long *empty = full + S;
    unsigned long long *accf = empty + S;
    unsigned long long *acce = accf + Cfg::NACC;
    uint32_t *tmem_word = reinterpret_cast<uint32_t *>(acce + Cfg::NACC);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_word + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = (long long)A.B * A.H * A.W;
    const int tiles = (int)(M / 128);
    const int per_row = A.W / 128;
    const int n0 = blockIdx.y * NT;
    const int nb = A.cin / CB;                     // channel blocks
    const int my_tiles = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int G = my_tiles * nb;
    if (G == 0) return;
    if (warp == 1) {
        tc05::tmem_alloc(tc05::smem_u32(tmem_word), Cfg::TMEM_COLS);
        tc05::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc05::mbar_init(tc05::smem_u32(&full[q]), 1);
            tc05::mbar_init(tc05::smem_u32(&empty[q]), 1);
        }
        for (int q = 0; q < Cfg::NACC; ++q) {
            tc05::mbar_init(tc05::smem_u32(&accf[q]), 1);
            tc05::mbar_init(tc05::smem_u32(&acce[q]), 32 * EPI_WARPS);
        }
        *abort = 0;
    }
    // resident weights and biases: K-major core matrices [k / 8][NT rows][8],
    // so the descriptor of weight column k is a linear step from column 0
    const uint32_t wbase = tc05::smem_u32(wsm);
    for (int v = tid; v < NT * (A.Kp / 8); v += Cfg::THREADS) {
        const int r = v % NT, kg = v / NT;
        cp_async16(wbase + (uint32_t)(kg * (NT * 16) + r * 16), A.w + (long long)(n0 + r) * A.Kp + kg * 8, 16u);
    }
    cp_async_commit();
    for (int i = tid; i < NT; i += Cfg::THREADS) sbias[i] = A.bias ? A.bias[n0 + i] : 0.0f;
    cp_async_wait<0>();
    tc05::fence_async_smem();
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    const uint32_t tmem = *tmem_word;
    const uint32_t sbase = tc05::smem_u32(base);

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
#pragma unroll 1
            for (int g = 0; g < G; ++g) {
                const int slot = g % S;
                if (!conv_wait(tc05::smem_u32(&empty[slot]), (uint32_t)(((g / S) & 1) ^ 1), abort)) break;
                const int lt = g / nb, cb = g - lt * nb;
                const int t = (int)blockIdx.x + lt * (int)gridDim.x;
                const int rowi = t / per_row, w0 = (t - rowi * per_row) * 128;
                const int b = rowi / A.H, h = rowi - b * A.H;
                const uint32_t bar = tc05::smem_u32(&full[slot]);
                tc05::mbar_arrive_expect_tx(bar, (uint32_t)Cfg::BOX_BYTES);
                tc05::tma_load_4d(sbase + slot * Cfg::STAGE_BYTES, &tmap, cb * CB, w0 - 1, h - 1, b, bar);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            const uint32_t idesc = tc05::idesc_bf16(128, NT);
            const uint64_t b_tap_step = (uint64_t)((A.cin * NT * 2) >> 4);   // weight columns tap*cin apart
            bool ok = true;
#pragma unroll 1
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                const int acc = lt % Cfg::NACC;
                if (!conv_wait(tc05::smem_u32(&acce[acc]), (uint32_t)(((lt / Cfg::NACC) & 1) ^ 1), abort)) break;
                tc05::fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * Cfg::TC);
#pragma unroll 1
                for (int cb = 0; cb < nb; ++cb) {
                    const int g = lt * nb + cb, slot = g % S;
                    if (!conv_wait(tc05::smem_u32(&full[slot]), (uint32_t)((g / S) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    tc05::fence_after();
                    // descriptors built once per stage and stepped by constants
                    // (descriptor address fields count 16-byte units): the
                    // single issuing thread spends ~2 instructions per MMA
                    const uint64_t a0 = tc05::sdesc_swz(sbase + slot * Cfg::STAGE_BYTES, Cfg::ROW_BYTES);
                    const uint64_t b0 = tc05::sdesc(wbase + (uint32_t)(cb * CB * NT * 2), NT * 16, 128);
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int ty = tap / 3, tx = tap % 3;
                        const uint64_t at = a0 + (uint64_t)(((ty * HALO_PX + tx) * Cfg::ROW_BYTES) >> 4);
                        const uint64_t bt = b0 + (uint64_t)tap * b_tap_step;
#pragma unroll
                        for (int q = 0; q < CB / 16; ++q)
                            tc05::mma_bf16(d, at + (uint64_t)(2 * q), bt + (uint64_t)(2 * q * NT), idesc,
                                           (cb > 0 || tap > 0 || q > 0) ? 1u : 0u);
                    }
                    tc05::mma_commit(tc05::smem_u32(&empty[slot]));
                }
                if (ok) tc05::mma_commit(tc05::smem_u32(&accf[acc]));
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        // two warps per TMEM lane quarter (warp % 4), each half of the columns
        // (16-column tiles: the first warp of the pair takes all 16)
        constexpr int PER = NT >= 32 ? NT / 2 : NT;
        const int quarter = warp & 3, e = warp - 2;
        const int cb = (e >> 2) * PER < NT ? (e >> 2) * PER : NT, ce = cb + PER < NT ? cb + PER : NT;
        uint8_t *wstg = stg + e * (epi_bufs(A.ystage) * 32 * A.ystage * 2);   // this warp's staging
        uint32_t nbuf = 0;
#pragma unroll 1
        for (int lt = 0; lt < my_tiles; ++lt) {
            const int acc = lt % Cfg::NACC;
            if (!conv_wait(tc05::smem_u32(&accf[acc]), (uint32_t)((lt / Cfg::NACC) & 1), abort)) break;
            tc05::fence_after();
            const long long m0 = ((long long)blockIdx.x + (long long)lt * gridDim.x) * 128;
            if (A.ystage)
                conv_tile_epilogue_tma<NT>(A, tmem, acc * Cfg::TC, quarter, m0, n0, sbias, &ymap, wstg, nbuf, cb, ce);
            else
                conv_tile_epilogue<NT>(A, tmem, acc * Cfg::TC, quarter, m0, n0, M, sbias, cb, ce);
            tc05::fence_before();
            mbar_arrive(tc05::smem_u32(&acce[acc]));
        }
        if (A.ystage && lane == 0) tc05::bulk_wait<0>();   // the output stores have landed
    }
    tc05::fence_before();
    __syncthreads();
    if (*abort && tid == 0 && A.err) atomicExch(A.err, 1);
    if (warp == 1) tc05::tmem_dealloc(tmem, Cfg::TMEM_COLS);
}


// ---------------------------------------------------------------------------
// Same-resolution convolutions (3x3 or 1x1) with both operands loaded by TMA.
// A 128-pixel tile is a box of the NHWC input: a segment of one image row
// (W a multiple of 128) or 128 / W whole rows (W dividing 128).  For each
// 64-wide K chunk the producer issues one box per 8-channel group -- the
// tile shifted by its tap (dx, dy), zero-filled outside the image -- which
// lands as 128 rows of 16 bytes, one K-major core-matrix plane; and one box
// per 8-column group of the weight rows.  No thread touches an operand.
// Warp roles as in k_conv_halo.  K columns past the last tap (zero weights)
// read whatever finite values the slot holds; the ring is zeroed at start.
// SW (cin a multiple of 64, so a 64-wide K chunk lies in one tap): the
// chunk's A operand is ONE box of 64 channels x 128 pixels and its weights
// one box of 64 columns x NT rows, both written by the TMA unit in the
// 128-byte-swizzled K-major layout -- two copies per chunk instead of 16.
template <int NT>
struct TmaCfg {
    static constexpr int STAGES = NT >= 256 ? 4 : 6;
    static constexpr int A_BYTES = 8 * 128 * 16;
    static constexpr int B_BYTES = 8 * NT * 16;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int TC = NT < 32 ? 32 : NT;
    static constexpr int NACC = TC <= 128 ? 4 : 2;        // TMEM accumulators (4 x TC <= 512 columns)
    static constexpr int TMEM_COLS = NACC * TC;
    static constexpr int THREADS = 32 * (2 + EPI_WARPS);   // producer, MMA issuer, epilogue warps
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 256 * 4 + (2 * STAGES + 2 * NACC) * 8 + 16 + 1024;
};

template <int NT, bool SW>
__global__ void __launch_bounds__(TmaCfg<NT>::THREADS)
    k_conv_tma(ConvArgs A, const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap wmap,
               const __grid_constant__ CUtensorMap ymap)
{
    using Cfg = TmaCfg<NT>;
    constexpr int S = Cfg::STAGES;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(smem_raw) & 1023)) & 1023);
    uint8_t *stg = base + S * Cfg::STAGE_BYTES;                        // TMA-store staging (1024-aligned)
    float *sbias = reinterpret_cast<float *>(stg + (A.ystage ? epi_stage_bytes(A.ystage) : 0));
    unsigned long long *full = reinterpret_cast<unsigned long long *>(sbias + 256);
    unsigned long long *empty = full + S;
    unsigned long long *accf = empty + S;
    unsigned long long *acce = accf + Cfg::NACC;
    uint32_t *tmem_word = reinterpret_cast<uint32_t *>(acce + Cfg::NACC);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_word + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = (long long)A.B * A.H * A.W;
    const int tiles = (int)(M / 128);
    const int n0 = blockIdx.y * NT;
    const int nk = A.Kp / 64;
    const int my_tiles = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int G = my_tiles * nk;
    if (G == 0) return;
    if (warp == 1) {
        tc05::tmem_alloc(tc05::smem_u32(tmem_word), Cfg::TMEM_COLS);
        tc05::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc05::mbar_init(tc05::smem_u32(&full[q]), 1);
            tc05::mbar_init(tc05::smem_u32(&empty[q]), 1);
        }
        for (int q = 0; q < Cfg::NACC; ++q) {
            tc05::mbar_init(tc05::smem_u32(&accf[q]), 1);
            tc05::mbar_init(tc05::smem_u32(&acce[q]), 32 * EPI_WARPS);
        }
        *abort = 0;
    }
    for (int i = tid; i < NT; i += Cfg::THREADS) sbias[i] = A.bias ? A.bias[n0 + i] : 0.0f;
    {
        uint4 *z = reinterpret_cast<uint4 *>(base);
        for (int i = tid; i < S * Cfg::STAGE_BYTES / 16; i += Cfg::THREADS) z[i] = make_uint4(0, 0, 0, 0);
    }
    tc05::fence_async_smem();
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    const uint32_t tmem = *tmem_word;
    const uint32_t sbase = tc05::smem_u32(base);

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            const int taps = A.ks * A.ks, half = A.ks >> 1;
            const int rows = A.W >= 128 ? 1 : 128 / A.W;          // image rows per tile
            const int segs = A.W >= 128 ? A.W / 128 : 1;          // tiles per image row
#pragma unroll 1
            for (int g = 0; g < G; ++g) {
                const int slot = g % S;
                if (!conv_wait(tc05::smem_u32(&empty[slot]), (uint32_t)(((g / S) & 1) ^ 1), abort)) break;
                const int lt = g / nk, kc = g - lt * nk;
                const int t = (int)blockIdx.x + lt * (int)gridDim.x;
                const int rowi = (t / segs) * rows, x0 = (t - (t / segs) * segs) * 128;
                const int b = rowi / A.H, y0 = rowi - b * A.H;
                const uint32_t sa = sbase + slot * Cfg::STAGE_BYTES, sb = sa + Cfg::A_BYTES;
                const uint32_t bar = tc05::smem_u32(&full[slot]);
                if constexpr (SW) {
                    const int k = kc * 64, tap = k >> A.cin_shift, c = k & (A.cin - 1);
                    const int ty = A.ks == 3 ? (tap * 11) >> 5 : 0;    // tap / 3 for tap < 9
                    const int dy = ty - half, dx = tap - ty * A.ks - half;
                    tc05::mbar_arrive_expect_tx(bar, (uint32_t)(Cfg::A_BYTES + Cfg::B_BYTES));
                    tc05::tma_load_4d(sa, &xmap, c, x0 + dx, y0 + dy, b, bar);
                    tc05::tma_load_2d(sb, &wmap, k, n0, bar);
                    continue;
                }
                int nA = 0;
                for (int j = 0; j < 8; ++j) nA += ((kc * 64 + 8 * j) >> A.cin_shift) < taps;
                tc05::mbar_arrive_expect_tx(bar, (uint32_t)(nA * 128 * 16 + 8 * NT * 16));
                for (int j = 0; j < 8; ++j) {
                    const int k = kc * 64 + 8 * j;
                    const int tap = k >> A.cin_shift, c = k & (A.cin - 1);
                    if (tap >= taps) continue;
                    const int ty = A.ks == 3 ? (tap * 11) >> 5 : 0;    // tap / 3 for tap < 9
                    const int dy = ty - half, dx = tap - ty * A.ks - half;
                    tc05::tma_load_4d(sa + j * 2048, &xmap, c, x0 + dx, y0 + dy, b, bar);
                }
                for (int j = 0; j < 8; ++j)
                    tc05::tma_load_2d(sb + j * (NT * 16), &wmap, kc * 64 + 8 * j, n0, bar);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            const uint32_t idesc = tc05::idesc_bf16(128, NT);
            bool ok = true;
#pragma unroll 1
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                const int acc = lt % Cfg::NACC;
                if (!conv_wait(tc05::smem_u32(&acce[acc]), (uint32_t)(((lt / Cfg::NACC) & 1) ^ 1), abort)) break;
                tc05::fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * Cfg::TC);
#pragma unroll 1
                for (int kc = 0; kc < nk; ++kc) {
                    const int g = lt * nk + kc, slot = g % S;
                    if (!conv_wait(tc05::smem_u32(&full[slot]), (uint32_t)((g / S) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    tc05::fence_after();
                    const uint32_t a0 = sbase + slot * Cfg::STAGE_BYTES, b0 = a0 + Cfg::A_BYTES;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if constexpr (SW)
                            tc05::mma_bf16(d, tc05::sdesc_sw128(a0) + (uint64_t)(2 * q), tc05::sdesc_sw128(b0) + (uint64_t)(2 * q),
                                           idesc, (kc > 0 || q > 0) ? 1u : 0u);
                        else
                            tc05::mma_bf16(d, tc05::sdesc(a0 + q * 2 * 2048, 2048, 128),
                                           tc05::sdesc(b0 + q * 2 * (NT * 16), NT * 16, 128), idesc,
                                           (kc > 0 || q > 0) ? 1u : 0u);
                    }
                    tc05::mma_commit(tc05::smem_u32(&empty[slot]));
                }
                if (ok) tc05::mma_commit(tc05::smem_u32(&accf[acc]));
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        // two warps per TMEM lane quarter (warp % 4), each half of the columns
        // (16-column tiles: the first warp of the pair takes all 16)
        constexpr int PER = NT >= 32 ? NT / 2 : NT;
        const int quarter = warp & 3, e = warp - 2;
        const int cb = (e >> 2) * PER < NT ? (e >> 2) * PER : NT, ce = cb + PER < NT ? cb + PER : NT;
        uint8_t *wstg = stg + e * (epi_bufs(A.ystage) * 32 * A.ystage * 2);   // this warp's staging
        uint32_t nbuf = 0;
#pragma unroll 1
        for (int lt = 0; lt < my_tiles; ++lt) {
            const int acc = lt % Cfg::NACC;
            if (!conv_wait(tc05::smem_u32(&accf[acc]), (uint32_t)((lt / Cfg::NACC) & 1), abort)) break;
            tc05::fence_after();
            const long long m0 = ((long long)blockIdx.x + (long long)lt * gridDim.x) * 128;
            if (A.ystage)
                conv_tile_epilogue_tma<NT>(A, tmem, acc * Cfg::TC, quarter, m0, n0, sbias, &ymap, wstg, nbuf, cb, ce);
            else
                conv_tile_epilogue<NT>(A, tmem, acc * Cfg::TC, quarter, m0, n0, M, sbias, cb, ce);
            tc05::fence_before();
            mbar_arrive(tc05::smem_u32(&acce[acc]));
        }
        if (A.ystage && lane == 0) tc05::bulk_wait<0>();   // the output stores have landed
    }
    tc05::fence_before();
    __syncthreads();
    if (*abort && tid == 0 && A.err) atomicExch(A.err, 1);
    if (warp == 1) tc05::tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

}  // namespace swof

namespace swof {

// ---------------------------------------------------------------------------
// Weight gradient:  dW[n][k] += sum_p G[p, n] * X[p, k], a GEMM with M' = n
// (output columns of the layer), N' = k, reduced over pixels p.  The pixel
// range is split over the grid's z dimension; split z writes its partial
// sum to part[z][n][k] and k_wgrad_sum adds the splits in index order, so
// the result does not depend on which CTA finishes first (training is
// reproducible bit for bit).  G is the layer's output gradient (bf16, [P][gc]) -- for the
// transposed conv gathered from the 2x-resolution tensor (row n = sub *
// cout + o); X is the layer's input, gathered like the forward A operand
// (3x3 taps or 1x1).  Both are staged transposed (pixels along K) with an
// 8 x 8 register transpose of bf16 blocks.
struct WgradArgs {
    const __nv_bfloat16 *g;    // output gradient
    int gc, gmode, cout_up;    // its channel stride; GATHER_SAME or GATHER_UP2 (transposed conv)
    const __nv_bfloat16 *x;    // layer input
    int cx, xc0, cin, ks;      // input channel stride / offset / count (a power of two), stencil (3 or 1)
    int cin_shift;             // log2(cin)
    int B, H, W;               // pixel grid of the reduction
    int nrows;                 // M' (number of valid rows n)
    int Kp;                    // row length of dW (padded K)
    float *dw;                 // [nrows][Kp] FP32, accumulated (+=) by k_wgrad_sum
    float *part;               // [splits][nrows][Kp] FP32 partial sums (scratch)
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

// Eight consecutive pixels p0 .. p0+7 of the output-gradient rows n .. n+7
// (16 bytes per pixel) into in[0..7]; zero beyond P or nrows.  The pixel
// coordinates are decoded once and stepped.
__device__ __forceinline__ void load_g8(const WgradArgs &A, int p0, int n, int P, uint4 (&in)[8])
{
    if (n >= A.nrows) {
#pragma unroll
        for (int i = 0; i < 8; ++i) in[i] = make_uint4(0, 0, 0, 0);
        return;
    }
    if (A.gmode == GATHER_SAME) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            in[i] = (p0 + i < P) ? *reinterpret_cast<const uint4 *>(A.g + (long long)(p0 + i) * A.gc + n)
                                 : make_uint4(0, 0, 0, 0);
        return;
    }
    const int hw = A.H * A.W;
    const int sub = n / A.cout_up, o = n - sub * A.cout_up;
    int b = p0 / hw, rem = p0 - b * hw;
    int y = rem / A.W, x = rem - y * A.W;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (p0 + i < P) {
            const long long q = ((long long)b * 2 * A.H + 2 * y + (sub >> 1)) * (2 * A.W) + 2 * x + (sub & 1);
            in[i] = *reinterpret_cast<const uint4 *>(A.g + q * A.gc + o);
        } else {
            in[i] = make_uint4(0, 0, 0, 0);
        }
        if (++x == A.W) {
            x = 0;
            if (++y == A.H) {
                y = 0;
                ++b;
            }
        }
    }
}

// Eight consecutive pixels p0 .. p0+7 of the gathered layer input at column
// k (tap k / cin, channels k % cin .. +7), zero outside the image or beyond
// the taps; decoded once and stepped.
__device__ __forceinline__ void load_x8(const WgradArgs &A, int p0, int k, int P, uint4 (&in)[8])
{
    const int taps = A.ks * A.ks;
    const int tap = k >> A.cin_shift, c = k & (A.cin - 1);
    if (tap >= taps) {
#pragma unroll
        for (int i = 0; i < 8; ++i) in[i] = make_uint4(0, 0, 0, 0);
        return;
    }
    const int half = A.ks >> 1;
    const int ty = A.ks == 3 ? (tap * 11) >> 5 : 0;      // tap / 3 for tap < 9
    const int dy = ty - half, dx = tap - ty * A.ks - half;
    const int hw = A.H * A.W;
    int b = p0 / hw, rem = p0 - b * hw;
    int y = rem / A.W, x = rem - y * A.W;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int sy = y + dy, sx = x + dx;
        if (p0 + i < P && sy >= 0 && sy < A.H && sx >= 0 && sx < A.W)
            in[i] = *reinterpret_cast<const uint4 *>(A.x + (long long)((b * A.H + sy) * A.W + sx) * A.cx + A.xc0 + c);
        else
            in[i] = make_uint4(0, 0, 0, 0);
        if (++x == A.W) {
            x = 0;
            if (++y == A.H) {
                y = 0;
                ++b;
            }
        }
    }
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
            load_g8(A, (int)p0 + pb * 8, nb0 + nb * 8, (int)P, in);
            transpose8(in, out);
#pragma unroll
            for (int r = 0; r < 8; ++r)
                *reinterpret_cast<uint4 *>(S.a[s] + tc05::canon_off(nb * 8 + r, pb * 8)) = out[r];
        }
        // B' = X^T: NT/8 row blocks (k) x 8 pixel blocks
        for (int blk = tid; blk < (NT / 8) * 8; blk += 128) {
            int kbk = blk % (NT / 8), pb = blk / (NT / 8);
            uint4 in[8], out[8];
            load_x8(A, (int)p0 + pb * 8, kb0 + kbk * 8, (int)P, in);
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
                float *row = A.part + ((long long)blockIdx.z * A.nrows + n) * A.Kp + kb0 + c0;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (kb0 + c0 + i < A.Kp) row[i] = v[i];
            }
        }
    } else if (tid == 0 && A.err) {
        atomicExch(A.err, 1);
    }
    tc05::fence_before();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, 256);
}

// dW[e] += sum over the splits z = 0, 1, ... of part[z][e], in that order.
__global__ void k_wgrad_sum(const float *part, int splits, long long n, float *dw)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < splits; ++z) s += part[(long long)z * n + e];
        dw[e] += s;
    }
}

}  // namespace swof

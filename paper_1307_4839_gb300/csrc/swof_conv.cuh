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

// ---- cp.async (16-byte copies global -> shared, zero-filled when the
// source size is 0) ----
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Pipeline depth and shared-memory footprint of k_conv<NT>.
template <int NT>
struct ConvCfg {
    static constexpr int STAGES = NT >= 256 ? 3 : 4;
    static constexpr int A_BYTES = 128 * 64 * 2;
    static constexpr int B_BYTES = NT * 64 * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int TMEM_COLS = NT < 32 ? 32 : NT;
    static constexpr int THREADS = 256;
    static constexpr int ROWS_PER_THREAD = 128 * 8 / THREADS;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 64 + 1024;
};

// Epilogue of one 128-pixel tile: TMEM -> + bias -> (pre-activation,
// activation) -> stores.  Each thread owns one pixel row.
template <int NT>
__device__ __forceinline__ void conv_epilogue(const ConvArgs &A, uint32_t tmem, long long m0, int n0, long long M)
{
    // warp w reads TMEM lanes 32 (w % 4) ..; the warps w / 4 = 0, 1 take
    // alternate 16-column groups
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lw = warp & 3, half = warp >> 2;
    const long long p = m0 + lw * 32 + lane;
    const int hw = A.H * A.W;
#pragma unroll 1
    for (int c0 = 16 * half; c0 < NT; c0 += 32) {
        float v[16];
        tc05::tmem_ld16(tmem + ((uint32_t)(lw * 32) << 16) + (uint32_t)c0, v);
        if (p >= M) continue;
        const int col0 = n0 + c0;
        if (A.bias) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += A.bias[col0 + i];
        }
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
            float4 *d = reinterpret_cast<float4 *>(A.yf + dst * A.cy + ch);
#pragma unroll
            for (int i = 0; i < 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
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
                float z = A.pre_round ? __bfloat162float(__float2bfloat16_rn(v[i])) : v[i];
                t[i] = __float2bfloat16_rn(A.act == ACT_GELU ? gelu_f(z) : z);
            }
            uint4 *d = reinterpret_cast<uint4 *>(A.y + dst * A.cy + ch);
            d[0] = reinterpret_cast<uint4 *>(t)[0];
            d[1] = reinterpret_cast<uint4 *>(t)[1];
        }
    }
}

// A persistent CTA: 128-pixel tiles m = blockIdx.x, blockIdx.x + gridDim.x,
// ... of column tile blockIdx.y (NT columns).  The K chunks of all its
// tiles form one stream fed by a STAGES-deep cp.async pipeline: while the
// tensor core works on chunk g, the copies of chunks g+1 .. g+STAGES-1 are
// in flight -- across tile boundaries, so the next tile's operands load
// during a tile's epilogue.  Each thread gathers the same 8 A rows (pixels)
// and 16-byte column j of every chunk; their coordinates are decoded once
// per tile.
template <int NT>
__global__ void __launch_bounds__(ConvCfg<NT>::THREADS) k_conv(ConvArgs A)
{
    using Cfg = ConvCfg<NT>;
    constexpr int RPT = Cfg::ROWS_PER_THREAD;
    constexpr int RSTEP = 128 / RPT;       // row step between a thread's rows
    constexpr int S = Cfg::STAGES;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(smem_raw) & 1023)) & 1023);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(base + S * Cfg::STAGE_BYTES);
    uint32_t *tmem_word = reinterpret_cast<uint32_t *>(bar + S);
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long M = (long long)A.B * A.H * A.W;
    const int tiles = (int)((M + 127) / 128);
    const int n0 = blockIdx.y * NT;
    const int nk = A.Kp / 64;
    const int my_tiles = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int G = my_tiles * nk;
    if (G == 0) return;             // uniform: nothing allocated yet
    if (warp == 0) {
        tc05::tmem_alloc(tc05::smem_u32(tmem_word), Cfg::TMEM_COLS);
        tc05::tmem_relinquish();
    }
    if (tid == 0)
        for (int q = 0; q < S; ++q) tc05::mbar_init(tc05::smem_u32(&bar[q]), 1);
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    const uint32_t tmem = *tmem_word;
    const uint32_t idesc = tc05::idesc_bf16(128, NT);
    const uint32_t sbase = tc05::smem_u32(base);

    const int j = tid & 7;
    const int taps = (A.gather == GATHER_SAME) ? A.ks * A.ks : 4;
    const int half = A.ks >> 1;
    const int hw = A.H * A.W;
    int ry[RPT], rx[RPT];
    int rbase[RPT];                  // pixel index of the tap origin (-1: row beyond M)
    int dec_tile = -1;
    // rows r_i = r0 + RSTEP i of a tile are RSTEP pixels apart: decode r0 once,
    // then step
    auto decode = [&](int ti) {
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
    auto issue = [&](int g) {
        const int ti = g / nk, kc = g - ti * nk;
        if (ti != dec_tile) decode(ti);
        const uint32_t sa = sbase + (g % S) * Cfg::STAGE_BYTES, sb = sa + Cfg::A_BYTES;
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
        for (int v = tid; v < NT * 8; v += Cfg::THREADS) {
            const int r = v >> 3, jj = v & 7;
            cp_async16(sb + tc05::canon_off(r, 8 * jj), A.w + (long long)(n0 + r) * A.Kp + kc * 64 + 8 * jj, 16u);
        }
    };
    // parity of the completion of chunk g on its slot's barrier (the
    // (g / S)-th completion of slot g % S); every completion is consumed
    // in order, at most once, before its slot is refilled
    auto wait_mma = [&](int g) -> bool {
        return tc05::mbar_wait(tc05::smem_u32(&bar[g % S]), (uint32_t)((g / S) & 1), CONV_WAIT_LIMIT);
    };

    int bad = 0;
    int waited = -1;               // chunks whose MMA completion has been consumed: 0 .. waited
#pragma unroll 1
    for (int q = 0; q < S - 1; ++q) {
        if (q < G) issue(q);
        cp_async_commit();
    }
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
        const int slot = g % S, ti = g / nk, kc = g - ti * nk;
        cp_async_wait<S - 2>();          // this thread's copies of chunk g have landed
        tc05::fence_async_smem();
        if (__syncthreads_or(bad)) break;
        if (tid == 0) {
            tc05::fence_after();
            const uint32_t a0 = sbase + slot * Cfg::STAGE_BYTES, b0 = a0 + Cfg::A_BYTES;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                tc05::mma_bf16(tmem, tc05::sdesc(a0 + q * 256, tc05::CANON_LBO, tc05::CANON_SBO),
                               tc05::sdesc(b0 + q * 256, tc05::CANON_LBO, tc05::CANON_SBO), idesc,
                               (kc > 0 || q > 0) ? 1u : 0u);
            tc05::mma_commit(tc05::smem_u32(&bar[slot]));
        }
        // refill the slot of chunk g-1 with chunk g+S-1 once its MMAs are done
        const int nxt = g + S - 1;
        if (nxt < G) {
            if (g >= 1 && waited < g - 1) {
                if (!wait_mma(g - 1)) bad = 1;
                waited = g - 1;
            }
            if (!bad) issue(nxt);
        }
        cp_async_commit();
        if (kc == nk - 1) {              // tile ti complete: its last commit covers all its MMAs
            if (!bad && waited < g) {
                if (!wait_mma(g)) bad = 1;
                waited = g;
            }
            tc05::fence_after();
            if (__syncthreads_or(bad)) break;
            conv_epilogue<NT>(A, tmem, ((long long)blockIdx.x + (long long)ti * gridDim.x) * 128, n0, M);
            tc05::fence_before();
        }
    }
    cp_async_wait<0>();
    if (bad && tid == 0 && A.err) atomicExch(A.err, 1);
    tc05::fence_before();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, Cfg::TMEM_COLS);
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

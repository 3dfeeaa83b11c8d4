// swof_tc.cu -- BF16 GEMM on the tcgen05 tensor cores (FP32 accumulation in
// tensor memory):  C[M x N] = A[M x K] . B[N x K]^T  (+ optional bias), both
// operands K-major bf16.  One CTA of 128 threads computes a 128 x N tile:
// the threads stage 64-wide K chunks of A and B into shared memory in the
// canonical no-swizzle layout (two buffers), one thread issues four
// K=16 MMAs per chunk and commits them to the chunk buffer's mbarrier, and
// after the last chunk the four warps read their TMEM lanes and write C.
// Every mbarrier wait is bounded; a timeout sets *err and the CTA still
// frees its tensor memory before returning.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/swof.h"
#include "tc05.cuh"

namespace swof {

constexpr long long TC_WAIT_LIMIT = 1LL << 22;

template <int N>
struct __align__(1024) GemmSmem {
    uint8_t a[2][128 * 64 * 2];     // A chunk, canonical layout (16 KB each)
    uint8_t b[2][256 * 64 * 2];     // B chunk sized for N <= 256 always
    unsigned long long bar[2];
    uint32_t tmem;
};

// Copy a [rows x 64] bf16 chunk (row stride ld elements, starting at column
// k0) into the canonical layout; rows >= nrows are zero-filled.
__device__ __forceinline__ void stage_chunk(uint8_t *dst, const __nv_bfloat16 *src, int rows, int nrows,
                                            long long ld, int k0, int kmax)
{
    for (int v = threadIdx.x; v < rows * 8; v += blockDim.x) {
        int r = v >> 3, j = v & 7;
        uint4 val = make_uint4(0, 0, 0, 0);
        int k = k0 + 8 * j;
        if (r < nrows && k < kmax) val = *reinterpret_cast<const uint4 *>(src + (long long)r * ld + k);
        *reinterpret_cast<uint4 *>(dst + tc05::canon_off(r, 8 * j)) = val;
    }
}

template <int N>
__global__ void __launch_bounds__(128) k_gemm_nt(const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *C,
                                                 const float *bias, int M, int K, int ldc, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    GemmSmem<N> &S = *reinterpret_cast<GemmSmem<N> *>(
        smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(smem_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128;
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
    const uint32_t idesc = tc05::idesc_bf16(128, N);
    const int nk = (K + 63) / 64;
    int bad = 0;
    uint32_t phase[2] = {0u, 0u};
    for (int kc = 0; kc < nk; ++kc) {
        const int s = kc & 1;
        if (kc >= 2) {   // the MMAs that read this buffer two chunks ago must be done
            if (!tc05::mbar_wait(tc05::smem_u32(&S.bar[s]), phase[s], TC_WAIT_LIMIT)) bad = 1;
            phase[s] ^= 1u;
        }
        if (__syncthreads_or(bad)) break;
        stage_chunk(S.a[s], A + (long long)m0 * K, 128, M - m0, K, kc * 64, K);
        stage_chunk(S.b[s], B, N, N, K, kc * 64, K);
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
    // wait for the last commit of each buffer still in flight
    if (!bad) {
        for (int kc = (nk >= 2 ? nk - 2 : 0); kc < nk; ++kc) {
            const int s = kc & 1;
            if (!tc05::mbar_wait(tc05::smem_u32(&S.bar[s]), phase[s], TC_WAIT_LIMIT)) bad = 1;
            phase[s] ^= 1u;
        }
    }
    tc05::fence_after();
    if (!__syncthreads_or(bad)) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc05::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) C[(long long)row * ldc + c0 + i] = v[i] + (bias ? bias[c0 + i] : 0.0f);
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    tc05::fence_before();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, 256);
}

template <int N>
int launch_gemm(const void *A, const void *B, float *C, const float *bias, int M, int K, int ldc, int *err,
                cudaStream_t s)
{
    size_t smem = sizeof(GemmSmem<N>) + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_nt<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return SWOF_ECUDA;
    k_gemm_nt<N><<<(M + 127) / 128, 128, smem, s>>>(static_cast<const __nv_bfloat16 *>(A),
                                                     static_cast<const __nv_bfloat16 *>(B), C, bias, M, K, ldc, err);
    return cudaGetLastError() == cudaSuccess ? SWOF_OK : SWOF_ECUDA;
}

}  // namespace swof

extern "C" int swof_gemm_bf16_nt(const void *A, const void *B, float *C, const float *bias, int M, int N, int K,
                                 int ldc, int *err, void *stream)
{
    if (!A || !B || !C || !err || M < 1 || K < 64 || (K % 64) || ldc < N) return SWOF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (N) {
    case 16: return swof::launch_gemm<16>(A, B, C, bias, M, K, ldc, err, s);
    case 32: return swof::launch_gemm<32>(A, B, C, bias, M, K, ldc, err, s);
    case 64: return swof::launch_gemm<64>(A, B, C, bias, M, K, ldc, err, s);
    case 128: return swof::launch_gemm<128>(A, B, C, bias, M, K, ldc, err, s);
    case 256: return swof::launch_gemm<256>(A, B, C, bias, M, K, ldc, err, s);
    default: return SWOF_EINVAL;
    }
}

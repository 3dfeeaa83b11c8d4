"""tcgen05 BF16 GEMM building block vs numpy (needs a GPU).

bf16 inputs are exact in FP32/FP64, so the only difference is the FP32
accumulation order: compared at 1e-5 relative to the magnitude of the sum.
"""
import ctypes

import numpy as np
import pytest

import paper_1307_4839_gb300 as sw

pytestmark = pytest.mark.gpu


def bf16_round(x):
    import torch
    return torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float32).numpy()


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (300, 64, 192), (257, 256, 128), (1000, 32, 576),
                                   (130, 128, 64)])
def test_gemm_bf16_nt_against_numpy(M, N, K):
    import torch
    sw.build()
    L = sw.load()
    rng = np.random.default_rng(M + N + K)
    A = bf16_round(rng.standard_normal((M, K)))
    B = bf16_round(rng.standard_normal((N, K)))
    bias = rng.standard_normal(N).astype(np.float32)
    dA = torch.tensor(A, device="cuda").to(torch.bfloat16).contiguous()
    dB = torch.tensor(B, device="cuda").to(torch.bfloat16).contiguous()
    dbias = torch.tensor(bias, device="cuda")
    C = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = L.swof_gemm_bf16_nt(ctypes.c_void_p(dA.data_ptr()), ctypes.c_void_p(dB.data_ptr()),
                             ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(dbias.data_ptr()), M, N, K, N,
                             ctypes.c_void_p(err.data_ptr()), None)
    assert st == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A.astype(np.float64) @ B.astype(np.float64).T + bias
    got = C.cpu().numpy()
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T + 1.0
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref) / scale) < 1e-5

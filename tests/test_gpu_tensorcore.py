"""Tensor-core (tcgen05) GEMM of the warm-start network against a plain FP32 product (GPU).

Row lengths that are multiples of 8 elements take the pipelined path (asynchronous 16-byte copies, three
64-wide K chunks in flight, ragged edges zero-filled); others (K = 100) the element-gather path.
"""

import numpy as np
import pytest

from paper_2510_16172_gb300 import fpt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2510_16172_gb300 import build

    build.build()
    return fpt.Context(0)


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (1, 16, 16), (300, 200, 100), (1000, 64, 256), (129, 256, 256),
                                   (4096, 16, 256), (256, 256, 4096), (200, 48, 1000), (130, 256, 136)])
def test_tc_gemm_matches_fp32_product(ctx, M, N, K):
    import torch

    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    W = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).float().cuda()
    C = fpt.tc_gemm_bf16(ctx, A, W, bias)
    ctx.sync()
    ref = (A.double() @ W.double().T + bias.double()).float()
    err = (C - ref).abs().max().item()
    scale = max(1.0, ref.abs().max().item())
    assert err <= 1e-4 * scale * np.sqrt(K), (err, scale)

"""Tensor-core (tcgen05) GEMM of the warm-start network against a plain FP32 product (GPU).

Row lengths that are multiples of 8 elements take the persistent warp-specialised kernel (TMA operand
boxes, ragged edges zero-filled by the copy engine); others (K = 100) the element-gather kernel.  The
last test drives the bounded mbarrier wait both kernels use into its poll limit.
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


def test_bounded_wait_reports_device_error_and_context_stays_usable(ctx):
    """A wait on an mbarrier that nothing arrives on gives up at its time limit and is reported by
    fpt_sync as FPT_EDEVICE; the word is then cleared, and the tensor cores still compute correctly."""
    import torch

    with pytest.raises(fpt.FptError, match="FPT_EINVAL"):
        fpt.check_bounded_wait(ctx, 1000001, arrive=False)
    with pytest.raises(fpt.FptError, match="FPT_EINVAL"):
        fpt.check_bounded_wait(ctx, 0, arrive=True)

    ns_ok = fpt.check_bounded_wait(ctx, 20000, arrive=True)
    ctx.sync()  # the arrival completed the phase: no error
    assert ns_ok < 1_000_000

    ns = fpt.check_bounded_wait(ctx, 20000, arrive=False)
    with pytest.raises(fpt.FptError, match="FPT_EDEVICE"):
        ctx.sync()
    ctx.sync()  # fpt_sync cleared the error word
    # the wait ends at its limit, not a poll count later (one poll suspends for microseconds)
    assert 20_000_000 <= ns < 100_000_000, ns
    print(f"wait with a 20 ms limit gave up after {ns / 1e6:.3f} ms")

    M, N, K = 300, 200, 100
    g = torch.Generator(device="cpu").manual_seed(5)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    W = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = fpt.tc_gemm_bf16(ctx, A, W)
    ctx.sync()
    ref = (A.double() @ W.double().T).float()
    assert (C - ref).abs().max().item() <= 1e-4 * max(1.0, ref.abs().max().item()) * np.sqrt(K)

"""The tcgen05 GEMM building block (TMA + 128B swizzle + TMEM) against float64 matmul of the
same rounded operands, on ragged shapes that exercise partial tiles and K below one atom."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(1, 128, 16, 16), (2, 200, 96, 40), (1, 128, 256, 64), (1, 256, 48, 96), (3, 130, 200, 136),
          (1, 64, 160, 8), (2, 300, 33, 72)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2401_04189_gb300 import build
    build.build()


def _round(x, prec):
    import torch
    if prec in ("bf16", "bf16x3"):
        hi = x.to(torch.bfloat16).float()
        lo = (x - hi).to(torch.bfloat16).float()
    else:
        u = x.view(torch.int32)
        hi = ((u + 0x1000) & ~0x1FFF).view(torch.float32)
        lo = x - hi
    return hi, lo


@pytest.mark.parametrize("prec", ["bf16", "tf32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("shape", SHAPES)
def test_tc_gemm_matches_float64(prec, shape):
    import torch
    import paper_2401_04189_gb300 as P
    b, M, N, K = shape
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(b, M, K, device="cuda", generator=g)
    B = torch.randn(b, N, K, device="cuda", generator=g)
    D = P.tx_selftest_gemm(prec, A, B)
    ah, al = _round(A, prec)
    bh, bl = _round(B, prec)
    if prec in ("bf16", "tf32"):
        ref = ah.double() @ bh.double().transpose(1, 2)
        tol = 2e-6
    else:
        ref = ah.double() @ bh.double().transpose(1, 2) + ah.double() @ bl.double().transpose(1, 2) + \
            al.double() @ bh.double().transpose(1, 2)
        tol = 2e-6
    err = ((D.double() - ref).norm() / ref.norm()).item()
    assert err < tol, f"{prec} {shape}: rel err {err:.3e}"

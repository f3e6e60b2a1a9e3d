"""The allocation-free apply entry point (tx_exchange_apply_static), for callers that cannot let
a library call cudaMalloc: applications whose device memory belongs to their own arena or pool
allocator, and loops that cannot afford the device-wide synchronisation cudaMalloc may cause.
It keeps all scratch in one fixed device array, so it must give the same result as the regular
entry point on consecutive calls (the array keeps the previous call's contents), allocate
nothing (the context's workspace stays empty and the device's free memory does not change),
and refuse sizes whose scratch does not fit.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as W
from _helpers import W_TOL, rel, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2401_04189_gb300 import build
    build.build()


def _call(P, ctx, psi, out):
    import torch
    return P.lib().tx_exchange_apply_static(ctx.handle, ctypes.c_void_p(psi.data_ptr()), psi.shape[0],
                                            ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_static_scratch_apply_matches_regular_apply_twice(prec):
    import torch
    import paper_2401_04189_gb300 as P
    s = W.config_small()
    psi = to_gpu(s.psi)
    # the reference: the regular float32 entry point, on a context of its own
    ref_ctx = P.Context.from_system(s, precision="fp32")
    ref = P.tx_exchange_apply(ref_ctx, psi).cpu().numpy()
    ref_ctx.destroy()
    # a fresh context that never runs the regular apply (so it holds no workspace)
    ctx = P.Context.from_system(s, precision=prec)
    assert ctx.workspace_bytes() == 0
    out = torch.empty_like(psi)
    torch.cuda.synchronize()
    for call in range(3):
        out.fill_(7.0)                          # stale output must not leak into the result
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = _call(P, ctx, psi, out)
        assert st == 0, P.lib().tx_last_error_message()
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        ctx.check_device_error()
        assert rel(out.cpu().numpy(), ref) < W_TOL["fp32"], f"call {call}"
        assert ctx.workspace_bytes() == 0, "the static entry point sized the context workspace"
        if call > 0:                            # after the first call every kernel is loaded
            assert free_after == free_before, f"call {call}: device free memory changed by {free_before - free_after}"


def test_static_scratch_apply_rejects_too_large_sizes():
    import torch
    import paper_2401_04189_gb300 as P
    n, r, T = 128, 64, 45                        # one pair needs ~95 MB of float32 scratch
    x, w = W.uniform_grid(n, 8.0)
    U = [np.linalg.qr(np.random.default_rng(d).standard_normal((n, r)))[0] for d in range(3)]
    theta, mu, _ = W.exp_sum_inverse_r(T, x[1] - x[0], 16 * 3 ** 0.5)
    ctx = P.Context([x] * 3, [w] * 3, U, theta, mu, precision="fp32")
    psi = torch.zeros((1, n, n, n), dtype=torch.float32, device="cuda")
    out = torch.empty_like(psi)
    st = _call(P, ctx, psi, out)
    assert st == -9
    msg = P.lib().tx_last_error_message().decode()
    assert "bytes of scratch" in msg and "33554432" in msg
    assert ctx.workspace_bytes() == 0

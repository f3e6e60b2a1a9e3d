"""Failure handling on the GPU without faulting it: non-finite inputs propagate (no trap, no
hang, the context stays usable), outputs are written inside their block only (canaries around
it stay intact), a bounded device wait that runs out is reported as TX_ERR_TIMEOUT and the
context works afterwards, and a captured batch graph whose buffers were replaced is refused."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _helpers import W_TOL, assert_close, rel, to_gpu

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16", "tf32", "tf32x3", "bf16x3"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2401_04189_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def small():
    s = W.config_small(n=16, n_orb=3, rank=6, T=4, L=5.0)
    S = O.Setup.from_system(s)
    return s, O.exchange_apply(s.psi, S)


@pytest.mark.parametrize("prec", PRECS)
def test_nan_input_propagates_and_context_stays_usable(prec, small):
    import paper_2401_04189_gb300 as P
    s, ref = small
    ctx = P.Context.from_system(s, precision=prec)
    bad = s.psi.copy()
    bad[1, 5, 6, 7] = np.nan
    out = P.tx_exchange_apply(ctx, to_gpu(bad)).cpu().numpy()
    ctx.check_device_error()                 # no wait gave up: the kernels ran to the end
    # every target pairs with orbital 1, whose pair densities carry the NaN into the core
    for i in range(out.shape[0]):
        assert np.isnan(out[i]).any(), f"target {i}: NaN did not propagate"
    e = float(P.tx_exchange_energy(ctx, to_gpu(bad)).item())
    assert not np.isfinite(e)
    # the same context on clean input
    got = P.tx_exchange_apply(ctx, to_gpu(s.psi)).cpu().numpy()
    ctx.check_device_error()
    assert_close(got, ref, prec, "after-nan")


@pytest.mark.parametrize("prec", PRECS)
def test_outputs_stay_inside_their_block(prec, small):
    """The output block sits between two canary orbitals; the apply writes its block only."""
    import torch
    import paper_2401_04189_gb300 as P
    s, ref = small
    ctx = P.Context.from_system(s, precision=prec)
    nt = s.psi.shape[0]
    buf = torch.full((nt + 2,) + tuple(s.psi.shape[1:]), 12345.0, dtype=torch.float32, device="cuda")
    out = buf[1:nt + 1]
    P.tx_exchange_apply(ctx, to_gpu(s.psi), out=out)
    ctx.check_device_error()
    b = buf.cpu().numpy()
    assert np.all(b[0] == 12345.0) and np.all(b[-1] == 12345.0)
    assert_close(b[1:nt + 1], ref, prec, "canary")


def test_bounded_wait_gives_up_and_context_recovers(small):
    """A wait on a barrier that nothing completes gives up after the context's limit, the host
    reads TX_ERR_TIMEOUT (where = the self-test's site), and the same context, with the limit
    restored, runs a correct tensor-core apply (the self-test freed its TMEM)."""
    import paper_2401_04189_gb300 as P
    s, ref = small
    ctx = P.Context.from_system(s, precision="bf16")
    with pytest.raises(P.TuckerExchangeError):
        ctx.set_wait_limit(10)               # below 1 us
    with pytest.raises(P.TuckerExchangeError):
        ctx.set_wait_limit(61 * 10 ** 9)     # above 60 s
    ctx.set_wait_limit(2_000_000)            # 2 ms
    for hold in (True, False):
        P.tx_selftest_wait(ctx, hold_tmem=hold)
        with pytest.raises(P.TuckerExchangeError) as ei:
            ctx.check_device_error()
        assert ei.value.status == -7
        assert "where 90" in str(ei.value)
        ctx.check_device_error()             # the word was cleared by the read
    ctx.set_wait_limit(0)
    got = P.tx_exchange_apply(ctx, to_gpu(s.psi)).cpu().numpy()
    ctx.check_device_error()
    assert_close(got, ref, "bf16", "after-timeout")


def test_replay_refused_after_workspace_replaced(small):
    """A captured batch graph holds raw workspace pointers: once a larger call on the same
    context replaces the workspace, replay is refused (TX_ERR_NOT_SETUP) until it is captured
    again; after the new capture the replay gives the individual call's result."""
    import torch
    import paper_2401_04189_gb300 as P
    s, ref = small
    ctx = P.Context.from_system(s, precision="bf16")
    psi = to_gpu(s.psi)
    plan = P.BatchPlan([dict(ctx=ctx, psi_occ=psi[:2])])
    st = torch.cuda.Stream()
    plan.capture(st)
    plan.replay(st)
    st.synchronize()
    before = ctx.workspace_bytes()
    P.tx_exchange_apply(ctx, psi)            # three orbitals: a larger workspace
    torch.cuda.synchronize()
    assert ctx.workspace_bytes() > before
    with pytest.raises(P.TuckerExchangeError) as ei:
        plan.replay(st)
    assert ei.value.status == -8
    plan.capture(st)
    plan.outputs()[0].zero_()
    plan.replay(st)
    st.synchronize()
    ctx.check_device_error()
    one = P.tx_exchange_apply(ctx, psi[:2]).cpu().numpy()
    assert rel(plan.outputs()[0].cpu().numpy(), one) < 1e-6
    # a destroyed context is refused too
    plan.capture(st)
    ctx.destroy()
    with pytest.raises(P.TuckerExchangeError) as ei:
        plan.replay(st)
    assert ei.value.status == -8
    with pytest.raises(P.TuckerExchangeError):
        plan.launch(st)

"""The torch.autograd wrappers (ExchangeEnergy, ExchangeApply) on the CPU: the library calls they
make are replaced by the oracle, so these tests check the wrappers' own logic (which call the
backward makes, which gradient goes to which input, scaling by the incoming gradient, the sum
autograd forms when one tensor is both the occupied and the target block) and, through
torch.autograd.gradcheck, that the backward is the derivative of the forward."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W


@pytest.fixture()
def wired(monkeypatch):
    import paper_2401_04189_gb300.autograd as A
    s = W.config_small(n=8, n_orb=3, rank=5, T=3, L=3.0)
    S = O.Setup.from_system(s)
    calls = []

    def energy(ctx, psi):
        calls.append("energy")
        return torch.tensor(O.exchange_energy(psi.detach().numpy(), S), dtype=torch.float64)

    def energy_grad(ctx, psi):
        calls.append("energy_grad")
        E, g = O.exchange_energy_grad(psi.detach().numpy(), S)
        return torch.tensor(E, dtype=torch.float64), torch.from_numpy(g).to(psi.dtype)

    def apply(ctx, occ, tgt):
        calls.append("apply")
        return torch.from_numpy(O.exchange_apply(occ.detach().numpy(), S, psi_tgt=tgt.detach().numpy())).to(occ.dtype)

    def vjp(ctx, occ, tgt, gW, need_occ=True, need_tgt=True):
        calls.append(("vjp", need_occ, need_tgt))
        go, gt = O.exchange_apply_vjp(occ.detach().numpy(), tgt.detach().numpy(), gW.detach().numpy(), S)
        return (torch.from_numpy(go).to(occ.dtype) if need_occ else None,
                torch.from_numpy(gt).to(tgt.dtype) if need_tgt else None)

    monkeypatch.setattr(A, "tx_exchange_energy", energy)
    monkeypatch.setattr(A, "tx_exchange_energy_grad", energy_grad)
    monkeypatch.setattr(A, "tx_exchange_apply", apply)
    monkeypatch.setattr(A, "tx_exchange_apply_vjp", vjp)
    return A, s, S, calls


def test_energy_backward_is_the_scaled_energy_gradient(wired):
    A, s, S, calls = wired
    x = torch.from_numpy(s.psi.astype(np.float64)).requires_grad_(True)
    E = A.exchange_energy(object(), x)
    E_ref, g_ref = O.exchange_energy_grad(s.psi, S)
    assert abs(float(E.detach()) - E_ref) <= 1e-12 * abs(E_ref)
    (2.5 * E).backward()
    assert calls == ["energy", "energy_grad"]
    np.testing.assert_allclose(x.grad.numpy(), 2.5 * g_ref, rtol=1e-12, atol=1e-14)


def test_apply_backward_routes_each_gradient(wired):
    A, s, S, calls = wired
    rng = np.random.default_rng(5)
    occ = torch.from_numpy(s.psi.astype(np.float64)).requires_grad_(True)
    tgt = torch.from_numpy(s.psi[:2] + 0.3 * rng.standard_normal(s.psi[:2].shape)).requires_grad_(True)
    cot = torch.from_numpy(rng.standard_normal(tgt.shape))
    (A.exchange_apply(object(), occ, tgt) * cot).sum().backward()
    go, gt = O.exchange_apply_vjp(occ.detach().numpy(), tgt.detach().numpy(), cot.numpy(), S)
    np.testing.assert_allclose(occ.grad.numpy(), go, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(tgt.grad.numpy(), gt, rtol=1e-12, atol=1e-14)
    # only the target needs a gradient: the occupied-block part is not requested
    calls.clear()
    tgt.grad = None
    (A.exchange_apply(object(), occ.detach(), tgt) * cot).sum().backward()
    assert calls == ["apply", ("vjp", False, True)]
    np.testing.assert_allclose(tgt.grad.numpy(), gt, rtol=1e-12, atol=1e-14)


def test_apply_with_one_tensor_as_both_blocks_sums_the_two_parts(wired):
    A, s, S, calls = wired
    rng = np.random.default_rng(6)
    x = torch.from_numpy(s.psi.astype(np.float64)).requires_grad_(True)
    cot = torch.from_numpy(rng.standard_normal(x.shape))
    (A.exchange_apply(object(), x, x) * cot).sum().backward()
    go, gt = O.exchange_apply_vjp(s.psi, s.psi, cot.numpy(), S)
    np.testing.assert_allclose(x.grad.numpy(), go + gt, rtol=1e-12, atol=1e-14)


def test_wrappers_pass_gradcheck(wired):
    """The backward of each wrapper against central differences of its forward (float64)."""
    A, s, S, calls = wired
    rng = np.random.default_rng(7)
    x = torch.from_numpy(s.psi[:2].astype(np.float64)).requires_grad_(True)
    t = torch.from_numpy(s.psi[2:3] + 0.2 * rng.standard_normal(s.psi[2:3].shape)).requires_grad_(True)
    ctx = object()
    assert torch.autograd.gradcheck(lambda a: A.exchange_energy(ctx, a), (x,), eps=1e-6, atol=1e-7, rtol=1e-5,
                                    fast_mode=True)
    assert torch.autograd.gradcheck(lambda a, b: A.exchange_apply(ctx, a, b), (x, t), eps=1e-6, atol=1e-7,
                                    rtol=1e-5, fast_mode=True)

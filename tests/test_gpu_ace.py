"""ACE construction on the GPU (the "ACE implementation" section, Eqs. ace1 and eta) against the
FP64 oracle: M_ij = <psi_i, W_j>_w, the projection vectors xi and the ACE operator applied to a
block.  W comes from the library's exchange apply in the context's precision on the GPU side and
from the oracle on the oracle side, so the comparisons carry the apply's own error."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _helpers import W_TOL, _log, rel, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2401_04189_gb300 import build
    build.build()


def _cases():
    return {
        "small": lambda: W.config_small(),
        "full-rank": lambda: W.config_small(n=16, n_orb=3, rank=16, T=6, L=5.0, full_rank=True),
        "six": lambda: W.config_small(n=24, n_orb=6, rank=10, T=8, L=6.0, seed=5),
    }


@pytest.mark.parametrize("case", ["small", "full-rank", "six"])
@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16"])
def test_ace_matches_oracle(prec, case):
    import paper_2401_04189_gb300 as P
    s = _cases()[case]()
    S = O.Setup.from_system(s)
    W_or = O.exchange_apply(s.psi, S)
    xi_or, M_or = O.ace_projectors(s.psi, S, W=W_or)
    V_or = O.ace_apply(xi_or, s.psi, S)
    ctx = P.Context.from_system(s, precision=prec)
    psi = to_gpu(s.psi)
    xi, M = P.tx_ace_projectors(ctx, psi)            # W = K psi computed by the library
    V = P.tx_ace_apply(ctx, xi, psi)
    ctx.check_device_error()
    errs = dict(M=rel(M.cpu().numpy(), M_or), xi=rel(xi.cpu().numpy(), xi_or), V=rel(V.cpu().numpy(), V_or))
    _log(dict(what=f"ace-{case}", prec=prec, **{k: float(v) for k, v in errs.items()}, frob=errs["V"], elem=0.0))
    # M and V_ACE psi carry the apply's error; xi also the conditioning of the Cholesky factor
    assert errs["M"] < W_TOL[prec], errs
    assert errs["V"] < 2 * W_TOL[prec], errs
    assert errs["xi"] < 20 * W_TOL[prec], errs
    if case == "full-rank":
        # exact on the occupied orbitals at full rank: V_ACE psi_j = W_j
        assert rel(V.cpu().numpy(), W_or) < 2 * W_TOL[prec]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16"])
def test_ace_on_the_pt_shaped_block_reproduces_its_exchange_potentials(prec):
    """The Pt-shaped block (64 orbitals): with -M_s = L L^T (M_s the symmetric part of M),
    V_ACE psi_a = sum_i W_i (M_s^-1 M^T)_ia exactly, which equals W_a up to the asymmetry of M (the
    identities the oracle's pins hold at any size), checked with the GPU's own W and M."""
    import paper_2401_04189_gb300 as P
    s = W.config_pt()
    ctx = P.Context.from_system(s, precision=prec)
    psi = to_gpu(s.psi)
    Wg = P.tx_exchange_apply(ctx, psi)
    xi, M = P.tx_ace_projectors(ctx, psi, Wg)
    V = P.tx_ace_apply(ctx, xi, psi)
    ctx.check_device_error()
    Mh = M.cpu().numpy()
    asym = np.linalg.norm(Mh - Mh.T) / np.linalg.norm(Mh)
    err = rel(V.cpu().numpy(), Wg.cpu().numpy())
    _log(dict(what="ace-pt", prec=prec, asym=float(asym), frob=err, elem=0.0))
    Ms = 0.5 * (Mh + Mh.T)
    assert np.all(np.linalg.eigvalsh(Ms) < 0)                          # negative definite
    assert err < 2 * asym + 2 * W_TOL[prec], (err, asym)
    B = np.linalg.solve(Ms, Mh.T)
    Wh = Wg.cpu().numpy().astype(np.float64)
    exact = np.tensordot(B, Wh, axes=(0, 0))
    e2 = rel(V.cpu().numpy(), exact)
    _log(dict(what="ace-pt-identity", prec=prec, frob=e2, elem=0.0))
    assert e2 < 1e-5, e2                                               # float32 products of the two mixes


def test_ace_refuses_a_matrix_that_is_not_negative_definite():
    """W = +psi makes M the (positive) overlap matrix: the factorisation reports
    TX_ERR_NOT_DEFINITE instead of returning projectors."""
    import torch
    import paper_2401_04189_gb300 as P
    s = W.config_small(n=16, n_orb=3, rank=6, T=4, L=5.0)
    ctx = P.Context.from_system(s, precision="fp32")
    psi = to_gpu(s.psi)
    with pytest.raises(P.TuckerExchangeError) as ei:
        P.tx_ace_projectors(ctx, psi, psi.clone())
    assert ei.value.status == -11
    # the context still works
    xi, _ = P.tx_ace_projectors(ctx, psi)
    assert torch.isfinite(xi).all()

"""GPU parity of the transfer between an unstructured finite-element mesh and the structured
grid (Eq. interpolate) against the oracle: both directions, element orders 1 to 3, a mesh
refined near two atoms (hanging nodes), more orbitals than one 32-orbital pass, and the
refusals of meshes that do not fit the grid."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from _helpers import _log, to_gpu

pytestmark = pytest.mark.gpu

L = 4.0
N_GRID = (19, 22, 25)          # n - 1 = 18, 21, 24: whole elements of orders 1 and 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2401_04189_gb300 import build
    build.build()


def _context(n=N_GRID, half=L):
    import paper_2401_04189_gb300 as P
    rng = np.random.default_rng(7)
    xs, ws = zip(*[W.uniform_grid(k, half) for k in n])
    U = [np.linalg.qr(rng.standard_normal((k, 4)))[0] for k in n]
    h = min(float(np.min(np.diff(v))) for v in xs)
    theta, mu, _ = W.exp_sum_inverse_r(6, h, math.sqrt(3) * 2 * half)
    return P.Context(list(xs), list(ws), U, theta, mu, precision="fp32"), list(xs)


def _orbitals(n_orb, seed=3):
    rng = np.random.default_rng(seed)
    cen = rng.uniform(-2.0, 2.0, size=(n_orb, 2, 3))
    exps = rng.uniform(0.3, 1.5, size=(n_orb, 2))
    coefs = rng.standard_normal(size=(n_orb, 2))
    return cen, exps, coefs


def _elem(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("order_u", [1, 2, 3])
def test_mesh_to_grid_matches_oracle(order_u):
    import torch
    import paper_2401_04189_gb300 as P
    ctx, xs = _context()
    X, conn = W.fe_mesh(L, 3, [[0.0, 0.0, 0.0], [1.5, -1.0, 0.5]], 2.0, order_u)
    cen, exps, coefs = _orbitals(37)
    psi_u = W.gaussian_sum_at_points(X, cen, exps, coefs).T.astype(np.float32)      # [n_nodes, 37]
    tr = P.Transfer(ctx, X, conn, order_u, 3)
    got = tr.u_to_s(torch.from_numpy(np.ascontiguousarray(psi_u)).cuda()).cpu().numpy()
    ref = O.transfer_u_to_s(psi_u.astype(np.float64), X, conn, order_u, xs)
    err = _elem(got, ref)
    _log(dict(what=f"transfer-u2s-p{order_u}", prec="fp32", frob=err, elem=err))
    assert err < 1e-6
    assert tr.map_bytes() > 0
    tr.destroy()


@pytest.mark.parametrize("order_s", [1, 3])
def test_grid_to_mesh_matches_oracle(order_s):
    import torch
    import paper_2401_04189_gb300 as P
    ctx, xs = _context()
    X, conn = W.fe_mesh(L, 3, [[0.0, 0.0, 0.0], [1.5, -1.0, 0.5]], 2.0, 2)
    cen, exps, coefs = _orbitals(37, seed=4)
    psi_s = W.gaussian_sum_orbitals(xs, cen, exps, coefs).astype(np.float32)
    tr = P.Transfer(ctx, X, conn, 2, order_s)
    got = tr.s_to_u(to_gpu(psi_s)).cpu().numpy()
    ref = O.transfer_s_to_u(psi_s.astype(np.float64), xs, order_s, X)
    err = _elem(got, ref)
    _log(dict(what=f"transfer-s2u-p{order_s}", prec="fp32", frob=err, elem=err))
    assert err < 1e-6
    tr.destroy()


def test_meshes_that_do_not_fit_the_grid_are_refused():
    import paper_2401_04189_gb300 as P
    X, conn = W.fe_mesh(L, 2, np.zeros((1, 3)), 0.0, 1, levels=0)
    ctx, _ = _context(half=5.0)                     # the grid reaches past the mesh
    with pytest.raises(P.TuckerExchangeError) as ei:
        P.Transfer(ctx, X, conn, 1, 3)
    assert ei.value.status == -2
    ctx2, _ = _context()
    for order_u, order_s, status in ((1, 2, -2), (4, 1, -1), (1, 0, -1)):   # 21 rows: no order-2 elements
        with pytest.raises((P.TuckerExchangeError, ValueError)) as ei:
            P.Transfer(ctx2, X, conn if order_u == 1 else np.zeros((1, (order_u + 1) ** 3), np.int32), order_u, order_s)
        if isinstance(ei.value, P.TuckerExchangeError):
            assert ei.value.status == status
    bad = conn.copy()
    bad[0, 0] = X.shape[0]
    with pytest.raises(P.TuckerExchangeError) as ei:
        P.Transfer(ctx2, X, bad, 1, 1)
    assert ei.value.status == -1

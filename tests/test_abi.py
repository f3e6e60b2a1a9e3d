"""The C ABI without a GPU: the library loads, exports every symbol include/tuxc.h declares,
and host-side validation rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2401_04189_gb300 as P
from paper_2401_04189_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names.update(re.findall(r"\b(tx_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_2401_04189_gb300 import build
    build.build()
    return P.lib()


def test_every_declared_symbol_is_exported(L):
    declared = _declared_symbols()
    assert len(declared) >= 14
    missing = [n for n in declared if not hasattr(L, n)]
    assert not missing, missing
    assert set(P.EXPORTED) <= set(declared)


def test_status_strings(L):
    for code, name in _lib.STATUS.items():
        assert L.tx_status_string(code).decode() == name


def _setup_args(n=(6, 7, 8), r=(2, 3, 4), T=3, seed=0):
    rng = np.random.default_rng(seed)
    xs = [np.linspace(-1, 1, k) for k in n]
    ws = [np.full(k, 2.0 / (k - 1)) for k in n]
    Us = [np.linalg.qr(rng.standard_normal((k, q)))[0] for k, q in zip(n, r)]
    th = np.linspace(0.5, 2.0, T)
    mu = np.full(T, 0.3)
    return xs, ws, Us, th, mu


def _call_setup(L, xs, ws, Us, th, mu, n=None, r=None, T=None, prec=0):
    n = n or [len(v) for v in xs]
    r = r or [u.shape[1] for u in Us]
    T = len(th) if T is None else T
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (*xs, *ws, *Us, th, mu)]
    pp = [a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
    h = ctypes.c_void_p()
    st = L.tx_tucker_setup(ctypes.byref(h), (ctypes.c_int * 3)(*n), *pp[0:3], *pp[3:6], (ctypes.c_int * 3)(*r),
                           *pp[6:9], T, pp[9], pp[10], prec, ctypes.c_void_p(0))
    return st, h


@pytest.mark.parametrize("case,expect", [
    ("not_orthonormal", -3), ("rank_too_big", -2), ("negative_weight", -1), ("zero_theta", -1),
    ("nan_mu", -1), ("bad_precision", -4), ("zero_T", -1),
])
def test_setup_validation_rejects_bad_arguments(L, case, expect):
    xs, ws, Us, th, mu = _setup_args()
    n = r = T = None
    prec = 0
    if case == "not_orthonormal":
        Us[1] = Us[1] * 1.001
    elif case == "rank_too_big":
        r = [2, 3, 9]
        Us[2] = np.zeros((8, 9))
    elif case == "negative_weight":
        ws[0] = ws[0].copy()
        ws[0][2] = -1.0
    elif case == "zero_theta":
        th = th.copy()
        th[1] = 0.0
    elif case == "nan_mu":
        mu = mu.copy()
        mu[0] = np.nan
    elif case == "bad_precision":
        prec = 17
    elif case == "zero_T":
        T = 0
    st, h = _call_setup(L, xs, ws, Us, th, mu, n=n, r=r, T=T, prec=prec)
    assert st == expect, L.tx_last_error_message()
    assert not h.value
    assert len(L.tx_last_error_message()) > 0


def test_calls_on_null_context_are_rejected(L):
    assert L.tx_exchange_apply(None, None, 1, None, 1, None, None) == -8
    assert L.tx_exchange_energy(None, None, 1, None, None) == -8
    assert L.tx_set_precision(None, 0, None) == -8
    L.tx_destroy(None)                     # no-op
    assert L.tx_workspace_bytes(None) == 0


def test_new_entry_points_reject_a_null_context(L):
    """The ACE, energy-share, quadrature, wait-limit and wait self-test entry points validate their context on
    the host before anything else (no device is touched)."""
    P_ = ctypes.c_void_p
    assert L.tx_ace_projectors(None, P_(0), 1, P_(0), P_(0), P_(0), P_(0)) == -8
    assert L.tx_ace_apply(None, P_(0), 1, P_(0), 1, P_(0), P_(0)) == -8
    assert L.tx_exchange_energy_from_w(None, P_(0), P_(0), 1, P_(0), P_(0)) == -8
    assert L.tx_set_wait_limit(None, 0) == -8
    assert L.tx_selftest_wait(None, 1, P_(0)) == -8
    assert L.tx_set_quadrature(None, 1, 3, P_(0)) == -8
    assert L.tx_exchange_apply_galerkin(None, P_(0), 1, P_(0), 1, P_(0), P_(0)) == -8
    assert L.tx_exchange_energy_galerkin(None, P_(0), 1, P_(0), P_(0)) == -8
    h = P_()
    assert L.tx_transfer_create(ctypes.byref(h), None, 1, P_(0), 1, P_(0), 1, 1) == -8
    assert L.tx_transfer_u_to_s(None, P_(0), 1, P_(0), P_(0)) == -8
    assert L.tx_transfer_s_to_u(None, P_(0), 1, P_(0), P_(0)) == -8
    assert L.tx_transfer_map_bytes(None) == 0
    L.tx_transfer_destroy(None)
    assert L.tx_exchange_apply_sthosvd(None, P_(0), 1, P_(0), 1, P_(0), P_(0)) == -8
    assert L.tx_status_string(-11).decode() == "TX_ERR_NOT_DEFINITE"

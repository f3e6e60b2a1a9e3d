"""ctypes binding of libtuxc.so: argument marshalling only.  Every step of the hot path runs
in the library's CUDA kernels; if the library is missing this module raises instead of
falling back to anything else."""
from __future__ import annotations

import ctypes
import enum
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtuxc.so")

TX_OK = 0
STATUS = {
    0: "TX_OK", -1: "TX_ERR_INVALID_ARG", -2: "TX_ERR_SHAPE", -3: "TX_ERR_NOT_ORTHONORMAL",
    -4: "TX_ERR_UNSUPPORTED_PRECISION", -5: "TX_ERR_CUDA", -6: "TX_ERR_OOM", -7: "TX_ERR_TIMEOUT",
    -8: "TX_ERR_NOT_SETUP", -9: "TX_ERR_UNSUPPORTED_SHAPE", -10: "TX_ERR_ALIGNMENT", -11: "TX_ERR_NOT_DEFINITE",
}
EXPORTED = [
    "tx_tucker_setup", "tx_destroy", "tx_set_precision", "tx_exchange_apply", "tx_exchange_energy",
    "tx_exchange_energy_grad", "tx_exchange_apply_vjp", "tx_workspace_bytes", "tx_set_workspace_limit",
    "tx_check_device_error", "tx_status_string", "tx_last_error_message", "tx_launch_count",
    "tx_reset_launch_count", "tx_exchange_apply_energy", "tx_profile_enable", "tx_profile_reset",
    "tx_profile_read", "tx_selftest_gemm", "tx_batch_plan", "tx_batch_launch", "tx_batch_capture",
    "tx_batch_replay", "tx_batch_item_plan", "tx_plan_destroy", "tx_set_tile_plan", "tx_set_accumulation_chunk", "tx_set_expansion_form",
    "tx_exchange_apply_static", "tx_describe_expansion_plan", "tx_set_wait_limit", "tx_selftest_wait",
    "tx_exchange_energy_from_w", "tx_ace_projectors", "tx_ace_apply", "tx_set_quadrature",
    "tx_exchange_apply_galerkin", "tx_exchange_energy_galerkin", "tx_transfer_create", "tx_transfer_u_to_s",
    "tx_transfer_s_to_u", "tx_transfer_map_bytes", "tx_transfer_destroy", "tx_exchange_apply_sthosvd",
]


class _BatchItem(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("psi_occ", ctypes.c_void_p), ("n_occ", ctypes.c_int),
                ("psi_tgt", ctypes.c_void_p), ("n_tgt", ctypes.c_int), ("out", ctypes.c_void_p),
                ("e_dev", ctypes.c_void_p)]


class Precision(enum.IntEnum):
    FP32 = 0
    BF16 = 1
    TF32 = 2
    TF32X3 = 3
    BF16X3 = 4

    @classmethod
    def parse(cls, p):
        if isinstance(p, str):
            return cls[p.upper()]
        return cls(int(p))


class TuckerExchangeError(RuntimeError):
    def __init__(self, status, where, message):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; call paper_2401_04189_gb300.build.build() first")
    L = ctypes.CDLL(LIB_PATH)
    L.tx_tucker_setup.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(_I), _P, _P, _P, _P, _P, _P,
                                  ctypes.POINTER(_I), _P, _P, _P, _I, _P, _P, _I, _P]
    L.tx_tucker_setup.restype = _I
    L.tx_destroy.argtypes = [_P]
    L.tx_destroy.restype = None
    L.tx_set_precision.argtypes = [_P, _I, _P]
    L.tx_set_precision.restype = _I
    L.tx_exchange_apply.argtypes = [_P, _P, _I, _P, _I, _P, _P]
    L.tx_exchange_apply.restype = _I
    L.tx_exchange_apply_galerkin.argtypes = [_P, _P, _I, _P, _I, _P, _P]
    L.tx_exchange_apply_galerkin.restype = _I
    L.tx_exchange_apply_sthosvd.argtypes = [_P, _P, _I, _P, _I, _P, _P]
    L.tx_exchange_apply_sthosvd.restype = _I
    L.tx_exchange_energy_galerkin.argtypes = [_P, _P, _I, _P, _P]
    L.tx_exchange_energy_galerkin.restype = _I
    L.tx_transfer_create.argtypes = [ctypes.POINTER(_P), _P, _I, _P, _I, _P, _I, _I]
    L.tx_transfer_create.restype = _I
    L.tx_transfer_u_to_s.argtypes = [_P, _P, _I, _P, _P]
    L.tx_transfer_u_to_s.restype = _I
    L.tx_transfer_s_to_u.argtypes = [_P, _P, _I, _P, _P]
    L.tx_transfer_s_to_u.restype = _I
    L.tx_transfer_map_bytes.argtypes = [_P]
    L.tx_transfer_map_bytes.restype = ctypes.c_long
    L.tx_transfer_destroy.argtypes = [_P]
    L.tx_transfer_destroy.restype = None
    L.tx_exchange_apply_energy.argtypes = [_P, _P, _I, _P, _P, _P]
    L.tx_exchange_apply_energy.restype = _I
    L.tx_profile_enable.argtypes = [_I]
    L.tx_profile_enable.restype = None
    L.tx_profile_reset.argtypes = []
    L.tx_profile_reset.restype = None
    L.tx_profile_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]
    L.tx_profile_read.restype = _I
    L.tx_batch_plan.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(_BatchItem), _I, ctypes.c_char_p, _I, _P]
    L.tx_batch_plan.restype = _I
    for name in ("tx_batch_launch", "tx_batch_capture", "tx_batch_replay"):
        getattr(L, name).argtypes = [_P, _P]
        getattr(L, name).restype = _I
    L.tx_batch_item_plan.argtypes = [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]
    L.tx_batch_item_plan.restype = _I
    L.tx_plan_destroy.argtypes = [_P]
    L.tx_plan_destroy.restype = None
    L.tx_exchange_apply_static.argtypes = [_P, _P, _I, _P, _P]
    L.tx_exchange_apply_static.restype = _I
    L.tx_set_tile_plan.argtypes = [_P, _I, _I]
    L.tx_set_tile_plan.restype = _I
    L.tx_set_accumulation_chunk.argtypes = [_P, _I]
    L.tx_set_accumulation_chunk.restype = _I
    L.tx_describe_expansion_plan.argtypes = [ctypes.POINTER(_I), ctypes.POINTER(_I), _I, _I, _I, ctypes.POINTER(_I), _I]
    L.tx_describe_expansion_plan.restype = _I
    L.tx_set_expansion_form.argtypes = [_P, _I]
    L.tx_set_expansion_form.restype = _I
    L.tx_selftest_gemm.argtypes = [_I, _I, _I, _I, _I, _P, _P, _P, _P]
    L.tx_selftest_gemm.restype = _I
    L.tx_exchange_energy.argtypes = [_P, _P, _I, _P, _P]
    L.tx_exchange_energy.restype = _I
    L.tx_exchange_energy_grad.argtypes = [_P, _P, _I, _P, _P, _P]
    L.tx_exchange_energy_grad.restype = _I
    L.tx_exchange_apply_vjp.argtypes = [_P, _P, _I, _P, _I, _P, _P, _P, _P]
    L.tx_exchange_apply_vjp.restype = _I
    L.tx_workspace_bytes.argtypes = [_P]
    L.tx_workspace_bytes.restype = ctypes.c_size_t
    L.tx_set_workspace_limit.argtypes = [_P, ctypes.c_size_t]
    L.tx_set_workspace_limit.restype = _I
    L.tx_check_device_error.argtypes = [_P]
    L.tx_check_device_error.restype = _I
    L.tx_set_wait_limit.argtypes = [_P, ctypes.c_uint64]
    L.tx_set_wait_limit.restype = _I
    L.tx_selftest_wait.argtypes = [_P, _I, _P]
    L.tx_selftest_wait.restype = _I
    L.tx_exchange_energy_from_w.argtypes = [_P, _P, _P, _I, _P, _P]
    L.tx_exchange_energy_from_w.restype = _I
    L.tx_ace_projectors.argtypes = [_P, _P, _I, _P, _P, _P, _P]
    L.tx_ace_projectors.restype = _I
    L.tx_ace_apply.argtypes = [_P, _P, _I, _P, _I, _P, _P]
    L.tx_ace_apply.restype = _I
    L.tx_set_quadrature.argtypes = [_P, _I, _I, _P]
    L.tx_set_quadrature.restype = _I
    L.tx_status_string.argtypes = [_I]
    L.tx_status_string.restype = ctypes.c_char_p
    L.tx_last_error_message.argtypes = []
    L.tx_last_error_message.restype = ctypes.c_char_p
    L.tx_launch_count.argtypes = []
    L.tx_launch_count.restype = ctypes.c_uint64
    L.tx_reset_launch_count.argtypes = []
    L.tx_reset_launch_count.restype = None
    _lib = L
    return L


def _check(status, where):
    if status != TX_OK:
        msg = lib().tx_last_error_message().decode(errors="replace")
        raise TuckerExchangeError(status, where, msg)


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Context:
    """Owns one tx_ctx: grid, weights, basis, Gaussian sum, operand copies, workspace."""

    def __init__(self, x, w, U, theta, mu, precision="fp32", stream=None):
        L = lib()
        self._host = [_f64(v) for v in (*x, *w, *U, theta, mu)]
        xs, ws, Us = self._host[0:3], self._host[3:6], self._host[6:9]
        th, m = self._host[9], self._host[10]
        self.n = tuple(int(v.shape[0]) for v in xs)
        self.r = tuple(int(u.shape[1]) for u in Us)
        self.T = int(th.shape[0])
        for d in range(3):
            if Us[d].shape != (self.n[d], self.r[d]) or ws[d].shape != (self.n[d],):
                raise ValueError(f"mode {d + 1}: inconsistent x / w / U shapes")
        if m.shape != th.shape:
            raise ValueError("theta and mu must have the same length")
        self.precision = Precision.parse(precision)
        n_arr = (_I * 3)(*self.n)
        r_arr = (_I * 3)(*self.r)
        h = _P()
        pp = [v.ctypes.data_as(_P) for v in self._host]
        st = L.tx_tucker_setup(ctypes.byref(h), n_arr, *pp[0:3], *pp[3:6], r_arr, *pp[6:9], self.T, pp[9], pp[10],
                               int(self.precision), _stream(stream))
        _check(st, "tx_tucker_setup")
        self._h = h

    @classmethod
    def from_system(cls, s, precision="fp32", stream=None):
        return cls(s.x, s.w, s.U, s.theta, s.mu, precision=precision, stream=stream)

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise RuntimeError("context was destroyed")
        return self._h

    def set_precision(self, precision, stream=None):
        p = Precision.parse(precision)
        _check(lib().tx_set_precision(self.handle, int(p), _stream(stream)), "tx_set_precision")
        self.precision = p

    def set_quadrature(self, order, points=0, stream=None):
        """1-D convolution integrals: order 0 = nodal quadrature (default); order p >= 1 =
        Lagrange elements of order p with `points` Gauss-Legendre points per element."""
        _check(lib().tx_set_quadrature(self.handle, int(order), int(points), _stream(stream)), "tx_set_quadrature")

    def set_workspace_limit(self, nbytes):
        _check(lib().tx_set_workspace_limit(self.handle, int(nbytes)), "tx_set_workspace_limit")

    def workspace_bytes(self):
        return int(lib().tx_workspace_bytes(self.handle))

    def check_device_error(self):
        _check(lib().tx_check_device_error(self.handle), "tx_check_device_error")

    def set_wait_limit(self, ns):
        """Time limit (ns) of the kernels' bounded device waits; 0 restores the default (2 s)."""
        _check(lib().tx_set_wait_limit(self.handle, int(ns)), "tx_set_wait_limit")

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tx_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # ---- checks -------------------------------------------------------------------
    def _block(self, t, name):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
            raise TypeError(f"{name} must be a float32 CUDA tensor")
        if t.dim() != 4 or tuple(t.shape[1:]) != self.n:
            raise ValueError(f"{name} must have shape [count, {self.n[0]}, {self.n[1]}, {self.n[2]}]")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t


def tx_tucker_setup(x, w, U, theta, mu, precision="fp32", stream=None) -> Context:
    return Context(x, w, U, theta, mu, precision=precision, stream=stream)


def tx_exchange_apply(ctx: Context, psi_occ, psi_tgt=None, out=None, stream=None, _fn="tx_exchange_apply"):
    """out = K psi_tgt (psi_tgt None: the occupied block itself)."""
    ctx._block(psi_occ, "psi_occ")
    n_tgt = psi_occ.shape[0] if psi_tgt is None else ctx._block(psi_tgt, "psi_tgt").shape[0]
    if out is None:
        out = torch.empty((n_tgt, *ctx.n), dtype=torch.float32, device=psi_occ.device)
    ctx._block(out, "out")
    if n_tgt == 0:
        return out          # no targets (an empty tensor has a NULL pointer, which the C call reads as "occupied")
    st = getattr(lib(), _fn)(ctx.handle, _ptr(psi_occ), psi_occ.shape[0], _ptr(psi_tgt),
                             0 if psi_tgt is None else n_tgt, _ptr(out), _stream(stream))
    _check(st, _fn)
    return out


def tx_exchange_apply_sthosvd(ctx: Context, psi_occ, psi_tgt=None, out=None, stream=None):
    """out = K psi_tgt with per-pair Tucker bases from a sequentially truncated HOSVD of every
    pair density (ranks = the context's ranks)."""
    return tx_exchange_apply(ctx, psi_occ, psi_tgt, out, stream, _fn="tx_exchange_apply_sthosvd")


def tx_exchange_apply_galerkin(ctx: Context, psi_occ, psi_tgt=None, out=None, stream=None):
    """out = K_G psi_tgt with the convolution projected onto the Tucker basis on both sides
    (P^* C P, P^* the weighted adjoint of the projector): an exactly symmetric, negative
    semi-definite exchange matrix at any rank."""
    return tx_exchange_apply(ctx, psi_occ, psi_tgt, out, stream, _fn="tx_exchange_apply_galerkin")


def tx_exchange_apply_energy(ctx: Context, psi_occ, out=None, e_out=None, stream=None):
    """(K psi_occ, E_x) in one pass."""
    ctx._block(psi_occ, "psi_occ")
    if out is None:
        out = torch.empty_like(psi_occ)
    ctx._block(out, "out")
    if e_out is None:
        e_out = torch.empty((), dtype=torch.float64, device=psi_occ.device)
    st = lib().tx_exchange_apply_energy(ctx.handle, _ptr(psi_occ), psi_occ.shape[0], _ptr(out), _ptr(e_out),
                                        _stream(stream))
    _check(st, "tx_exchange_apply_energy")
    return out, e_out


def tx_exchange_energy_from_w(ctx: Context, psi, W, e_out=None, stream=None):
    """1/2 sum_i sum_x w(x) psi_i(x) W_i(x) as a float64 device scalar."""
    ctx._block(psi, "psi")
    ctx._block(W, "W")
    if W.shape[0] != psi.shape[0]:
        raise ValueError("psi and W must hold the same number of orbitals")
    if e_out is None:
        e_out = torch.empty((), dtype=torch.float64, device=psi.device)
    st = lib().tx_exchange_energy_from_w(ctx.handle, _ptr(psi), _ptr(W), psi.shape[0], _ptr(e_out), _stream(stream))
    _check(st, "tx_exchange_energy_from_w")
    return e_out


def tx_ace_projectors(ctx: Context, psi_occ, W=None, stream=None):
    """(xi, M): the ACE projection vectors and M_ij = <psi_i, W_j>_w (float64 device tensor).
    W = K psi_occ is computed with the context's precision when not given."""
    ctx._block(psi_occ, "psi_occ")
    if W is None:
        W = tx_exchange_apply(ctx, psi_occ, stream=stream)
    ctx._block(W, "W")
    if W.shape[0] != psi_occ.shape[0]:
        raise ValueError("psi_occ and W must hold the same number of orbitals")
    xi = torch.empty_like(psi_occ)
    M = torch.empty((psi_occ.shape[0], psi_occ.shape[0]), dtype=torch.float64, device=psi_occ.device)
    st = lib().tx_ace_projectors(ctx.handle, _ptr(psi_occ), psi_occ.shape[0], _ptr(W), _ptr(xi), _ptr(M),
                                 _stream(stream))
    _check(st, "tx_ace_projectors")
    return xi, M


def tx_ace_apply(ctx: Context, xi, psi, out=None, stream=None):
    """V_ACE psi = - sum_k xi_k <xi_k, psi>_w for every orbital of the block psi."""
    ctx._block(xi, "xi")
    ctx._block(psi, "psi")
    if out is None:
        out = torch.empty_like(psi)
    ctx._block(out, "out")
    st = lib().tx_ace_apply(ctx.handle, _ptr(xi), xi.shape[0], _ptr(psi), psi.shape[0], _ptr(out), _stream(stream))
    _check(st, "tx_ace_apply")
    return out


def tx_selftest_wait(ctx: Context, hold_tmem=True, stream=None):
    """Launches the bounded-wait self-test (a wait nothing completes); see include/tuxc.h."""
    _check(lib().tx_selftest_wait(ctx.handle, 1 if hold_tmem else 0, _stream(stream)), "tx_selftest_wait")


def tx_profile_enable(enable=True):
    lib().tx_profile_enable(1 if enable else 0)


def tx_profile_reset():
    lib().tx_profile_reset()


def tx_profile_read(name):
    """(launches, total device ms) of one kernel class since the last reset."""
    n = _I()
    ms = ctypes.c_double()
    _check(lib().tx_profile_read(name.encode(), ctypes.byref(n), ctypes.byref(ms)), "tx_profile_read")
    return int(n.value), float(ms.value)


def tx_exchange_energy(ctx: Context, psi_occ, e_out=None, stream=None, _fn="tx_exchange_energy"):
    """E_x as a float64 device scalar."""
    ctx._block(psi_occ, "psi_occ")
    if e_out is None:
        e_out = torch.empty((), dtype=torch.float64, device=psi_occ.device)
    st = getattr(lib(), _fn)(ctx.handle, _ptr(psi_occ), psi_occ.shape[0], _ptr(e_out), _stream(stream))
    _check(st, _fn)
    return e_out


def tx_exchange_energy_galerkin(ctx: Context, psi_occ, e_out=None, stream=None):
    """E_x with the two-sided projection, evaluated in core space (O(T r^4) per pair)."""
    return tx_exchange_energy(ctx, psi_occ, e_out, stream, _fn="tx_exchange_energy_galerkin")


def tx_exchange_energy_grad(ctx: Context, psi_occ, grad=None, e_out=None, stream=None):
    """(E_x, dE_x/dpsi)."""
    ctx._block(psi_occ, "psi_occ")
    if grad is None:
        grad = torch.empty_like(psi_occ)
    if e_out is None:
        e_out = torch.empty((), dtype=torch.float64, device=psi_occ.device)
    st = lib().tx_exchange_energy_grad(ctx.handle, _ptr(psi_occ), psi_occ.shape[0], _ptr(grad), _ptr(e_out),
                                       _stream(stream))
    _check(st, "tx_exchange_energy_grad")
    return e_out, grad


def tx_exchange_apply_vjp(ctx: Context, psi_occ, psi_tgt, grad_out, need_occ=True, need_tgt=True, stream=None):
    """(grad_occ, grad_tgt) of sum(grad_out * K psi_tgt)."""
    ctx._block(psi_occ, "psi_occ")
    ctx._block(psi_tgt, "psi_tgt")
    ctx._block(grad_out, "grad_out")
    g_occ = torch.empty_like(psi_occ) if need_occ else None
    g_tgt = torch.empty_like(psi_tgt) if need_tgt else None
    st = lib().tx_exchange_apply_vjp(ctx.handle, _ptr(psi_occ), psi_occ.shape[0], _ptr(psi_tgt), psi_tgt.shape[0],
                                     _ptr(grad_out), _ptr(g_occ), _ptr(g_tgt), _stream(stream))
    _check(st, "tx_exchange_apply_vjp")
    return g_occ, g_tgt


def tx_selftest_gemm(precision, A, B, stream=None):
    """D[b] = A[b] @ B[b]^T on the tensor cores (A [batch][M][K], B [batch][N][K] float32 CUDA)."""
    batch, M, K = A.shape
    N = B.shape[1]
    D = torch.empty((batch, M, N), dtype=torch.float32, device=A.device)
    st = lib().tx_selftest_gemm(int(Precision.parse(precision)), batch, M, N, K, _ptr(A.contiguous()),
                                _ptr(B.contiguous()), _ptr(D), _stream(stream))
    _check(st, "tx_selftest_gemm")
    return D


class BatchPlan:
    """tx_batch_plan over a list of items: dict(ctx=Context, psi_occ=tensor, psi_tgt=None|tensor,
    out=None|tensor, energy=False).  Outputs (and energies) are allocated here when absent."""

    def __init__(self, items, tune_table=None, autotune=False, stream=None):
        self.items = []
        arr = (_BatchItem * len(items))()
        for k, it in enumerate(items):
            ctx = it["ctx"]
            occ = ctx._block(it["psi_occ"], "psi_occ")
            tgt = it.get("psi_tgt")
            if tgt is not None:
                ctx._block(tgt, "psi_tgt")
            n_tgt = occ.shape[0] if tgt is None else tgt.shape[0]
            out = it.get("out")
            if out is None:
                out = torch.empty((n_tgt, *ctx.n), dtype=torch.float32, device=occ.device)
            e = torch.empty((), dtype=torch.float64, device=occ.device) if it.get("energy") else None
            self.items.append(dict(ctx=ctx, psi_occ=occ, psi_tgt=tgt, out=out, e=e))
            arr[k] = _BatchItem(ctx.handle.value, occ.data_ptr(), occ.shape[0], 0 if tgt is None else tgt.data_ptr(),
                                0 if tgt is None else n_tgt, out.data_ptr(), 0 if e is None else e.data_ptr())
        self._arr = arr
        h = _P()
        st = lib().tx_batch_plan(ctypes.byref(h), arr, len(items),
                                 None if tune_table is None else str(tune_table).encode(), 1 if autotune else 0,
                                 _stream(stream))
        _check(st, "tx_batch_plan")
        self._h = h

    def launch(self, stream=None):
        _check(lib().tx_batch_launch(self._h, _stream(stream)), "tx_batch_launch")

    def capture(self, stream):
        _check(lib().tx_batch_capture(self._h, _stream(stream)), "tx_batch_capture")

    def replay(self, stream=None):
        _check(lib().tx_batch_replay(self._h, _stream(stream)), "tx_batch_replay")

    def item_plan(self, i):
        bx, ns = _I(), _I()
        st = lib().tx_batch_item_plan(self._h, i, ctypes.byref(bx), ctypes.byref(ns))
        if st < 0:
            _check(st, "tx_batch_item_plan")
        return bx.value, ns.value

    def outputs(self):
        return [it["out"] for it in self.items]

    def energies(self):
        return [it["e"] for it in self.items]

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tx_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def tx_set_tile_plan(ctx, bx, nstage):
    _check(lib().tx_set_tile_plan(ctx.handle, int(bx), int(nstage)), "tx_set_tile_plan")


def tx_set_accumulation_chunk(ctx, terms):
    """Split precisions: Gaussian terms per tensor-core accumulation chunk of phi (0 = default)."""
    _check(lib().tx_set_accumulation_chunk(ctx.handle, int(terms)), "tx_set_accumulation_chunk")


def tx_set_expansion_form(ctx, form):
    """Single-pass precisions: 0 = automatic (persistent expansion kernel where it applies, short
    last y tiles of several planes packed into one item; default), 1 = one CTA per item,
    2 = persistent with stage 3 in bf16 (bf16 only), 3 = automatic without the packing,
    4 = persistent with Y rounded to bf16 in TMEM so that stage 3 runs in bf16 (bf16 only),
    5 = persistent with two stage-2 and two stage-3 MMA issuing warps (bf16 only)."""
    _check(lib().tx_set_expansion_form(ctx.handle, int(form)), "tx_set_expansion_form")


PLAN_FIELDS = ("kernel", "planes", "stages2", "stages3", "ybuffers", "tmem_cols", "smem_bytes", "threads",
               "ksteps2", "ksteps3", "n3p", "items_per_pair", "tail_planes", "z_parts")
PLAN_KERNELS = {0: "float32", 1: "converter", 2: "per_item", 3: "persistent", 4: "persistent_bf16",
                5: "persistent_bf16_tmem", 6: "persistent_dual_issue"}


def tx_describe_expansion_plan(n, r, T, precision, form=0):
    """The expansion kernel and tile plan a context of this shape would launch (host only, no
    device needed): a dict over PLAN_FIELDS, with "kernel" named as in PLAN_KERNELS."""
    out = (_I * len(PLAN_FIELDS))()
    st = lib().tx_describe_expansion_plan((_I * 3)(*[int(v) for v in n]), (_I * 3)(*[int(v) for v in r]), int(T),
                                          int(Precision.parse(precision)), int(form), out, len(PLAN_FIELDS))
    _check(st, "tx_describe_expansion_plan")
    d = dict(zip(PLAN_FIELDS, (int(v) for v in out)))
    d["kernel"] = PLAN_KERNELS[d["kernel"]]
    return d


def tx_launch_count() -> int:
    return int(lib().tx_launch_count())


def tx_reset_launch_count():
    lib().tx_reset_launch_count()


class Transfer:
    """Transfer of orbitals between an unstructured finite-element mesh (nodes X [n_nodes, 3],
    cells conn [n_cells, (order_u + 1)^3]) and the structured grid of a context, whose elements
    have order `order_s` (Eq. interpolate).  Orbitals on the mesh are [n_nodes, n_orb] (orbital
    index fastest); on the grid [n_orb, n1, n2, n3]."""

    def __init__(self, ctx: "Context", X, conn, order_u, order_s):
        X = np.ascontiguousarray(X, dtype=np.float64)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        if X.ndim != 2 or X.shape[1] != 3 or conn.ndim != 2 or conn.shape[1] != (int(order_u) + 1) ** 3:
            raise ValueError("X must be [n_nodes, 3] and conn [n_cells, (order_u + 1)^3]")
        self.ctx = ctx
        self.n_nodes = X.shape[0]
        h = _P()
        _check(lib().tx_transfer_create(ctypes.byref(h), ctx.handle, int(order_s), X.ctypes.data, X.shape[0],
                                        conn.ctypes.data, conn.shape[0], int(order_u)), "tx_transfer_create")
        self.handle = h

    def map_bytes(self) -> int:
        return int(lib().tx_transfer_map_bytes(self.handle))

    def u_to_s(self, psi_u, out=None, stream=None):
        if psi_u.dtype != torch.float32 or not psi_u.is_contiguous() or psi_u.dim() != 2 or psi_u.shape[0] != self.n_nodes:
            raise ValueError("psi_u must be contiguous float32 [n_nodes, n_orb]")
        n_orb = psi_u.shape[1]
        if out is None:
            out = torch.empty((n_orb, *self.ctx.n), dtype=torch.float32, device=psi_u.device)
        self.ctx._block(out, "psi_s")
        _check(lib().tx_transfer_u_to_s(self.handle, _ptr(psi_u), n_orb, _ptr(out), _stream(stream)), "tx_transfer_u_to_s")
        return out

    def s_to_u(self, psi_s, out=None, stream=None):
        self.ctx._block(psi_s, "psi_s")
        n_orb = psi_s.shape[0]
        if out is None:
            out = torch.empty((self.n_nodes, n_orb), dtype=torch.float32, device=psi_s.device)
        if out.dtype != torch.float32 or not out.is_contiguous() or tuple(out.shape) != (self.n_nodes, n_orb):
            raise ValueError("out must be contiguous float32 [n_nodes, n_orb]")
        _check(lib().tx_transfer_s_to_u(self.handle, _ptr(psi_s), n_orb, _ptr(out), _stream(stream)), "tx_transfer_s_to_u")
        return out

    def destroy(self):
        if getattr(self, "handle", None):
            lib().tx_transfer_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

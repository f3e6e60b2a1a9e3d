"""Shared helpers for the GPU parity tests (the oracle is the reference everywhere)."""
import json
import os

import numpy as np

import oracle as O

# Relative Frobenius tolerances of W (and relative tolerances of E_x) against the FP64 oracle,
# per GEMM arithmetic.  bf16 keeps 8 significant bits (unit roundoff 2^-9) and the chain rounds
# its operands about five times; tf32 keeps 11 (2^-12 per rounding after round-to-nearest).
# The split (3-pass) forms carry ~22 (tf32) or ~16 (bf16) bits per tensor-core operand; their
# projection onto the core and first expansion mode run in float32, the cross products of every
# tensor-core product accumulate separately, and the final contraction is folded into a float32
# register accumulator after every Gaussian term, so the tensor core's truncating float32
# accumulator never sums more than one term.  Measured worst cases: tf32x3 5.9e-7 (TiO2-shaped
# rows, 45 terms), bf16x3 4.6e-6.  The tf32x3 bound is the 1e-6 target of the split form.
W_TOL = {"fp32": 2e-6, "tf32x3": 1e-6, "bf16x3": 1e-5, "tf32": 5e-3, "bf16": 2e-2}
E_TOL = {"fp32": 1e-6, "tf32x3": 1e-6, "bf16x3": 1e-5, "tf32": 5e-3, "bf16": 1e-2}


# Elementwise bound: max |W_gpu - W_ref| / max |W_ref| over the compared block, per GEMM
# arithmetic.  The largest errors sit where |W| is largest, so this is of the order of the
# Frobenius error; the bound catches a wrong ragged tile or a dropped slab that carries little
# of the norm, which the Frobenius check alone would let through.
# Measured worst cases over the parity suite (GB300): fp32 1.4e-6 (TiO2-shaped rows), bf16
# 7.7e-3, tf32 2.0e-3, tf32x3 7.7e-7 (TiO2-shaped rows), bf16x3 8.1e-6 (100 x 200 planes in y/z
# items; gradients take 5x the bound).
ELEM_TOL = {"fp32": 2e-6, "tf32x3": 1.5e-6, "bf16x3": 1.5e-5, "tf32": 5e-3, "bf16": 1.6e-2}


def elem_rel(a, b):
    """(max |a - b| / max |b|, index of the largest |a - b|)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.abs(a - b)
    k = int(np.argmax(d))
    return float(d.ravel()[k] / np.abs(b).max()), np.unravel_index(k, d.shape)


def log_energy(prec, what, got, ref):
    _log(dict(what=what, prec=prec, energy_rel=abs(got - ref) / abs(ref)))


def _log(entry):
    path = os.environ.get("TX_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(entry) + "\n")


def assert_close(got, ref, prec, what="W", scale=1.0):
    """Frobenius and elementwise parity against the oracle at the precision's tolerances
    (times `scale`); the message names the worst element."""
    fr = rel(got, ref)
    el, idx = elem_rel(got, ref)
    _log(dict(what=what, prec=prec, frob=fr, elem=el))
    assert fr < scale * W_TOL[prec], f"{what} [{prec}]: Frobenius error {fr:.3e} >= {scale * W_TOL[prec]:.1e}"
    assert el < scale * ELEM_TOL[prec], (
        f"{what} [{prec}]: elementwise error {el:.3e} >= {scale * ELEM_TOL[prec]:.1e} at index {tuple(int(v) for v in idx)}"
        f" (got {np.asarray(got).ravel()[np.ravel_multi_index(idx, np.shape(got))]:.6e},"
        f" oracle {np.asarray(ref).ravel()[np.ravel_multi_index(idx, np.shape(ref))]:.6e})")
    return fr, el


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def max_row_rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return max(float(np.linalg.norm((a[i] - b[i]).ravel()) / np.linalg.norm(b[i].ravel())) for i in range(len(a)))


def oracle_setup(s):
    return O.Setup.from_system(s)


def to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()

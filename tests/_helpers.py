"""Shared helpers for the GPU parity tests (the oracle is the reference everywhere)."""
import numpy as np

import oracle as O

# Relative Frobenius tolerances of W (and relative tolerances of E_x) against the FP64 oracle,
# per GEMM arithmetic.  bf16 keeps 8 significant bits (unit roundoff 2^-9) and the chain rounds
# its operands about five times; tf32 keeps 11 (2^-12 per rounding after round-to-nearest).
# The 3-pass forms carry ~22 (tf32) or ~16 (bf16) bits per operand (2^-22 ~ 2.4e-7 per stored
# value and per product), rounded again at each of ~7 chained tensor-core stages; the tensor
# core's float32 accumulator adds an error that grows with the accumulation length, which the
# library bounds by splitting K over several accumulators and by folding the final contraction
# every 5 Gaussian terms.  Measured worst cases: tf32x3 2.9e-6 (Pt-shaped block), bf16x3 5e-6.
W_TOL = {"fp32": 2e-6, "tf32x3": 5e-6, "bf16x3": 1e-5, "tf32": 5e-3, "bf16": 2e-2}
E_TOL = {"fp32": 1e-6, "tf32x3": 5e-6, "bf16x3": 1e-5, "tf32": 5e-3, "bf16": 1e-2}


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

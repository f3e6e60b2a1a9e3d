"""Shared helpers for the GPU parity tests (the oracle is the reference everywhere)."""
import numpy as np

import oracle as O

# relative Frobenius tolerances of W against the FP64 oracle, per GEMM arithmetic
# (FP32 accumulation everywhere; see the design doc for the derivation)
W_TOL = {"fp32": 2e-6, "tf32x3": 2e-6, "bf16x3": 6e-5, "tf32": 5e-3, "bf16": 2e-2}
E_TOL = {"fp32": 1e-6, "tf32x3": 1e-6, "bf16x3": 5e-5, "tf32": 5e-3, "bf16": 1e-2}


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

"""The seeded input generators: the device form of make_system (used where the block is too large
for the host, e.g. the TiO2-shaped one) draws and computes the same inputs as the host form."""
import numpy as np
import pytest

import workloads as W


def test_device_generator_matches_the_host_generator():
    pytest.importorskip("torch")
    args = ("t", 24, 6.0, 6, 10, 12, 4, W.rutile_cluster(40), 2, (0.2, 3.0))
    host = W.make_system(*args, centres_per_orbital=8)
    dev, psi = W.make_system_on_device(*args, centres_per_orbital=8, device="cpu", chunk=5000)
    p = psi.numpy()
    assert p.dtype == np.float32 and p.shape == host.psi.shape
    assert np.linalg.norm(p - host.psi) <= 1e-6 * np.linalg.norm(host.psi)
    for u, v in zip(dev.U, host.U):
        assert np.abs(u - v).max() < 1e-10
    assert np.array_equal(dev.theta, host.theta) and np.array_equal(dev.mu, host.mu)
    # the orbitals are orthonormal in the trapezoid inner product
    w = host.w
    w3 = (w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]).reshape(-1)
    P = p.reshape(p.shape[0], -1).astype(np.float64)
    assert np.abs((P * w3) @ P.T - np.eye(p.shape[0])).max() < 1e-5

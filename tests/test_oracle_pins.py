"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms, brute-force direct sums with 3-D distances, textbook bounds, exact
invariants of the operator at full rank, transposes and finite differences.

Each pin is chosen to fail on a plausible mistake: a transposed convolution matrix
(non-uniform weights in the brute-force test), a mixed-up mode (different n per mode),
a dropped mu_t or a wrong theta_t (brute force and closed form), a wrong sign or factor
(energy of a Gaussian orbital), a wrong adjoint (dot-product and finite-difference tests).
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _random_setup(rng, n, r, T, uniform=False, full_rank=False):
    xs, ws, Us = [], [], []
    for d in range(3):
        if uniform:
            x, w = W.uniform_grid(n[d], 3.0)
        else:
            x = np.sort(rng.uniform(-3.0, 3.0, n[d]))
            w = rng.uniform(0.2, 0.8, n[d])
        xs.append(x)
        ws.append(w)
        if full_rank:
            Us.append(np.eye(n[d]))
        else:
            Q, _ = np.linalg.qr(rng.standard_normal((n[d], r[d])))
            Us.append(Q)
    theta = rng.uniform(0.05, 2.0, T)
    mu = rng.uniform(0.1, 1.0, T)
    return O.Setup(xs, ws, Us, theta, mu)


# ---------------------------------------------------------------------------------
# Gaussian-sum approximation of 1/r (Eq. gauss): error on [r1, r2] against 1/r itself
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("T,n,L,tol", [(30, 32, 8.0, 3e-6), (35, 64, 10.0, 2e-6),
                                       (40, 96, 12.0, 1e-6), (45, 160, 16.0, 1e-6)])
def test_exp_sum_matches_inverse_r_on_grid_range(T, n, L, tol):
    h = 2 * L / (n - 1)
    r1, r2 = h, 2 * L * math.sqrt(3)
    theta, mu, reported = W.exp_sum_inverse_r(T, r1, r2)
    assert np.all(theta > 0) and np.all(mu > 0)
    r = np.geomspace(r1, r2, 20001)                       # denser than the fit's own sample
    approx = np.exp(-np.outer(r * r, theta)) @ mu
    err = np.max(np.abs(approx * r - 1.0))
    assert err < tol
    assert abs(err - reported) < 0.2 * reported + 1e-12
    # the paper notes the fit fails below r1 (1/r is singular there)
    r_small = np.array([0.05 * r1])
    assert abs((np.exp(-np.outer(r_small ** 2, theta)) @ mu)[0] * r_small[0] - 1) > 10 * tol


# ---------------------------------------------------------------------------------
# 1-D convolution matrices (Eq. discInteg) against the closed-form Gaussian convolution
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("a,theta", [(1.0, 0.5), (0.3, 2.0), (2.5, 0.01)])
def test_conv_matrix_resolved_gaussian_closed_form(a, theta):
    x, w = W.uniform_grid(97, 12.0)           # h = 0.25; (a + theta) h^2 <= 0.3: resolved
    C = O.conv_matrix(x, w, theta)
    f = np.exp(-a * x * x)
    got = C @ f
    exact = math.sqrt(math.pi / (a + theta)) * np.exp(-a * theta * x * x / (a + theta))
    inner = np.abs(x) <= 4.0
    assert np.max(np.abs(got - exact)[inner]) < 1e-10


# ---------------------------------------------------------------------------------
# Projection: textbook HOSVD error bound, idempotence, exactness in the span
# ---------------------------------------------------------------------------------
def test_projection_hosvd_error_bound():
    s = W.config_small()
    rho = s.psi[0].astype(np.float64) ** 2
    for r in (4, 8, 12):
        U = W.density_hosvd_basis(s.psi[:1], (r, r, r))      # HOSVD of rho = psi_0^2 itself
        P = O.project(rho, U)
        for d in range(3):
            P = O.mode_product(P, U[d], d)
        err2 = np.sum((rho - P) ** 2)
        bound = 0.0
        for d in range(3):
            M = np.moveaxis(rho, d, 0).reshape(rho.shape[d], -1)
            sv = np.linalg.svd(M, compute_uv=False)
            bound += np.sum(sv[r:] ** 2)
        # truncated HOSVD: ||rho - P rho||^2 <= sum_d sum_{discarded} sigma_d^2
        assert err2 <= bound * (1 + 1e-9)
        assert err2 > 0


def test_projection_idempotent_and_exact_on_span():
    rng = np.random.default_rng(5)
    n, r = (9, 11, 13), (4, 5, 6)
    S = _random_setup(rng, n, r, 2)
    rho = rng.standard_normal(n)
    G = O.project(rho, S.U)
    P1 = G
    for d in range(3):
        P1 = O.mode_product(P1, S.U[d], d)
    G2 = O.project(P1, S.U)
    assert _rel(G2, G) < 1e-13
    # a separable field whose factors lie in span(U_d) is reproduced exactly
    f = [S.U[d] @ rng.standard_normal(r[d]) for d in range(3)]
    sep = np.einsum("a,b,c->abc", *f)
    G = O.project(sep, S.U)
    back = G
    for d in range(3):
        back = O.mode_product(back, S.U[d], d)
    assert _rel(back, sep) < 1e-13


# ---------------------------------------------------------------------------------
# Whole potential at full rank against the brute-force O(n^6 T) sum with 3-D distances
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1])
def test_full_rank_potential_equals_direct_sum(seed):
    rng = np.random.default_rng(seed)
    n = (7, 9, 11)                                # different per mode: catches mode mix-ups
    S = _random_setup(rng, n, n, 3, full_rank=True)
    rho = rng.standard_normal(n)
    phi = O.apply_L(rho, S)
    ref = O.direct_gaussian_kernel_potential(rho, S.x, S.w, S.theta, S.mu)
    assert _rel(phi, ref) < 1e-12


def test_truncated_rank_potential_on_the_span_equals_direct_sum():
    """At truncated rank the operator is L = sum_t mu_t (x)_d C_td U_d U_d^T: a density whose
    mode factors lie in span(U_d) passes the projection unchanged, so its potential is the
    brute-force sum; a density orthogonal to the span in one mode has none.  Catches a wrong
    composition A_td = C_td U_d (transposed or swapped factors) that full rank (U = I) hides."""
    rng = np.random.default_rng(11)
    n, r = (7, 8, 9), (3, 4, 5)
    S = _random_setup(rng, n, r, 3)
    rho = np.zeros(n)
    for _ in range(2):
        f = [S.U[d] @ rng.standard_normal(r[d]) for d in range(3)]
        rho += np.einsum("a,b,c->abc", *f)
    ref = O.direct_gaussian_kernel_potential(rho, S.x, S.w, S.theta, S.mu)
    assert _rel(O.apply_L(rho, S), ref) < 1e-12
    # the mode-2 factor orthogonal to span(U_2): nothing survives the projection
    g = rng.standard_normal(n[1])
    g -= S.U[1] @ (S.U[1].T @ g)
    perp = np.einsum("a,b,c->abc", S.U[0][:, 0], g, S.U[2][:, 1])
    full = O.direct_gaussian_kernel_potential(perp, S.x, S.w, S.theta, S.mu)
    assert np.linalg.norm(O.apply_L(perp, S)) < 1e-12 * np.linalg.norm(full)


def test_direct_sum_reference_is_sensitive_to_transposed_weights():
    # the brute-force reference must tell C = K D apart from C = D K on a non-uniform grid
    rng = np.random.default_rng(3)
    n = (7, 8, 9)
    S = _random_setup(rng, n, n, 2, full_rank=True)
    rho = rng.standard_normal(n)
    ref = O.direct_gaussian_kernel_potential(rho, S.x, S.w, S.theta, S.mu)
    wrong = 0
    for t in range(S.T):
        Y = rho
        for d in range(3):
            Ct = O.conv_matrix(S.x[d], S.w[d], S.theta[t])
            Ct = Ct / S.w[d][None, :] * S.w[d][:, None]          # weights on the wrong index
            Y = O.mode_product(Y, Ct, d)
        wrong = wrong + S.mu[t] * Y
    assert _rel(wrong, ref) > 1e-3


# ---------------------------------------------------------------------------------
# Physics: potential of a Gaussian charge is erf(sqrt(a) r)/r (O(h^2) on the grid)
# ---------------------------------------------------------------------------------
def test_gaussian_charge_potential_closed_form_and_convergence():
    a, L = 1.0, 7.0
    errs, sep_errs = [], []
    for n in (15, 29, 57):
        x, w = W.uniform_grid(n, L)
        h = x[1] - x[0]
        theta, mu, _ = W.exp_sum_inverse_r(30, h, 2 * L * math.sqrt(3))
        S = O.Setup([x] * 3, [w] * 3, [np.eye(n)] * 3, theta, mu)
        X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1)
        r = np.linalg.norm(X, axis=-1)
        rho = (a / math.pi) ** 1.5 * np.exp(-a * r * r)
        phi = O.apply_L(rho, S)
        exact = O.gaussian_charge_potential(a, r)
        inner = r <= 3.0
        errs.append(np.max(np.abs(phi - exact)[inner]) / np.max(exact))
        # the continuous convolution with the fitted kernel: its error comes only from
        # distances below r1 = h, where the fit departs from 1/r, so it is also O(h^2)
        sep = O.gaussian_kernel_charge_potential(a, r[inner], theta, mu)
        sep_errs.append(np.max(np.abs(sep - exact[inner])) / np.max(exact))
    assert errs[-1] < 1e-2 and sep_errs[-1] < 5e-3
    # second order in h: halving h cuts the error by about 4
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 2.5
    assert sep_errs[0] / sep_errs[1] > 2.5 and sep_errs[1] / sep_errs[2] > 2.5


def test_gaussian_orbital_exchange_energy_closed_form():
    # psi = (2a/pi)^{3/4} exp(-a r^2): rho = psi^2 is a unit Gaussian charge of exponent 2a,
    # whose Coulomb self-energy is J = sqrt(2 * 2a / pi); one orbital gives E_x = -J/2.
    a, L = 0.8, 7.0
    errs = []
    for n in (15, 29, 57):
        x, w = W.uniform_grid(n, L)
        theta, mu, _ = W.exp_sum_inverse_r(30, x[1] - x[0], 2 * L * math.sqrt(3))
        S = O.Setup([x] * 3, [w] * 3, [np.eye(n)] * 3, theta, mu)
        X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1)
        psi = (2 * a / math.pi) ** 0.75 * np.exp(-a * np.sum(X * X, -1))
        E = O.exchange_energy(psi[None], S)
        errs.append(abs(E + 0.5 * math.sqrt(4 * a / math.pi)))
        assert E < 0
    assert errs[-1] / (0.5 * math.sqrt(4 * a / math.pi)) < 5e-3
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 2.5


def test_true_coulomb_brute_force_agrees_within_self_cell_error():
    a, L, n = 1.0, 5.0, 13
    x, w = W.uniform_grid(n, L)
    h = x[1] - x[0]
    theta, mu, _ = W.exp_sum_inverse_r(30, h, 2 * L * math.sqrt(3))
    S = O.Setup([x] * 3, [w] * 3, [np.eye(n)] * 3, theta, mu)
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1)
    r = np.linalg.norm(X, axis=-1)
    rho = (a / math.pi) ** 1.5 * np.exp(-a * r * r)
    phi = O.apply_L(rho, S)
    bf = O.direct_coulomb_potential(rho, S.x, S.w)
    # away from r < h the two sums differ only by the fit error and the self/near cells
    far = r > 2 * h
    rel = np.max(np.abs(phi - bf)[far]) / np.max(np.abs(bf))
    assert rel < 0.2


# ---------------------------------------------------------------------------------
# Operator invariants: symmetric and negative semidefinite exactly at full rank
# ---------------------------------------------------------------------------------
def test_exchange_matrix_symmetric_nsd_at_full_rank():
    s = W.config_small(n=14, n_orb=3, rank=14, T=8, L=5.0, full_rank=True)
    S = O.Setup.from_system(s)
    psi = s.psi.astype(np.float64)
    Wk = O.exchange_apply(psi, S)
    M = np.einsum("axyz,bxyz->ab", psi * S.w3[None], Wk)
    assert np.max(np.abs(M - M.T)) / np.max(np.abs(M)) < 1e-12
    assert np.max(np.linalg.eigvalsh(0.5 * (M + M.T))) < 1e-12 * np.max(np.abs(M))


def test_exchange_matrix_nearly_symmetric_at_truncated_rank():
    s = W.config_small(n=14, n_orb=3, rank=10, T=8, L=5.0)
    S = O.Setup.from_system(s)
    psi = s.psi.astype(np.float64)
    M = np.einsum("axyz,bxyz->ab", psi * S.w3[None], O.exchange_apply(psi, S))
    asym = np.max(np.abs(M - M.T)) / np.max(np.abs(M))
    assert 0 < asym < 0.05


def test_pair_potential_symmetric_in_the_pair():
    s = W.config_small(n=12, n_orb=2, rank=6, T=4, L=5.0)
    S = O.Setup.from_system(s)
    a, b = s.psi.astype(np.float64)
    assert _rel(O.pair_potential(a, b, S), O.pair_potential(b, a, S)) < 1e-14


# ---------------------------------------------------------------------------------
# Transposes and derivatives
# ---------------------------------------------------------------------------------
def test_transpose_dot_product():
    rng = np.random.default_rng(7)
    n, r = (8, 10, 12), (3, 4, 5)
    S = _random_setup(rng, n, r, 3)
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    lhs = np.sum(O.apply_L(x, S) * y)
    rhs = np.sum(x * O.apply_LT(y, S))
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + np.linalg.norm(x) * np.linalg.norm(y))


def test_energy_gradient_finite_differences():
    s = W.config_small(n=10, n_orb=3, rank=6, T=4, L=5.0)
    S = O.Setup.from_system(s)
    psi = s.psi.astype(np.float64)
    E, g = O.exchange_energy_grad(psi, S)
    rng = np.random.default_rng(11)
    for _ in range(5):
        v = rng.standard_normal(psi.shape)
        v /= np.linalg.norm(v)
        eps = 1e-4
        fd = (O.exchange_energy(psi + eps * v, S) - O.exchange_energy(psi - eps * v, S)) / (2 * eps)
        assert abs(fd - np.sum(g * v)) < 1e-6 * max(1.0, abs(fd))


def test_energy_gradient_full_rank_is_twice_weighted_W():
    s = W.config_small(n=10, n_orb=2, rank=10, T=4, L=5.0, full_rank=True)
    S = O.Setup.from_system(s)
    psi = s.psi.astype(np.float64)
    _, g = O.exchange_energy_grad(psi, S)
    Wk = O.exchange_apply(psi, S)
    assert _rel(g, 2 * S.w3[None] * Wk) < 1e-12


def test_apply_vjp_finite_differences():
    s = W.config_small(n=10, n_orb=3, rank=6, T=4, L=5.0)
    S = O.Setup.from_system(s)
    occ = s.psi.astype(np.float64)
    tgt = occ[:2] * 1.3 + 0.1 * occ[1:3]
    rng = np.random.default_rng(13)
    Wb = rng.standard_normal(tgt.shape)
    g_occ, g_tgt = O.exchange_apply_vjp(occ, tgt, Wb, S)

    def f(o, t):
        return np.sum(Wb * O.exchange_apply(o, S, psi_tgt=t))

    eps = 1e-4
    for _ in range(3):
        vo = rng.standard_normal(occ.shape)
        vt = rng.standard_normal(tgt.shape)
        fd_o = (f(occ + eps * vo, tgt) - f(occ - eps * vo, tgt)) / (2 * eps)
        fd_t = (f(occ, tgt + eps * vt) - f(occ, tgt - eps * vt)) / (2 * eps)
        assert abs(fd_o - np.sum(g_occ * vo)) < 1e-6 * max(1.0, abs(fd_o))
        assert abs(fd_t - np.sum(g_tgt * vt)) < 1e-6 * max(1.0, abs(fd_t))


def test_apply_linear_in_target_quadratic_in_occupied():
    s = W.config_small(n=10, n_orb=2, rank=6, T=3, L=5.0)
    S = O.Setup.from_system(s)
    occ = s.psi.astype(np.float64)
    W1 = O.exchange_apply(occ, S, psi_tgt=occ[:1])
    assert _rel(O.exchange_apply(occ, S, psi_tgt=2 * occ[:1]), 2 * W1) < 1e-14
    assert _rel(O.exchange_apply(3 * occ, S, psi_tgt=occ[:1]), 9 * W1) < 1e-14


# ---------------------------------------------------------------------------------
# Adaptively compressed exchange (section "ACE implementation"): exact on the occupied space
# ---------------------------------------------------------------------------------
def _w_inner(S, a, b):
    return float(np.sum(S.w3 * a * b))


def test_ace_reproduces_the_exchange_operator_on_the_occupied_orbitals():
    """At full rank M is symmetric negative definite and V_ACE psi_j = K psi_j = W_j for every
    occupied j (the defining property of ACE), so its exchange energy is E_x."""
    s = W.config_small(n=12, n_orb=3, rank=12, T=4, L=4.0, full_rank=True)
    S = O.Setup.from_system(s)
    Wx = O.exchange_apply(s.psi, S)
    xi, M = O.ace_projectors(s.psi, S, W=Wx)
    assert np.abs(M - M.T).max() < 1e-12 * np.abs(M).max()
    assert np.all(np.linalg.eigvalsh(0.5 * (M + M.T)) < 0)
    V = O.ace_apply(xi, s.psi, S)
    assert _rel(V, Wx) < 1e-12
    e_ace = 0.5 * sum(_w_inner(S, s.psi[i], V[i]) for i in range(len(s.psi)))
    e = O.exchange_energy(s.psi, S, W=Wx)
    assert abs(e_ace - e) < 1e-12 * abs(e)


def test_ace_operator_is_symmetric_negative_semidefinite_of_rank_n():
    """V_ACE = - sum_k xi_k xi_k^T (with the quadrature weights) at any rank: symmetric, NSD, and
    zero on fields w-orthogonal to every W_j."""
    s = W.config_small(n=10, n_orb=3, rank=6, T=4, L=5.0)
    S = O.Setup.from_system(s)
    Wx = O.exchange_apply(s.psi, S)
    xi, _ = O.ace_projectors(s.psi, S, W=Wx)
    rng = np.random.default_rng(17)
    f, g = rng.standard_normal((2,) + s.psi.shape[1:])
    Vf, Vg = O.ace_apply(xi, np.stack([f, g]), S)
    assert abs(_w_inner(S, f, Vg) - _w_inner(S, g, Vf)) < 1e-13 * abs(_w_inner(S, f, Vf))
    assert _w_inner(S, f, Vf) < 0 and _w_inner(S, g, Vg) < 0
    # remove from h its w-projection onto span(W): V_ACE h must vanish
    h = rng.standard_normal(s.psi.shape[1:])
    G = np.array([[_w_inner(S, a, b) for b in Wx] for a in Wx])
    c = np.linalg.solve(G, np.array([_w_inner(S, a, h) for a in Wx]))
    h = h - np.tensordot(c, Wx, axes=(0, 0))
    assert np.linalg.norm(O.ace_apply(xi, h[None], S)) < 1e-12 * np.linalg.norm(Vf)


def test_ace_at_truncated_rank_is_exact_up_to_the_asymmetry_of_M():
    """At truncated rank M = <psi_i, W_j> is slightly asymmetric (one-sided projection) and the
    symmetrised factorisation reproduces W_j up to an error of the size of that asymmetry."""
    s = W.config_small(n=12, n_orb=3, rank=7, T=5, L=4.0)
    S = O.Setup.from_system(s)
    Wx = O.exchange_apply(s.psi, S)
    xi, M = O.ace_projectors(s.psi, S, W=Wx)
    asym = np.linalg.norm(M - M.T) / np.linalg.norm(M)
    assert 0 < asym < 1e-2
    V = O.ace_apply(xi, s.psi, S)
    assert _rel(V, Wx) < 2 * asym
    # algebra: with L L^T = -Ms (Ms the symmetric part of M), V_ACE psi_a = sum_i W_i (Ms^-1 M^T)_ia,
    # which reduces to W_a exactly when M is symmetric
    Ms = 0.5 * (M + M.T)
    B = np.linalg.solve(Ms, M.T)
    assert _rel(V, np.tensordot(B, Wx, axes=(0, 0))) < 1e-10


# ------------------------------------------------------------------------------------------
# Finite-element quadrature of the 1-D convolutions (Eqs. quadVal, discInteg)
# ------------------------------------------------------------------------------------------
def test_fe_linear_elements_match_the_closed_form():
    """Linear elements: Gauss-Legendre quadrature inside every element against the exact integral
    of the hat function times the Gaussian (erf on each interval), on a non-uniform grid."""
    rng = np.random.default_rng(11)
    x = np.sort(np.concatenate([[-4.0, 4.0], rng.uniform(-4, 4, 15)]))
    for th in (0.05, 0.6, 4.0):
        C = O.conv_matrix_fe(x, th, 1, 24)
        E = O.conv_matrix_p1_exact(x, th)
        assert np.abs(C - E).max() < 1e-12 * np.abs(E).max(), th


@pytest.mark.parametrize("order", [1, 2, 3])
def test_fe_elements_reproduce_polynomials_of_their_order(order):
    """Lagrange elements of order p interpolate x^k (k <= p) exactly, so sum_b C[a,b] x_b^k is the
    convolution integral of x^k over the whole interval, computed here by adaptive quadrature
    (scipy.integrate.quad) of the continuous integrand."""
    from scipy.integrate import quad
    x = np.linspace(-3.0, 3.0, 6 * order + 1)
    th = 0.8
    C = O.conv_matrix_fe(x, th, order, 20)
    for k in range(order + 1):
        for a in (0, len(x) // 3, len(x) - 1):
            ref, _ = quad(lambda u: u ** k * np.exp(-th * (x[a] - u) ** 2), x[0], x[-1], epsabs=1e-14, epsrel=1e-13)
            got = float(C[a] @ x ** k)
            assert abs(got - ref) < 1e-11 * max(1.0, abs(ref)), (order, k, a, got, ref)


def test_fe_quadrature_of_a_flat_kernel_gives_the_element_weights():
    """For theta -> 0 the kernel is 1 and C[a, b] -> integral of N_b: the trapezoid weights for
    linear elements, Simpson's 1/6, 4/6, 1/6 pattern (times the element length) for quadratic."""
    x = np.linspace(-2.0, 2.0, 9)
    h = x[1] - x[0]
    C1 = O.conv_matrix_fe(x, 1e-12, 1, 8)
    trap = np.full(9, h)
    trap[[0, -1]] = h / 2
    assert np.abs(C1 - trap[None, :]).max() < 1e-9
    C2 = O.conv_matrix_fe(x, 1e-12, 2, 8)
    simp = np.array([1, 4, 2, 4, 2, 4, 2, 4, 1]) * (2 * h) / 6
    assert np.abs(C2 - simp[None, :]).max() < 1e-9


def test_fe_setup_changes_only_the_convolution_matrices():
    """A Setup with FE quadrature of linear elements on a resolved Gaussian sum gives nearly the
    same potential as the nodal rule (both converge to the same integral) and exactly
    conv_matrix_fe @ U for its A_td."""
    s = W.config_small(n=16, n_orb=2, rank=6, T=3, L=4.0)
    Sn = O.Setup.from_system(s)
    Sf = O.Setup.from_system(s, quadrature=("fe", 1, 12))
    for t in range(s.T):
        for d in range(3):
            assert np.abs(Sf.A[t][d] - O.conv_matrix_fe(s.x[d], s.theta[t], 1, 12) @ s.U[d]).max() < 1e-14
    Wn = O.exchange_apply(s.psi, Sn)
    Wf = O.exchange_apply(s.psi, Sf)
    assert 0 < _rel(Wf, Wn) < 0.2


# ---------------------------------------------------------------------------------
# Two-sided (Galerkin) projection: P^* C P with P^* = D^-1 P D the w-adjoint of P
# ---------------------------------------------------------------------------------
def _explicit_pieces(S):
    """The n^3 x n^3 matrices of the separable convolution and of the projection, built by
    Kronecker products straight from the grid (independent of the oracle's mode products), and
    the 3-D weight vector (C-order flattening: z fastest)."""
    def kron3(m):
        return np.kron(m[0], np.kron(m[1], m[2]))
    K = sum(S.mu[t] * kron3([np.exp(-S.theta[t] * (S.x[d][:, None] - S.x[d][None, :]) ** 2) * S.w[d][None, :]
                            for d in range(3)]) for t in range(S.T))
    P = kron3([S.U[d] @ S.U[d].T for d in range(3)])
    Dv = kron3([S.w[d][:, None] for d in range(3)]).ravel()
    return K, P, Dv


def test_galerkin_operator_equals_its_explicit_matrix():
    rng = np.random.default_rng(21)
    n, r = (4, 5, 6), (2, 3, 4)
    S = _random_setup(rng, n, r, 3)
    K, P, Dv = _explicit_pieces(S)
    LG = (P @ (Dv[:, None] * (K @ P))) / Dv[:, None]          # D^-1 P D K P
    rho = rng.standard_normal(n)
    assert _rel(O.apply_L_galerkin(rho, S), (LG @ rho.ravel()).reshape(n)) < 1e-12
    assert _rel(O.apply_L(rho, S), (K @ P @ rho.ravel()).reshape(n)) < 1e-12    # one-sided: K P


def test_galerkin_at_full_rank_equals_the_one_sided_operator():
    rng = np.random.default_rng(22)
    n = (5, 6, 7)
    S = _random_setup(rng, n, n, 3)              # square orthogonal U_d, not the identity
    rho = rng.standard_normal(n)
    assert _rel(O.apply_L_galerkin(rho, S), O.apply_L(rho, S)) < 1e-12


def test_galerkin_form_is_symmetric_and_positive_semidefinite_at_truncated_rank():
    """<e_k, P^* C P e_l>_w over all grid points is a symmetric positive semi-definite matrix
    (so E_x <= 0 exactly); the one-sided form at the same rank is not symmetric."""
    rng = np.random.default_rng(23)
    n, r = (4, 4, 5), (2, 3, 3)
    S = _random_setup(rng, n, r, 3)
    _, _, Dv = _explicit_pieces(S)
    N = int(np.prod(n))
    E = np.eye(N)
    LG = np.array([O.apply_L_galerkin(E[k].reshape(n), S).ravel() for k in range(N)]).T
    L1 = np.array([O.apply_L(E[k].reshape(n), S).ravel() for k in range(N)]).T
    MG, M1 = Dv[:, None] * LG, Dv[:, None] * L1
    scale = np.max(np.abs(MG))
    assert np.max(np.abs(MG - MG.T)) < 1e-12 * scale
    assert np.min(np.linalg.eigvalsh(0.5 * (MG + MG.T))) > -1e-12 * scale
    assert np.max(np.abs(M1 - M1.T)) > 1e-3 * np.max(np.abs(M1))


def test_galerkin_agrees_with_the_one_sided_form_on_the_span():
    """For sigma and rho whose mode factors lie in span(U_d), P sigma = sigma and P rho = rho,
    so <sigma, P^* C P rho>_w = <sigma, C P rho>_w."""
    rng = np.random.default_rng(24)
    n, r = (6, 7, 8), (3, 3, 4)
    S = _random_setup(rng, n, r, 4)
    _, _, Dv = _explicit_pieces(S)
    Dv = Dv.reshape(n)

    def in_span():
        f = [S.U[d] @ rng.standard_normal(r[d]) for d in range(3)]
        return np.einsum("a,b,c->abc", *f)
    sig, rho = in_span() + in_span(), in_span()
    a = float(np.sum(Dv * sig * O.apply_L_galerkin(rho, S)))
    b = float(np.sum(Dv * sig * O.apply_L(rho, S)))
    assert abs(a - b) < 1e-12 * abs(b)


def test_galerkin_energy_in_core_space_equals_the_grid_energy():
    s = W.config_small(n=10, n_orb=3, rank=6, T=5, L=5.0)
    S = O.Setup.from_system(s)
    psi = s.psi.astype(np.float64)
    Wg = O.exchange_apply_galerkin(psi, S)
    e_grid = 0.5 * float(np.sum(S.w3[None] * psi * Wg))
    e_core = O.exchange_energy_galerkin(psi, S)
    assert e_core < 0
    assert abs(e_core - e_grid) < 1e-12 * abs(e_grid)
    # the exchange matrix <psi_a, W_b>_w is exactly symmetric and negative semi-definite
    M = np.einsum("axyz,bxyz->ab", psi * S.w3[None], Wg)
    assert np.max(np.abs(M - M.T)) < 1e-12 * np.max(np.abs(M))
    assert np.max(np.linalg.eigvalsh(0.5 * (M + M.T))) < 1e-12 * np.max(np.abs(M))


# ---------------------------------------------------------------------------------
# Transfer between the unstructured and structured finite-element bases (Eq. interpolate)
# ---------------------------------------------------------------------------------
def _poly(deg):
    """A polynomial of degree `deg` in each coordinate, different along every axis."""
    cx = [1.0, 2.0, 0.5, -0.1][: deg + 1]
    cy = [1.0, -1.0, 0.3, 0.05][: deg + 1]
    cz = [2.0, 1.0, -0.7, 0.02][: deg + 1]
    return lambda x, y, z: (sum(c * x ** k for k, c in enumerate(cx)) * sum(c * y ** k for k, c in enumerate(cy))
                            * sum(c * z ** k for k, c in enumerate(cz)))


def _transfer_case():
    X, conn = W.fe_mesh(4.0, 3, [[0.0, 0.0, 0.0], [1.5, -1.0, 0.5]], 2.0, 2)
    xs = [np.linspace(-4, 4, 19), np.linspace(-4, 4, 22), np.linspace(-4, 4, 25)]
    return X, conn, xs


def test_transfer_to_the_grid_reproduces_polynomials_of_the_element_order():
    """Lagrange elements of order 2 reproduce any polynomial of degree 2 in each coordinate, on
    refined and unrefined cells alike; one of degree 3 is not reproduced."""
    X, conn, xs = _transfer_case()
    G = np.meshgrid(*xs, indexing="ij")
    for deg, exact in ((2, True), (3, False)):
        f = _poly(deg)
        got = O.transfer_u_to_s(f(X[:, 0], X[:, 1], X[:, 2])[:, None], X, conn, 2, xs)[0]
        err = np.max(np.abs(got - f(*G))) / np.max(np.abs(f(*G)))
        assert (err < 1e-12) if exact else (err > 1e-6)


def test_transfer_to_the_mesh_reproduces_polynomials_of_the_element_order():
    X, conn, xs = _transfer_case()
    xs = [np.linspace(-4, 4, 19), np.linspace(-4, 4, 22), np.linspace(-4, 4, 25)]   # 18, 21, 24: order 3
    G = np.meshgrid(*xs, indexing="ij")
    for deg in (1, 3):
        f = _poly(deg)
        got = O.transfer_s_to_u(f(*G)[None], xs, 3, X)[:, 0]
        ref = f(X[:, 0], X[:, 1], X[:, 2])
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    f = _poly(2)
    got = O.transfer_s_to_u(f(*G)[None], xs, 1, X)[:, 0]      # linear elements: not exact for degree 2
    ref = f(X[:, 0], X[:, 1], X[:, 2])
    assert np.max(np.abs(got - ref)) > 1e-6 * np.max(np.abs(ref))


def test_transfer_between_matching_meshes_is_the_identity():
    """Unstructured cells that are the structured elements themselves (same nodes, same order):
    both transfers only renumber the values."""
    p = 2
    xs = [np.linspace(-2, 2, 5), np.linspace(-3, 3, 7), np.linspace(-1, 1, 9)]
    cells, Xl, index = [], [], {}
    for ex in range(2):
        for ey in range(3):
            for ez in range(4):
                ids = []
                for lx in range(p + 1):
                    for ly in range(p + 1):
                        for lz in range(p + 1):
                            key = (p * ex + lx, p * ey + ly, p * ez + lz)
                            if key not in index:
                                index[key] = len(Xl)
                                Xl.append([xs[0][key[0]], xs[1][key[1]], xs[2][key[2]]])
                            ids.append(index[key])
                cells.append(ids)
    X, conn = np.array(Xl), np.array(cells, dtype=np.int32)
    rng = np.random.default_rng(31)
    psi_s = rng.standard_normal((3, 5, 7, 9))
    psi_u = O.transfer_s_to_u(psi_s, xs, p, X)
    for key, g in index.items():
        assert np.allclose(psi_u[g], psi_s[:, key[0], key[1], key[2]], rtol=0, atol=1e-13)
    assert np.max(np.abs(O.transfer_u_to_s(psi_u, X, conn, p, xs) - psi_s)) < 1e-13


def test_transfer_of_a_smooth_orbital_converges_at_the_element_order():
    """A Gaussian sampled on the unstructured nodes and carried to the grid: halving the cells
    divides the error by about 2^(order + 1) (order 2: ~8)."""
    xs = [np.linspace(-4, 4, 33)] * 3
    G = np.meshgrid(*xs, indexing="ij")
    cen = np.array([[[0.3, -0.2, 0.1]]])
    f = lambda pts: W.gaussian_sum_at_points(pts, cen, np.array([[0.5]]), np.array([[1.0]]))[0]
    exact = f(np.stack([g.ravel() for g in G], axis=1)).reshape(G[0].shape)
    errs = []
    for base in (4, 8):
        X, conn = W.fe_mesh(4.0, base, np.zeros((1, 3)), 0.0, 2, levels=0)
        got = O.transfer_u_to_s(f(X)[:, None], X, conn, 2, xs)[0]
        errs.append(np.max(np.abs(got - exact)))
    assert 5.0 < errs[0] / errs[1] < 12.0


# ---------------------------------------------------------------------------------
# Per-pair Tucker bases (sequentially truncated HOSVD, Eq. TuckerDecompField)
# ---------------------------------------------------------------------------------
def test_sthosvd_error_is_the_sum_of_the_discarded_eigenvalues():
    """For the sequentially truncated HOSVD the squared error of the reconstruction is exactly
    the sum over modes of the eigenvalues discarded at that mode's step (each step removes an
    orthogonal part); truncating nothing reconstructs the tensor."""
    rng = np.random.default_rng(41)
    rho = rng.standard_normal((9, 10, 11)) + np.einsum("a,b,c->abc", *[rng.standard_normal(k) for k in (9, 10, 11)]) * 4
    ranks = (4, 5, 6)
    G, Us = O.sthosvd(rho, ranks)
    rec = G
    for d in range(3):
        rec = O.mode_product(rec, Us[d], d)
    discarded = 0.0
    T = rho
    for d in range(3):
        M = np.moveaxis(T, d, 0).reshape(T.shape[d], -1)
        ev = np.sort(np.linalg.eigvalsh(M @ M.T))[::-1]
        discarded += ev[ranks[d]:].sum()
        T = O.mode_product(T, Us[d].T, d)
    err2 = float(np.sum((rho - rec) ** 2))
    assert abs(err2 - discarded) < 1e-10 * np.sum(rho ** 2)
    G, Us = O.sthosvd(rho, rho.shape)
    rec = G
    for d in range(3):
        rec = O.mode_product(rec, Us[d], d)
    assert _rel(rec, rho) < 1e-12


def test_per_pair_bases_at_full_rank_give_the_direct_sum():
    rng = np.random.default_rng(42)
    n = (6, 7, 8)
    S = _random_setup(rng, n, (3, 3, 3), 3)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    phi = O.pair_potential_sthosvd(a, b, S, n)
    ref = O.direct_gaussian_kernel_potential(a * b, S.x, S.w, S.theta, S.mu)
    assert _rel(phi, ref) < 1e-12


def test_per_pair_bases_capture_a_separable_density_at_rank_one():
    """A rank-(1,1,1) pair density (a product of separable orbitals) is reproduced exactly by
    rank-1 per-pair bases, whatever the shared basis, so its potential is the direct sum."""
    rng = np.random.default_rng(43)
    n = (7, 8, 9)
    S = _random_setup(rng, n, (2, 2, 2), 3)
    fa = [rng.standard_normal(k) for k in n]
    fb = [rng.standard_normal(k) for k in n]
    a, b = np.einsum("a,b,c->abc", *fa), np.einsum("a,b,c->abc", *fb)
    phi = O.pair_potential_sthosvd(a, b, S, (1, 1, 1))
    ref = O.direct_gaussian_kernel_potential(a * b, S.x, S.w, S.theta, S.mu)
    assert _rel(phi, ref) < 1e-12
    # the shared rank-2 random basis does not capture it
    assert _rel(O.pair_potential(a, b, S), ref) > 1e-3

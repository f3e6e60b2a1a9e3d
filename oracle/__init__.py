"""FP64 CPU oracle for the Tucker-tensor Fock-exchange hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code with the CUDA library.

It follows the paper (arXiv 2401.04189, "Convolution operation" section) step by step, in
plain numpy float64, with ``np.tensordot`` as the only library primitive (one mode-n
product = one tensordot):

  rho_ij = psi_i * psi_j                                  pair density (the step before Eq. TuckerDecompField)
  G_ij   = rho_ij x1 U1^T x2 U2^T x3 U3^T                 Tucker core on a shared basis (Eq. TuckerDecompField)
  C_td[a,b] = w_b exp(-theta_t (x_a - x_b)^2)             1-D convolution matrix, nodal quadrature (Eq. discInteg)
  A_td   = C_td U_d                                       1-D convolutions of the basis functions (Eq. final)
  phi_ij = sum_t mu_t G_ij x1 A_t1 x2 A_t2 x3 A_t3        separable convolution (Eqs. gauss, final)
  W_i    = - sum_j psi_j * phi_ij                         action of the exchange operator (Eqs. ExchangeOperator, hadam)
  E_x    = 1/2 sum_i sum_x w(x) psi_i(x) W_i(x)           exact-exchange energy with alpha = 1 (Eq. for S[phi])

Readings of the paper (it is silent on these): the basis U_d is shared by all pairs and
orthonormal in the Euclidean inner product on nodal values; the 1-D integrals use the
nodal trapezoid quadrature of the uniform grid; occupations are 1 and alpha = 1.

Gradients are not in the paper; they are derived from the definitions above with
L = sum_t mu_t (x)_d (A_td U_d^T), so that phi_ij = L rho_ij:
  L^T y          = (sum_t mu_t y x1 A_t1^T x2 A_t2^T x3 A_t3^T) x1 U1 x2 U2 x3 U3
  dE/dpsi_k      = w * W_k - sum_j psi_j * L^T(w * rho_kj)
  VJP of W for a cotangent Wbar over the targets:
    grad_tgt_k   = - sum_j psi_j * L^T(Wbar_k * psi_j)
    grad_occ_j   = - sum_k Wbar_k * phi_kj - sum_k psi_k * L^T(Wbar_k * psi_j)

A second set-up variant follows Eqs. quadVal and discInteg with finite-element quadrature: the
1-D field is interpolated by Lagrange elements of order p on the nodes (elements of p + 1
consecutive nodes sharing their end nodes), and each 1-D convolution integral is evaluated by
Gauss-Legendre quadrature inside every element:
  C_td[a,b] = sum_e sum_q J_e w_q N_b(x_q) exp(-theta_t (x_a - x_q)^2)
(conv_matrix_fe; Setup(..., quadrature=("fe", p, points))).

A per-pair variant follows the paper's own decomposition (Eq. TuckerDecompField): every pair
density gets its own bases from a sequentially truncated HOSVD (modes 1, 2, 3 in turn; the r_d
leading eigenvectors of the mode-d Gram matrix of the partly projected tensor), and the
convolution uses A_td,ij = C_td U_d,ij (sthosvd, pair_potential_sthosvd, exchange_apply_sthosvd).

A two-sided (Galerkin) variant of the convolution, which the paper does not describe: the
one-sided operator C P (P = (x)_d U_d U_d^T) is not symmetric in the w inner product at a
truncated rank.  Projecting the output too, with the w-adjoint P^* = D^-1 P D, gives
P^* C P, whose form <sigma, P^* C P rho>_w = (U^T sigma)^T [sum_t mu_t (x)_d B_td] (U^T rho) is
symmetric and positive semi-definite (B_td = U_d^T D_d K_td D_d U_d), so E_x <= 0 exactly and it
is computable in core space (galerkin_core_matrices, apply_L_galerkin, exchange_apply_galerkin,
exchange_energy_galerkin).

The transfer of orbitals between the unstructured finite-element basis of a DFT code and the
structured grid (section "Transfer of wavefunctions", Eq. interpolate): every structured node
takes the value of the unstructured cell containing it, psi_s[i, a] = sum_b N_ab psi_u[b, i]
with N_ab the cell's shape function of node b at a (transfer_u_to_s), and every unstructured
node the value of the structured element containing it (transfer_s_to_u).

The adaptively compressed exchange operator built from W (section "ACE implementation",
Eqs. eta, ace1): M_ij = <psi_i, W_j>_w, M = -L L^T, xi_k = sum_i W_i (L^-1)_ki and
V_ACE psi = - sum_k xi_k <xi_k, psi>_w (M symmetrised first where a truncated rank leaves it
slightly asymmetric).

Independent references used by the pins (brute force and closed forms) are at the end.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "Setup", "conv_matrix", "mode_product", "project", "expand", "expand_transpose",
    "apply_L", "apply_LT", "pair_potential", "exchange_apply", "exchange_energy",
    "exchange_energy_grad", "exchange_apply_vjp", "ace_projectors", "ace_apply",
    "direct_gaussian_kernel_potential", "direct_coulomb_potential",
    "gaussian_charge_potential", "gaussian_kernel_charge_potential", "conv_matrix_fe",
    "conv_matrix_p1_exact", "galerkin_core_matrices", "galerkin_core_convolve", "apply_L_galerkin",
    "exchange_apply_galerkin", "exchange_energy_galerkin", "lagrange_basis", "transfer_u_to_s",
    "transfer_s_to_u", "sthosvd", "pair_potential_sthosvd", "exchange_apply_sthosvd",
]


# ----------------------------------------------------------------------------------
# set-up: 1-D convolution matrices (Eqs. quadVal / discInteg, with nodal quadrature)
# ----------------------------------------------------------------------------------
def conv_matrix(x, w, theta):
    """C[a, b] = w_b * exp(-theta * (x_a - x_b)^2): the 1-D convolution integral of a
    nodal field evaluated at node a by the trapezoid rule (Eq. discInteg)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    d = x[:, None] - x[None, :]
    return np.exp(-float(theta) * d * d) * w[None, :]


def conv_matrix_fe(x, theta, order, points):
    """C[a, b] = integral of N_b(x') exp(-theta (x_a - x')^2) dx' (Eqs. quadVal, discInteg) with
    N_b the Lagrange basis function of node b on elements of `order` + 1 consecutive nodes
    (element e holds nodes order*e .. order*e + order), each element integrated by
    Gauss-Legendre quadrature with `points` points on its interval.  len(x) - 1 must be a
    multiple of `order`."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    p = int(order)
    if p < 1 or (n - 1) % p:
        raise ValueError("len(x) - 1 must be a multiple of the element order")
    xi, wq = np.polynomial.legendre.leggauss(int(points))
    C = np.zeros((n, n))
    for e in range((n - 1) // p):
        nodes = x[p * e: p * e + p + 1]
        xl, xr = nodes[0], nodes[-1]
        half = 0.5 * (xr - xl)
        xq = 0.5 * (xl + xr) + half * xi                    # quadrature points in the element
        # Lagrange basis of the element's nodes at the quadrature points: L[k, q]
        L = np.ones((p + 1, len(xq)))
        for k in range(p + 1):
            for m in range(p + 1):
                if m != k:
                    L[k] *= (xq - nodes[m]) / (nodes[k] - nodes[m])
        K = np.exp(-float(theta) * (x[:, None] - xq[None, :]) ** 2)   # [a, q]
        C[:, p * e: p * e + p + 1] += (K * (half * wq)[None, :]) @ L.T
    return C


def conv_matrix_p1_exact(x, theta):
    """The same integral for linear elements (order 1) in closed form: the hat function of node b
    times the Gaussian, integrated exactly with erf on each of its two intervals."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    th = float(theta)
    s = math.sqrt(th)
    C = np.zeros((n, n))

    def lin_gauss(xa, u0, u1):
        # integral over [u0, u1] of (u - u0) exp(-th (xa - u)^2) du
        erf = math.erf
        g = 0.5 * math.sqrt(math.pi / th) * (erf(s * (u1 - xa)) - erf(s * (u0 - xa)))   # int exp
        m = (math.exp(-th * (u0 - xa) ** 2) - math.exp(-th * (u1 - xa) ** 2)) / (2 * th)   # int (u - xa) exp
        return m + (xa - u0) * g

    for a in range(n):
        xa = x[a]
        for b in range(n):
            v = 0.0
            if b > 0:                                           # rising part on [x_{b-1}, x_b]
                u0, u1 = x[b - 1], x[b]
                v += lin_gauss(xa, u0, u1) / (u1 - u0)
            if b < n - 1:                                       # falling part on [x_b, x_{b+1}]
                u0, u1 = x[b], x[b + 1]
                erf = math.erf
                g = 0.5 * math.sqrt(math.pi / th) * (erf(s * (u1 - xa)) - erf(s * (u0 - xa)))
                v += g - lin_gauss(xa, u0, u1) / (u1 - u0)
            C[a, b] = v
    return C


class Setup:
    """Everything that does not depend on the orbitals: grid, weights, basis, and the
    Gaussian-sum coefficients of 1/r, plus the derived A_td = C_td U_d.  quadrature: ("nodal",)
    for the trapezoid rule on the nodes, or ("fe", order, points) for finite-element quadrature
    (conv_matrix_fe)."""

    def __init__(self, x, w, U, theta, mu, quadrature=("nodal",)):
        self.x = [np.asarray(v, dtype=np.float64) for v in x]
        self.w = [np.asarray(v, dtype=np.float64) for v in w]
        self.U = [np.asarray(u, dtype=np.float64) for u in U]
        self.theta = np.asarray(theta, dtype=np.float64)
        self.mu = np.asarray(mu, dtype=np.float64)
        self.T = len(self.theta)
        self.quadrature = tuple(quadrature)

        def C(d, t):
            if self.quadrature[0] == "fe":
                return conv_matrix_fe(self.x[d], self.theta[t], self.quadrature[1], self.quadrature[2])
            return conv_matrix(self.x[d], self.w[d], self.theta[t])

        # C[t][d], the 1-D convolution matrices, and A[t][d] = C_td U_d, an [n_d, r_d] matrix
        self.C = [[C(d, t) for d in range(3)] for t in range(self.T)]
        self.A = [[self.C[t][d] @ self.U[d] for d in range(3)] for t in range(self.T)]
        self.w3 = self.w[0][:, None, None] * self.w[1][None, :, None] * self.w[2][None, None, :]

    @classmethod
    def from_system(cls, s, quadrature=("nodal",)):
        return cls(s.x, s.w, s.U, s.theta, s.mu, quadrature=quadrature)


# ----------------------------------------------------------------------------------
# tensor algebra
# ----------------------------------------------------------------------------------
def mode_product(X, M, mode):
    """(X x_mode M)[..., i, ...] = sum_k M[i, k] X[..., k, ...]."""
    return np.moveaxis(np.tensordot(M, X, axes=(1, mode)), 0, mode)


def project(rho, U):
    """Core of rho on the shared basis: G = rho x1 U1^T x2 U2^T x3 U3^T (Eq. TuckerDecompField)."""
    G = rho
    for d in range(3):
        G = mode_product(G, U[d].T, d)
    return G


def expand(G, S: Setup):
    """phi = sum_t mu_t G x1 A_t1 x2 A_t2 x3 A_t3 (Eq. final: a weighted sum over the
    Gaussian terms of tensor products of 1-D convolutions applied to the Tucker core)."""
    phi = None
    for t in range(S.T):
        Y = G
        for d in range(3):
            Y = mode_product(Y, S.A[t][d], d)
        phi = S.mu[t] * Y if phi is None else phi + S.mu[t] * Y
    return phi


def expand_transpose(y, S: Setup):
    """H = sum_t mu_t y x1 A_t1^T x2 A_t2^T x3 A_t3^T (the adjoint of `expand`)."""
    H = None
    for t in range(S.T):
        Y = y
        for d in range(3):
            Y = mode_product(Y, S.A[t][d].T, d)
        H = S.mu[t] * Y if H is None else H + S.mu[t] * Y
    return H


def apply_L(rho, S: Setup):
    """phi = L rho: project onto the core, then the separable Gaussian-sum convolution."""
    return expand(project(rho, S.U), S)


def apply_LT(y, S: Setup):
    """L^T y = (sum_t mu_t y x_d A_td^T) x_d U_d."""
    H = expand_transpose(y, S)
    for d in range(3):
        H = mode_product(H, S.U[d], d)
    return H


def pair_potential(psi_a, psi_b, S: Setup):
    """phi_ab for one orbital pair: rho = psi_a * psi_b, then L rho."""
    return apply_L(np.asarray(psi_a, np.float64) * np.asarray(psi_b, np.float64), S)


# ----------------------------------------------------------------------------------
# the operator, its energy and derivatives
# ----------------------------------------------------------------------------------
def exchange_apply(psi_occ, S: Setup, psi_tgt=None):
    """W_i = - sum_j psi_j * phi_ij for every target i (Eqs. ExchangeOperator, hadam).
    psi_tgt defaults to psi_occ.  Every ordered pair is computed separately."""
    occ = np.asarray(psi_occ, dtype=np.float64)
    tgt = occ if psi_tgt is None else np.asarray(psi_tgt, dtype=np.float64)
    W = np.zeros_like(tgt)
    for i in range(tgt.shape[0]):
        for j in range(occ.shape[0]):
            W[i] -= occ[j] * pair_potential(tgt[i], occ[j], S)
    return W


def exchange_energy(psi_occ, S: Setup, W=None):
    """E_x = 1/2 sum_i sum_x w(x) psi_i(x) W_i(x) (the exchange term of S[phi], alpha = 1)."""
    occ = np.asarray(psi_occ, dtype=np.float64)
    if W is None:
        W = exchange_apply(occ, S)
    return 0.5 * float(np.sum(S.w3[None] * occ * W))


def exchange_energy_grad(psi_occ, S: Setup):
    """(E_x, dE_x/dpsi): dE/dpsi_k = w * W_k - sum_j psi_j * L^T(w * rho_kj)."""
    occ = np.asarray(psi_occ, dtype=np.float64)
    W = exchange_apply(occ, S)
    g = S.w3[None] * W
    for k in range(occ.shape[0]):
        for j in range(occ.shape[0]):
            g[k] -= occ[j] * apply_LT(S.w3 * occ[k] * occ[j], S)
    return exchange_energy(occ, S, W), g


def exchange_apply_vjp(psi_occ, psi_tgt, grad_out, S: Setup):
    """(grad_occ, grad_tgt) of f = sum_k <grad_out_k, W_k> (plain sum over grid points)."""
    occ = np.asarray(psi_occ, dtype=np.float64)
    tgt = np.asarray(psi_tgt, dtype=np.float64)
    Wb = np.asarray(grad_out, dtype=np.float64)
    g_occ = np.zeros_like(occ)
    g_tgt = np.zeros_like(tgt)
    for k in range(tgt.shape[0]):
        for j in range(occ.shape[0]):
            zeta = apply_LT(Wb[k] * occ[j], S)
            g_tgt[k] -= occ[j] * zeta
            g_occ[j] -= Wb[k] * pair_potential(tgt[k], occ[j], S) + tgt[k] * zeta
    return g_occ, g_tgt


# ----------------------------------------------------------------------------------
# per-pair Tucker bases: sequentially truncated HOSVD of every pair density (Eq. TuckerDecompField)
# ----------------------------------------------------------------------------------
def sthosvd(rho, ranks):
    """Sequentially truncated HOSVD: for d = 1, 2, 3 in turn, U_d = the r_d leading eigenvectors
    (eigenvalues descending) of the Gram matrix of the mode-d unfolding of the current tensor,
    which is then projected onto them in mode d.  Returns (G, [U1, U2, U3]) with
    rho ~ G x1 U1 x2 U2 x3 U3."""
    G = np.asarray(rho, dtype=np.float64)
    Us = []
    for d in range(3):
        M = np.moveaxis(G, d, 0).reshape(G.shape[d], -1)
        ev, V = np.linalg.eigh(M @ M.T)
        U = V[:, ::-1][:, : int(ranks[d])]
        G = mode_product(G, U.T, d)
        Us.append(U)
    return G, Us


def pair_potential_sthosvd(psi_a, psi_b, S: Setup, ranks):
    """phi_ab with the pair's own Tucker bases (Eqs. TuckerDecompField, final):
    phi = sum_t mu_t G x1 (C_t1 U1) x2 (C_t2 U2) x3 (C_t3 U3) with (G, U_d) = sthosvd(rho_ab)."""
    G, Us = sthosvd(np.asarray(psi_a, np.float64) * np.asarray(psi_b, np.float64), ranks)
    phi_p = np.zeros(np.shape(psi_a))
    for t in range(S.T):
        Yp = G
        for d in range(3):
            Yp = mode_product(Yp, S.C[t][d] @ Us[d], d)
        phi_p += S.mu[t] * Yp
    return phi_p


def exchange_apply_sthosvd(psi_occ, S: Setup, ranks, psi_tgt=None):
    """W_i = - sum_j psi_j * phi_ij with per-pair Tucker bases of ranks (r1, r2, r3)."""
    occ = np.asarray(psi_occ, dtype=np.float64)
    tgt = occ if psi_tgt is None else np.asarray(psi_tgt, dtype=np.float64)
    W = np.zeros_like(tgt)
    for i in range(tgt.shape[0]):
        for j in range(occ.shape[0]):
            W[i] -= occ[j] * pair_potential_sthosvd(tgt[i], occ[j], S, ranks)
    return W


# ----------------------------------------------------------------------------------
# two-sided (Galerkin) projection of the convolution onto the Tucker basis
# ----------------------------------------------------------------------------------
def galerkin_core_matrices(S: Setup):
    """B[t][d] = U_d^T D_d C_td U_d = U_d^T D_d A_td, an [r_d, r_d] matrix: the 1-D convolution
    of Eq. final compressed onto the basis on both sides (D_d = diag(w_d)).  With the nodal
    quadrature D_d C_td = D_d K_td D_d, so B[t][d] is symmetric and positive semi-definite."""
    return [[S.U[d].T @ (S.w[d][:, None] * S.A[t][d]) for d in range(3)] for t in range(S.T)]


def galerkin_core_convolve(G, S: Setup, B=None):
    """H = sum_t mu_t G x1 B_t1 x2 B_t2 x3 B_t3 (the core-space convolution)."""
    B = galerkin_core_matrices(S) if B is None else B
    Hc = np.zeros_like(G)
    for t in range(S.T):
        Yc = G
        for d in range(3):
            Yc = mode_product(Yc, B[t][d], d)
        Hc += S.mu[t] * Yc
    return Hc


def apply_L_galerkin(rho, S: Setup, B=None):
    """phi = P^* C P rho, where P = (x)_d U_d U_d^T projects onto the basis, C is the separable
    Gaussian-sum convolution and P^* = D^-1 P D is the adjoint of P in the w inner product:
    phi = (sum_t mu_t G x_d B_td) x_d (D_d^-1 U_d) with G = rho x_d U_d^T."""
    H = galerkin_core_convolve(project(rho, S.U), S, B)
    for d in range(3):
        H = mode_product(H, S.U[d] / S.w[d][:, None], d)
    return H


def exchange_apply_galerkin(psi_occ, S: Setup, psi_tgt=None):
    """W_i = - sum_j psi_j * (P^* C P)(psi_i psi_j): the exchange action with the two-sided
    projection (every ordered pair separately)."""
    occ = np.asarray(psi_occ, dtype=np.float64)
    tgt = occ if psi_tgt is None else np.asarray(psi_tgt, dtype=np.float64)
    B = galerkin_core_matrices(S)
    W = np.zeros_like(tgt)
    for i in range(tgt.shape[0]):
        for j in range(occ.shape[0]):
            W[i] -= occ[j] * apply_L_galerkin(tgt[i] * occ[j], S, B)
    return W


def exchange_energy_galerkin(psi_occ, S: Setup):
    """E_x = - 1/2 sum_ij <G_ij, sum_t mu_t G_ij x_d B_td>, evaluated in core space: O(T r^4) per
    pair instead of a reconstruction on the grid."""
    occ = np.asarray(psi_occ, dtype=np.float64)
    B = galerkin_core_matrices(S)
    E = 0.0
    for i in range(occ.shape[0]):
        for j in range(occ.shape[0]):
            G = project(occ[i] * occ[j], S.U)
            E -= 0.5 * float(np.sum(G * galerkin_core_convolve(G, S, B)))
    return E


# ----------------------------------------------------------------------------------
# adaptively compressed exchange (section "ACE implementation": Eqs. eta, ace1)
# ----------------------------------------------------------------------------------
def ace_projectors(psi_occ, S: Setup, W=None):
    """(xi, M) of the ACE operator V_ACE(r, r') = - sum_k xi_k(r) xi_k(r'):
    W_i = K psi_i (Eq. ace1), M_ij = <psi_i, W_j>_w (the integral by the grid's quadrature),
    M = - L L^T (Cholesky), xi_k = sum_i W_i (L^-1)_ki (Eq. eta).  The paper is silent on the
    asymmetry of M that a truncated Tucker rank leaves; M is symmetrised, (M + M^T) / 2, before
    the factorisation."""
    occ = np.asarray(psi_occ, dtype=np.float64)
    if W is None:
        W = exchange_apply(occ, S)
    N = occ.shape[0]
    M = np.array([[np.sum(S.w3 * occ[i] * W[j]) for j in range(N)] for i in range(N)])
    Ms = 0.5 * (M + M.T)
    L = np.linalg.cholesky(-Ms)
    Linv = np.linalg.inv(L)
    xi = np.tensordot(Linv, W, axes=(1, 0))          # xi[k] = sum_i Linv[k, i] W[i]
    return xi, M


def ace_apply(xi, psi, S: Setup):
    """V_ACE psi_a = - sum_k xi_k <xi_k, psi_a>_w for every orbital psi_a of the block."""
    psi = np.asarray(psi, dtype=np.float64)
    C = np.array([[np.sum(S.w3 * xi[k] * psi[a]) for a in range(psi.shape[0])] for k in range(xi.shape[0])])
    return -np.tensordot(C, xi, axes=(0, 0))          # [a] = - sum_k C[k, a] xi[k]


# ----------------------------------------------------------------------------------
# transfer between the unstructured and the structured finite-element bases (Eq. interpolate)
# ----------------------------------------------------------------------------------
def lagrange_basis(nodes, x):
    """L[k, j] = value at x[j] of the 1-D Lagrange polynomial that is 1 at nodes[k] and 0 at the
    other nodes."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    L = np.ones((nodes.size, x.size))
    for k in range(nodes.size):
        for m in range(nodes.size):
            if m != k:
                L[k] *= (x - nodes[m]) / (nodes[k] - nodes[m])
    return L


def transfer_u_to_s(psi_u, X, conn, order, xs):
    """psi_s[i, a] = sum_b N_ab psi_u[b, i] (Eq. interpolate): every node a of the structured
    grid xs (three 1-D node arrays) is interpolated from the unstructured cell that contains
    it, N_ab being the value of that cell's shape function of node b at a.  Cells are
    tensor-product Lagrange elements of `order` on axis-aligned boxes (local node (lx, ly, lz) at
    index (lx (order+1) + ly) (order+1) + lz).  Where several cells contain a node (a shared face,
    or a face with hanging nodes) the cell listed first is used.  psi_u: [n_nodes, N];
    returns [N, n1, n2, n3]."""
    p = int(order)
    psi_u = np.asarray(psi_u, dtype=np.float64)
    xs = [np.asarray(v, dtype=np.float64) for v in xs]
    n = [v.size for v in xs]
    P = np.stack(np.meshgrid(*xs, indexing="ij"), axis=-1).reshape(-1, 3)     # [n1 n2 n3, 3]
    out = np.zeros((psi_u.shape[1], P.shape[0]))
    done = np.zeros(P.shape[0], dtype=bool)
    for c in range(conn.shape[0]):
        nodes = X[conn[c]].reshape(p + 1, p + 1, p + 1, 3)
        ax = [nodes[:, 0, 0, 0], nodes[0, :, 0, 1], nodes[0, 0, :, 2]]      # 1-D node coordinates
        lo = np.array([a.min() for a in ax])
        hi = np.array([a.max() for a in ax])
        tol = 1e-9 * (hi - lo)
        inside = ~done & np.all((P >= lo - tol) & (P <= hi + tol), axis=1)
        idx = np.nonzero(inside)[0]
        if idx.size == 0:
            continue
        Lx, Ly, Lz = (lagrange_basis(ax[d], P[idx, d]) for d in range(3))
        N = (Lx[:, None, None, :] * Ly[None, :, None, :] * Lz[None, None, :, :]).reshape(-1, idx.size)
        out[:, idx] = (N.T @ psi_u[conn[c]]).T
        done[idx] = True
    if not done.all():
        raise ValueError("the unstructured mesh does not cover every structured node")
    return out.reshape(psi_u.shape[1], *n)


def transfer_s_to_u(psi_s, xs, order, X):
    """psi_u[b, i] = sum_a M_ba psi_s[i, a]: every unstructured node b is interpolated from the
    structured element that contains it, the structured mesh being the tensor product of 1-D
    Lagrange elements of `order` on the nodes xs (element e of an axis holds nodes
    order e .. order e + order).  psi_s: [N, n1, n2, n3]; returns [n_nodes, N]."""
    p = int(order)
    psi_s = np.asarray(psi_s, dtype=np.float64)
    xs = [np.asarray(v, dtype=np.float64) for v in xs]
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros((X.shape[0], psi_s.shape[0]))
    for b in range(X.shape[0]):
        sel, wts = [], []
        for d in range(3):
            x = xs[d]
            nel = (x.size - 1) // p
            e = 0
            while e < nel - 1 and X[b, d] > x[p * (e + 1)]:
                e += 1
            nodes = x[p * e: p * (e + 1) + 1]
            sel.append(np.arange(p * e, p * e + p + 1))
            wts.append(lagrange_basis(nodes, [X[b, d]])[:, 0])
        block = psi_s[:, sel[0][:, None, None], sel[1][None, :, None], sel[2][None, None, :]]
        W3 = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
        out[b] = np.tensordot(block, W3, axes=([1, 2, 3], [0, 1, 2]))
    return out


# ----------------------------------------------------------------------------------
# independent references for the pins
# ----------------------------------------------------------------------------------
def direct_gaussian_kernel_potential(rho, x, w, theta, mu):
    """Brute force O(n^6 T): phi(r) = sum_{r'} w(r') rho(r') sum_t mu_t exp(-theta_t |r - r'|^2),
    with 3-D distances and product weights -- no separation of variables."""
    X = np.stack(np.meshgrid(*x, indexing="ij"), -1).reshape(-1, 3)
    wq = (w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]).reshape(-1)
    q = wq * np.asarray(rho, np.float64).reshape(-1)
    d2 = np.sum((X[:, None, :] - X[None, :, :]) ** 2, axis=-1)
    K = np.zeros_like(d2)
    for th, m in zip(theta, mu):
        K += m * np.exp(-th * d2)
    return (K @ q).reshape(np.shape(rho))


def direct_coulomb_potential(rho, x, w):
    """Brute force phi(r) = sum_{r' != r} w(r') rho(r') / |r - r'| (self term skipped)."""
    X = np.stack(np.meshgrid(*x, indexing="ij"), -1).reshape(-1, 3)
    wq = (w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]).reshape(-1)
    q = wq * np.asarray(rho, np.float64).reshape(-1)
    d = np.sqrt(np.sum((X[:, None, :] - X[None, :, :]) ** 2, axis=-1))
    np.fill_diagonal(d, np.inf)
    return ((1.0 / d) @ q).reshape(np.shape(rho))


def gaussian_charge_potential(a, r):
    """Potential of the unit charge (a/pi)^{3/2} exp(-a r^2): erf(sqrt(a) r) / r,
    with the limit 2 sqrt(a/pi) at r = 0."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    small = r < 1e-12
    from math import erf
    out[~small] = np.vectorize(erf)(math.sqrt(a) * r[~small]) / r[~small]
    out[small] = 2.0 * math.sqrt(a / math.pi)
    return out


def gaussian_kernel_charge_potential(a, r, theta, mu):
    """Continuous convolution of the unit Gaussian charge with the Gaussian-sum kernel:
    sum_t mu_t (a / (a + theta_t))^{3/2} exp(-a theta_t r^2 / (a + theta_t))."""
    r = np.asarray(r, dtype=np.float64)
    out = np.zeros_like(r)
    for th, m in zip(theta, mu):
        out += m * (a / (a + th)) ** 1.5 * np.exp(-a * th * r * r / (a + th))
    return out

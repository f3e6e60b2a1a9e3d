"""The pins must catch plausible mistakes in the oracle.  One at a time, a mistake is planted in
a copy of the oracle's source (one changed line, loaded as a separate module on the CPU; the
oracle itself is untouched) and the pins of test_oracle_pins run against that copy: at least
one of them must fail.  The mistakes are the kinds a reader checking the oracle against the
paper would look for: a wrong sign or factor, a dropped term or weight, a transposed or
skipped operand, a wrong index."""
import inspect
import os
import types

import pytest

import oracle
import test_oracle_pins as PINS

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "__init__.py")).read()

MUTATIONS = [
    ("W has the wrong sign",
     "            W[i] -= occ[j] * pair_potential(tgt[i], occ[j], S)",
     "            W[i] += occ[j] * pair_potential(tgt[i], occ[j], S)"),
    ("W multiplies by psi_i instead of psi_j",
     "            W[i] -= occ[j] * pair_potential(tgt[i], occ[j], S)",
     "            W[i] -= tgt[i] * pair_potential(tgt[i], occ[j], S)"),
    ("E_x without the factor 1/2",
     "    return 0.5 * float(np.sum(S.w3[None] * occ * W))",
     "    return 1.0 * float(np.sum(S.w3[None] * occ * W))"),
    ("E_x without the quadrature weights",
     "    return 0.5 * float(np.sum(S.w3[None] * occ * W))",
     "    return 0.5 * float(np.sum(occ * W))"),
    ("energy gradient without the L^T term",
     "            g[k] -= occ[j] * apply_LT(S.w3 * occ[k] * occ[j], S)",
     "            pass"),
    ("energy gradient without the weight inside L^T",
     "            g[k] -= occ[j] * apply_LT(S.w3 * occ[k] * occ[j], S)",
     "            g[k] -= occ[j] * apply_LT(occ[k] * occ[j], S)"),
    ("VJP of the occupied block without the potential term",
     "            g_occ[j] -= Wb[k] * pair_potential(tgt[k], occ[j], S) + tgt[k] * zeta",
     "            g_occ[j] -= tgt[k] * zeta"),
    ("VJP of the occupied block without the L^T term",
     "            g_occ[j] -= Wb[k] * pair_potential(tgt[k], occ[j], S) + tgt[k] * zeta",
     "            g_occ[j] -= Wb[k] * pair_potential(tgt[k], occ[j], S)"),
    ("VJP of the targets with the wrong sign",
     "            g_tgt[k] -= occ[j] * zeta",
     "            g_tgt[k] += occ[j] * zeta"),
    ("expansion drops mu_t",
     "        phi = S.mu[t] * Y if phi is None else phi + S.mu[t] * Y",
     "        phi = Y if phi is None else phi + Y"),
    ("expansion applies mu_t twice",
     "        phi = S.mu[t] * Y if phi is None else phi + S.mu[t] * Y",
     "        phi = S.mu[t] ** 2 * Y if phi is None else phi + S.mu[t] ** 2 * Y"),
    ("adjoint expansion drops mu_t",
     "        H = S.mu[t] * Y if H is None else H + S.mu[t] * Y",
     "        H = Y if H is None else H + Y"),
    ("expansion keeps only the first Gaussian term",
     "    for t in range(S.T):\n        Y = G\n",
     "    for t in range(1):\n        Y = G\n"),
    ("FE elements stepped by order + 1 nodes instead of order",
     "        nodes = x[p * e: p * e + p + 1]",
     "        nodes = x[(p + 1) * e: (p + 1) * e + p + 1] if (p + 1) * e + p < len(x) else x[p * e: p * e + p + 1]"),
    ("FE quadrature without the element Jacobian",
     "        C[:, p * e: p * e + p + 1] += (K * (half * wq)[None, :]) @ L.T",
     "        C[:, p * e: p * e + p + 1] += (K * wq[None, :]) @ L.T"),
    ("FE basis function of the wrong node",
     "                    L[k] *= (xq - nodes[m]) / (nodes[k] - nodes[m])",
     "                    L[k] *= (xq - nodes[m]) / (nodes[m] - nodes[k])"),
    ("1-D kernel in |x - x'| instead of its square",
     "    return np.exp(-float(theta) * d * d) * w[None, :]",
     "    return np.exp(-float(theta) * np.abs(d)) * w[None, :]"),
    ("1-D convolution without quadrature weights",
     "    return np.exp(-float(theta) * d * d) * w[None, :]",
     "    return np.exp(-float(theta) * d * d)"),
    ("1-D convolution with the weight on the output node",
     "    return np.exp(-float(theta) * d * d) * w[None, :]",
     "    return np.exp(-float(theta) * d * d) * w[:, None]"),
    ("A_td built from the transposed convolution",
     "            return conv_matrix(self.x[d], self.w[d], self.theta[t])",
     "            return conv_matrix(self.x[d], self.w[d], self.theta[t]).T"),
    ("projection skips mode 3",
     "    for d in range(3):\n        G = mode_product(G, U[d].T, d)",
     "    for d in range(2):\n        G = mode_product(G, U[d].T, d)"),
    ("L^T does not map the core back with U_d",
     "    for d in range(3):\n        H = mode_product(H, S.U[d], d)\n    return H",
     "    return H"),
    ("ACE projectors with L instead of L^-1",
     "    xi = np.tensordot(Linv, W, axes=(1, 0))          # xi[k] = sum_i Linv[k, i] W[i]",
     "    xi = np.tensordot(L, W, axes=(1, 0))          # xi[k] = sum_i Linv[k, i] W[i]"),
    ("ACE projectors with L^-T instead of L^-1",
     "    xi = np.tensordot(Linv, W, axes=(1, 0))          # xi[k] = sum_i Linv[k, i] W[i]",
     "    xi = np.tensordot(Linv.T, W, axes=(1, 0))          # xi[k] = sum_i Linv[k, i] W[i]"),
    ("ACE operator with the wrong sign",
     "    return -np.tensordot(C, xi, axes=(0, 0))          # [a] = - sum_k C[k, a] xi[k]",
     "    return np.tensordot(C, xi, axes=(0, 0))          # [a] = - sum_k C[k, a] xi[k]"),
    ("ACE overlap M without quadrature weights",
     "    M = np.array([[np.sum(S.w3 * occ[i] * W[j]) for j in range(N)] for i in range(N)])",
     "    M = np.array([[np.sum(occ[i] * W[j]) for j in range(N)] for i in range(N)])"),
    ("ACE without symmetrising M",
     "    Ms = 0.5 * (M + M.T)",
     "    Ms = M"),
    ("Galerkin reconstruction without the inverse weights",
     "        H = mode_product(H, S.U[d] / S.w[d][:, None], d)",
     "        H = mode_product(H, S.U[d], d)"),
    ("Galerkin core matrices without the weights",
     "    return [[S.U[d].T @ (S.w[d][:, None] * S.A[t][d]) for d in range(3)] for t in range(S.T)]",
     "    return [[S.U[d].T @ S.A[t][d] for d in range(3)] for t in range(S.T)]"),
    ("Galerkin core convolution drops mu_t",
     "        Hc += S.mu[t] * Yc",
     "        Hc += Yc"),
    ("Galerkin energy without the factor 1/2",
     "            E -= 0.5 * float(np.sum(G * galerkin_core_convolve(G, S, B)))",
     "            E -= float(np.sum(G * galerkin_core_convolve(G, S, B)))"),
    ("transfer: Lagrange basis of the wrong node",
     "                L[k] *= (x - nodes[m]) / (nodes[k] - nodes[m])",
     "                L[k] *= (x - nodes[m]) / (nodes[m] - nodes[k])"),
    ("transfer to the grid with the y and z node coordinates swapped",
     "        ax = [nodes[:, 0, 0, 0], nodes[0, :, 0, 1], nodes[0, 0, :, 2]]      # 1-D node coordinates",
     "        ax = [nodes[:, 0, 0, 0], nodes[0, 0, :, 2], nodes[0, :, 0, 1]]      # 1-D node coordinates"),
    ("transfer to the mesh with elements stepped by order + 1 nodes",
     "            nodes = x[p * e: p * (e + 1) + 1]",
     "            nodes = x[(p + 1) * e: (p + 1) * e + p + 1] if (p + 1) * e + p < x.size else x[p * e: p * (e + 1) + 1]"),
    ("transfer to the mesh always from the first element",
     "            while e < nel - 1 and X[b, d] > x[p * (e + 1)]:",
     "            while False:"),
    ("STHOSVD keeps the trailing eigenvectors",
     "        U = V[:, ::-1][:, : int(ranks[d])]",
     "        U = V[:, : int(ranks[d])]"),
    ("STHOSVD computes every mode's Gram matrix from the original density",
     "        G = mode_product(G, U.T, d)\n        Us.append(U)",
     "        Us.append(U)"),
    ("per-pair potential drops mu_t",
     "        phi_p += S.mu[t] * Yp",
     "        phi_p += Yp"),
    ("per-pair potential with the convolution matrix transposed",
     "            Yp = mode_product(Yp, S.C[t][d] @ Us[d], d)",
     "            Yp = mode_product(Yp, S.C[t][d].T @ Us[d], d)"),
    ("quadrature weight of mode 2 on mode 3",
     "        self.w3 = self.w[0][:, None, None] * self.w[1][None, :, None] * self.w[2][None, None, :]",
     "        self.w3 = self.w[0][:, None, None] * self.w[2][None, None, :] * self.w[2][None, None, :]"),
]


def _pins():
    """Every pin of test_oracle_pins, with the first parameter set of the parametrized ones."""
    calls = []
    for name, fn in inspect.getmembers(PINS, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        kw = {}
        if marks:
            names = [a.strip() for a in marks[0].args[0].split(",")]
            first = marks[0].args[1][0]
            kw = dict(zip(names, first if len(names) > 1 else (first,)))
        calls.append((name, fn, kw))
    return calls


def _mutant(old, new):
    assert SRC.count(old) == 1, old
    mod = types.ModuleType("oracle_with_a_planted_mistake")
    exec(compile(SRC.replace(old, new), mod.__name__, "exec"), mod.__dict__)
    return mod


def test_pins_pass_on_the_oracle_itself(monkeypatch):
    """The control: the same calls on the unchanged oracle all pass (so a failure below comes
    from the planted mistake, not from the harness)."""
    monkeypatch.setattr(PINS, "O", oracle)
    for name, fn, kw in _pins():
        fn(**kw)


@pytest.mark.parametrize("what,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_a_planted_mistake_fails_a_pin(monkeypatch, what, old, new):
    monkeypatch.setattr(PINS, "O", _mutant(old, new))
    for name, fn, kw in _pins():
        try:
            fn(**kw)
        except Exception:
            return
    pytest.fail(f"no pin fails with the planted mistake: {what}")

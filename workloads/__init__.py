"""Seeded synthetic inputs for the Tucker-tensor exchange hot path.

This module builds the inputs that both the FP64 oracle and the CUDA path receive:
1-D grids with trapezoid weights, orthonormal Gaussian-sum orbitals, the shared
Tucker basis U_d and the Gaussian-sum coefficients (theta_t, mu_t) of 1/r.  It
holds none of the exchange arithmetic itself (no pair densities, projections,
convolutions or Hadamard products): those live in ``oracle/`` and in the CUDA
library, which share no code.

The paper's Pt and TiO2 wavefunctions, finite-element meshes and pseudopotentials
are not available, so orbitals are random sums of s-type Gaussians placed on
cluster-shaped centre sets, orthonormalised in the trapezoid inner product and
rounded to float32 once.  Both paths then use the same float32 values.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "uniform_grid", "fcc_cluster", "rutile_cluster", "gaussian_sum_orbitals",
    "lowdin_orthonormalise", "density_hosvd_basis", "exp_sum_inverse_r",
    "System", "make_system", "make_system_on_device", "config_tio2_on_device", "CONFIGS",
    "batched_system_specs", "batched_system_args", "fe_mesh", "gaussian_sum_at_points",
]


# ----------------------------------------------------------------------------------
# grids
# ----------------------------------------------------------------------------------
def uniform_grid(n: int, L: float):
    """Endpoint-inclusive uniform nodes on [-L, L] with trapezoid weights (h, ends h/2)."""
    if n < 2:
        raise ValueError("a trapezoid grid needs at least 2 nodes")
    x = np.linspace(-L, L, n)
    h = 2.0 * L / (n - 1)
    w = np.full(n, h)
    w[0] = w[-1] = 0.5 * h
    return x, w


# ----------------------------------------------------------------------------------
# centre sets shaped like the paper's clusters
# ----------------------------------------------------------------------------------
def fcc_cluster(count: int, spacing: float) -> np.ndarray:
    """The `count` fcc lattice points (nearest-neighbour distance `spacing`) closest to
    the origin, re-centred on their centroid."""
    a = spacing * math.sqrt(2.0)
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    m = int(math.ceil(count ** (1 / 3))) + 2
    rng = np.arange(-m, m + 1)
    cells = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    pts = (cells[:, None, :] + basis[None]).reshape(-1, 3) * a
    off = np.array([0.11, 0.07, 0.03]) * a          # break distance ties deterministically
    order = np.lexsort((pts[:, 2], pts[:, 1], pts[:, 0], np.round(np.linalg.norm(pts - off, axis=1), 9)))
    sel = pts[order[:count]]
    return sel - sel.mean(0)


def rutile_cluster(count: int, a: float = 8.68, c: float = 5.59, u: float = 0.3) -> np.ndarray:
    """The `count` sites of a rutile-like TiO2 supercell (2 Ti + 4 O per cell) closest to
    the origin, re-centred on their centroid."""
    frac = np.array([[0, 0, 0], [.5, .5, .5],
                     [u, u, 0], [1 - u, 1 - u, 0], [.5 + u, .5 - u, .5], [.5 - u, .5 + u, .5]])
    m = int(math.ceil((count / 6) ** (1 / 3))) + 3
    rng = np.arange(-m, m + 1)
    cells = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    pts = (cells[:, None, :] + frac[None]).reshape(-1, 3) * np.array([a, a, c])
    off = np.array([0.013, 0.007, 0.003])
    order = np.lexsort((pts[:, 2], pts[:, 1], pts[:, 0], np.round(np.linalg.norm(pts - off, axis=1), 9)))
    sel = pts[order[:count]]
    return sel - sel.mean(0)


# ----------------------------------------------------------------------------------
# orbitals
# ----------------------------------------------------------------------------------
def gaussian_sum_orbitals(grids, centres, exps, coefs, dtype=np.float64):
    """psi_i(x,y,z) = sum_k coefs[i,k] * exp(-exps[i,k] * |r - centres[i,k]|^2).

    grids: three 1-D node arrays; centres: [N, K, 3]; exps, coefs: [N, K].
    Each Gaussian is separable, so an orbital is a sum of K rank-1 tensors.
    Returns an array [N, n1, n2, n3].
    """
    x1, x2, x3 = (np.asarray(g, dtype=np.float64) for g in grids)
    N, K = exps.shape
    out = np.empty((N, x1.size, x2.size, x3.size), dtype=dtype)
    for i in range(N):
        a = exps[i][:, None]
        ex = coefs[i][:, None] * np.exp(-a * (x1[None, :] - centres[i, :, 0:1]) ** 2)   # [K, n1]
        ey = np.exp(-a * (x2[None, :] - centres[i, :, 1:2]) ** 2)                         # [K, n2]
        ez = np.exp(-a * (x3[None, :] - centres[i, :, 2:3]) ** 2)                         # [K, n3]
        t = (ex[:, :, None] * ey[:, None, :]).reshape(K, -1)                             # [K, n1 n2]
        out[i] = (t.T @ ez).reshape(x1.size, x2.size, x3.size)
    return out


def lowdin_orthonormalise(psi: np.ndarray, weights) -> np.ndarray:
    """Psi <- Psi S^{-1/2} with S_ij = sum_x w(x) psi_i(x) psi_j(x), in float64."""
    N = psi.shape[0]
    w1, w2, w3 = (np.asarray(v, dtype=np.float64) for v in weights)
    w3d = (w1[:, None, None] * w2[None, :, None] * w3[None, None, :]).reshape(-1)
    P = psi.reshape(N, -1).astype(np.float64)
    S = (P * w3d[None, :]) @ P.T
    ev, V = np.linalg.eigh(0.5 * (S + S.T))
    if ev.min() <= 1e-12 * ev.max():
        raise ValueError("orbitals are numerically linearly dependent")
    X = (V * ev[None, :] ** -0.5) @ V.T
    return (X @ P).reshape(psi.shape)


def density_hosvd_basis(psi: np.ndarray, ranks):
    """Shared Tucker basis: for each mode d, the r_d leading left singular vectors of
    the mode-d unfolding of rho_tot = sum_i psi_i^2 on nodal values (no weights).
    Column signs are fixed so the largest-magnitude entry of each column is positive."""
    rho = np.zeros(psi.shape[1:], dtype=np.float64)
    for p in psi:
        rho += p.astype(np.float64) ** 2
    Us = []
    for d in range(3):
        M = np.moveaxis(rho, d, 0).reshape(rho.shape[d], -1)
        ev, V = np.linalg.eigh(M @ M.T)
        V = V[:, ::-1][:, : ranks[d]]
        s = np.sign(V[np.argmax(np.abs(V), axis=0), np.arange(V.shape[1])])
        Us.append(np.ascontiguousarray(V * s[None, :]))
    return Us


# ----------------------------------------------------------------------------------
# Gaussian-sum coefficients of 1/r (the canonical approximation of the paper's Eq. gauss)
# ----------------------------------------------------------------------------------
@functools.lru_cache(maxsize=64)
def _exp_sum_cached(T: int, r_min: float, r_max: float):
    # 1/r = (2/sqrt(pi)) * int_R exp(-r^2 e^{2s} + s) ds.  The trapezoid (sinc) rule on
    # s_t = s_hi - (T-1-t) * delta gives theta_t = e^{2 s_t}, mu_t = (2/sqrt(pi)) delta e^{s_t}.
    # Below the lowest node exp(-r^2 e^{2s}) ~ 1 on [r_min, r_max], so the rest of the rule
    # there is a geometric series that is folded into mu_0.  (delta, s_hi) are picked by a
    # coarse-then-fine grid search on the maximum relative error over [r_min, r_max].
    rs = np.geomspace(r_min, r_max, 1200)
    c = 2.0 / math.sqrt(math.pi)

    def build(delta, s_hi_off):
        s = (-math.log(r_min) + s_hi_off) - delta * np.arange(T)[::-1]
        th = np.exp(2.0 * s)
        mu = c * delta * np.exp(s)
        mu[0] += c * delta * math.exp(s[0]) * math.exp(-delta) / (1.0 - math.exp(-delta))
        return th, mu

    def err(delta, s_hi_off):
        th, mu = build(delta, s_hi_off)
        return float(np.max(np.abs(rs * (np.exp(-np.outer(rs * rs, th)) @ mu) - 1.0)))

    best = None
    for delta in np.linspace(0.15, 1.5, 28):
        for off in np.linspace(-0.5, 3.0, 15):
            e = err(delta, off)
            if best is None or e < best[0]:
                best = (e, delta, off)
    _, d0, o0 = best
    for delta in np.linspace(d0 - 0.05, d0 + 0.05, 21):
        if delta <= 0.05:
            continue
        for off in np.linspace(o0 - 0.25, o0 + 0.25, 11):
            e = err(delta, off)
            if e < best[0]:
                best = (e, delta, off)
    e, d, o = best
    th, mu = build(d, o)
    return th, mu, e


def exp_sum_inverse_r(T: int, r_min: float, r_max: float):
    """(theta[T], mu[T], max relative error on [r_min, r_max]) with
    1/r ~ sum_t mu_t exp(-theta_t r^2); theta_t, mu_t > 0, theta ascending."""
    if T < 1 or not (0 < r_min < r_max):
        raise ValueError("need T >= 1 and 0 < r_min < r_max")
    th, mu, e = _exp_sum_cached(int(T), float(r_min), float(r_max))
    return th.copy(), mu.copy(), e


# ----------------------------------------------------------------------------------
# whole systems
# ----------------------------------------------------------------------------------
@dataclass
class System:
    name: str
    x: list            # three float64 node arrays
    w: list            # three float64 trapezoid-weight arrays
    U: list            # three float64 [n_d, r_d] orthonormal bases
    theta: np.ndarray  # float64 [T]
    mu: np.ndarray     # float64 [T]
    psi: np.ndarray    # float32 [N, n1, n2, n3]
    fit_error: float   # max relative error of the Gaussian sum vs 1/r on [r1, r2]
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return tuple(len(v) for v in self.x)

    @property
    def r(self):
        return tuple(u.shape[1] for u in self.U)

    @property
    def T(self):
        return len(self.theta)


def _fit_range(xs, Ls):
    h = min(float(np.min(np.diff(v))) for v in xs)
    diag = math.sqrt(sum((2 * L) ** 2 for L in Ls))
    return h, diag


def make_system(name: str, n: int, L: float, n_orb: int, rank: int, T: int, seed: int,
                centres: np.ndarray, n_gauss_per_centre: int, exp_range, centres_per_orbital=None,
                full_rank=False) -> System:
    """Build one synthetic system.  Orbital i is a sum over its centres of
    `n_gauss_per_centre` s-Gaussians with exponents U[exp_range] and N(0,1) coefficients."""
    rng = np.random.default_rng(seed)
    x, w = uniform_grid(n, L)
    xs, ws = [x, x.copy(), x.copy()], [w, w.copy(), w.copy()]
    C = centres.shape[0]
    if centres_per_orbital is None:
        idx = np.broadcast_to(np.arange(C), (n_orb, C))
    else:
        idx = np.stack([rng.choice(C, size=centres_per_orbital, replace=False) for _ in range(n_orb)])
    k = idx.shape[1] * n_gauss_per_centre
    cen = np.repeat(centres[idx], n_gauss_per_centre, axis=1).reshape(n_orb, k, 3)
    exps = rng.uniform(exp_range[0], exp_range[1], size=(n_orb, k))
    coefs = rng.standard_normal(size=(n_orb, k))
    psi64 = gaussian_sum_orbitals(xs, cen, exps, coefs)
    psi64 = lowdin_orthonormalise(psi64, ws)
    psi = psi64.astype(np.float32)
    del psi64
    if full_rank:
        U = [np.eye(n) for _ in range(3)]
    else:
        U = density_hosvd_basis(psi, (rank, rank, rank))
    r1, r2 = _fit_range(xs, (L, L, L))
    theta, mu, ferr = exp_sum_inverse_r(T, r1, r2)
    return System(name, xs, ws, U, theta, mu, psi, ferr,
                  meta=dict(seed=seed, L=L, n_orb=n_orb, rank=rank, fit_range=(r1, r2)))


def make_system_on_device(name: str, n: int, L: float, n_orb: int, rank: int, T: int, seed: int,
                          centres: np.ndarray, n_gauss_per_centre: int, exp_range, centres_per_orbital=None,
                          device="cuda", chunk=1 << 20):
    """make_system with the orbital arithmetic on a torch device, for blocks too large for the
    host (the TiO2-shaped block: 1842 orbitals of 160^3 points, 60 GB in float64): the same
    seeded draws, Gaussian sums, Loewdin orthonormalisation and density HOSVD, in float64 on the
    device.  Returns (System with psi=None, psi as a float32 device tensor [N, n, n, n])."""
    import torch
    rng = np.random.default_rng(seed)
    x, w = uniform_grid(n, L)
    xs, ws = [x, x.copy(), x.copy()], [w, w.copy(), w.copy()]
    C = centres.shape[0]
    if centres_per_orbital is None:
        idx = np.broadcast_to(np.arange(C), (n_orb, C))
    else:
        idx = np.stack([rng.choice(C, size=centres_per_orbital, replace=False) for _ in range(n_orb)])
    k = idx.shape[1] * n_gauss_per_centre
    cen = np.repeat(centres[idx], n_gauss_per_centre, axis=1).reshape(n_orb, k, 3)
    exps = rng.uniform(exp_range[0], exp_range[1], size=(n_orb, k))
    coefs = rng.standard_normal(size=(n_orb, k))
    f64 = dict(dtype=torch.float64, device=device)
    xg = torch.tensor(x, **f64)
    N3 = n ** 3
    P = torch.empty((n_orb, N3), **f64)
    for i in range(n_orb):
        a = torch.tensor(exps[i], **f64)[:, None]
        c = torch.tensor(cen[i], **f64)
        ex = torch.tensor(coefs[i], **f64)[:, None] * torch.exp(-a * (xg[None, :] - c[:, 0:1]) ** 2)
        ey = torch.exp(-a * (xg[None, :] - c[:, 1:2]) ** 2)
        ez = torch.exp(-a * (xg[None, :] - c[:, 2:3]) ** 2)
        t = (ex[:, :, None] * ey[:, None, :]).reshape(k, -1)
        P[i] = (t.T @ ez).reshape(-1)
    wg = torch.tensor(w, **f64)
    w3d = (wg[:, None, None] * wg[None, :, None] * wg[None, None, :]).reshape(-1)
    S = torch.zeros((n_orb, n_orb), **f64)
    for c0 in range(0, N3, chunk):
        Pc = P[:, c0:c0 + chunk]
        S += (Pc * w3d[None, c0:c0 + chunk]) @ Pc.T
    # the small eigenproblems run on the host (LAPACK): the device solver library is not always
    # loadable (e.g. under a profiler's injection)
    ev, V = (v.to(device) for v in torch.linalg.eigh((0.5 * (S + S.T)).cpu()))
    if float(ev.min()) <= 1e-12 * float(ev.max()):
        raise ValueError("orbitals are numerically linearly dependent")
    X = (V * ev[None, :] ** -0.5) @ V.T
    psi = torch.empty((n_orb, N3), dtype=torch.float32, device=device)
    for c0 in range(0, N3, chunk):
        psi[:, c0:c0 + chunk] = (X @ P[:, c0:c0 + chunk]).to(torch.float32)
    del P
    psi = psi.reshape(n_orb, n, n, n)
    rho = torch.zeros((n, n, n), **f64)
    for p in psi:
        rho += p.to(torch.float64) ** 2
    Us = []
    for d in range(3):
        M = torch.movedim(rho, d, 0).reshape(n, -1)
        evd, Vd = (v.to(device) for v in torch.linalg.eigh((M @ M.T).cpu()))
        Vd = Vd.flip(1)[:, :rank].cpu().numpy()
        sgn = np.sign(Vd[np.argmax(np.abs(Vd), axis=0), np.arange(Vd.shape[1])])
        Us.append(np.ascontiguousarray(Vd * sgn[None, :]))
    r1, r2 = _fit_range(xs, (L, L, L))
    theta, mu, ferr = exp_sum_inverse_r(T, r1, r2)
    return (System(name, xs, ws, Us, theta, mu, None, ferr,
                   meta=dict(seed=seed, L=L, n_orb=n_orb, rank=rank, fit_range=(r1, r2))), psi)


def config_tio2_on_device(n=160, L=16.0, n_orb=1842, rank=64, T=45, seed=4, device="cuda"):
    """The TiO2-shaped block of config_tio2, generated on a torch device."""
    return make_system_on_device("tio2", n, L, n_orb, rank, T, seed, rutile_cluster(240), 2, (0.2, 3.0),
                                 centres_per_orbital=16, device=device)


def _small(seed=0, n=32, n_orb=4, rank=16, T=30, L=8.0, full_rank=False):
    rng = np.random.default_rng(seed)
    # orbital i is a sum of 3 Gaussians, each with its own centre
    cen = rng.uniform(-2.0, 2.0, size=(3 * n_orb, 3))
    x, w = uniform_grid(n, L)
    xs, ws = [x, x.copy(), x.copy()], [w, w.copy(), w.copy()]
    exps = rng.uniform(0.3, 2.0, size=(n_orb, 3))
    coefs = rng.standard_normal(size=(n_orb, 3))
    psi = lowdin_orthonormalise(gaussian_sum_orbitals(xs, cen.reshape(n_orb, 3, 3), exps, coefs), ws)
    psi = psi.astype(np.float32)
    U = [np.eye(n) for _ in range(3)] if full_rank else density_hosvd_basis(psi, (rank,) * 3)
    r1, r2 = _fit_range(xs, (L, L, L))
    theta, mu, ferr = exp_sum_inverse_r(T, r1, r2)
    return System("small", xs, ws, U, theta, mu, psi, ferr,
                  meta=dict(seed=seed, L=L, n_orb=n_orb, rank=rank, fit_range=(r1, r2)))


def config_small(**kw) -> System:
    """32^3 on [-8,8]^3, 4 orbitals of 3 s-Gaussians each (exponents U[0.3,2], centres
    U[-2,2]^3, seed 0), Tucker rank 16 from the density HOSVD, 30 Gaussian terms."""
    return _small(**kw)


def config_pt(n=96, L=12.0, n_orb=64, rank=40, T=40, seed=1) -> System:
    """Pt-cluster-shaped block: 96^3 on [-12,12]^3, 64 orbitals over 8 fcc centres
    (spacing 2.6 bohr), 3 Gaussians per centre with exponents U[0.2,3], rank 40, 40 terms."""
    return make_system("pt", n, L, n_orb, rank, T, seed, fcc_cluster(8, 2.6), 3, (0.2, 3.0))


def config_diff(n=64, L=10.0, n_orb=32, rank=32, T=35, seed=2) -> System:
    """Differentiation case: 64^3 on [-10,10]^3, 32 orbitals, rank 32, 35 terms."""
    return make_system("diff", n, L, n_orb, rank, T, seed, fcc_cluster(8, 2.6), 3, (0.2, 3.0))


def config_tio2(n=160, L=16.0, n_orb=1842, rank=64, T=45, seed=4) -> System:
    """TiO2-cluster-shaped scale: 160^3 on [-16,16]^3, 1842 orbitals, each a Gaussian sum
    over 16 of 240 rutile-like centres with 2 exponents U[0.2,3] per centre; rank 64, 45 terms.
    (float32 psi alone is 30 GB; build it only where the memory exists.)"""
    return make_system("tio2", n, L, n_orb, rank, T, seed, rutile_cluster(240), 2, (0.2, 3.0),
                       centres_per_orbital=16)


def batched_system_specs(count=16, base_seed=100):
    """Shapes of the uneven batch: per system n in {48..112}, N in U{8..128}, r in U{20..48},
    T in U{30..40}; box half-width n/8 so the spacing matches the Pt-shaped block."""
    specs = []
    for s in range(count):
        rng = np.random.default_rng(base_seed + s)
        n = int(rng.choice([48, 64, 80, 96, 112]))
        specs.append(dict(n=n, L=n / 8.0, n_orb=int(rng.integers(8, 129)), rank=int(rng.integers(20, 49)),
                          T=int(rng.integers(30, 41)), seed=base_seed + s))
    return specs


# orbitals of the uneven batch: Gaussian sums on 4 of the 32 atoms of an fcc cluster, 3 per atom,
# so that blocks of up to 128 orbitals stay linearly independent (the overlap matrix of 128
# orbitals drawn on one 8-atom cluster is singular to working precision)
BATCH_CENTRES, BATCH_GAUSS_PER_CENTRE, BATCH_CENTRES_PER_ORBITAL = 32, 3, 4


def batched_system_args(spec):
    """Positional and keyword arguments of make_system / make_system_on_device for one system
    of the uneven batch."""
    return ((spec["n"], spec["L"], spec["n_orb"], spec["rank"], spec["T"], spec["seed"],
             fcc_cluster(BATCH_CENTRES, 2.6), BATCH_GAUSS_PER_CENTRE, (0.2, 3.0)),
            dict(centres_per_orbital=BATCH_CENTRES_PER_ORBITAL))


def config_batched_system(spec) -> System:
    a, kw = batched_system_args(spec)
    return make_system("batched", *a, **kw)


CONFIGS = {
    "small": config_small,
    "pt": config_pt,
    "diff": config_diff,
    "tio2": config_tio2,
}


# ----------------------------------------------------------------------------------
# finite-element meshes for the transfer between the unstructured and structured bases
# ----------------------------------------------------------------------------------
def fe_mesh(L: float, base: int, centres, radius: float, order: int, levels: int = 1):
    """A hexahedral finite-element mesh of [-L, L]^3 that is refined near atoms: base^3 cubic
    cells, then `levels` times every cell whose centre lies within `radius` of a centre is split
    into eight.  Refined cells next to unrefined ones leave hanging nodes (the mesh is
    non-conforming there).  Every cell carries (order + 1)^3 equispaced Lagrange nodes, local
    node (lx, ly, lz) at index (lx (order + 1) + ly) (order + 1) + lz; nodes at the same place
    are one global node.  Returns (X [n_nodes, 3] float64, conn [n_cells, (order+1)^3] int32).
    Cells are listed coarse first, in the order they were made."""
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    h = 2.0 * L / base
    cells = [(np.array([-L + i * h, -L + j * h, -L + k * h]), h) for i in range(base) for j in range(base)
             for k in range(base)]
    for _ in range(levels):
        out = []
        for lo, w in cells:
            c = lo + 0.5 * w
            if np.min(np.linalg.norm(centres - c[None, :], axis=1)) < radius:
                hw = 0.5 * w
                out.extend((lo + hw * np.array([a, b, d]), hw) for a in (0, 1) for b in (0, 1) for d in (0, 1))
            else:
                out.append((lo, w))
        cells = sorted(out, key=lambda cw: -cw[1])        # coarse cells first
    p = int(order)
    q = np.arange(p + 1) / p
    index = {}
    X = []
    conn = np.empty((len(cells), (p + 1) ** 3), dtype=np.int32)
    tol = 1e-9 * L
    for ci, (lo, w) in enumerate(cells):
        l = 0
        for lx in range(p + 1):
            for ly in range(p + 1):
                for lz in range(p + 1):
                    pt = lo + w * np.array([q[lx], q[ly], q[lz]])
                    key = tuple(np.round(pt / tol).astype(np.int64))
                    g = index.get(key)
                    if g is None:
                        g = len(X)
                        index[key] = g
                        X.append(pt)
                    conn[ci, l] = g
                    l += 1
    return np.asarray(X, dtype=np.float64), conn


def gaussian_sum_at_points(points, centres, exps, coefs):
    """psi_i at arbitrary points [P, 3] (the orbitals of gaussian_sum_orbitals): [N, P]."""
    pts = np.asarray(points, dtype=np.float64)
    N, K = exps.shape
    out = np.zeros((N, pts.shape[0]))
    for i in range(N):
        for k in range(K):
            d2 = np.sum((pts - centres[i, k][None, :]) ** 2, axis=1)
            out[i] += coefs[i, k] * np.exp(-exps[i, k] * d2)
    return out

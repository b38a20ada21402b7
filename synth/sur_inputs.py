"""Seeded synthetic SUR problems (shared input generators).

This module only DRAWS inputs: regressor blocks X_i, the covariance factor
of Omega, the true parameters beta and the disturbances.  It contains none of
the estimation arithmetic (no projection, no Sigma-apply, no solve); both the
CPU oracle and the CUDA path consume its output.

Every problem is drawn from numpy's counter-based Philox4x32-10 generator
(Salmon et al., SC'11), keyed by ``seed`` so that a (seed, shape) pair always
yields the same bytes on every machine.

Model (SUR, paper Sec. 1 and Sec. 4.3, eq. SURdefs):
    y = vec(Y),  X = (+)_i X_i,  Sigma = Omega (x) I_M,
    y = X beta + eps,  eps = (F (x) I_M) z,  z iid N(0, 1),  Omega = F F^T.
With vec stacking columns, (F (x) I_M) vec(Z) = vec(Z F^T) for Z of shape
M x r, so the disturbance matrix of one right-hand side is E = Z F^T (M x G).

Layouts returned (all float64, C-contiguous numpy arrays):
    X_blocks : list of G arrays, X_i of shape (M, n_i)
    Omega    : (G, G) symmetric positive semi-definite
    Y        : (m, k) with m = G*M, column j = vec(Y_j) (block i = rows i*M..)
    beta     : (n, k) true parameters, n = sum(n_i)
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

SEED_BASE = 2510014471


def rng(seed: int) -> np.random.Generator:
    """Philox4x32-10 stream keyed by ``seed``."""
    return np.random.Generator(np.random.Philox(key=int(seed)))


@dataclass
class SurProblem:
    X_blocks: list
    Omega: np.ndarray
    Y: np.ndarray
    beta: np.ndarray
    M: int
    noise_factor: np.ndarray          # F with Omega = F F^T (G x r)
    C: np.ndarray | None = None       # optional restrictions C beta = d (kc x n)
    d: np.ndarray | None = None       # (kc, k)
    meta: dict = field(default_factory=dict)

    @property
    def G(self) -> int:
        return len(self.X_blocks)

    @property
    def n_i(self) -> list:
        return [int(x.shape[1]) for x in self.X_blocks]

    @property
    def n(self) -> int:
        return int(sum(self.n_i))

    @property
    def m(self) -> int:
        return self.G * self.M

    @property
    def k(self) -> int:
        return int(self.Y.shape[1])


# ----------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------

def gaussian_blocks(g: np.random.Generator, M: int, n_i, cond_max: float | None = None):
    """X_i with iid N(0,1) entries; if ``cond_max`` is given, columns are
    rescaled by log-spaced factors so that cond(X_i) <= cond_max.

    The spread rho of the column scales is chosen from the drawn block's own
    2-norm condition number kappa_Z as rho = 0.9 * cond_max / kappa_Z, so
    cond(X_i) <= kappa_Z * rho < cond_max by submultiplicativity."""
    blocks = []
    for ni in n_i:
        Z = g.standard_normal((M, ni))
        if cond_max is not None and ni > 1:
            kappa_z = np.linalg.cond(Z)
            rho = max(1.0, 0.9 * cond_max / kappa_z)
            s = np.logspace(0.0, -np.log10(rho), ni)
            Z = Z * s[None, :]
        blocks.append(np.ascontiguousarray(Z))
    return blocks


def lower_factor(g: np.random.Generator, G: int, offdiag_std: float = 0.3):
    """Lower-triangular L with diag U(0.5, 2) and off-diagonal N(0, offdiag_std^2)."""
    L = np.tril(g.standard_normal((G, G)) * offdiag_std, -1)
    L[np.diag_indices(G)] = g.uniform(0.5, 2.0, G)
    return L


def draw_responses(g: np.random.Generator, X_blocks, F: np.ndarray, M: int, k: int,
                   beta: np.ndarray | None = None):
    """y^(j) = X beta^(j) + vec(Z_j F^T) for j < k, each column with its own
    beta^(j) ~ N(0, I) (unless ``beta`` is given) and its own noise."""
    G = len(X_blocks)
    n = sum(x.shape[1] for x in X_blocks)
    r = F.shape[1]
    if beta is None:
        beta = g.standard_normal((n, k))
    Y = np.empty((G * M, k))
    for j in range(k):
        Z = g.standard_normal((M, r))
        E = Z @ F.T                                   # M x G disturbance matrix
        off = 0
        for i, Xi in enumerate(X_blocks):
            ni = Xi.shape[1]
            Y[i * M:(i + 1) * M, j] = Xi @ beta[off:off + ni, j] + E[:, i]
            off += ni
    return Y, beta


# ----------------------------------------------------------------------------
# generic problem families (used by tests at small sizes)
# ----------------------------------------------------------------------------

def make_problem(G: int, M: int, n_i, k: int = 1, seed: int = 0, omega: str = "chol",
                 rank: int | None = None, cond_max: float | None = None,
                 equal_X: bool = False, n_constraints: int = 0) -> SurProblem:
    """Small generic SUR problem.

    omega: "chol"     Omega = L L^T, L as ``lower_factor``
           "lowrank"  Omega = A A^T, A G x rank iid N(0,1) (singular if rank < G)
           "diag"     Omega diagonal, entries U(0.5, 2)
           "ident"    Omega = 2.5 I
           "spectrum" Omega = V diag(lam) V^T, lam log-uniform in [0.1, 10], V Haar
           "wishart"  Omega = B B^T / tr, B G x (G+4) iid N(0,1)
    """
    g = rng(seed)
    if equal_X:
        X0 = gaussian_blocks(g, M, [n_i[0]], cond_max)[0]
        X_blocks = [X0.copy() for _ in range(G)]
    else:
        X_blocks = gaussian_blocks(g, M, n_i, cond_max)
    F = omega_factor(g, G, omega, rank)
    Omega = F @ F.T
    Omega = 0.5 * (Omega + Omega.T)
    Y, beta = draw_responses(g, X_blocks, F, M, k)
    C = d = None
    if n_constraints:
        n = beta.shape[0]
        C = g.standard_normal((n_constraints, n))
        d = C @ beta
    return SurProblem(X_blocks, Omega, Y, beta, M, F, C, d,
                      meta=dict(seed=seed, omega=omega, rank=rank))


def omega_factor(g: np.random.Generator, G: int, kind: str, rank: int | None = None):
    if kind == "chol":
        return lower_factor(g, G)
    if kind == "lowrank":
        return g.standard_normal((G, rank if rank is not None else G))
    if kind == "diag":
        return np.diag(np.sqrt(g.uniform(0.5, 2.0, G)))
    if kind == "ident":
        return np.sqrt(2.5) * np.eye(G)
    if kind == "spectrum":
        V = haar_orthogonal(g, G)
        lam = np.exp(g.uniform(np.log(0.1), np.log(10.0), G))
        return V * np.sqrt(lam)[None, :]
    if kind == "wishart":
        B = g.standard_normal((G, G + 4))
        return B / np.sqrt(np.sum(B * B))
    raise ValueError(kind)


def haar_orthogonal(g: np.random.Generator, G: int):
    """Haar-distributed orthogonal matrix: QR of a Gaussian with the signs of
    diag(R) made positive (Mezzadri 2007)."""
    A = g.standard_normal((G, G))
    Qm, Rm = np.linalg.qr(A)
    return Qm * np.sign(np.diag(Rm))[None, :]


# ----------------------------------------------------------------------------
# the five named workloads
# ----------------------------------------------------------------------------

def small_g3_m200(seed_offset: int = 0) -> SurProblem:
    """Plain SUR, FP64, one RHS: G=3, M=200, n_i=(5,4,6), Omega = L L^T."""
    g = rng(SEED_BASE + 0 + 1000 * seed_offset)
    X = gaussian_blocks(g, 200, [5, 4, 6])
    L = lower_factor(g, 3)
    Y, beta = draw_responses(g, X, L, 200, 1)
    return SurProblem(X, L @ L.T, Y, beta, 200, L, meta=dict(name="sur-g3-m200"))


def singular_g64_m20000(k: int = 1, M: int = 20000, G: int = 64, rank: int = 56,
            nmin: int = 8, nmax: int = 32) -> SurProblem:
    """Singular covariance: G=64, M=20000, n_i ~ U{8..32}, cond(X_i) <= 1e3,
    Omega = A A^T with A 64 x 56 (rank 56)."""
    g = rng(SEED_BASE + 1)
    n_i = g.integers(nmin, nmax + 1, G).tolist()
    X = gaussian_blocks(g, M, n_i, cond_max=1e3)
    A = g.standard_normal((G, rank))
    Y, beta = draw_responses(g, X, A, M, k)
    Om = A @ A.T
    return SurProblem(X, 0.5 * (Om + Om.T), Y, beta, M, A,
                      meta=dict(name=f"sur-singular-g{G}-m{M}-k{k}"))


def batched_uneven_instances(count: int = 2048, k: int = 8, Gmin: int = 2, Gmax: int = 12,
                      Mmin: int = 200, Mmax: int = 4000, nmin: int = 2, nmax: int = 10,
                      first: int = 0):
    """Batched uneven SUR instances (list of SurProblem): G ~ U{2..12},
    M ~ U{200..4000}, n_i ~ U{2..10}, Omega = Wishart(G, G+4) / trace.
    Instance j is drawn from its own stream so that any subset can be
    regenerated alone."""
    out = []
    for j in range(first, first + count):
        g = rng(SEED_BASE + 2 + 7919 * (j + 1))
        G = int(g.integers(Gmin, Gmax + 1))
        M = int(g.integers(Mmin, Mmax + 1))
        n_i = g.integers(nmin, nmax + 1, G).tolist()
        X = gaussian_blocks(g, M, n_i)
        B = g.standard_normal((G, G + 4))
        Fm = B / np.sqrt(np.sum(B * B))
        Y, beta = draw_responses(g, X, Fm, M, k)
        out.append(SurProblem(X, Fm @ Fm.T, Y, beta, M, Fm, meta=dict(instance=j)))
    return out


def constrained_g32_m50000(k: int = 1, M: int = 50000, G: int = 32, ni: int = 16, kc: int = 64) -> SurProblem:
    """Constrained SUR: G=32, M=50000, n_i=16, C (64 x 512) iid N(0,1),
    d = C beta, Omega = V diag(lam) V^T, lam log-uniform [0.1, 10]."""
    g = rng(SEED_BASE + 3)
    X = gaussian_blocks(g, M, [ni] * G)
    F = omega_factor(g, G, "spectrum")
    Y, beta = draw_responses(g, X, F, M, k)
    n = G * ni
    C = g.standard_normal((kc, n))
    Om = F @ F.T
    return SurProblem(X, 0.5 * (Om + Om.T), Y, beta, M, F, C, C @ beta,
                      meta=dict(name=f"sur-constrained-g{G}-m{M}-k{k}"))


def differentiable_g128_m40000(M: int = 40000, G: int = 128, nmin: int = 4, nmax: int = 24):
    """Differentiable SUR: G=128, M=40000, n_i ~ U{4..24}, Omega = L L^T,
    beta_target iid N(0,1).  Returns (problem, L, beta_target)."""
    g = rng(SEED_BASE + 4)
    n_i = g.integers(nmin, nmax + 1, G).tolist()
    X = gaussian_blocks(g, M, n_i, cond_max=1e3)
    L = lower_factor(g, G)
    Y, beta = draw_responses(g, X, L, M, 1)
    target = g.standard_normal((sum(n_i), 1))
    return SurProblem(X, L @ L.T, Y, beta, M, L, meta=dict(name=f"sur-grad-g{G}-m{M}")), L, target


def monte_carlo_problem(count: int, seed: int = SEED_BASE + 77):
    """The Monte-Carlo setup of the statistical study (Sec. 3.4): m = 80,
    n = 20, Sigma with the four distinct eigenvalues 0.01, 0.1, 10, 50, read
    as a SUR model G = 4, M = 20, n_i = 5, Omega = V diag(0.01, 0.1, 10, 50) V^T
    (V Haar), so that each eigenvalue of Sigma = Omega (x) I_M has
    multiplicity 20.  X iid N(0, 1) and beta fixed; `count` replications of
    the disturbance as the columns of Y (G M x count).
    Returns (X_blocks, Omega, beta (n, 1), Y, Xbeta (G M, 1))."""
    g = rng(seed)
    G, M = 4, 20
    X = gaussian_blocks(g, M, [5, 5, 5, 5])
    V = haar_orthogonal(g, G)
    Omega = V @ np.diag([0.01, 0.1, 10.0, 50.0]) @ V.T
    Omega = 0.5 * (Omega + Omega.T)
    F = np.linalg.cholesky(Omega)
    beta = g.standard_normal((20, 1))
    Xb = np.vstack([X[i] @ beta[5 * i:5 * i + 5] for i in range(G)])
    Z = g.standard_normal((G, M * count))
    E = (F @ Z).reshape(G, M, count).reshape(G * M, count)   # rows of equation i: Z F^T, column by column
    return X, Omega, beta, Xb + E, Xb

"""Seeded synthetic restricted VAR problems (shared input generators).

Like ``sur_inputs`` this module only DRAWS inputs; it holds none of the
estimation arithmetic.  It stands in for the VAR data of the paper's second
experiment (Sec. "Experimental Tests", Table tab:varStats), which are not
available: G = 12 series, M = 300 observations, N = 60 regressors.

Recipe (the readings are listed in the design notes):
  * the series follows a VAR(4) y_t = sum_{l=1..4} A_l y_{t-l} + u_t with
    u_t ~ N(0, Omega0) and y_t = 0 before the first of ``burn`` + M + 5 steps
    (burn = 50 for a stationary series, 0 for an explosive one);
  * the regressors of row t are the five lags [y_{t-1}^T ... y_{t-5}^T], so
    N = 5 G = 60 and the true B (N x G, Y = Z0 B + U) has zero lag-5 rows;
  * a sparsity factor s makes a fraction s of the N G entries of B zero:
    all lag-5 entries, then entries of lags 1..4 drawn at random; the
    restrictions are exactly these exclusions, b_ij = 0 (selection rows C_i
    with gamma_i = 0, Sec. "GLMs with linear restrictions on the
    parameters");
  * the nonzero entries are N(0, 1), then A_l is scaled by c^l so that the
    largest modulus of the roots of the VAR (the eigenvalues of its
    companion matrix) is ``lam_max`` (0.90 stationary, 1.05 explosive);
  * Omega0 = V diag(logspace(0, log10(omega_cond), G)) V^T / mean, V Haar;
  * right-hand side 0 is the series itself (Y_0 = its last M values); the
    others keep Z0 and draw new disturbances: Y_j = Z0 B + U_j.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .sur_inputs import rng, haar_orthogonal


@dataclass
class VarProblem:
    Z0: np.ndarray          # (M, N) regressors
    Y: np.ndarray           # (M, G, k) responses
    Omega0: np.ndarray      # (G, G)
    B: np.ndarray           # (N, G) true coefficients
    C_list: list            # G selection matrices (k_i, N): the zero entries of column i of B
    gamma_list: list        # G arrays (k_i, k) of zeros
    free: list              # G index arrays: the unrestricted regressors of equation i

    @property
    def G(self) -> int:
        return self.Y.shape[1]

    @property
    def M(self) -> int:
        return self.Y.shape[0]

    @property
    def N(self) -> int:
        return self.Z0.shape[1]

    @property
    def k(self) -> int:
        return self.Y.shape[2]

    @property
    def k_i(self) -> list:
        return [int(c.shape[0]) for c in self.C_list]

    def y_vec(self) -> np.ndarray:
        """vec(Y_j) per right-hand side: (G M, k), equation i in rows i M .. (i+1) M - 1."""
        return np.ascontiguousarray(self.Y.transpose(1, 0, 2).reshape(self.G * self.M, self.k))

    def free_blocks(self) -> list:
        """The SUR regressor blocks of the same model with the exclusions
        substituted: X_i = Z0[:, free_i]."""
        return [np.ascontiguousarray(self.Z0[:, f]) for f in self.free]


def var_problem(G: int = 12, M: int = 300, lags: int = 5, true_lags: int = 4, sparsity: float = 0.26,
                lam_max: float = 0.90, omega_cond: float = 4.48, k: int = 1, burn: int | None = None,
                seed: int = 0) -> VarProblem:
    g = rng(seed)
    if burn is None:
        burn = 50 if lam_max < 1.0 else 0     # an explosive series starts at the first observations
    N = lags * G
    # zero pattern of B: every entry of the lags beyond true_lags, then random entries
    zero = np.zeros((N, G), dtype=bool)
    zero[true_lags * G:, :] = True
    need = int(round(sparsity * N * G)) - int(zero.sum())
    if need > 0:
        cand = np.flatnonzero(~zero.ravel())
        pick = g.choice(cand, size=min(need, cand.size - G), replace=False)   # keep >= G free entries
        zero.ravel()[pick] = True
    # every equation keeps at least one regressor
    for i in range(G):
        if zero[:, i].all():
            zero[0, i] = False
    A = g.standard_normal((N, G))
    A[zero] = 0.0
    # A_l = B[lag block l]^T; scale the VAR roots to lam_max
    blocks = [A[l * G:(l + 1) * G, :].T.copy() for l in range(true_lags)]
    comp = np.zeros((true_lags * G, true_lags * G))
    for l in range(true_lags):
        comp[:G, l * G:(l + 1) * G] = blocks[l]
    comp[G:, :-G] = np.eye((true_lags - 1) * G)
    rho = np.max(np.abs(np.linalg.eigvals(comp)))
    c = lam_max / rho
    blocks = [blocks[l] * c ** (l + 1) for l in range(true_lags)]
    B = np.zeros((N, G))
    for l in range(true_lags):
        B[l * G:(l + 1) * G, :] = blocks[l].T
    # Omega0 with the requested condition number
    V = haar_orthogonal(g, G)
    Om = V @ np.diag(np.logspace(0.0, np.log10(omega_cond), G)) @ V.T
    Om = Om / np.mean(np.diag(Om))
    Om = 0.5 * (Om + Om.T)
    F = np.linalg.cholesky(Om)
    T = burn + M + lags
    ys = np.zeros((T, G))
    for t in range(T):
        acc = F @ g.standard_normal(G)
        for l in range(true_lags):
            if t - l - 1 >= 0:
                acc = acc + blocks[l] @ ys[t - l - 1]
        ys[t] = acc
    rows = np.arange(burn + lags, T)
    Z0 = np.hstack([ys[rows - l - 1] for l in range(lags)])
    Y = np.empty((M, G, k))
    Y[:, :, 0] = ys[rows]
    for j in range(1, k):
        Y[:, :, j] = Z0 @ B + g.standard_normal((M, G)) @ F.T
    C_list, gamma_list, free = [], [], []
    for i in range(G):
        zi = np.flatnonzero(zero[:, i])
        C = np.zeros((zi.size, N))
        C[np.arange(zi.size), zi] = 1.0
        C_list.append(C)
        gamma_list.append(np.zeros((zi.size, k)))
        free.append(np.flatnonzero(~zero[:, i]))
    return VarProblem(Z0=np.ascontiguousarray(Z0), Y=Y, Omega0=Om, B=B, C_list=C_list, gamma_list=gamma_list,
                      free=free)

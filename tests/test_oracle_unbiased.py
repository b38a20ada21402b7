"""Pins of Theorem t:glmPcgUnbiased (Sec. 3.4): with w_1 = 0 the iterates
w_i of Algorithm glmpcg2 are odd functions of the disturbance, so z_i =
X*^T (y - Sigma w_i) satisfies z_i(X beta + eps) + z_i(X beta - eps) =
2 beta at every step, and E[z_i] = beta; the PCG-NE iterates (CG on the
normal equations from beta_1 = 0) are not odd and are biased (the
comparison of the paper's Monte-Carlo experiment).  CPU only."""
import numpy as np
import pytest

from oracle import sur_oracle as O
from synth import sur_inputs as S


@pytest.fixture(scope="module")
def mc():
    return S.monte_carlo_problem(2000)


@pytest.mark.parametrize("steps", [1, 2, 3, 6])
def test_pcg_aug_iterates_are_odd_in_the_disturbance(mc, steps):
    X, Om, beta, Y, Xb = mc
    eps = Y[:, :1] - Xb
    Ypm = np.hstack([Xb + eps, Xb - eps])
    res = O.sur_pcg_aug(X, Om, Ypm, tol=0.0, maxit=steps, stag_window=1000)
    s = res["b"][:, 0] + res["b"][:, 1] - 2.0 * beta[:, 0]
    assert np.linalg.norm(s) <= 1e-12 * np.linalg.norm(beta)
    w = res["w"]
    assert np.linalg.norm(w[:, 0] + w[:, 1]) <= 1e-12 * np.linalg.norm(w[:, 0])
    # a PCG-NE iterate is not odd: its error has an even part
    ne = O.pcg_ne(X, Om, Ypm, tol=0.0, maxit=steps)
    s_ne = ne["b"][:, 0] + ne["b"][:, 1] - 2.0 * beta[:, 0]
    assert np.linalg.norm(s_ne) >= 0.1 * np.linalg.norm(beta)


@pytest.mark.parametrize("steps", [1, 3])
def test_monte_carlo_means(mc, steps):
    # 2000 replications: the mean of z_i - beta is within 4.5 standard errors
    # of zero in every coordinate; the PCG-NE mean is hundreds of standard
    # errors away
    X, Om, beta, Y, Xb = mc
    N = Y.shape[1]
    aug = O.sur_pcg_aug(X, Om, Y, tol=0.0, maxit=steps, stag_window=1000)["b"] - beta
    ne = O.pcg_ne(X, Om, Y, tol=0.0, maxit=steps)["b"] - beta
    t_aug = aug.mean(axis=1) / (aug.std(axis=1, ddof=1) / np.sqrt(N))
    t_ne = ne.mean(axis=1) / (ne.std(axis=1, ddof=1) / np.sqrt(N))
    assert np.max(np.abs(t_aug)) <= 4.5, t_aug
    assert np.max(np.abs(t_ne)) >= 50.0, t_ne

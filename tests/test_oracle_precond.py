"""Pins of the oracle's general preconditioner block D and of Algorithms
glmpcg and glmpcg3 (Sec. 3.2, eq. invprec, eq. Xstar; the scaling study of
Sec. 3.3 and the VAR experiments use D = alpha I and D = diag(Sigma)).
CPU only.

For the SUR model D = diag(delta) (x) I_M; the pins build the augmented
matrix G and the preconditioner K = [D X; X^T 0]^-1 densely and run the
generic Algorithm pcg on them, which fixes both the w- and the z-iterates."""
import numpy as np
import pytest

from oracle import sur_oracle as O
from synth import sur_inputs as S


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dense_pcg_iterates(p, delta, iters):
    Sigma, X = O.sur_dense(p.X_blocks, p.Omega)
    m, n = X.shape
    D = np.diag(np.repeat(np.asarray(delta, dtype=float), p.M))
    Gm = O.augmented_matrix(Sigma, X)
    Km = np.linalg.inv(O.augmented_matrix(D, X))            # eq. (invprec)
    h = np.concatenate([p.Y[:, 0], np.zeros(n)])
    xs = O.pcg(Gm, Km, h, np.zeros(m + n), iters)
    return [x[:m] for x in xs], [x[m:] for x in xs]


@pytest.mark.parametrize("delta", [[1.0, 1.0, 1.0], [0.3, 2.0, 5.0], [4.0, 4.0, 4.0]])
def test_general_d_matches_generic_pcg(delta):
    # glmpcg2 with D = diag(delta) (x) I reproduces the w-iterates of Algorithm
    # pcg on the dense (G, K); the z-iterates of Algorithm glmpcg (carried as
    # z) reproduce its z-iterates
    p = S.make_problem(G=3, M=12, n_i=[2, 3, 2], k=1, seed=17, omega="chol")
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=6, stag_window=100, record=True,
                        delta=delta)
    ws, zs = dense_pcg_iterates(p, delta, 6)
    for i in range(1, len(ws)):
        assert rel(res["history"]["w"][i][:, 0], ws[i]) < 1e-9, i
    assert rel(res["z"][:, 0], zs[-1]) < 1e-8


@pytest.mark.parametrize("delta", [None, [0.5, 3.0, 1.5, 8.0]])
def test_glmpcg3_iterates_equal_glmpcg2(delta):
    # Algorithm glmpcg3 carries s_i in place of u_i, v_i; in exact arithmetic
    # its w-iterates and c_i are those of Algorithm glmpcg2
    p = S.make_problem(G=4, M=30, n_i=[3, 2, 4, 2], k=2, seed=23, omega="chol")
    a = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=10, stag_window=100, record=True, delta=delta)
    b = O.sur_pcg_aug3(p.X_blocks, p.Omega, p.Y, 10, delta=delta)
    for i in range(1, 11):
        assert rel(b["history"]["w"][i], a["history"]["w"][i]) < 1e-9, i
        assert rel(b["history"]["c"][i], a["history"]["c"][i]) < 1e-8, i


def test_d_equal_sigma_converges_in_one_step():
    # D = Sigma makes GK = I (Sec. 3.2, after eq. invprec): one step.  For the
    # SUR model with diagonal Omega, D = diag(Sigma) = Sigma.
    p = S.make_problem(G=4, M=25, n_i=[2, 3, 4, 2], k=3, seed=31, omega="diag")
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=1e-12, delta=O.jacobi_delta(p.Omega))
    assert list(res["iters"]) == [1, 1, 1]
    assert rel(res["b"], O.ols_blocks(p.X_blocks, p.Y)) < 1e-12


def test_scaled_identity_keeps_the_iterates():
    # D = alpha I scales Pi by 1/alpha: c, d and lambda rescale and the
    # w-iterates are those of D = I
    p = S.make_problem(G=4, M=40, n_i=[3, 2, 4, 3], k=2, seed=37, omega="chol")
    a = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=12, stag_window=100, record=True)
    b = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=12, stag_window=100, record=True,
                      delta=O.scaled_identity_delta(p.Omega))
    for i in range(1, 13):
        assert rel(b["history"]["w"][i], a["history"]["w"][i]) < 1e-10, i


def test_jacobi_block_helps_a_badly_scaled_omega():
    # Omega = S R S with equation scales spread over two orders of magnitude
    # and a well-conditioned correlation R: D = diag(Omega) (x) I removes the
    # scales (B^-1 A on null(X^T) becomes the correlation operator) and
    # converges to the GLS estimate in a few dozen steps, while D = I is still
    # far from it after m - n + 1 steps (the effect of the choice of D that
    # Sec. 3.3 and the VAR experiments show)
    g = S.rng(5)
    G, M = 6, 60
    X = S.gaussian_blocks(g, M, [3, 2, 4, 3, 2, 3])
    A = g.standard_normal((G, G))
    R = A @ A.T / G + np.eye(G)
    d = np.sqrt(np.diag(R))
    R = R / np.outer(d, d)
    sc = np.logspace(-1, 1, G)
    Om = np.outer(sc, sc) * R
    F = np.linalg.cholesky(Om)
    Y, _ = S.draw_responses(g, X, F, M, 1)
    _, b_dense = O.aug_dense_solve(X, Om, Y)
    jac = O.sur_pcg_aug(X, Om, Y, tol=1e-12, stag_window=1000, delta=O.jacobi_delta(Om))
    plain = O.sur_pcg_aug(X, Om, Y, tol=1e-12, stag_window=1000)
    assert jac["status"] == [O.STATUS_CONVERGED] and jac["iters"][0] <= 30, jac["iters"]
    assert rel(jac["b"], b_dense) < 1e-11
    assert rel(plain["b"], b_dense) > 1e3 * rel(jac["b"], b_dense)


# ---------------------------------------------------------------- PCG-NE comparator

def test_pcg_ne_matches_generic_cg_on_the_normal_matrix():
    # Algorithm pcg with K = I on the dense normal matrix A = X^T Sigma^-1 X
    # fixes the iterates of the matrix-free SUR version
    p = S.make_problem(G=3, M=20, n_i=[2, 3, 2], k=1, seed=51, omega="chol")
    Sigma, X = O.sur_dense(p.X_blocks, p.Omega)
    Sinv = np.linalg.inv(Sigma)
    A = X.T @ Sinv @ X
    h = X.T @ Sinv @ p.Y[:, 0]
    xs = O.pcg(A, np.eye(A.shape[0]), h, np.zeros(A.shape[0]), 5)
    res = O.pcg_ne(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=5, record=True)
    for i in range(1, len(xs)):
        assert rel(res["history"][i][:, 0], xs[i]) < 1e-9, i


def test_pcg_ne_converges_to_gls_within_n_steps():
    # exact arithmetic: at most n steps (n distinct eigenvalues at most);
    # the limit is eq. (GLS)
    p = S.make_problem(G=4, M=50, n_i=[3, 2, 4, 3], k=2, seed=53, omega="spectrum")
    res = O.pcg_ne(p.X_blocks, p.Omega, p.Y, tol=1e-13, maxit=4 * p.n)
    assert all(s == O.STATUS_CONVERGED for s in res["status"])
    assert max(res["iters"]) <= p.n + 2
    assert rel(res["b"], O.gls_formula(p.X_blocks, p.Omega, p.Y)) < 1e-10


def test_pcg_ne_steps_equal_the_distinct_eigenvalues():
    # orthonormal X_i and diagonal Omega: X^T Sigma^-1 X = blockdiag(I / omega_ii),
    # whose distinct eigenvalues are the distinct omega_ii; CG ends after
    # exactly that many steps
    g = S.rng(59)
    G, M = 5, 40
    X = [np.linalg.qr(x)[0] for x in S.gaussian_blocks(g, M, [3, 2, 3, 2, 3])]
    Om = np.diag([1.0, 2.0, 5.0, 5.0, 0.5])
    Y, _ = S.draw_responses(g, X, np.linalg.cholesky(Om), M, 2)
    res = O.pcg_ne(X, Om, Y, tol=1e-12)
    assert list(res["iters"]) == [4, 4]
    assert rel(res["b"], O.gls_formula(X, Om, Y)) < 1e-12


def test_pcg_ne_loses_finite_termination_on_ill_conditioned_x():
    # regressors with singular values over five orders: cond(X^T Sigma^-1 X)
    # ~ 1e10 and PCG-NE needs several times n steps, while PCG-Aug (whose
    # projection does not see cond(X)) needs fewer than n + 10 (the VAR
    # experiments: PCG-NE stalls on ill-conditioned normal systems)
    g = S.rng(57)
    G, M = 5, 40
    X = S.gaussian_blocks(g, M, [3, 2, 3, 2, 3])
    for i in range(G):
        U, s, Vt = np.linalg.svd(X[i], full_matrices=False)
        X[i] = U @ np.diag(np.logspace(0, -5, len(s))) @ Vt
    A = g.standard_normal((G, G))
    Om = A @ A.T / G + np.eye(G)
    Y, _ = S.draw_responses(g, X, np.linalg.cholesky(Om), M, 1)
    n = 13
    ne = O.pcg_ne(X, Om, Y, tol=1e-10, maxit=10 * n)
    aug = O.sur_pcg_aug(X, Om, Y, tol=1e-10, stag_window=1000)
    assert aug["status"] == [O.STATUS_CONVERGED] and aug["iters"][0] < n + 10
    assert ne["iters"][0] > 3 * n, ne["iters"]
    cut = O.pcg_ne(X, Om, Y, tol=1e-10, maxit=n)
    bg = O.gls_formula(X, Om, Y)
    assert rel(cut["b"], bg) > 0.5

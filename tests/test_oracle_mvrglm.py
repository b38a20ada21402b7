"""Pins of the oracle's MVRGLM (Sec. "Multivariate linear models with
parameters restrictions"): model reduction by the QR of Z0, the updating
QRDs [R0; C_i] = Qt_i R_i and Algorithm glmpcg2 with the block-diagonal X*
and Pi.  Each pin ties it to something other than itself: the closed-form
restricted GLS estimator, the dense augmented solve of the unreduced model,
the generic Algorithm pcg on the densely built (G, K) of eq. (invprec), the
step bound k + 1, OLS when nothing is restricted, and the SUR model with the
excluded regressors removed.  CPU only."""
import numpy as np
import pytest

from oracle import sur_oracle as O
from synth import sur_inputs as S
from synth import var_inputs as V


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def small_model(seed, G=3, M=40, N=6, k_i=(2, 0, 3), k=2):
    g = S.rng(seed)
    Z0 = g.standard_normal((M, N))
    A = g.standard_normal((G, G))
    Om = A @ A.T / G + 0.5 * np.eye(G)
    C_list = [g.standard_normal((ki, N)) for ki in k_i]
    B = g.standard_normal((N, G))
    gamma = [C_list[i] @ B[:, i:i + 1] * np.ones((1, k)) for i in range(G)]
    U = np.einsum("mgk,hg->mhk", g.standard_normal((M, G, k)), np.linalg.cholesky(Om))
    Y = np.einsum("mn,ng->mg", Z0, B)[:, :, None] + U
    return Z0, Y, Om, C_list, gamma


def vec_y(Y):
    M, G, k = Y.shape
    return Y.transpose(1, 0, 2).reshape(G * M, k)


def blockdiag(mats, N):
    rows = sum(m.shape[0] for m in mats)
    out = np.zeros((rows, N * len(mats)))
    r = 0
    for i, m in enumerate(mats):
        out[r:r + m.shape[0], i * N:(i + 1) * N] = m
        r += m.shape[0]
    return out


def restricted_gls_closed_form(Z0, Y, Om, C_list, gamma):
    # b_R = b - A^-1 C^T (C A^-1 C^T)^-1 (C b - gamma), A = X^T Sigma^-1 X,
    # b the GLS estimate of the unrestricted model (Sigma positive definite)
    M, G, k = Y.shape
    N = Z0.shape[1]
    X = np.kron(np.eye(G), Z0)
    Si = np.kron(np.linalg.inv(Om), np.eye(M))
    A = X.T @ Si @ X
    Ai = np.linalg.inv(A)
    b = Ai @ X.T @ Si @ vec_y(Y)
    C = blockdiag(C_list, N)
    gam = np.vstack([gi.reshape(-1, k) for gi in gamma])
    corr = Ai @ C.T @ np.linalg.solve(C @ Ai @ C.T, C @ b - gam)
    return b - corr


def test_mvrglm_equals_restricted_gls():
    Z0, Y, Om, C_list, gamma = small_model(3)
    res = O.mvrglm_pcg_aug(Z0, Y, Om, C_list, gamma, tol=1e-13, stag_window=100)
    assert all(s == O.STATUS_CONVERGED for s in res["status"])
    cf = restricted_gls_closed_form(Z0, Y, Om, C_list, gamma)
    assert rel(res["b"], cf) < 1e-10
    # the dense augmented system of the unreduced model (eq. RGLM1setup)
    G = Y.shape[1]
    C = blockdiag(C_list, Z0.shape[1])
    d = np.vstack([gi.reshape(-1, Y.shape[2]) for gi in gamma])
    _, b_dense = O.aug_dense_solve([Z0] * G, Om, vec_y(Y), C=C, d=d)
    assert rel(res["b"], b_dense) < 1e-10
    # the restrictions hold
    for i in range(G):
        assert np.allclose(C_list[i] @ res["B"][:, i, :], gamma[i], atol=1e-11)


def test_mvrglm_equals_sec51_fold_in_of_the_unreduced_model():
    # model reduction is exact: Algorithm glmpcg2 on the unreduced restricted
    # model (X_aug = [I (x) Z0; C], eq. rglm1m) reaches the same estimate
    Z0, Y, Om, C_list, gamma = small_model(5, k=1)
    G = Y.shape[1]
    C = blockdiag(C_list, Z0.shape[1])
    d = np.vstack([gi.reshape(-1, 1) for gi in gamma])
    full = O.rglm_pcg_aug([Z0] * G, Om, vec_y(Y), C, d, tol=1e-13, stag_window=200)
    red = O.mvrglm_pcg_aug(Z0, Y, Om, C_list, gamma, tol=1e-13, stag_window=100)
    assert rel(red["b"], full["b"]) < 1e-10


def test_mvrglm_iterates_equal_generic_pcg_on_dense_g_and_k():
    # G and K = [D X; X^T 0]^-1 (D = I) built densely in the equation-by-
    # equation order; Algorithm pcg on them fixes the w-iterates
    Z0, Y, Om, C_list, gamma = small_model(7, k=1)
    res = O.mvrglm_pcg_aug(Z0, Y, Om, C_list, gamma, tol=0.0, maxit=5, stag_window=100, record=True)
    N = Z0.shape[1]
    G = len(C_list)
    R0 = np.linalg.qr(Z0)[1]
    rows = [N + c.shape[0] for c in C_list]
    roff = np.cumsum([0] + rows)
    m = int(roff[-1])
    Sig = np.zeros((m, m))
    for i in range(G):
        for h in range(G):
            Sig[roff[i]:roff[i] + N, roff[h]:roff[h] + N] = Om[i, h] * np.eye(N)
    X = np.zeros((m, G * N))
    for i in range(G):
        X[roff[i]:roff[i + 1], i * N:(i + 1) * N] = np.vstack([R0, C_list[i]])
    Gm = O.augmented_matrix(Sig, X)
    Km = np.linalg.inv(O.augmented_matrix(np.eye(m), X))
    h = np.concatenate([res["yaug"][:, 0], np.zeros(G * N)])
    xs = O.pcg(Gm, Km, h, np.zeros(m + G * N), 5)
    for i in range(1, len(xs)):
        assert rel(res["history"]["w"][i][:, 0], xs[i][:m]) < 1e-9, i


@pytest.mark.parametrize("k_i", [(2, 0, 3), (1, 1, 1), (4, 2, 5)])
def test_mvrglm_ends_within_total_restrictions_plus_one(k_i):
    # m + k - n + 1 = G N + sum k_i - G N + 1 steps in exact arithmetic: the
    # relative residual collapses by then (in floating point a step or two
    # more reach the rounding floor)
    Z0, Y, Om, C_list, gamma = small_model(11, k_i=k_i, k=1)
    kk = sum(k_i)
    cut = O.mvrglm_pcg_aug(Z0, Y, Om, C_list, gamma, tol=1e-12, maxit=kk + 1, stag_window=100)
    assert cut["relres"][0] <= 1e-8, cut["relres"]
    res = O.mvrglm_pcg_aug(Z0, Y, Om, C_list, gamma, tol=1e-12, maxit=2 * kk + 4, stag_window=100)
    assert res["status"] == [O.STATUS_CONVERGED] and res["iters"][0] <= kk + 3, (res["iters"], kk)
    assert rel(res["b"], restricted_gls_closed_form(Z0, Y, Om, C_list, gamma)) < 1e-11


def test_reduced_form_iterates_equal_glmpcg2_on_sur():
    # eq. (urwProj): the reduced recursion takes the w-iterates of Algorithm
    # glmpcg2 (compared on a SUR model, where the literal r-recursion is
    # stable: lambda_i near 1)
    p = S.make_problem(G=4, M=30, n_i=[3, 2, 4, 2], k=2, seed=23, omega="chol")
    for delta in (None, [0.5, 3.0, 1.5, 8.0]):
        a = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=10, stag_window=100, record=True, delta=delta)
        b = O.pcg_aug_reduced(O.SurOps(p.X_blocks, p.Omega, delta), p.Y, tol=0.0, maxit=10, stag_window=100,
                              record=True)
        for i in range(1, 11):
            assert rel(b["history"]["w"][i], a["history"]["w"][i]) < 1e-9, i


def test_mvrglm_without_restrictions_is_ols():
    # [R0] square: Pi = 0, no step is taken and b = R0^-1 Q0^T y = OLS
    # (OLS = GLS for the multivariate model with a common Z0)
    Z0, Y, Om, _, _ = small_model(13)
    res = O.mvrglm_pcg_aug(Z0, Y, Om, [np.zeros((0, Z0.shape[1]))] * 3)
    assert list(res["iters"]) == [0, 0]
    B_ols = np.stack([np.linalg.lstsq(Z0, Y[:, :, j], rcond=None)[0] for j in range(Y.shape[2])], axis=2)
    assert rel(res["B"], B_ols) < 1e-12


def test_var_exclusions_equal_sur_without_the_excluded_regressors():
    # b_ij = 0 restrictions: the estimate is the SUR GLS estimate of X_i =
    # Z0[:, free_i], scattered back, and the excluded entries are zero
    p = V.var_problem(G=4, M=90, lags=3, true_lags=2, sparsity=0.45, k=2, seed=17)
    res = O.mvrglm_pcg_aug(p.Z0, p.Y, p.Omega0, p.C_list, p.gamma_list, tol=1e-13, stag_window=200)
    assert all(s == O.STATUS_CONVERGED for s in res["status"])
    b_free = O.gls_formula(p.free_blocks(), p.Omega0, p.y_vec())
    B = np.zeros((p.N, p.G, p.k))
    off = 0
    for i, f in enumerate(p.free):
        B[f, i, :] = b_free[off:off + f.size]
        off += f.size
    assert rel(res["B"], B) < 1e-10
    for i, f in enumerate(p.free):
        mask = np.ones(p.N, dtype=bool)
        mask[f] = False
        assert np.max(np.abs(res["B"][mask, i, :])) <= 1e-12 * np.max(np.abs(res["B"]))


@pytest.mark.parametrize("delta_fn", [O.scaled_identity_delta, O.jacobi_delta])
def test_mvrglm_preconditioner_block_keeps_the_estimate(delta_fn):
    # D = D0 (x) I on the reduced rows and D0 on the restriction rows (the
    # choices K1 and K2 of the VAR experiments): same estimate, same bound
    Z0, Y, Om, C_list, gamma = small_model(19, k=1)
    Om = np.diag([0.1, 1.0, 30.0]) @ Om @ np.diag([0.1, 1.0, 30.0])
    a = O.mvrglm_pcg_aug(Z0, Y, Om, C_list, gamma, tol=1e-12, stag_window=100)
    b = O.mvrglm_pcg_aug(Z0, Y, Om, C_list, gamma, tol=1e-12, stag_window=100, delta=delta_fn(Om))
    assert b["status"] == [O.STATUS_CONVERGED] and b["iters"][0] <= 5 + 3
    assert rel(b["b"], restricted_gls_closed_form(Z0, Y, Om, C_list, gamma)) < 1e-9
    assert rel(a["b"], b["b"]) < 1e-9

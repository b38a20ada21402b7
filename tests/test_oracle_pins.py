"""Pins of the FP64 CPU oracle to facts fixed by the paper and by mathematics
(brute force, closed forms, invariants, printed values).  CPU only."""
import json
import os

import numpy as np
import pytest

from oracle import sur_oracle as O
from synth import sur_inputs as S

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dense_aug_equals_gls_formula_pd(seed):
    # eq. (aug1) with PD Sigma is equivalent to eq. (GLS)
    p = S.make_problem(G=3, M=20, n_i=[3, 2, 4], k=2, seed=seed, omega="chol")
    _, b1 = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    b2 = O.gls_formula(p.X_blocks, p.Omega, p.Y)
    assert rel(b1, b2) < 1e-12


@pytest.mark.parametrize("omega,rank", [("chol", None), ("lowrank", 3)])
def test_dense_aug_equals_lemma(omega, rank):
    # Lemma thm:AugBLUE closed form (eq. augsol); the low-rank case has
    # Q_N^T Sigma Q_N non-singular because (G - rank) * M = 20 <= n = 24 is
    # not required: we check the condition directly below.
    p = S.make_problem(G=4, M=20, n_i=[6, 6, 6, 6], k=1, seed=5, omega=omega, rank=rank)
    Sigma, X = O.sur_dense(p.X_blocks, p.Omega)
    Qf, _ = np.linalg.qr(X, mode="complete")
    QN = Qf[:, X.shape[1]:]
    assert np.linalg.matrix_rank(QN.T @ Sigma @ QN) == QN.shape[1]
    w1, b1 = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    w2, b2 = O.aug_lemma(p.X_blocks, p.Omega, p.Y)
    assert rel(b1, b2) < 1e-11
    assert rel(w1, w2) < 1e-10


def test_rotated_system_solution_lemma_proof():
    # Appendix proof of Lemma thm:AugBLUE: in the rotated system w_R = 0.
    p = S.make_problem(G=3, M=15, n_i=[2, 3, 2], k=1, seed=9, omega="chol")
    Sigma, X = O.sur_dense(p.X_blocks, p.Omega)
    w, _ = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    Qf, _ = np.linalg.qr(X, mode="complete")
    wR = Qf[:, :X.shape[1]].T @ w
    assert np.linalg.norm(wR) < 1e-12 * max(1.0, np.linalg.norm(w))


# ---------------------------------------------------------------- closed forms

def test_diagonal_omega_gives_blockwise_ols():
    # Omega diagonal -> Sigma block diagonal -> equations decouple, GLS = OLS (Sec. 1)
    p = S.make_problem(G=4, M=25, n_i=[2, 3, 4, 2], k=2, seed=3, omega="diag")
    b_ols = O.ols_blocks(p.X_blocks, p.Y)
    _, b1 = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    b2 = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=1e-14)
    assert rel(b1, b_ols) < 1e-12
    assert rel(b2, b_ols) < 1e-12
    assert rel(res["b"], b_ols) < 1e-12
    # A = Q_N^T Sigma Q_N = (+) omega_ii I  ->  at most #distinct(omega_ii) steps
    assert max(res["iters"]) <= len(np.unique(np.round(np.diag(p.Omega), 12))) + 1


def test_equal_regressors_give_ols():
    # all X_i equal (multivariate model, Sec. 1 / Sec. 4.2): GLS = OLS
    p = S.make_problem(G=4, M=30, n_i=[3], k=1, seed=4, omega="chol", equal_X=True)
    b_ols = O.ols_blocks(p.X_blocks, p.Y)
    _, b1 = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    b2 = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=1e-14)
    assert rel(b1, b_ols) < 1e-11
    assert rel(b2, b_ols) < 1e-11
    assert rel(res["b"], b_ols) < 1e-11
    # Sigma and Pi commute: A = Omega (x) I on null(X_0^T) -> <= G distinct eigenvalues
    assert max(res["iters"]) <= p.G + 1


def test_omega_scaled_identity_one_step():
    # D = Sigma up to scale -> GK has one eigenvalue on null(X^T): one step
    p = S.make_problem(G=3, M=20, n_i=[2, 2, 3], k=3, seed=6, omega="ident")
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=1e-13)
    assert list(res["iters"]) == [1, 1, 1]
    assert rel(res["b"], O.ols_blocks(p.X_blocks, p.Y)) < 1e-12


def test_singular_omega_recovers_beta_exactly():
    # Omega = A A^T with rank r < G and noise (A (x) I) z: every null vector v
    # of Omega gives sum_i v_i y_i = sum_i v_i X_i beta_i exactly, and the
    # stacked regressors have full column rank, so b = beta_true.
    p = S.make_problem(G=6, M=40, n_i=[3, 4, 2, 5, 3, 4], k=2, seed=11, omega="lowrank", rank=4)
    _, b1 = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    b2 = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=1e-14, record=True)
    assert rel(b1, p.beta) < 1e-10
    assert rel(b2, p.beta) < 1e-10
    # A = Q_N^T Sigma Q_N is singular here (eq. SigmaPosXNull fails): the
    # recursive residual of the iteration reaches a floor near 1e-10 and then
    # grows again, and the stagnation rule (no new minimum of c for W = 25
    # steps) ends it W steps after the floor.  The iterate at the floor gives
    # beta_true; the last iterate has drifted by at most a few 1e-9.
    assert all(s == O.STATUS_STAGNATED for s in res["status"])
    hist = res["history"]
    c = np.array(hist["c"])
    ops = O.SurOps(p.X_blocks, p.Omega)
    for j in range(p.k):
        best = int(np.argmin(c[:, j]))
        w = hist["w"][best][:, j:j + 1]
        b_best = ops.xstar_t(p.Y[:, j:j + 1] - ops.sigma(w))
        assert rel(b_best, p.beta[:, j:j + 1]) < 1e-9, j
        assert res["iters"][j] == best + 25, (j, best, res["iters"][j])
    assert rel(res["b"], p.beta) < 1e-8


# ---------------------------------------------------------------- structured direct vs brute force

@pytest.mark.parametrize("omega,rank,seed", [("chol", None, 1), ("spectrum", None, 2),
                                             ("wishart", None, 3), ("lowrank", 2, 4)])
def test_structured_equals_dense(omega, rank, seed):
    p = S.make_problem(G=4, M=18, n_i=[2, 3, 1, 3], k=2, seed=seed, omega=omega, rank=rank)
    _, b1 = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    b2 = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
    assert rel(b2, b1) < 1e-10


def test_structured_reduction_when_W_rank_deficient():
    # M < n: range(W) is all of R^M, the reduction keeps every row
    p = S.make_problem(G=3, M=8, n_i=[3, 4, 3], k=1, seed=21, omega="chol")
    _, b1 = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    b2 = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
    assert rel(b2, b1) < 1e-9


# ---------------------------------------------------------------- PCG-Aug (Algorithm glmpcg2)

def _dense_pcg_w_iterates(p, iters):
    Sigma, X = O.sur_dense(p.X_blocks, p.Omega)
    m, n = X.shape
    Gm = O.augmented_matrix(Sigma, X)
    Km = np.linalg.inv(O.augmented_matrix(np.eye(m), X))    # eq. (invprec), D = I
    h = np.concatenate([p.Y[:, 0], np.zeros(n)])
    xs = O.pcg(Gm, Km, h, np.zeros(m + n), iters)
    return [x[:m] for x in xs]


def test_glmpcg2_matches_generic_pcg_iterates():
    # Algorithm glmpcg2 in the SUR form of Sec. 4.3 must reproduce the
    # w-iterates of Algorithm pcg on (G, K) built densely (eq. Gaug, invprec).
    p = S.make_problem(G=3, M=12, n_i=[2, 3, 2], k=1, seed=7, omega="chol")
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=6, stag_window=100,
                        record=True)
    ws = _dense_pcg_w_iterates(p, 6)
    for i in range(len(ws)):
        assert rel(res["history"]["w"][i][:, 0], ws[i]) < 1e-9 or np.linalg.norm(ws[i]) == 0


def test_glmpcg2_invariants():
    p = S.make_problem(G=3, M=16, n_i=[3, 2, 3], k=1, seed=8, omega="chol")
    op = O.SurOps(p.X_blocks, p.Omega)
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=8, stag_window=100,
                        record=True)
    H = res["history"]
    w_exact, _ = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    Sigma, _ = O.sur_dense(p.X_blocks, p.Omega)
    errs = []
    for i, w in enumerate(H["w"]):
        # X^T w_i = 0 for every iterate (w_1 = 0, Sec. 3.2)
        assert np.linalg.norm(op.xt(w)) < 1e-11 * max(1.0, np.linalg.norm(w))
        e = w[:, 0] - w_exact[:, 0]
        errs.append(e @ Sigma @ e)
    # eq. (wOptim): Sigma-norm error non-increasing
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) + 1e-20 for i in range(len(errs) - 1))
    # Property orth: residuals Pi-orthogonal, directions Sigma-conjugate (j < i)
    Pr = [op.pi(r) for r in H["r"]]
    for i in range(1, 6):
        for j in range(i):
            ri = H["r"][i][:, 0]
            assert abs(ri @ Pr[j][:, 0]) < 1e-8 * np.linalg.norm(ri) * np.linalg.norm(Pr[j])
            ui, uj = H["u"][i][:, 0], H["u"][j][:, 0]
            assert abs(uj @ Sigma @ ui) < 1e-8 * np.sqrt((ui @ Sigma @ ui) * (uj @ Sigma @ uj))


def test_finite_termination_distinct_eigenvalues():
    # Property finite: #steps = #distinct eigenvalues of A = Q_N^T Sigma Q_N.
    # Omega = diag with 2 distinct values repeated -> 2 steps.
    g = S.rng(123)
    X = S.gaussian_blocks(g, 15, [2, 3, 2, 2])
    Om = np.diag([1.0, 3.0, 1.0, 3.0])
    F = np.sqrt(Om)
    Y, _ = S.draw_responses(g, X, F, 15, 1)
    res = O.sur_pcg_aug(X, Om, Y, tol=1e-12)
    assert res["iters"][0] == 2
    # general case: bound G + (G-1) n counts eigenvalues of A with multiplicity
    p = S.make_problem(G=2, M=9, n_i=[2, 2], k=1, seed=12, omega="chol")
    Sigma, Xd = O.sur_dense(p.X_blocks, p.Omega)
    Qf, _ = np.linalg.qr(Xd, mode="complete")
    QN = Qf[:, Xd.shape[1]:]
    ev = np.linalg.eigvalsh(QN.T @ Sigma @ QN)
    distinct = 1 + int(np.sum(np.diff(np.sort(ev)) > 1e-9 * ev.max()))
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=1e-12, stag_window=100)
    assert res["iters"][0] <= distinct + 1
    assert distinct <= p.G + (p.G - 1) * p.n


def test_scaling_experiment_condition_numbers_printed_in_paper():
    # Sec. 3.3 prints cond(KG) = 4 (alpha = 1) and 8 (alpha = 1/4, 4) for
    # m = 300, n = 50, D = I and Sigma with eigenvalues alpha{1/2,1,3/2,2}
    # (multiplicity 75).  A SUR with G = 4, M = 75, Omega = alpha diag(1/2,1,3/2,2)
    # has exactly that spectrum of Sigma.
    gold = json.load(open(os.path.join(HERE, "golden", "scaling_condKG.json")))
    g = S.rng(77)
    X = S.gaussian_blocks(g, 75, [13, 13, 12, 12])
    for alpha_s, expect in gold["cond_KG"].items():
        alpha = float(alpha_s)
        Om = alpha * np.diag([0.5, 1.0, 1.5, 2.0])
        Sigma, Xd = O.sur_dense(X, Om)
        assert Xd.shape == (gold["m"], gold["n"])
        Gm = O.augmented_matrix(Sigma, Xd)
        Km = np.linalg.inv(O.augmented_matrix(np.eye(Xd.shape[0]), Xd))
        ev = np.abs(np.linalg.eigvals(Km @ Gm))
        assert abs(ev.max() / ev.min() - expect) < 1e-6 * expect


def test_pcg_matches_dense_on_the_small_workload():
    p = S.small_g3_m200()
    _, b1 = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    b2 = O.gls_formula(p.X_blocks, p.Omega, p.Y)
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=1e-13)
    assert rel(b1, b2) < 1e-12
    assert rel(res["b"], b1) < 1e-11
    assert res["status"][0] == O.STATUS_CONVERGED


# ---------------------------------------------------------------- restrictions (Sec. 4.1)

def test_restricted_models_agree_and_satisfy_constraints():
    p = S.make_problem(G=3, M=14, n_i=[3, 3, 2], k=2, seed=31, omega="spectrum", n_constraints=3)
    _, b1 = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y, p.C, p.d)
    b2 = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y, p.C, p.d)
    res = O.rglm_pcg_aug(p.X_blocks, p.Omega, p.Y, p.C, p.d, tol=1e-14)
    assert rel(b2, b1) < 1e-10
    assert rel(res["b"], b1) < 1e-9
    for b in (b1, b2, res["b"]):
        assert np.linalg.norm(p.C @ b - p.d) < 1e-10 * np.linalg.norm(p.d)
    # at most m + k - n + 1 steps (Sec. 4.1)
    assert max(res["iters"]) <= p.m + 3 - p.n + 1


def test_selection_restriction_fixes_parameters():
    # C a selection matrix, d = 0: the restricted elements of b are zero
    p = S.make_problem(G=3, M=14, n_i=[3, 3, 2], k=1, seed=32, omega="chol")
    C = np.zeros((2, p.n)); C[0, 1] = 1; C[1, 6] = 1
    d = np.zeros((2, 1))
    b = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y, C, d)
    _, b1 = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y, C, d)
    assert abs(b[1, 0]) < 1e-13 and abs(b[6, 0]) < 1e-13
    assert rel(b, b1) < 1e-10


# ---------------------------------------------------------------- adjoint

def test_gradient_matches_finite_differences():
    p = S.make_problem(G=3, M=10, n_i=[2, 2, 3], k=1, seed=41, omega="chol")
    target = S.rng(5).standard_normal((p.n, 1))

    def loss(Y, Om):
        _, b = O.aug_dense_solve(p.X_blocks, Om, Y)
        return float(np.sum((b - target) ** 2))

    _, b = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    lam, gO = O.sur_gls_gradient(p.X_blocks, p.Omega, p.Y, 2 * (b - target))
    # adjoint identity X^T lam = dL/db
    _, X = O.sur_dense(p.X_blocks, p.Omega)
    assert rel(X.T @ lam, 2 * (b - target)) < 1e-10
    h = 1e-6
    g = S.rng(6)
    for _ in range(4):
        dY = g.standard_normal(p.Y.shape)
        fd = (loss(p.Y + h * dY, p.Omega) - loss(p.Y - h * dY, p.Omega)) / (2 * h)
        assert abs(fd - np.sum(lam * dY)) < 1e-6 * max(1.0, abs(fd))
        E = g.standard_normal((p.G, p.G)); E = E + E.T
        fd = (loss(p.Y, p.Omega + h * E) - loss(p.Y, p.Omega - h * E)) / (2 * h)
        assert abs(fd - np.sum(gO * E)) < 1e-6 * max(1.0, abs(fd))


def test_kron_gradient_matches_dense_adjoint():
    # the Kronecker-inverse adjoint against the dense augmented-system adjoint
    for seed, omega in ((42, "chol"), (43, "wishart"), (44, "spectrum")):
        p = S.make_problem(G=4, M=9, n_i=[2, 3, 1, 2], k=2, seed=seed, omega=omega)
        gb = S.rng(seed + 100).standard_normal((p.n, 2))
        w_d, b_d = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
        lam_d, gO_d = O.sur_gls_gradient(p.X_blocks, p.Omega, p.Y, gb)
        b, w, lam, gO = O.sur_gls_gradient_kron(p.X_blocks, p.Omega, p.Y, gb)
        assert rel(b, b_d) < 1e-10 and rel(w, w_d) < 1e-9
        assert rel(lam, lam_d) < 1e-9 and rel(gO, gO_d) < 1e-9


def test_kron_gradient_finite_differences_medium():
    # directional central differences of L(b) = ||b - target||^2 at G = 8, M = 60
    p = S.make_problem(G=8, M=60, n_i=[3, 5, 2, 4, 6, 3, 2, 5], k=1, seed=45, omega="chol")
    target = S.rng(46).standard_normal((p.n, 1))

    def loss(Y, Om):
        return float(np.sum((O.gls_formula(p.X_blocks, Om, Y) - target) ** 2))

    b, w, lam, gO = O.sur_gls_gradient_kron(p.X_blocks, p.Omega, p.Y, 0 * target)
    b, w, lam, gO = O.sur_gls_gradient_kron(p.X_blocks, p.Omega, p.Y, 2 * (b - target))
    # adjoint identity X^T lam = dL/db
    xtl = np.concatenate([p.X_blocks[i].T @ lam[i * p.M:(i + 1) * p.M, 0] for i in range(p.G)])
    assert rel(xtl, 2 * (b - target)[:, 0]) < 1e-10
    h, g = 1e-6, S.rng(47)
    for _ in range(3):
        dY = g.standard_normal(p.Y.shape)
        fd = (loss(p.Y + h * dY, p.Omega) - loss(p.Y - h * dY, p.Omega)) / (2 * h)
        assert abs(fd - np.sum(lam * dY)) < 1e-6 * max(1.0, abs(fd))
        E = g.standard_normal((p.G, p.G)); E = E + E.T
        fd = (loss(p.Y, p.Omega + h * E) - loss(p.Y, p.Omega - h * E)) / (2 * h)
        assert abs(fd - np.sum(gO * E)) < 1e-6 * max(1.0, abs(fd))


def test_refined_solution_matches_dense_and_converges():
    # extended-precision refinement: equal to the dense brute force on tiny
    # inputs; the corrections fall to the float64 rounding level
    p = S.make_problem(G=4, M=9, n_i=[2, 3, 1, 2], k=2, seed=48, omega="chol")
    gb = S.rng(49).standard_normal((p.n, 2))
    out = O.sur_gls_refined(p.X_blocks, p.Omega, p.Y, gb, steps=3)
    w_d, b_d = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    lam_d, gO_d = O.sur_gls_gradient(p.X_blocks, p.Omega, p.Y, gb)
    assert rel(out["b"], b_d) < 1e-12 and rel(out["w"], w_d) < 1e-11
    assert rel(out["lam"], lam_d) < 1e-11 and rel(out["dOmega"], gO_d) < 1e-11
    # an ill-conditioned Omega (G = 128, cond ~ 5e6): the first correction is
    # the normal equations' error, the later ones settle below 1e-15
    q, Lf, _ = S.differentiable_g128_m40000(M=20, G=128, nmin=2, nmax=4)
    assert np.linalg.cond(q.Omega) > 1e6
    out = O.sur_gls_refined(q.X_blocks, q.Omega, q.Y, steps=3)
    c = out["corrections"][0]
    assert c[1] > 1e-12 and c[-1] < 1e-15 and c[-2] < 1e-15, c
    assert rel(out["b"], O.gls_formula(q.X_blocks, q.Omega, q.Y)) < 1e-8


def test_augmented_residual_of_exact_solution_is_zero():
    p = S.make_problem(G=3, M=12, n_i=[2, 3, 2], k=2, seed=51, omega="chol")
    w, b = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    top, bot = O.augmented_residual(p.X_blocks, p.Omega, p.Y, w, b)
    assert np.linalg.norm(top) < 1e-11 * np.linalg.norm(p.Y)
    assert np.linalg.norm(bot) < 1e-11 * np.linalg.norm(p.Y)
    top, _ = O.augmented_residual(p.X_blocks, p.Omega, p.Y, w, b + 1e-3)
    assert np.linalg.norm(top) > 1e-5


# ---------------------------------------------------------------- planted mistakes

def test_planted_sign_error_in_sigma_apply_is_caught():
    # A plausible bug (transposed Omega in the Sigma-apply) must fail the
    # brute-force comparison: Omega non-symmetric input exposes it.
    p = S.make_problem(G=3, M=12, n_i=[2, 3, 2], k=1, seed=61, omega="chol")
    op = O.SurOps(p.X_blocks, p.Omega)
    Sigma, _ = O.sur_dense(p.X_blocks, p.Omega)
    u = S.rng(1).standard_normal((p.m, 1))
    assert rel(op.sigma(u), Sigma @ u) < 1e-14
    A = S.rng(2).standard_normal((3, 3))
    op.Omega = A
    Sg, _ = O.sur_dense(p.X_blocks, A)
    # (U Omega)_h = sum_g U_g omega_gh  <->  Sigma = Omega^T (x) I acting on vec(U)
    assert rel(op.sigma(u), Sg.T @ u) < 1e-14


# ---------------------------------------------------------------- invariances

def test_scaling_omega_leaves_b_and_scales_w():
    # Sigma -> c Sigma: (w, b) -> (w / c, b) solves eq. (aug1) again
    p = S.make_problem(G=3, M=20, n_i=[2, 3, 2], k=2, seed=71, omega="chol")
    w, b = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
    w2, b2 = O.aug_dense_solve(p.X_blocks, 7.5 * p.Omega, p.Y)
    assert rel(b2, b) < 1e-12 and rel(7.5 * w2, w) < 1e-11
    res = O.sur_pcg_aug(p.X_blocks, 7.5 * p.Omega, p.Y, tol=1e-14)
    assert rel(res["b"], b) < 1e-10


def test_permuting_equations_permutes_b():
    # reordering the equations (blocks of X and y, rows/columns of Omega)
    # reorders the blocks of b and nothing else
    p = S.make_problem(G=4, M=25, n_i=[2, 3, 1, 2], k=1, seed=72, omega="chol")
    perm = [2, 0, 3, 1]
    Xp = [p.X_blocks[i] for i in perm]
    Op = p.Omega[np.ix_(perm, perm)]
    Yp = np.vstack([p.Y[i * p.M:(i + 1) * p.M] for i in perm])
    b = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
    bp = O.sur_gls_structured(Xp, Op, Yp)
    offs = np.cumsum([0] + p.n_i)
    b_perm = np.vstack([b[offs[i]:offs[i + 1]] for i in perm])
    assert rel(bp, b_perm) < 1e-12
    res = O.sur_pcg_aug(Xp, Op, Yp, tol=1e-14)
    assert rel(res["b"], b_perm) < 1e-10


def test_row_reduction_leaves_b_unchanged():
    # Remark rem:reduction: rotating the rows of every equation onto range(W),
    # W = [X_1 ... X_G], gives a model with the same estimate (dense brute force
    # on both models; singular and regular Omega)
    for seed, omega, rank in ((73, "chol", None), (74, "lowrank", 2)):
        p = S.make_problem(G=3, M=30, n_i=[2, 3, 2], k=2, seed=seed, omega=omega, rank=rank)
        B = O.range_basis(np.hstack(p.X_blocks))
        Xr = [B.T @ x for x in p.X_blocks]
        Yr = np.vstack([B.T @ p.Y[i * p.M:(i + 1) * p.M] for i in range(p.G)])
        _, b = O.aug_dense_solve(p.X_blocks, p.Omega, p.Y)
        _, br = O.aug_dense_solve(Xr, p.Omega, Yr)
        assert rel(br, b) < 1e-10


def test_reduced_projected_residual_plus_complement_energy_is_the_full_one():
    # Remark rem:reduction: with Q an orthonormal basis of range(W) the rows
    # outside range(W) carry no regressor, so for each equation
    # ||Pi y_i||^2 = ||Pi' y_i'||^2 + ||y_i||^2 - ||Q^T y_i||^2 (y_i' = Q^T y_i,
    # X_i' = Q^T X_i): the reference of the reduced solve's tolerance
    # The identity holds equation by equation, so it also holds under the row
    # scaling of a preconditioner block (equation i weighted by 1/delta_i).
    p = S.make_problem(G=4, M=300, n_i=[3, 5, 2, 4], k=3, seed=91, omega="chol")
    Q = O.range_basis(np.hstack(p.X_blocks))
    delta = O.jacobi_delta(p.Omega)
    tot = np.zeros((2, p.k))
    for i, X in enumerate(p.X_blocks):
        y = p.Y[i * p.M:(i + 1) * p.M]
        Qi = O.range_basis(X)
        full = np.sum((y - Qi @ (Qi.T @ y)) ** 2, axis=0)
        yr, Xr = Q.T @ y, Q.T @ X
        Qri = O.range_basis(Xr)
        red = np.sum((yr - Qri @ (Qri.T @ yr)) ** 2, axis=0)
        comp = np.sum(y ** 2, axis=0) - np.sum(yr ** 2, axis=0)
        assert np.all(comp > 0.5 * full)       # most of the noise lies outside range(W)
        assert np.max(np.abs(full - (red + comp)) / full) < 1e-12
        tot += np.vstack([full, red + comp]) / delta[i]
    assert np.max(np.abs(tot[0] - tot[1]) / tot[0]) < 1e-12

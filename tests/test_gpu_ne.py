"""PCG-NE (glm_sur_solve_ne) on the GPU against the oracle's PCG-NE and the
direct GLS solvers: CG with K = I on X^T Sigma^-1 X beta = X^T Sigma^-1 y
(Sec. "Statistical properties of the PCG-Aug estimator", the comparator of
the Monte-Carlo study and of Sec. "Experimental Tests").  Tolerance: relative
||b - b_ref|| <= 1e-9 per right-hand side at convergence; the step counts of
the GPU and of the oracle agree within 2 (CG in float64, different sum
orders)."""
import numpy as np
import pytest

from oracle import sur_oracle as O
from synth import sur_inputs as S

pytestmark = pytest.mark.gpu

TOL_B = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_14471_gb300 import build
    build.build()


def relcols(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300))


def solve_ne(X, Om, Y, **kw):
    from paper_2510_14471_gb300.sur import GlmSur
    h = GlmSur(X, Om, precision="fp64", **kw)
    r = h.solve_ne(Y)
    out = dict(b=r.b.cpu().numpy(), iters=r.iters.cpu().numpy(), status=r.status,
               relres=r.relres.cpu().numpy())
    h.close()
    return out


@pytest.mark.parametrize("G,M,n_i,k,omega", [
    (3, 200, [5, 4, 6], 1, "chol"),
    (4, 997, [5, 3, 9, 2], 3, "chol"),
    (8, 3001, [7, 12, 3, 9, 16, 5, 8, 11], 16, "spectrum"),
    (16, 2500, [8] * 16, 4, "wishart"),
])
def test_ne_matches_oracle_and_gls(G, M, n_i, k, omega):
    p = S.make_problem(G=G, M=M, n_i=n_i, k=k, seed=G * 7 + M, omega=omega)
    r = solve_ne(p.X_blocks, p.Omega, p.Y, tol=1e-12)
    ref = O.pcg_ne(p.X_blocks, p.Omega, p.Y, tol=1e-12, maxit=4 * p.n)
    assert r["status"] == [0] * k, r["status"]
    assert np.all(np.abs(r["iters"].astype(int) - np.asarray(ref["iters"])) <= 2), (r["iters"], ref["iters"])
    assert relcols(r["b"], O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)) <= TOL_B
    assert relcols(r["b"], ref["b"]) <= TOL_B


def test_ne_iterates_follow_the_oracle():
    # a fixed number of steps (maxit, tol 0): the partial iterate equals the
    # oracle's CG iterate after the same steps
    p = S.make_problem(G=5, M=800, n_i=[4, 6, 3, 5, 7], k=2, seed=61, omega="chol")
    for steps in (1, 3, 7):
        r = solve_ne(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=steps)
        ref = O.pcg_ne(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=steps)
        assert list(r["iters"]) == [steps, steps]
        assert r["status"] == [5, 5]          # GLM_SUR_NOT_CONVERGED at maxit
        assert relcols(r["b"], ref["b"]) <= 1e-10, steps
        assert np.allclose(r["relres"], ref["relres"], rtol=1e-8)


def test_ne_steps_equal_the_distinct_eigenvalues():
    # orthonormal X_i, diagonal Omega with 4 distinct values: 4 steps
    g = S.rng(59)
    X = [np.linalg.qr(x)[0] for x in S.gaussian_blocks(g, 500, [3, 2, 3, 2, 3])]
    Om = np.diag([1.0, 2.0, 5.0, 5.0, 0.5])
    Y, _ = S.draw_responses(g, X, np.linalg.cholesky(Om), 500, 2)
    r = solve_ne(X, Om, Y, tol=1e-12)
    assert list(r["iters"]) == [4, 4]
    assert relcols(r["b"], O.gls_formula(X, Om, Y)) <= 1e-12


def test_ne_on_ill_conditioned_regressors_needs_more_than_n_steps():
    g = S.rng(57)
    G, M = 5, 400
    X = S.gaussian_blocks(g, M, [3, 2, 3, 2, 3])
    for i in range(G):
        U, s, Vt = np.linalg.svd(X[i], full_matrices=False)
        X[i] = U @ np.diag(np.logspace(0, -5, len(s))) @ Vt
    A = g.standard_normal((G, G))
    Om = A @ A.T / G + np.eye(G)
    Y, _ = S.draw_responses(g, X, np.linalg.cholesky(Om), M, 1)
    r = solve_ne(X, Om, Y, tol=1e-10, maxit=130)
    ref = O.pcg_ne(X, Om, Y, tol=1e-10, maxit=130)
    # cond(X^T Sigma^-1 X) ~ 1e10: the step count depends on the rounding of
    # every sum (oracle: 45 on one host, 46 on another), so only the property
    # the paper draws is pinned, with the counts within 25 %, and the
    # estimate's error against GLS within 10x the oracle's own
    it_gpu, it_ref = int(r["iters"][0]), int(ref["iters"][0])
    assert r["status"] == [0] and it_gpu > 3 * 13 and it_ref > 3 * 13
    assert abs(it_gpu - it_ref) <= 0.25 * it_ref, (it_gpu, it_ref)
    bg = O.gls_formula(X, Om, Y)
    assert relcols(r["b"], bg) <= 10 * relcols(ref["b"], bg) + 1e-12


def test_ne_row_reduced_handle():
    p = S.make_problem(G=4, M=5000, n_i=[3, 5, 4, 2], k=3, seed=67, omega="chol")
    r = solve_ne(p.X_blocks, p.Omega, p.Y, tol=1e-12, reduce_rows=True)
    assert r["status"] == [0, 0, 0]
    assert relcols(r["b"], O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)) <= TOL_B


def test_ne_refusals():
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur
    # singular Omega: the normal equations need Sigma^-1
    p = S.make_problem(G=5, M=300, n_i=[3, 4, 2, 5, 3], k=1, seed=71, omega="lowrank", rank=3)
    h = GlmSur(p.X_blocks, p.Omega, precision="fp64")
    with pytest.raises(L.GlmSurError):
        h.solve_ne(p.Y)
    # the w of a PCG-Aug solve is gone after PCG-NE: backward is refused
    q = S.make_problem(G=3, M=300, n_i=[3, 4, 2], k=1, seed=73, omega="chol")
    h2 = GlmSur(q.X_blocks, q.Omega, precision="fp64")
    h2.solve(q.Y)
    h2.solve_ne(q.Y)
    with pytest.raises(L.GlmSurError):
        h2.backward(np.ones((q.n, 1)))
    h.close()
    h2.close()

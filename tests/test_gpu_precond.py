"""The preconditioner block D = D0 (x) I_M of eq. (invprec) on the GPU
(opts.precond: D0 = alpha I with alpha = max omega_ii, or D0 = diag(Omega)),
against the oracle: the estimate against the direct solvers, the step counts
against the oracle's Algorithm glmpcg2 run with the same D.  Tolerance:
relative ||b - b_oracle|| <= 1e-9 per right-hand side."""
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


def solve(p, precond, precision="fp64", **kw):
    from paper_2510_14471_gb300.sur import GlmSur
    h = GlmSur(p.X_blocks, p.Omega, precision=precision, precond=precond, **kw)
    r = h.solve(p.Y)
    return h, dict(b=r.b.cpu().numpy(), iters=r.iters.cpu().numpy(), status=r.status)


@pytest.mark.parametrize("precond", ["scaled", "diag"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("G,M,n_i,k,omega,rank", [
    (4, 997, [5, 3, 9, 2], 3, "chol", None),
    (6, 1501, [4, 4, 7, 3, 8, 5], 16, "spectrum", None),
    (5, 800, [3, 4, 2, 5, 3], 2, "lowrank", 3),      # singular Omega
])
def test_precond_matches_oracle(precond, precision, G, M, n_i, k, omega, rank):
    p = S.make_problem(G=G, M=M, n_i=n_i, k=k, seed=G * 101 + M, omega=omega, rank=rank)
    b_ref = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
    h, r = solve(p, precond, precision, tol=1e-13)
    assert all(s in (0, 4) for s in r["status"]), r["status"]
    assert relcols(r["b"], b_ref) <= TOL_B, (relcols(r["b"], b_ref), r["iters"])
    h.close()


@pytest.mark.parametrize("precond,delta_fn", [("scaled", O.scaled_identity_delta), ("diag", O.jacobi_delta)])
def test_precond_step_counts_match_reference_pcg(precond, delta_fn):
    p = S.make_problem(G=5, M=400, n_i=[3, 5, 2, 4, 6], k=4, seed=41, omega="chol")
    ref = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=1e-10, delta=delta_fn(p.Omega))
    h, r = solve(p, precond, tol=1e-10)
    assert np.all(np.abs(r["iters"].astype(int) - ref["iters"].astype(int)) <= 2), (r["iters"], ref["iters"])
    assert relcols(r["b"], ref["b"]) <= TOL_B
    h.close()


def test_diagonal_block_on_a_badly_scaled_omega():
    # equation scales over two orders of magnitude: D = diag(Sigma) converges
    # in a few dozen steps to the GLS estimate (the oracle's pin shows D = I
    # still far from it after m - n + 1 steps)
    g = S.rng(5)
    G, M = 6, 600
    X = S.gaussian_blocks(g, M, [3, 2, 4, 3, 2, 3])
    A = g.standard_normal((G, G))
    R = A @ A.T / G + np.eye(G)
    d = np.sqrt(np.diag(R))
    R = R / np.outer(d, d)
    sc = np.logspace(-1, 1, G)
    Om = np.outer(sc, sc) * R
    Y, _ = S.draw_responses(g, X, np.linalg.cholesky(Om), M, 2)
    from paper_2510_14471_gb300.sur import GlmSur
    h = GlmSur(X, Om, precision="fp64", precond="diag", tol=1e-12, stagnation_window=1000)
    r = h.solve(Y)
    b_ref = O.gls_formula(X, Om, Y)
    assert r.status == [0, 0]
    assert int(r.iters.max()) <= 40
    assert relcols(r.b.cpu().numpy(), b_ref) <= TOL_B
    h.close()


def test_precond_refusals():
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur
    p = S.make_problem(G=3, M=60, n_i=[3, 2, 3], k=1, seed=43, omega="chol", n_constraints=2)
    h = GlmSur(p.X_blocks, p.Omega, precision="fp64", precond="diag")
    h.solve(p.Y)
    h.set_restrictions(p.C)
    with pytest.raises(L.GlmSurError):
        h.solve(p.Y, d=p.d)
    h.close()


@pytest.mark.parametrize("precond,precision,reduce_rows",
                         [("diag", "fp64", False), ("scaled", "fp64", False), ("diag", "fp32_refine", False),
                          ("diag", "fp64", True)])
def test_precond_w_and_adjoint_match_oracle(precond, precision, reduce_rows):
    """A preconditioner block changes the iteration's model, not b: get_w
    returns the given model's w = S w~ and the adjoint its dL/dy = S dL/dy~
    and dL/dOmega = D0^-1/2 dL/dOmega~ D0^-1/2, compared with the oracle's
    Kronecker-inverse adjoint (eq. (GLS), Sigma^-1 = Omega^-1 (x) I_M) on an
    Omega whose diagonal spans two decades."""
    from paper_2510_14471_gb300.sur import GlmSur
    n_i = [3, 7, 2, 9, 5, 4, 8, 6, 1, 10, 3, 5]
    p = S.make_problem(G=12, M=700, n_i=n_i, k=2, seed=74, omega="chol")
    dsc = np.logspace(-1.0, 1.0, p.G)
    Om = p.Omega * np.sqrt(np.outer(dsc, dsc))
    Y = p.Y.copy()
    for i in range(p.G):
        Y[i * p.M:(i + 1) * p.M] *= np.sqrt(dsc[i])
    gb = S.rng(9).standard_normal((p.n, 2))
    b_o, w_o, lam_o, gO = O.sur_gls_gradient_kron(p.X_blocks, Om, Y, gb)
    h = GlmSur(p.X_blocks, Om, precision=precision, precond=precond, tol=1e-13, stagnation_window=1000,
               reduce_rows=reduce_rows)
    r = h.solve(Y)
    assert relcols(r.b.cpu().numpy(), b_o) <= TOL_B
    if not reduce_rows:                       # w of the rows outside range(W) is not formed on a reduced handle
        assert relcols(h.w(2).cpu().numpy(), w_o) <= TOL_B
    dY, dO, iters, relres, status = h.backward(gb)
    assert all(s in (0, 4) for s in status), status
    lam = dY.cpu().numpy()
    assert relcols(lam, lam_o) <= TOL_B
    gs = 0.5 * (gO + gO.T)
    assert np.linalg.norm(dO.cpu().numpy() - gs) <= TOL_B * np.linalg.norm(gs)
    h.close()

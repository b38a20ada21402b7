"""Row reduction of the model (Remark rem:reduction: the rows of each
equation rotated onto range(W), W = [X_1 ... X_G]) against the float64
oracle and against the unreduced GPU path: the estimate, the restricted
estimate and the adjoint are those of the full model (relative 1e-9)."""
import numpy as np
import pytest

from oracle import sur_oracle as O
from synth import sur_inputs as S

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_14471_gb300 import build
    build.build()


def relcols(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300))


def solver(p, **kw):
    from paper_2510_14471_gb300.sur import GlmSur
    h = GlmSur(p.X_blocks, p.Omega, **kw)
    assert h.setup_status() == 0
    return h


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("omega,rank", [("chol", None), ("lowrank", 3), ("wishart", None)])
def test_reduced_estimate_matches_oracle(precision, omega, rank):
    p = S.make_problem(G=5, M=1500, n_i=[4, 7, 3, 9, 5], k=3, seed=601, omega=omega, rank=rank)
    r = solver(p, precision=precision, reduce_rows=True).solve(p.Y)
    assert all(s in (0, 4) for s in r.status), r.status
    b = r.b.cpu().numpy()
    if omega == "lowrank":
        assert relcols(b, p.beta) <= TOL          # singular Omega: b = beta exactly
    else:
        assert relcols(b, O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)) <= TOL
    b_full = solver(p, precision=precision).solve(p.Y).b.cpu().numpy()
    assert relcols(b, b_full) <= TOL


def test_reduction_falls_back_when_w_is_rank_deficient():
    # equal regressors in every equation: W has rank n_1 < n, the model is kept whole
    p = S.make_problem(G=3, M=800, n_i=[4, 4, 4], k=2, seed=602, omega="chol", equal_X=True)
    h = solver(p, reduce_rows=True)
    r = h.solve(p.Y)
    assert relcols(r.b.cpu().numpy(), O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)) <= TOL
    # the handle is the unreduced one: its factors are available (a reduced
    # handle refuses glm_sur_get_factors) and Q has the model's M rows
    Q, Rs = h.factors()
    assert Q.shape == (800, 12)
    Qn = Q.cpu().numpy()
    assert np.allclose(Qn[:, :4] @ Rs[0].cpu().numpy(), p.X_blocks[0], atol=1e-10)


def test_reduced_restricted_estimate():
    p = S.make_problem(G=4, M=1200, n_i=[5, 3, 6, 4], k=2, seed=603, omega="spectrum", n_constraints=5)
    h = solver(p, reduce_rows=True)
    h.set_restrictions(p.C)
    r = h.solve(p.Y, d=p.d)
    ref = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y, C=p.C, d=p.d)
    assert relcols(r.b.cpu().numpy(), ref) <= TOL


def test_reduced_adjoint_matches_oracle():
    p = S.make_problem(G=6, M=900, n_i=[3, 5, 2, 6, 4, 3], k=2, seed=604, omega="chol")
    gb = S.rng(605).standard_normal((p.n, 2))
    h = solver(p, reduce_rows=True)
    h.solve(p.Y)
    dY, dO, _, _, status = h.backward(gb)
    assert all(s in (0, 4) for s in status), status
    _, _, lam, gO = O.sur_gls_gradient_kron(p.X_blocks, p.Omega, p.Y, gb)
    assert relcols(dY.cpu().numpy(), lam) <= TOL
    assert np.linalg.norm(dO.cpu().numpy() - 0.5 * (gO + gO.T)) <= TOL * np.linalg.norm(gO + gO.T) / 2


def test_reduced_full_size_singular_workload():
    # the benchmark workload (M = 20000 rows reduced to n = 1234)
    p = S.singular_g64_m20000(k=16)
    r = solver(p, precision="fp32_refine", reduce_rows=True).solve(p.Y)
    assert all(s in (0, 4) for s in r.status), r.status
    assert relcols(r.b.cpu().numpy(), p.beta) <= TOL


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_reduced_tolerance_refers_to_the_full_model(precision):
    # y = X beta + e with e almost all outside range(W): ||Pi y|| of the
    # M-row model is about 1e8 times ||Pi' y'|| of the reduced one.  A
    # tolerance relative to ||Pi y|| (the full model's) is met at the start
    # of the reduced solve; one relative to ||Pi' y'|| would have to iterate.
    p = S.make_problem(G=4, M=2000, n_i=[3, 5, 2, 4], k=2, seed=604, omega="chol")
    Q = O.range_basis(np.hstack(p.X_blocks))
    g = S.rng(605)
    Y = np.empty_like(p.Y)
    for i, X in enumerate(p.X_blocks):
        z = g.standard_normal((p.M, p.k))
        e = z - Q @ (Q.T @ z) + 1e-8 * g.standard_normal((p.M, p.k))
        off = sum(p.n_i[:i])
        Y[i * p.M:(i + 1) * p.M] = X @ p.beta[off:off + X.shape[1]] + e
    h = solver(p, precision=precision, reduce_rows=True, tol=1e-6)
    r = h.solve(Y)
    assert list(r.status) == [0] * p.k, r.status
    assert int(r.iters.max()) == 0, r.iters
    assert float(r.relres.max()) <= 1e-6
    assert relcols(r.b.cpu().numpy(), O.sur_gls_structured(p.X_blocks, p.Omega, Y)) <= 1e-6

"""Edge cases of the boundary on the GPU: the largest k and G a solve takes
(and the first ones it refuses), responses exactly in range(X), one
equation, and a batched instance at the batch limits.  Each result is
compared with the float64 oracle (relative 1e-9 per right-hand side)."""
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


def solver(p, **kw):
    from paper_2510_14471_gb300.sur import GlmSur
    h = GlmSur(p.X_blocks, p.Omega, **kw)
    assert h.setup_status() == 0
    return h


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_largest_k(precision):
    p = S.make_problem(G=3, M=150, n_i=[2, 3, 4], k=64, seed=501, omega="chol")
    r = solver(p, precision=precision).solve(p.Y)
    assert all(s in (0, 4) for s in r.status)
    assert relcols(r.b.cpu().numpy(), O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)) <= TOL_B


def test_k_beyond_limit_is_refused():
    from paper_2510_14471_gb300 import _lib as L
    p = S.make_problem(G=2, M=40, n_i=[2, 3], k=65, seed=502, omega="chol")
    with pytest.raises(L.GlmSurError):
        solver(p).solve(p.Y)


def test_largest_g_and_first_refused():
    from paper_2510_14471_gb300 import _lib as L
    p = S.make_problem(G=156, M=24, n_i=[1] * 156, k=1, seed=503, omega="diag")
    r = solver(p).solve(p.Y)
    # diagonal Omega: GLS is per-block OLS (Sec. 1)
    assert relcols(r.b.cpu().numpy(), O.ols_blocks(p.X_blocks, p.Y)) <= TOL_B
    q = S.make_problem(G=157, M=24, n_i=[1] * 157, k=1, seed=504, omega="diag")
    with pytest.raises(L.GlmSurError):
        solver(q).solve(q.Y)


def test_response_in_range_of_x():
    # y = X beta exactly: P y vanishes up to rounding, w ~ 0 and b = beta
    p = S.make_problem(G=4, M=300, n_i=[3, 2, 5, 4], k=2, seed=505, omega="chol")
    Y = np.vstack([p.X_blocks[i] @ p.beta[sum(x.shape[1] for x in p.X_blocks[:i]):][:p.X_blocks[i].shape[1]]
                   for i in range(p.G)])
    for precision in ("fp64", "fp32_refine"):
        r = solver(p, precision=precision).solve(Y)
        assert all(s in (0, 4) for s in r.status), (precision, r.status)
        assert relcols(r.b.cpu().numpy(), p.beta) <= 1e-12, precision


def test_single_equation_is_ols():
    p = S.make_problem(G=1, M=500, n_i=[7], k=3, seed=506, omega="chol")
    r = solver(p, precision="fp32_refine").solve(p.Y)
    assert relcols(r.b.cpu().numpy(), O.ols_blocks(p.X_blocks, p.Y)) <= TOL_B


def test_batched_instance_at_the_limits():
    # G = 32 equations of 16 columns (n' = 512) with k = 8 in one batch with a small instance
    from paper_2510_14471_gb300.sur import GlmSurBatch
    big = S.make_problem(G=32, M=600, n_i=[16] * 32, k=8, seed=507, omega="wishart")
    small = S.make_problem(G=2, M=40, n_i=[1, 2], k=8, seed=508, omega="chol")
    bt = GlmSurBatch([(big.X_blocks, big.Omega), (small.X_blocks, small.Omega)])
    assert bt.setup_status() == 0
    b, iters, relres, status = bt.solve([big.Y, small.Y], 8)
    assert all(s in (0, 4) for s in status), status
    for q, bq in zip((big, small), b):
        assert relcols(bq.cpu().numpy(), O.sur_gls_structured(q.X_blocks, q.Omega, q.Y)) <= TOL_B


def test_scaling_omega_leaves_b_unchanged():
    p = S.make_problem(G=5, M=700, n_i=[3, 4, 2, 5, 3], k=2, seed=509, omega="chol")
    h = solver(p)
    b1 = h.solve(p.Y).b.cpu().numpy()
    h.set_omega(12.5 * p.Omega)
    b2 = h.solve(p.Y).b.cpu().numpy()
    assert relcols(b2, b1) <= TOL_B
    assert relcols(b1, O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)) <= TOL_B


def test_permuting_equations_permutes_b():
    p = S.make_problem(G=5, M=700, n_i=[3, 4, 2, 5, 3], k=3, seed=510, omega="spectrum")
    perm = [3, 0, 4, 2, 1]
    q_blocks = [p.X_blocks[i] for i in perm]
    q_omega = p.Omega[np.ix_(perm, perm)]
    q_y = np.vstack([p.Y[i * p.M:(i + 1) * p.M] for i in perm])
    from paper_2510_14471_gb300.sur import GlmSur
    b = solver(p, precision="fp32_refine").solve(p.Y).b.cpu().numpy()
    bq = GlmSur(q_blocks, q_omega, precision="fp32_refine").solve(q_y).b
    offs = np.cumsum([0] + p.n_i)
    b_perm = np.vstack([b[offs[i]:offs[i + 1]] for i in perm])
    assert relcols(bq.cpu().numpy(), b_perm) <= TOL_B


def test_one_handle_many_solves_and_precisions():
    # k grows and shrinks and the precision changes on one handle; every
    # result against the oracle
    p = S.make_problem(G=4, M=900, n_i=[6, 3, 8, 5], k=8, seed=511, omega="wishart")
    ref = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
    h = solver(p)
    for precision, cols in (("fp64", [0, 1]), ("fp64", list(range(8))), ("fp32_refine", [2, 3, 4, 5]),
                            ("fp32_refine", [7]), ("fp64", [6, 1, 0])):
        h.set_options(precision=precision)
        r = h.solve(p.Y[:, cols])
        assert all(s in (0, 4) for s in r.status), (precision, cols, r.status)
        assert relcols(r.b.cpu().numpy(), ref[:, cols]) <= TOL_B, (precision, cols)

"""Algorithm glmpcg3 on the GPU (opts.algorithm = GLMPCG3, float64) against
the oracle's glmpcg3 and the direct solvers: the estimate at convergence,
the iterate after a fixed number of steps (equal to the oracle's glmpcg3
and glmpcg2 iterates in exact arithmetic), the preconditioner blocks, and
the refusals.  Tolerance: relative ||b - b_ref|| <= 1e-9 per right-hand side."""
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


@pytest.mark.parametrize("G,M,n_i,k,omega,precond", [
    (4, 997, [5, 3, 9, 2], 3, "chol", "identity"),
    (8, 2001, [7, 12, 3, 9, 16, 5, 8, 11], 8, "spectrum", "identity"),
    (6, 1501, [4, 4, 7, 3, 8, 5], 4, "chol", "diag"),
])
def test_glmpcg3_converges_to_the_gls_estimate(G, M, n_i, k, omega, precond):
    from paper_2510_14471_gb300.sur import GlmSur
    p = S.make_problem(G=G, M=M, n_i=n_i, k=k, seed=G * 13 + M, omega=omega)
    h = GlmSur(p.X_blocks, p.Omega, precision="fp64", tol=1e-12, algorithm="glmpcg3", precond=precond)
    r = h.solve(p.Y)
    assert r.status == [0] * k, (r.status, r.iters)
    assert relcols(r.b.cpu().numpy(), O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)) <= TOL_B
    # the step counts of glmpcg2 on the same handle (the same iterates in exact arithmetic)
    h2 = GlmSur(p.X_blocks, p.Omega, precision="fp64", tol=1e-12, precond=precond)
    r2 = h2.solve(p.Y)
    assert np.all(np.abs(r.iters.cpu().numpy().astype(int) - r2.iters.cpu().numpy().astype(int)) <= 3)
    h.close()
    h2.close()


@pytest.mark.parametrize("steps", [1, 4, 9])
def test_glmpcg3_iterate_after_fixed_steps_equals_the_oracle(steps):
    from paper_2510_14471_gb300.sur import GlmSur
    p = S.make_problem(G=5, M=600, n_i=[3, 5, 2, 4, 6], k=2, seed=131, omega="chol")
    h = GlmSur(p.X_blocks, p.Omega, precision="fp64", tol=0.0, maxit=steps, algorithm="glmpcg3")
    r = h.solve(p.Y)
    assert list(r.iters.cpu().numpy()) == [steps, steps]
    ref3 = O.sur_pcg_aug3(p.X_blocks, p.Omega, p.Y, steps)["b"]
    ref2 = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=steps, stag_window=1000)["b"]
    b = r.b.cpu().numpy()
    assert relcols(b, ref3) <= TOL_B
    assert relcols(b, ref2) <= TOL_B
    h.close()


def test_glmpcg3_refusals():
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur
    p = S.make_problem(G=3, M=200, n_i=[3, 2, 3], k=1, seed=137, omega="chol", n_constraints=2)
    h = GlmSur(p.X_blocks, p.Omega, precision="fp32_refine", algorithm="glmpcg3")
    with pytest.raises(L.GlmSurError):
        h.solve(p.Y)
    h.close()
    h = GlmSur(p.X_blocks, p.Omega, precision="fp64", algorithm="glmpcg3")
    h.set_restrictions(p.C)
    with pytest.raises(L.GlmSurError):
        h.solve(p.Y, d=p.d)
    h.close()

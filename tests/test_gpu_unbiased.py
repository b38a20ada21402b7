"""Theorem t:glmPcgUnbiased (Sec. 3.4) on the GPU path: with w_1 = 0 the
float64 iterate after any number of steps is an odd function of the
disturbance, z_i(X beta + eps) + z_i(X beta - eps) = 2 beta (the two signs
as two right-hand sides of one solve; the even stop statistics c_i take the
same decisions for both), and the iterate is one of the oracle's iterates;
the PCG-NE iterates of the GPU are not odd.  Tolerance: 1e-10 relative to
||beta|| for the sum (P X beta vanishes only to rounding), 1e-9 for the
iterates."""
import numpy as np
import pytest

from oracle import sur_oracle as O
from synth import sur_inputs as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_14471_gb300 import build
    build.build()


@pytest.mark.parametrize("steps", [1, 2, 3, 7])
def test_gpu_iterates_are_odd_and_follow_the_oracle(steps):
    from paper_2510_14471_gb300.sur import GlmSur
    X, Om, beta, Y, Xb = S.monte_carlo_problem(4)
    eps = Y[:, :1] - Xb
    Ypm = np.hstack([Xb + eps, Xb - eps])
    h = GlmSur(X, Om, precision="fp64", tol=0.0, maxit=steps, stagnation_window=1000)
    r = h.solve(Ypm)
    b = r.b.cpu().numpy()
    assert list(r.iters.cpu().numpy()) == [steps, steps]
    s = b[:, 0] + b[:, 1] - 2.0 * beta[:, 0]
    assert np.linalg.norm(s) <= 1e-10 * np.linalg.norm(beta), np.linalg.norm(s)
    # the returned iterate (the last one, or the best saved one) is an oracle iterate
    errs = []
    for j in range(1, steps + 1):
        ref = O.sur_pcg_aug(X, Om, Ypm, tol=0.0, maxit=j, stag_window=1000)["b"]
        errs.append(np.linalg.norm(b - ref) / np.linalg.norm(ref))
    assert min(errs) <= 1e-9, errs
    # PCG-NE on the GPU: not odd
    ne = h.solve_ne(Ypm)
    bn = ne.b.cpu().numpy()
    assert np.linalg.norm(bn[:, 0] + bn[:, 1] - 2.0 * beta[:, 0]) >= 0.1 * np.linalg.norm(beta)
    h.close()

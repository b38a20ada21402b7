"""The allocation-free entry point glm_sur_ols_static, called through the C
ABI, against the existing solver and the oracle's per-block least squares.

glm_sur_ols_static returns the per-block least-squares estimate
R_i^-1 Q_i^T y_i from a handle's factors using only the library's fixed
scratch array (for callers that cannot allocate device memory).  With a
diagonal Omega the GLS estimate of glm_sur_solve is exactly that per-block
estimate (the equations decouple), so the two entry points must agree to the
parity tolerance of the other GPU tests.  Collected last on purpose: it runs
after every other test, and also passes alone in a fresh process."""
import ctypes

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


def test_ols_static_matches_solver_on_two_calls_in_a_row():
    import torch
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur

    p = S.make_problem(G=6, M=3001, n_i=[3, 8, 5, 12, 7, 4], k=4, seed=71, omega="diag")
    h = GlmSur(p.X_blocks, p.Omega, precision="fp64", tol=1e-13)
    ref = h.solve(p.Y).b.cpu().numpy()                      # existing entry point
    ols = O.ols_blocks(p.X_blocks, p.Y)                     # Sec. 1: b_i = (X_i^T X_i)^-1 X_i^T y_i
    Ycm = torch.as_tensor(np.ascontiguousarray(p.Y.T), device="cuda")
    m, k = p.Y.shape
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        b = torch.full((k, p.n), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.glm_sur_ols_static(h.handle, Ycm.data_ptr(), m, k, b.data_ptr(), p.n, stream)
        assert rc == L.GLM_SUR_OK, (call, rc)
        torch.cuda.synchronize()
        got = b.t().cpu().numpy()
        err = np.max(np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0))
        assert err <= TOL_B, (call, err)
        err_o = np.max(np.linalg.norm(got - ols, axis=0) / np.linalg.norm(ols, axis=0))
        assert err_o <= TOL_B, (call, err_o)


def test_ols_static_rejects_requests_beyond_its_scratch():
    import torch
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur

    # n' = 160 * 32 = 5120 padded columns; k = 64 needs 2 * 5120 * 64 > 2^19 doubles
    p = S.make_problem(G=160, M=40, n_i=[32] * 160, k=1, seed=72, omega="diag")
    h = GlmSur(p.X_blocks, p.Omega, precision="fp64")
    m = p.m
    Y = torch.zeros((64, m), dtype=torch.float64, device="cuda")
    b = torch.zeros((64, p.n), dtype=torch.float64, device="cuda")
    rc = L.glm_sur_ols_static(h.handle, Y.data_ptr(), m, 64, b.data_ptr(), p.n,
                              torch.cuda.current_stream().cuda_stream)
    assert rc == L.GLM_SUR_INVALID_ARG

"""The fused float32 step with the Sigma-apply on the tensor cores (tcgen05,
three tf32 products accumulated in tensor memory) inside the float64
iterative refinement, against the structured float64 oracle and against the
four-launch SIMT step on the same inputs.

Shapes cover both operand paddings (G <= 32 -> 32, G <= 64 -> 64), k = 8 and
16 (row tiles of 16 and 8 observations), CTAs whose row range is shorter
than one tile or empty (M below 152 x tile), ragged last tiles, blocks of
32 columns, and a singular Omega.  Tolerance: relative ||b - b_oracle|| <=
1e-9 per right-hand side, the bar of every GPU parity test."""
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


def solve(p, step_kernels):
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur
    h = GlmSur(p.X_blocks, p.Omega, precision="fp32_refine", tol=1e-13, step_kernels=step_kernels)
    r = h.solve(p.Y)
    path = L.glm_sur_step_path(h.handle)
    out = dict(b=r.b.cpu().numpy(), iters=r.iters.cpu().numpy(), status=r.status, path=path)
    h.close()
    return out


def n_list(seed, G, lo, hi):
    return [int(v) for v in np.random.default_rng(seed).integers(lo, hi + 1, size=G)]


CASES = [
    # G, M, n_i, k, omega, rank
    (64, 3001, n_list(1, 64, 8, 32), 16, "spectrum", None),  # Gp = 64, several tiles per CTA, ragged
    (40, 1999, n_list(2, 40, 2, 32), 8, "wishart", None),    # Gp = 64 with padding, tiles of 16 rows
    (17, 2500, n_list(3, 17, 1, 32), 16, "spectrum", None),  # Gp = 32
    (3, 777, [5, 32, 9], 8, "chol", None),                   # fewer rows per CTA than one tile
    (64, 150, n_list(4, 64, 2, 6), 16, "diag", None),        # M < 152: CTAs without rows
    (24, 1201, n_list(5, 24, 3, 20), 16, "lowrank", 20),     # singular Omega
]


@pytest.mark.parametrize("G,M,n_i,k,omega,rank", CASES)
def test_tensor_core_step_matches_oracle(G, M, n_i, k, omega, rank):
    p = S.make_problem(G=G, M=M, n_i=n_i, k=k, seed=G * 13 + M, omega=omega, rank=rank)
    b_ref = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
    r = solve(p, "auto")
    assert r["path"] == 1, "the tensor-core step was not selected"
    assert all(s in (0, 4) for s in r["status"]), r["status"]
    assert relcols(r["b"], b_ref) <= TOL_B, (relcols(r["b"], b_ref), r["iters"], r["status"])


def test_tensor_core_and_simt_steps_agree():
    p = S.make_problem(G=32, M=4099, n_i=n_list(6, 32, 4, 28), k=16, seed=77, omega="chol")
    a = solve(p, "auto")
    b = solve(p, "simt")
    assert a["path"] == 1 and b["path"] == 0
    assert a["status"] == [0] * 16 and b["status"] == [0] * 16, (a["status"], b["status"])
    assert relcols(a["b"], b["b"]) <= TOL_B
    # the same float32 iteration up to rounding; per-column step totals of
    # the refinement's inner solves differ by rounding, their sums stay close
    assert abs(int(a["iters"].sum()) - int(b["iters"].sum())) <= 0.2 * int(b["iters"].sum()), \
        (a["iters"], b["iters"])


def test_ineligible_shapes_keep_the_simt_step():
    # G > 64 and k = 4: the four-launch SIMT step
    p = S.make_problem(G=70, M=300, n_i=[2] * 70, k=16, seed=5, omega="diag")
    assert solve(p, "auto")["path"] == 0
    p = S.make_problem(G=8, M=500, n_i=[3] * 8, k=4, seed=6, omega="chol")
    assert solve(p, "auto")["path"] == 0

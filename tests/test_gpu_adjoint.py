"""Adjoint solve (glm_sur_backward) and the autograd function against the
float64 oracle: dense adjoint on tiny inputs, the Kronecker-inverse adjoint
on larger ones, the adjoint identity X^T lam = dL/db, and central finite
differences of the GPU forward path itself.  Tolerance 1e-9 relative for
oracle comparisons (as for b), 1e-6 for finite differences (h = 1e-6: the
truncation and rounding floor of a central difference)."""
import numpy as np
import pytest
import torch

from oracle import sur_oracle as O
from synth import sur_inputs as S

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_14471_gb300 import build
    build.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def sym(A):
    return 0.5 * (A + A.T)


def xt_lam(p, lam):
    """X^T lam (n, k) for lam (m, k) in the vec layout."""
    return np.vstack([p.X_blocks[i].T @ lam[i * p.M:(i + 1) * p.M] for i in range(p.G)])


def solver_for(p, precision="fp64", **kw):
    from paper_2510_14471_gb300.sur import GlmSur
    h = GlmSur(p.X_blocks, p.Omega, precision=precision, **kw)
    assert h.setup_status() == 0
    return h


@pytest.mark.parametrize("k", [1, 2])
def test_backward_matches_dense_adjoint_tiny(k):
    p = S.make_problem(G=3, M=10, n_i=[2, 2, 3], k=k, seed=41, omega="chol")
    gb = S.rng(7).standard_normal((p.n, k))
    h = solver_for(p)
    r = h.solve(p.Y)
    dY, dO, iters, relres, status = h.backward(gb)
    lam, gO = O.sur_gls_gradient(p.X_blocks, p.Omega, p.Y, gb)
    assert all(s in (0, 4) for s in status), status
    assert rel(dY.cpu().numpy(), lam) <= TOL
    assert rel(dO.cpu().numpy(), sym(gO)) <= TOL
    # the forward w is back in place: a second backward gives the same result
    dY2, dO2, *_ = h.backward(gb)
    assert torch.equal(dY, dY2) and torch.equal(dO, dO2)


@pytest.mark.parametrize("precision,omega,k", [("fp64", "chol", 3), ("fp64", "spectrum", 1),
                                               ("fp32_refine", "wishart", 2)])
def test_backward_matches_kron_adjoint(precision, omega, k):
    n_i = [3, 7, 2, 9, 5, 4, 8, 6, 1, 10, 3, 5]
    p = S.make_problem(G=12, M=700, n_i=n_i, k=k, seed=71, omega=omega)
    gb = S.rng(8).standard_normal((p.n, k))
    h = solver_for(p, precision)
    h.solve(p.Y)
    dY, dO, iters, relres, status = h.backward(gb)
    assert all(s in (0, 4) for s in status), status
    b, w, lam, gO = O.sur_gls_gradient_kron(p.X_blocks, p.Omega, p.Y, gb)
    lam_gpu = dY.cpu().numpy()
    assert rel(lam_gpu, lam) <= TOL
    assert rel(xt_lam(p, lam_gpu), gb) <= TOL
    assert rel(dO.cpu().numpy(), sym(gO)) <= TOL


def test_backward_rejects_mismatched_calls():
    from paper_2510_14471_gb300 import _lib as L
    p = S.make_problem(G=3, M=40, n_i=[2, 3, 2], k=2, seed=72, omega="chol")
    h = solver_for(p)
    with pytest.raises(L.GlmSurError):              # no solve yet
        h.backward(np.ones((p.n, 2)))
    h.solve(p.Y)
    with pytest.raises(L.GlmSurError):              # k differs from the solve
        h.backward(np.ones((p.n, 1)))
    h.set_omega(p.Omega)
    with pytest.raises(L.GlmSurError):              # Omega set after the solve
        h.backward(np.ones((p.n, 2)))
    h.solve(p.Y)
    h.set_options(precision="fp32_refine")
    with pytest.raises(L.GlmSurError):              # precision changed after the solve
        h.backward(np.ones((p.n, 2)))


def _autograd_case(p, precision, target, Lfac):
    from paper_2510_14471_gb300.sur import SurGLSFunction
    h = solver_for(p, precision)
    Y = torch.tensor(p.Y, dtype=torch.float64, device="cuda", requires_grad=True)
    Lt = torch.tensor(Lfac, dtype=torch.float64, device="cuda", requires_grad=True)
    tgt = torch.tensor(target, dtype=torch.float64, device="cuda")

    def loss_of(Yv, Lv):
        b = SurGLSFunction.apply(Yv, Lv @ Lv.T, h)
        return ((b - tgt) ** 2).sum()

    loss = loss_of(Y, torch.tril(Lt))
    loss.backward()
    return h, loss_of, Y, Lt


def test_autograd_cholesky_factor_vs_oracle_and_finite_differences():
    # Omega = L L^T parametrised by its lower factor; loss ||b - target||^2
    g = S.rng(80)
    p, Lfac, target = S.differentiable_g128_m40000(M=300, G=10, nmin=2, nmax=6)
    h, loss_of, Y, Lt = _autograd_case(p, "fp64", target, Lfac)
    gL = torch.tril(Lt.grad).cpu().numpy()
    gY = Y.grad.cpu().numpy()
    # oracle: dL/dOmega (symmetric) -> dL/dL = (G + G^T) L, lower triangle
    b = O.sur_gls_gradient_kron(p.X_blocks, p.Omega, p.Y, np.zeros_like(target))[0]
    _, _, lam, gO = O.sur_gls_gradient_kron(p.X_blocks, p.Omega, p.Y, 2 * (b - target))
    assert rel(gY, lam) <= TOL
    assert rel(gL, np.tril(2 * sym(gO) @ Lfac)) <= TOL
    # central differences of the GPU path itself, along random directions
    hstep = 1e-6
    with torch.no_grad():
        for _ in range(8):
            E = np.tril(g.standard_normal(Lfac.shape))
            Et = torch.tensor(E, device="cuda")
            L0 = torch.tensor(Lfac, device="cuda")
            fd = (loss_of(Y.detach(), L0 + hstep * Et) - loss_of(Y.detach(), L0 - hstep * Et)).item() / (2 * hstep)
            an = float(np.sum(gL * E))
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)
            dYd = g.standard_normal(p.Y.shape)
            Dt = torch.tensor(dYd, device="cuda")
            fd = (loss_of(Y.detach() + hstep * Dt, L0) - loss_of(Y.detach() - hstep * Dt, L0)).item() / (2 * hstep)
            an = float(np.sum(gY * dYd))
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_autograd_refuses_stale_forward():
    from paper_2510_14471_gb300.sur import SurGLSFunction
    p = S.make_problem(G=3, M=40, n_i=[2, 3, 2], k=1, seed=73, omega="chol")
    h = solver_for(p)
    Om = torch.tensor(p.Omega, device="cuda", requires_grad=True)
    b = SurGLSFunction.apply(torch.tensor(p.Y, device="cuda"), Om, h)
    h.solve(p.Y)                                  # a later solve replaces w
    with pytest.raises(RuntimeError):
        b.sum().backward()


# ---------------------------------------------------------------- differentiable workload
# Omega = L L^T with G = 128 (cond ~ 1e6).  The float64 PCG's recursive
# residual drifts from the true one on this problem (b error ~2e-9 at full
# size), so the workload runs float32 steps inside float64 refinement, with
# a stagnation window of 1000 steps (the residual of such an ill-conditioned
# run can go hundreds of steps without a new minimum).  Reference values come
# from the oracle's extended-precision refinement.
CFG4_OPTS = dict(precision="fp32_refine", stagnation_window=1000, max_refine=20)


def test_differentiable_workload_m2000_vs_refined_oracle():
    p, Lfac, target = S.differentiable_g128_m40000(M=2000)
    ref = O.sur_gls_refined(p.X_blocks, p.Omega, p.Y, steps=3)
    gb = 2 * (ref["b"] - target)
    adj = O.sur_gls_refined(p.X_blocks, p.Omega, p.Y, gb, steps=3)
    h = solver_for(p, **CFG4_OPTS)
    r = h.solve(p.Y)
    assert all(s in (0, 4) for s in r.status), r.status
    assert rel(r.b.cpu().numpy(), ref["b"]) <= TOL
    dY, dO, iters, relres, status = h.backward(gb)
    assert all(s in (0, 4) for s in status), status
    assert rel(dY.cpu().numpy(), adj["lam"]) <= TOL
    assert rel(dO.cpu().numpy(), sym(adj["dOmega"])) <= TOL


def test_differentiable_workload_full_size_vs_reference_values():
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "differentiable_g128_m40000_reference.json")))
    p, Lfac, target = S.differentiable_g128_m40000()
    assert (p.G, p.M, p.n) == (gold["G"], gold["M"], gold["n"])
    h = solver_for(p, **CFG4_OPTS)
    r = h.solve(p.Y)
    b = r.b.cpu().numpy()
    assert all(s in (0, 4) for s in r.status), r.status
    bref = np.asarray(gold["b"])[:, None]
    assert rel(b, bref) <= TOL
    gb = 2 * (b - target)
    dY, dO, iters, relres, status = h.backward(gb)
    assert all(s in (0, 4) for s in status), status
    lam = dY.cpu().numpy()[:, 0]
    om = dO.cpu().numpy().reshape(-1)
    # gb differs from the reference's 2 (b_ref - target) by 2 (b - b_ref): a
    # relative change below TOL, passed on to lam and dOmega at most linearly
    assert abs(np.linalg.norm(lam) / gold["lam_norm"] - 1) <= TOL
    assert rel(lam[gold["lam_idx"]], np.asarray(gold["lam"])) <= TOL
    assert abs(np.linalg.norm(om) / gold["dOmega_sym_norm"] - 1) <= TOL
    assert rel(om[gold["dOmega_idx"]], np.asarray(gold["dOmega_sym"])) <= TOL
    # adjoint identity X^T lam = dL/db
    assert rel(xt_lam(p, lam[:, None]), gb) <= TOL


def test_differentiable_workload_full_size_reduced_diag_with_central_differences():
    """The differentiable workload through the path its benchmark times: the
    row-reduced model (Remark rem:reduction) with the preconditioner block D
    = diag(Sigma), float64 steps.  b, dL/dy and dL/dOmega against the stored
    reference values, then central differences (h = 1e-6) of the GPU loss
    along 8 directions of Y and 8 of the Cholesky factor L of Omega = L L^T.
    Two forward solves whose b is within TOL move a difference quotient by at
    most 2 ||b - t|| ||b|| TOL / h; the loss is quadratic in Y and smooth in
    L, so that bound (plus 1e-6 relative for truncation) is the tolerance."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "differentiable_g128_m40000_reference.json")))
    p, Lfac, target = S.differentiable_g128_m40000()
    h = solver_for(p, precision="fp64", precond="diag", stagnation_window=1000, reduce_rows=True)
    r = h.solve(p.Y)
    assert all(s == 0 for s in r.status), r.status
    b = r.b.cpu().numpy()
    assert rel(b, np.asarray(gold["b"])[:, None]) <= TOL
    gb = 2 * (b - target)
    dY, dO, iters, relres, status = h.backward(gb)
    assert all(s == 0 for s in status), status
    lam = dY.cpu().numpy()[:, 0]
    gO = dO.cpu().numpy()
    om = gO.reshape(-1)
    assert abs(np.linalg.norm(lam) / gold["lam_norm"] - 1) <= TOL
    assert rel(lam[gold["lam_idx"]], np.asarray(gold["lam"])) <= TOL
    assert abs(np.linalg.norm(om) / gold["dOmega_sym_norm"] - 1) <= TOL
    assert rel(om[gold["dOmega_idx"]], np.asarray(gold["dOmega_sym"])) <= TOL
    gL = np.tril(2 * gO @ Lfac)                    # dL/dL for Omega = L L^T (gO symmetric)

    def loss(Y):
        bb = h.solve(Y).b.cpu().numpy()
        return float(np.sum((bb - target) ** 2))

    hstep = 1e-6
    noise = 2 * np.linalg.norm(b - target) * np.linalg.norm(b) * TOL / hstep
    g = S.rng(81)
    for _ in range(8):
        D = g.standard_normal(p.Y.shape)
        fd = (loss(p.Y + hstep * D) - loss(p.Y - hstep * D)) / (2 * hstep)
        an = float(np.sum(lam * D[:, 0]))
        assert abs(fd - an) <= noise + 1e-6 * abs(an), (fd, an, noise)
    for _ in range(8):
        E = np.tril(g.standard_normal(Lfac.shape))
        Lp, Lm = Lfac + hstep * E, Lfac - hstep * E
        h.set_omega(Lp @ Lp.T)
        lp = loss(p.Y)
        h.set_omega(Lm @ Lm.T)
        lm = loss(p.Y)
        fd = (lp - lm) / (2 * hstep)
        an = float(np.sum(gL * E))
        assert abs(fd - an) <= noise + 1e-6 * abs(an), (fd, an, noise)
    h.close()

"""PyTorch-facing wrapper of the C ABI: torch tensors hold device memory,
the library does every step of the method."""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _lib as L

PRECISIONS = {"fp64": L.GLM_SUR_PREC_FP64, "fp32_refine": L.GLM_SUR_PREC_FP32_REFINE}
STEP_KERNELS = {"auto": L.GLM_SUR_STEP_AUTO, "simt": L.GLM_SUR_STEP_SIMT}
ALGORITHMS = {"glmpcg2": L.GLM_SUR_ALG_GLMPCG2, "glmpcg3": L.GLM_SUR_ALG_GLMPCG3}
PRECONDS = {"identity": L.GLM_SUR_PRECOND_IDENTITY, "scaled": L.GLM_SUR_PRECOND_SCALED,
            "diag": L.GLM_SUR_PRECOND_DIAG}


def _dev_f64(x, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.float64)
    return torch.as_tensor(x, dtype=torch.float64, device=device)


@dataclass
class SolveResult:
    b: torch.Tensor          # (n, k) float64, device
    iters: torch.Tensor      # (k,) int32, device
    relres: torch.Tensor     # (k,) float64, device
    status: list             # k glm_sur_status codes (host)


class GlmSur:
    """SUR model handle: X_i factored once (TSQR on the device), Omega kept
    on the device; ``solve`` runs PCG-Aug for k right-hand sides."""

    def __init__(self, X_blocks, Omega, precision: str = "fp64", tol: float = 1e-13, maxit: int = 0,
                 stagnation_window: int = 25, inner_tol: float = 1e-5, max_refine: int = 8,
                 chunk: int = 16, inner_shift: float = 0.0, reduce_rows: bool = False,
                 step_kernels: str = "auto", precond: str = "identity", algorithm: str = "glmpcg2",
                 device="cuda"):
        self.device = torch.device(device)
        blocks = [_dev_f64(x, self.device) for x in X_blocks]
        self.n_i = [int(x.shape[1]) for x in blocks]
        self.M = int(blocks[0].shape[0])
        self.G = len(blocks)
        self.n = sum(self.n_i)
        # [X_1 ... X_G] column-major (M x n, ld = M) == row-major (n, M)
        self._X = torch.cat([x.t() for x in blocks], dim=0).contiguous()
        self._Omega = _dev_f64(Omega, self.device).contiguous()
        self.opts = L.default_opts()
        self.opts.precision = PRECISIONS[precision]
        self.opts.tol = tol
        self.opts.maxit = maxit
        self.opts.stagnation_window = stagnation_window
        self.opts.inner_tol = inner_tol
        self.opts.max_refine = max_refine
        self.opts.chunk = chunk
        self.opts.inner_shift = inner_shift
        self.opts.reduce_rows = int(bool(reduce_rows))
        self.opts.step_kernels = STEP_KERNELS[step_kernels]
        self.opts.precond = PRECONDS[precond]
        self.opts.algorithm = ALGORITHMS[algorithm]
        self.generation = 0     # number of solves so far (the adjoint belongs to the last one)
        self._h = L.glm_sur_setup(self.G, self.M, self.n_i, self._X.data_ptr(), self.M, self._Omega.data_ptr(),
                                  self.opts, self._stream())

    @staticmethod
    def _stream() -> int:
        return torch.cuda.current_stream().cuda_stream

    @property
    def handle(self) -> int:
        return self._h

    def setup_status(self) -> int:
        return L.glm_sur_get_setup_status(self._h)

    def set_omega(self, Omega) -> None:
        self._Omega = _dev_f64(Omega, self.device).contiguous()
        L.glm_sur_set_omega(self._h, self._Omega.data_ptr(), self._stream())

    def set_options(self, **kw) -> None:
        for key, v in kw.items():
            if key == "precision":
                v = PRECISIONS[v]
            setattr(self.opts, key, v)
        L.glm_sur_set_opts(self._h, self.opts)

    def set_restrictions(self, C) -> None:
        """Linear restrictions C b = d (C: (kc, n)); None or an empty C removes them."""
        if C is None or len(C) == 0:
            L.glm_sur_set_restrictions(self._h, 0, 1, 0, self._stream())
            self._C = None
            return
        Cd = _dev_f64(C, self.device)
        self._C = Cd.t().contiguous()                  # column-major kc x n
        L.glm_sur_set_restrictions(self._h, self._C.data_ptr(), Cd.shape[0], Cd.shape[0], self._stream())

    def solve(self, Y, d=None) -> SolveResult:
        """Y: (m, k) (column j = vec(Y_j)) or (m,); d: (kc, k) right-hand sides of
        the restrictions (restricted handles only).  Returns b as (n, k)."""
        Y = _dev_f64(Y, self.device)
        if Y.dim() == 1:
            Y = Y[:, None]
        m, k = Y.shape
        Ycm = Y.t().contiguous()                     # column-major m x k
        b = torch.empty((k, self.n), dtype=torch.float64, device=self.device)
        iters = torch.zeros(k, dtype=torch.int32, device=self.device)
        relres = torch.zeros(k, dtype=torch.float64, device=self.device)
        if d is not None:
            dd = _dev_f64(d, self.device).reshape(-1, k)
            dcm = dd.t().contiguous()
            L.glm_sur_solve_restricted(self._h, Ycm.data_ptr(), m, dcm.data_ptr(), dd.shape[0], k, b.data_ptr(),
                                       self.n, iters.data_ptr(), relres.data_ptr(), self._stream())
        else:
            L.glm_sur_solve(self._h, Ycm.data_ptr(), m, k, b.data_ptr(), self.n, iters.data_ptr(),
                            relres.data_ptr(), self._stream())
        status = L.glm_sur_get_status(self._h, k)
        self.generation += 1
        return SolveResult(b.t(), iters, relres, status)

    def solve_ne(self, Y) -> SolveResult:
        """PCG-NE: conjugate gradients on X^T Sigma^-1 X beta = X^T Sigma^-1 y
        (float64, positive definite Omega).  Y as in ``solve``; b as (n, k)."""
        Y = _dev_f64(Y, self.device)
        if Y.dim() == 1:
            Y = Y[:, None]
        m, k = Y.shape
        Ycm = Y.t().contiguous()
        b = torch.empty((k, self.n), dtype=torch.float64, device=self.device)
        iters = torch.zeros(k, dtype=torch.int32, device=self.device)
        relres = torch.zeros(k, dtype=torch.float64, device=self.device)
        L.glm_sur_solve_ne(self._h, Ycm.data_ptr(), m, k, b.data_ptr(), self.n, iters.data_ptr(),
                           relres.data_ptr(), self._stream())
        status = L.glm_sur_get_status(self._h, k)
        self.generation += 1
        return SolveResult(b.t(), iters, relres, status)

    def backward(self, dL_db, want_y: bool = True, want_omega: bool = True):
        """Adjoint of the last solve (same k, no restrictions, Omega unchanged).
        dL_db: (n, k) or (n,).  Returns (dL_dY (m, k) or None, dL_dOmega (G, G)
        symmetrised or None, iters, relres, status) of the adjoint solve."""
        g = _dev_f64(dL_db, self.device)
        if g.dim() == 1:
            g = g[:, None]
        k = g.shape[1]
        gcm = g.t().contiguous()
        m = self.M * self.G
        dY = torch.empty((k, m), dtype=torch.float64, device=self.device) if want_y else None
        dO = torch.empty((self.G, self.G), dtype=torch.float64, device=self.device) if want_omega else None
        iters = torch.zeros(k, dtype=torch.int32, device=self.device)
        relres = torch.zeros(k, dtype=torch.float64, device=self.device)
        L.glm_sur_backward(self._h, gcm.data_ptr(), self.n, k, dY.data_ptr() if want_y else 0, m,
                           dO.data_ptr() if want_omega else 0, self.G, iters.data_ptr(), relres.data_ptr(),
                           self._stream())
        status = L.glm_sur_get_status(self._h, k)
        # dO is written column-major; it is symmetric, so its transpose is itself
        return (dY.t() if want_y else None), dO, iters, relres, status

    def w(self, k: int) -> torch.Tensor:
        out = torch.empty((k, self.M * self.G), dtype=torch.float64, device=self.device)
        L.glm_sur_get_w(self._h, out.data_ptr(), self.M * self.G, self._stream())
        return out.t()

    def factors(self):
        """(Q (M, n) with Q_i side by side, [R_i] list of (n_i, n_i))."""
        Q = torch.empty((self.n, self.M), dtype=torch.float64, device=self.device)
        R = torch.empty(sum(v * v for v in self.n_i), dtype=torch.float64, device=self.device)
        L.glm_sur_get_factors(self._h, Q.data_ptr(), self.M, R.data_ptr(), self._stream())
        Rs, off = [], 0
        for v in self.n_i:
            Rs.append(R[off:off + v * v].view(v, v))
            off += v * v
        return Q.t(), Rs

    def close(self) -> None:
        if getattr(self, "_h", None):
            L.glm_sur_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GlmMvrglm:
    """The restricted multivariate GLM Y = Z0 B + U (Sec. "Multivariate linear
    models with parameters restrictions"), MVRGLM: model reduction by the QR
    of Z0, the updating QRDs [R0; C_i] and PCG-Aug with the block-diagonal X*
    and Pi.  Z0: (M, N); Omega0: (G, G); C_list: G matrices (k_i, N) (k_i = 0
    allowed).  ``solve(Y, gamma=None)`` takes Y as (M, G) or (M, G, k) and
    gamma as a list of G arrays (k_i,) or (k_i, k), and returns B as (N, G, k)."""

    def __init__(self, Z0, Omega0, C_list, precision: str = "fp64", tol: float = 1e-13, maxit: int = 0,
                 stagnation_window: int = 25, inner_tol: float = 1e-5, max_refine: int = 8, chunk: int = 16,
                 precond: str = "identity", device="cuda"):
        self.device = torch.device(device)
        Z = _dev_f64(Z0, self.device)
        self.M, self.N = Z.shape
        Om = _dev_f64(Omega0, self.device)
        self.G = Om.shape[0]
        self.k_i = [int(torch.as_tensor(c).reshape(-1, self.N).shape[0]) for c in C_list]
        self.ktot = sum(self.k_i)
        Zcm = Z.t().contiguous()
        Cs = [_dev_f64(c, self.device).reshape(-1, self.N) for c in C_list]
        Ccm = torch.cat(Cs, dim=0).t().contiguous() if self.ktot > 0 else None
        self.opts = L.default_opts()
        self.opts.precision = PRECISIONS[precision]
        self.opts.tol = tol
        self.opts.maxit = maxit
        self.opts.stagnation_window = stagnation_window
        self.opts.inner_tol = inner_tol
        self.opts.max_refine = max_refine
        self.opts.chunk = chunk
        self.opts.precond = PRECONDS[precond]
        self._h = L.glm_sur_mvrglm_setup(self.G, self.M, self.N, Zcm.data_ptr(), self.M, Om.contiguous().data_ptr(),
                                         self.k_i, Ccm.data_ptr() if Ccm is not None else 0, max(self.ktot, 1),
                                         self.opts, GlmSur._stream())
        torch.cuda.synchronize(self.device)
        st = L.glm_sur_get_setup_status(self._h)
        if st != L.GLM_SUR_OK:
            self.close()
            raise L.GlmSurError(st, "glm_sur_mvrglm_setup (updating QRDs)")

    @property
    def handle(self) -> int:
        return self._h

    def set_omega(self, Omega0) -> None:
        O = _dev_f64(Omega0, self.device).contiguous()
        L.glm_sur_set_omega(self._h, O.data_ptr(), GlmSur._stream())

    def solve(self, Y, gamma=None) -> SolveResult:
        Y = _dev_f64(Y, self.device)
        if Y.dim() == 2:
            Y = Y[:, :, None]
        M, G, k = Y.shape
        Ycm = Y.permute(2, 1, 0).contiguous()          # column j = vec(Y_j)
        b = torch.empty((k, G * self.N), dtype=torch.float64, device=self.device)
        iters = torch.zeros(k, dtype=torch.int32, device=self.device)
        relres = torch.zeros(k, dtype=torch.float64, device=self.device)
        if gamma is not None and self.ktot > 0:
            gs = [_dev_f64(gi, self.device).reshape(ki, -1).expand(ki, k) for gi, ki in zip(gamma, self.k_i)
                  if ki > 0]
            gcm = torch.cat(gs, dim=0).t().contiguous()
            L.glm_sur_solve_restricted(self._h, Ycm.data_ptr(), M * G, gcm.data_ptr(), self.ktot, k, b.data_ptr(),
                                       G * self.N, iters.data_ptr(), relres.data_ptr(), GlmSur._stream())
        else:
            L.glm_sur_solve(self._h, Ycm.data_ptr(), M * G, k, b.data_ptr(), G * self.N, iters.data_ptr(),
                            relres.data_ptr(), GlmSur._stream())
        status = L.glm_sur_get_status(self._h, k)
        B = b.view(k, G, self.N).permute(2, 1, 0)
        return SolveResult(B, iters, relres, status)

    def close(self) -> None:
        if getattr(self, "_h", None):
            L.glm_sur_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GlmSurBatch:
    """Many independent SUR instances solved in one persistent launch.

    problems: list of (X_blocks, Omega) pairs (numpy or torch, float64).
    reduce_rows: solve every instance with M >= 2 n on its n rotated rows
    (Remark rem:reduction; tol then refers to the reduced system).
    tol defaults to 1e-12: the float64 residual of a refined batched solve
    settles at a few 1e-13, below which refinement steps buy nothing."""

    def __init__(self, problems, tol: float = 1e-12, inner_tol: float = 1e-5, max_refine: int = 8,
                 reduce_rows: bool = False, device="cuda"):
        self.device = torch.device(device)
        self.G = [len(xb) for xb, _ in problems]
        self.M = [int(xb[0].shape[0]) for xb, _ in problems]
        self.n_i = [int(x.shape[1]) for xb, _ in problems for x in xb]
        self.n = [sum(int(x.shape[1]) for x in xb) for xb, _ in problems]
        self.m = [g * mm for g, mm in zip(self.G, self.M)]
        xs = []
        for xb, _ in problems:
            xs.append(torch.cat([_dev_f64(x, self.device).t() for x in xb], dim=0).reshape(-1))
        self._X = torch.cat(xs).contiguous()
        self._Om = torch.cat([_dev_f64(om, self.device).t().reshape(-1) for _, om in problems]).contiguous()
        self.opts = L.default_opts()
        self.opts.tol = tol
        self.opts.inner_tol = inner_tol
        self.opts.max_refine = max_refine
        self.opts.reduce_rows = int(bool(reduce_rows))
        self._h = L.glm_sur_batch_setup(len(problems), self.G, self.M, self.n_i, self._X.data_ptr(),
                                        self._Om.data_ptr(), self.opts, torch.cuda.current_stream().cuda_stream)

    @property
    def handle(self) -> int:
        return self._h

    def setup_status(self) -> int:
        return L.glm_sur_batch_get_setup_status(self._h)

    def pack_y(self, Ys):
        """List of (m_j, k) arrays -> one device buffer in the ABI layout."""
        return torch.cat([_dev_f64(y, self.device).t().reshape(-1) for y in Ys]).contiguous()

    def solve(self, Ys, k: int):
        Y = self.pack_y(Ys) if isinstance(Ys, (list, tuple)) else Ys
        b = torch.empty(sum(self.n) * k, dtype=torch.float64, device=self.device)
        cnt = len(self.G)
        iters = torch.zeros(cnt * k, dtype=torch.int32, device=self.device)
        relres = torch.zeros(cnt * k, dtype=torch.float64, device=self.device)
        L.glm_sur_batch_solve(self._h, Y.data_ptr(), k, b.data_ptr(), iters.data_ptr(), relres.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
        status = L.glm_sur_batch_get_status(self._h, cnt * k)
        out, off = [], 0
        for nj in self.n:
            out.append(b[off:off + nj * k].view(k, nj).t())
            off += nj * k
        return out, iters.view(cnt, k), relres.view(cnt, k), status

    def close(self) -> None:
        if getattr(self, "_h", None):
            L.glm_sur_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SurGLSFunction(torch.autograd.Function):
    """b = GLS estimate of the SUR model of ``solver`` (its X_i) for responses
    Y (m, k) and covariance Omega (G, G, symmetric), differentiable in Y and
    Omega through ``GlmSur.backward``.  Usage: SurGLSFunction.apply(Y, Omega,
    solver).  The backward pass must run before the solver's next solve."""

    @staticmethod
    def forward(ctx, Y, Omega, solver):
        solver.set_omega(Omega.detach())
        r = solver.solve(Y.detach())
        bad = [s for s in r.status if s not in (L.GLM_SUR_OK, L.GLM_SUR_STAGNATED)]
        if bad:
            raise RuntimeError(f"forward solve ended with status {bad}")
        ctx.solver, ctx.token, ctx.vec = solver, solver.generation, Y.dim() == 1
        return r.b[:, 0] if ctx.vec else r.b

    @staticmethod
    def backward(ctx, gb):
        solver = ctx.solver
        if solver.generation != ctx.token:
            raise RuntimeError("the solver ran another solve after this forward; its w is gone")
        need_y, need_om = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_y or need_om):
            return None, None, None
        dY, dO, _, _, status = solver.backward(gb, want_y=need_y, want_omega=need_om)
        bad = [s for s in status if s not in (L.GLM_SUR_OK, L.GLM_SUR_STAGNATED)]
        if bad:
            raise RuntimeError(f"adjoint solve ended with status {bad}")
        if dY is not None and ctx.vec:
            dY = dY[:, 0]
        return dY, dO, None

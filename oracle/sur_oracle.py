"""Plain, slow FP64 CPU oracle for GLS estimation of SUR models by PCG-Aug.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module: only the test-suite, the package's smoke check and the benchmark's
CPU-baseline leg use it.  It shares no code with the CUDA library; its inputs
come from the seeded generators in ``synth.sur_inputs``.

Everything here is float64 numpy, written for a reader to check against the
paper (Foschi, "Preconditioned Conjugate Gradient methods for the estimation
of General Linear Models"):

  * ``aug_dense_solve``   -- brute force: the augmented system eq. (aug1)
                             built densely and solved (min-norm LS if singular).
  * ``gls_formula``       -- eq. (GLS), b = (X^T S^-1 X)^-1 X^T S^-1 y (PD only).
  * ``aug_lemma``         -- Lemma thm:AugBLUE closed form (eq. augsol).
  * ``ols_blocks``        -- per-block OLS of the SUR model (Sec. 1).
  * ``sur_gls_structured``-- structured direct GLS: Remark rem:reduction, then
                             an eigen-split of Omega; zero-variance directions
                             become exact restrictions (Sec. 4.1 idea).
  * ``pcg``               -- Algorithm pcg on dense (G, K, h).
  * ``sur_pcg_aug``       -- Algorithm glmpcg2 (PCG-Aug) in the SUR form of
                             Sec. 4.3 (per-block QR, Sigma u = vec(U Omega)),
                             D = I or D = diag(delta) (x) I_M (alpha I, diag(Sigma));
                             also carries the z-iterates of Algorithm glmpcg.
  * ``sur_pcg_aug3``      -- Algorithm glmpcg3 (s-recurrence), fixed steps.
  * ``pcg_ne``            -- the PCG-NE comparator: CG on the normal equations
                             with Sigma^-1 = Omega^-1 (x) I_M (PD Omega).
  * ``pcg_aug_reduced``   -- Algorithm glmpcg2 in the reduced form of
                             eq. (urwProj) (null-space PCG, no v_i).
  * ``mvrglm_pcg_aug``    -- MVRGLM: model reduction by QR of Z0, updating
                             QRDs [R0; C_i] = Qt_i R_i, Algorithm glmpcg2 with
                             the block-diagonal X* and Pi.
  * ``rglm_pcg_aug``      -- the same algorithm on the restricted GLM of
                             Sec. 4.1 (eq. RGLM1setup, eq. rglm1m with D = I).
  * ``sur_gls_gradient``  -- adjoint of eq. (aug1) for L(b): dL/dy and dL/dOmega.
  * ``sur_gls_gradient_kron`` -- the same adjoint for positive definite Omega
    through Sigma^-1 = Omega^-1 (x) I_M (medium sizes, no m x m matrix).
  * ``sur_gls_refined``  -- eq. (aug1) and its adjoint for positive definite
    Omega by iterative refinement with residuals in extended precision
    (for ill-conditioned Omega, where the normal equations lose digits).

Layouts: X_blocks list of (M, n_i); Omega (G, G); Y (m, k) with column j =
vec(Y_j) (block i occupies rows i*M .. (i+1)*M); b (n, k).

Parity status: every function above is pinned by tests/test_oracle_pins.py
against brute force, closed forms, invariants or textbook special cases.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "sur_dense", "augmented_matrix", "aug_dense_solve", "gls_formula", "aug_lemma",
    "ols_blocks", "sur_gls_structured", "pcg", "sur_pcg_aug", "rglm_pcg_aug",
    "sur_gls_gradient", "sur_gls_gradient_kron", "sur_gls_refined", "augmented_residual", "lse_solve",
    "sur_pcg_aug3", "jacobi_delta", "scaled_identity_delta", "pcg_ne", "MvOps", "mvrglm_pcg_aug",
    "pcg_aug_reduced",
]


# ----------------------------------------------------------------------------
# dense building blocks (Sec. 1 SUR structure; eq. aug1)
# ----------------------------------------------------------------------------

def sur_dense(X_blocks, Omega):
    """Dense Sigma = Omega (x) I_M and X = (+)_i X_i (Sec. 1)."""
    M = X_blocks[0].shape[0]
    Sigma = np.kron(Omega, np.eye(M))
    n = sum(x.shape[1] for x in X_blocks)
    X = np.zeros((len(X_blocks) * M, n))
    off = 0
    for i, Xi in enumerate(X_blocks):
        X[i * M:(i + 1) * M, off:off + Xi.shape[1]] = Xi
        off += Xi.shape[1]
    return Sigma, X


def augmented_matrix(Sigma, X):
    """[[Sigma, X], [X^T, 0]] of eq. (aug1)."""
    m, n = X.shape
    K = np.zeros((m + n, m + n))
    K[:m, :m] = Sigma
    K[:m, m:] = X
    K[m:, :m] = X.T
    return K


def _pinv_solve(K, H):
    """Minimum-norm least-squares solution of K x = H via the SVD (handles a
    singular augmented matrix; the b-part of any solution is unique when X
    has full column rank)."""
    U, s, Vt = np.linalg.svd(K)
    r = int(np.sum(s > s[0] * max(K.shape) * np.finfo(float).eps))
    return Vt[:r].T @ ((U[:, :r].T @ H) / s[:r, None])


def aug_dense_solve(X_blocks, Omega, Y, C=None, d=None):
    """Brute force (O1): build eq. (aug1) densely and solve it.

    With restrictions C b = d the model is the GLM of eq. (RGLM1setup):
    Sigma_aug = diag(Sigma, 0), X_aug = [X; C], y_aug = [y; d].
    Returns (w, b): w of length m (+ kc), b (n, k)."""
    Sigma, X = sur_dense(X_blocks, Omega)
    Y = np.asarray(Y, dtype=float).reshape(Sigma.shape[0], -1)
    if C is not None:
        kc = C.shape[0]
        m = Sigma.shape[0]
        S2 = np.zeros((m + kc, m + kc))
        S2[:m, :m] = Sigma
        Sigma = S2
        X = np.vstack([X, C])
        Y = np.vstack([Y, np.asarray(d, dtype=float).reshape(kc, -1)])
    m, n = X.shape
    K = augmented_matrix(Sigma, X)
    H = np.vstack([Y, np.zeros((n, Y.shape[1]))])
    try:
        x = np.linalg.solve(K, H)
        if not np.all(np.isfinite(x)) or np.linalg.cond(K) > 1e14:
            raise np.linalg.LinAlgError
    except np.linalg.LinAlgError:
        x = _pinv_solve(K, H)
    return x[:m], x[m:]


def gls_formula(X_blocks, Omega, Y):
    """eq. (GLS): b = (X^T Sigma^-1 X)^-1 X^T Sigma^-1 y with
    Sigma^-1 = Omega^-1 (x) I_M (Omega positive definite only)."""
    M = X_blocks[0].shape[0]
    _, X = sur_dense(X_blocks, Omega)
    Si = np.kron(np.linalg.inv(Omega), np.eye(M))
    A = X.T @ Si @ X
    return np.linalg.solve(A, X.T @ Si @ np.asarray(Y).reshape(X.shape[0], -1))


def aug_lemma(X_blocks, Omega, Y):
    """Lemma thm:AugBLUE (eq. augsol): with the full QR X = [Q_R Q_N][R; 0],
    w = Q_N (Q_N^T Sigma Q_N)^-1 Q_N^T y,
    b = R^-1 Q_R^T P_N y,  P_N = I - Sigma Q_N (Q_N^T Sigma Q_N)^-1 Q_N^T."""
    Sigma, X = sur_dense(X_blocks, Omega)
    m, n = X.shape
    Y = np.asarray(Y).reshape(m, -1)
    Qf, Rf = np.linalg.qr(X, mode="complete")
    QR_, QN = Qf[:, :n], Qf[:, n:]
    R = Rf[:n]
    A = QN.T @ Sigma @ QN
    w = QN @ np.linalg.solve(A, QN.T @ Y)
    PN_y = Y - Sigma @ QN @ np.linalg.solve(A, QN.T @ Y)
    b = np.linalg.solve(R, QR_.T @ PN_y)
    return w, b


def ols_blocks(X_blocks, Y):
    """Per-block OLS of the SUR model (Sec. 1): b_i = (X_i^T X_i)^-1 X_i^T y_i."""
    M = X_blocks[0].shape[0]
    Y = np.asarray(Y).reshape(len(X_blocks) * M, -1)
    out = []
    for i, Xi in enumerate(X_blocks):
        out.append(np.linalg.solve(Xi.T @ Xi, Xi.T @ Y[i * M:(i + 1) * M]))
    return np.vstack(out)


# ----------------------------------------------------------------------------
# structured direct GLS (Remark rem:reduction + eigen-split of Omega)
# ----------------------------------------------------------------------------

def lse_solve(A, a, B=None, bc=None):
    """min ||A x - a|| subject to B x = bc (B consistent, may be tall or
    rank deficient), by the null-space method with an SVD of B."""
    if B is None or B.shape[0] == 0:
        return np.linalg.lstsq(A, a, rcond=None)[0]
    U, s, Vt = np.linalg.svd(B, full_matrices=True)
    r = int(np.sum(s > s[0] * max(B.shape) * np.finfo(float).eps * 16))
    xp = Vt[:r].T @ ((U[:, :r].T @ bc) / s[:r, None])
    N = Vt[r:].T
    if N.shape[1] == 0 or A.shape[0] == 0:
        return xp
    t = np.linalg.lstsq(A @ N, a - A @ xp, rcond=None)[0]
    return xp + N @ t


def range_basis(W):
    """Orthonormal basis of range(W): thin Householder QR when W is tall with
    full column rank, otherwise the left singular vectors above a threshold."""
    M, n = W.shape
    if M >= n:
        Qw, Rw = np.linalg.qr(W)
        dg = np.abs(np.diag(Rw))
        if dg.min() > 1e-10 * dg.max():
            return Qw
    U, s, _ = np.linalg.svd(W, full_matrices=False)
    r = int(np.sum(s > s[0] * max(W.shape) * np.finfo(float).eps))
    return U[:, :r]


def sur_gls_structured(X_blocks, Omega, Y, C=None, d=None, tau_rel=None):
    """Structured direct GLS (O2).

    1. Remark rem:reduction: with B an orthonormal basis of range(W),
       W = [X_1 ... X_G], replace y_i, X_i by B^T y_i, B^T X_i (q rows each).
       Rows orthogonal to range(W) carry no regressor and, as Sigma = Omega (x) I
       keeps rows independent, no information on beta.
    2. Omega = V diag(lam) V^T.  Right-multiplying the reduced M x G model by
       V decouples it into G independent regressions: equation j has
       regressor [v_1j X_1, ..., v_Gj X_G] and disturbance variance lam_j.
    3. lam_j > tau: weighted LS rows (scaled by lam_j^-1/2);  lam_j <= tau:
       exact (zero-variance) restrictions, as in eq. (RGLM1setup).
       Rows [C | d] are appended as restrictions.
    4. Solve the equality-constrained LS problem (``lse_solve``).
    tau = tau_rel * lam_max with tau_rel = sqrt(eps) by default."""
    G = len(X_blocks)
    M = X_blocks[0].shape[0]
    n_i = [x.shape[1] for x in X_blocks]
    n = sum(n_i)
    Y = np.asarray(Y, dtype=float).reshape(G * M, -1)
    k = Y.shape[1]
    Bw = range_basis(np.hstack(X_blocks))
    Xr = [Bw.T @ Xi for Xi in X_blocks]                       # q x n_i
    lam, V = np.linalg.eigh(0.5 * (Omega + Omega.T))
    if tau_rel is None:
        tau_rel = np.sqrt(np.finfo(float).eps)
    tau = tau_rel * max(lam.max(), 0.0)
    offs = np.cumsum([0] + n_i)
    ls_A, con_A, ls_j, con_j = [], [], [], []
    for j in range(G):
        Aj = np.zeros((Bw.shape[1], n))
        for i in range(G):
            Aj[:, offs[i]:offs[i + 1]] = V[i, j] * Xr[i]
        if lam[j] > tau:
            ls_A.append(Aj / np.sqrt(lam[j]))
            ls_j.append(j)
        else:
            con_A.append(Aj)
            con_j.append(j)
    A = np.vstack(ls_A) if ls_A else np.zeros((0, n))
    Bc = np.vstack(con_A) if con_A else np.zeros((0, n))
    if C is not None:
        Bc = np.vstack([Bc, C])
    out = np.empty((n, k))
    for c in range(k):
        Yr = Bw.T @ Y[:, c].reshape(G, M).T                   # q x G reduced responses
        Yt = Yr @ V                                           # decoupled responses
        a = np.concatenate([Yt[:, j] / np.sqrt(lam[j]) for j in ls_j]) if ls_j else np.zeros(0)
        bc = np.concatenate([Yt[:, j] for j in con_j]) if con_j else np.zeros(0)
        if C is not None:
            bc = np.concatenate([bc, np.asarray(d, dtype=float).reshape(C.shape[0], -1)[:, c]])
        out[:, c] = lse_solve(A, a[:, None], Bc if Bc.shape[0] else None,
                              bc[:, None] if Bc.shape[0] else None)[:, 0]
    return out


# ----------------------------------------------------------------------------
# PCG (Algorithm pcg) and PCG-Aug (Algorithm glmpcg2) in the SUR form
# ----------------------------------------------------------------------------

def pcg(Gm, Km, h, x1, iters):
    """Algorithm pcg, verbatim in the paper's notation, for ``iters`` steps on
    dense symmetric G and K; residual convention f = G x - h.  Returns the list
    of iterates x_1 .. x_{iters+1} (stops early if d_i == 0)."""
    x = x1.copy()
    f = Gm @ x - h
    p = Km @ f
    c = f @ (Km @ f)
    xs = [x.copy()]
    for _ in range(iters):
        Gp = Gm @ p
        dd = p @ Gp
        if dd == 0.0:
            break
        lam = c / dd
        x = x - lam * p
        f = f - lam * Gp
        Kf = Km @ f
        c_new = f @ Kf
        mu = c_new / c
        p = Kf + mu * p
        c = c_new
        xs.append(x.copy())
    return xs


class SurOps:
    """The SUR applies of Sec. 4.3 from thin QRs X_i = Q_i R_i, with the
    preconditioner block D = D_0 (x) I_M, D_0 = diag(delta) (D = I when delta
    is not given).  From eq. (Xstar): X* = D^-1 X (X^T D^-1 X)^-1 and
    Pi = (I - X* X^T) D^-1; with block i of D equal to delta_i I the delta_i
    cancel in X* and
      Pi xi      = vec((xi_i - Q_i Q_i^T xi_i) / delta_i)
      P xi       = vec(xi_i - Q_i Q_i^T xi_i)      (orthogonal projector; Pi = P D^-1)
      X*^T xi    = vec(R_i^-1 Q_i^T xi_i)
      X v        = vec(X_i v_i)
      Sigma u    = vec(U Omega),  u = vec(U)."""

    def __init__(self, X_blocks, Omega, delta=None):
        self.X = X_blocks
        self.Omega = np.asarray(Omega, dtype=float)
        self.G = len(X_blocks)
        self.M = X_blocks[0].shape[0]
        self.n_i = [x.shape[1] for x in X_blocks]
        self.offs = np.cumsum([0] + self.n_i)
        self.QR = [np.linalg.qr(Xi) for Xi in X_blocks]
        self.delta = np.ones(self.G) if delta is None else np.asarray(delta, dtype=float)
        self.m = self.G * self.M

    def sigma(self, u):
        # (U Omega)_h = sum_g U_g omega_gh: with the G columns of every U_j as
        # the rows of a (G, M*k) matrix this is one matrix product Omega^T U.
        k = u.shape[1]
        U = u.reshape(self.G, self.M * k)
        return (self.Omega.T @ U).reshape(self.G * self.M, k)

    def proj(self, xi):
        out = np.empty_like(xi)
        M = self.M
        for i, (Qi, _) in enumerate(self.QR):
            blk = xi[i * M:(i + 1) * M]
            out[i * M:(i + 1) * M] = blk - Qi @ (Qi.T @ blk)
        return out

    def dinv(self, xi):
        """D^-1 xi (block i divided by delta_i)."""
        return xi / np.repeat(self.delta, self.M)[:, None]

    def pi(self, xi):
        return self.dinv(self.proj(xi))

    def xstar_t(self, xi):
        M = self.M
        parts = []
        for i, (Qi, Ri) in enumerate(self.QR):
            parts.append(np.linalg.solve(Ri, Qi.T @ xi[i * M:(i + 1) * M]))
        return np.vstack(parts)

    def xmul(self, v):
        M = self.M
        out = np.empty((self.G * M, v.shape[1]))
        for i, Xi in enumerate(self.X):
            out[i * M:(i + 1) * M] = Xi @ v[self.offs[i]:self.offs[i + 1]]
        return out

    def xt(self, w):
        M = self.M
        return np.vstack([Xi.T @ w[i * M:(i + 1) * M] for i, Xi in enumerate(self.X)])


STATUS_CONVERGED = "converged"
STATUS_BREAKDOWN = "breakdown"
STATUS_STAGNATED = "stagnated"
STATUS_NOT_CONVERGED = "not_converged"


def sur_pcg_aug(X_blocks, Omega, Y, tol=1e-13, maxit=None, stag_window=25,
                record=False, ops=None, w1=None, delta=None):
    """Algorithm glmpcg2 (PCG-Aug) in the SUR form of Sec. 4.3 (O3), with the
    preconditioner block D = diag(delta) (x) I_M (D = I by default; Sec. 3.3
    and the VAR experiments use D = alpha I and D = diag(Sigma)).

    One independent PCG per column of Y (each with its own c, d, lambda, mu).
    Start: w_1 = 0 (or ``w1`` with X^T w_1 = 0), z_1 = 0.
    Pi = P D^-1 with P the orthogonal projector onto null(X^T) and D commuting
    with P block by block, so c = r^T Pi r is evaluated as (P r)^T D^-1 (P r):
    the same quantity, without the cancellation of the large range-space
    part of r against Pi r (which floors sqrt(c/c_1) near sqrt(eps) when
    written as r . (Pi r)).
    The z-iterates of Algorithm glmpcg (z_{i+1} = z_i - lambda_i v_i) are
    carried too and returned as ``z``.
    Stop a column when sqrt(c_{i+1}/c_1) <= tol (converged), when d_i <= 0 or
    is not finite (breakdown), when c has not reached a new minimum for W
    steps (stagnation: c no longer decreases, Sec. 3.2; c_i need
    not decrease monotonically, so a window over the running minimum is
    used), or at ``maxit``.  Every column returns its last iterate w and
    z_hat = X*^T (y - Sigma w) (step 10 of the algorithm).
    Returns dict(b, w, iters, status, relres[, history])."""
    op = ops if ops is not None else SurOps(X_blocks, Omega, delta)
    m = op.m
    Y = np.asarray(Y, dtype=float).reshape(m, -1)
    k = Y.shape[1]
    n = int(op.offs[-1])
    if maxit is None:
        maxit = m - n + 1
    w = np.zeros((m, k)) if w1 is None else np.array(w1, dtype=float).reshape(m, k)
    z = np.zeros((n, k))
    r = op.sigma(w) + op.xmul(z) - Y                          # step 2
    Pr = op.proj(r)
    Pir = op.dinv(Pr)                                         # Pi r
    c = np.sum(Pr * Pir, axis=0)                              # r^T Pi r
    u = Pir.copy()                                            # step 3
    v = op.xstar_t(r)
    c1 = c.copy()
    active = c1 > 0
    iters = np.zeros(k, dtype=int)
    status = np.array([STATUS_CONVERGED if not a else STATUS_NOT_CONVERGED for a in active],
                      dtype=object)
    relres = np.where(c1 > 0, 1.0, 0.0)
    cbest = c.copy()
    itbest = np.zeros(k, dtype=int)
    hist = {"w": [w.copy()], "r": [r.copy()], "u": [u.copy()], "c": [c.copy()]} if record else None
    for it in range(1, maxit + 1):
        if not active.any():
            break
        Su = op.sigma(u)
        dd = np.sum(u * Su, axis=0)                           # step 5
        bad = active & (~np.isfinite(dd) | (dd <= 0))
        for j in np.where(bad)[0]:
            status[j] = STATUS_BREAKDOWN
        active &= ~bad
        lam = np.where(active, c / np.where(active, dd, 1.0), 0.0)
        w = w - lam * u                                       # step 6
        z = z - lam * v                                       # (Algorithm glmpcg)
        r = r - lam * (Su + op.xmul(v))                       # step 7
        Pr = op.proj(r)
        Pir = op.dinv(Pr)
        c_new = np.where(active, np.sum(Pr * Pir, axis=0), c)  # step 8
        iters = iters + active
        rr = np.sqrt(np.maximum(c_new, 0.0) / np.where(c1 > 0, c1, 1.0))
        relres = np.where(active, rr, relres)
        bad_c = active & (~np.isfinite(c_new) | (c_new < 0))
        for j in np.where(bad_c)[0]:
            status[j] = STATUS_BREAKDOWN
        active &= ~bad_c
        conv = active & (rr <= tol)
        for j in np.where(conv)[0]:
            status[j] = STATUS_CONVERGED
        active &= ~conv
        better = active & (c_new < cbest)
        cbest = np.where(better, c_new, cbest)
        itbest = np.where(better, it, itbest)
        stag = active & (it - itbest >= stag_window)
        for j in np.where(stag)[0]:
            status[j] = STATUS_STAGNATED
        active &= ~stag
        mu = np.where(active, c_new / np.where(c > 0, c, 1.0), 0.0)
        v = op.xstar_t(r) + mu * v                            # step 12
        u = np.where(active, Pir + mu * u, u)
        c = np.where(active, c_new, c)
        if record:
            hist["w"].append(w.copy()); hist["r"].append(r.copy())
            hist["u"].append(u.copy()); hist["c"].append(c_new.copy())
    b = op.xstar_t(Y - op.sigma(w))                           # step 10
    out = dict(b=b, w=w, z=z, iters=iters, status=list(status), relres=relres)
    if record:
        out["history"] = hist
    return out


def pcg_aug_reduced(ops, Y, tol=1e-13, maxit=None, stag_window=25, record=False):
    """Algorithm glmpcg2 in the reduced form of eq. (urwProj): with r_i, u_i,
    w_i split on range(X) and null(X^T), the null-space parts follow PCG on
    A w~ = Q_N^T y (A = Q_N^T Sigma Q_N, preconditioner B^-1, B = Q_N^T D Q_N)
    and the directions v_i are not needed.  In the full space, with D
    commuting with P (block i of D equal to delta_i I), this reads
      g_1 = P r_1 = -P y,  u_1 = D^-1 g_1,  c_1 = g_1^T D^-1 g_1,
      d_i = u_i^T Sigma u_i,  lambda_i = c_i / d_i,  w_{i+1} = w_i - lambda_i u_i,
      g_{i+1} = g_i - lambda_i P Sigma u_i,  c_{i+1} = g_{i+1}^T D^-1 g_{i+1},
      u_{i+1} = D^-1 g_{i+1} + (c_{i+1} / c_i) u_i,
    and b = X*^T (y - Sigma w) at the end (step 10).  Unlike the literal
    recursion r_{i+1} = r_i - lambda_i (Sigma u_i + X v_i), nothing here
    grows with the range-space part z_i of the iterate, which is multiplied
    by about (1 - lambda_i) per step: when lambda_i >> 1 (a Sigma whose
    Rayleigh quotients on null(X^T) are far below those of D, as with the
    zero-variance restriction rows) that recursion loses P r to rounding.
    Stopping rules as ``sur_pcg_aug``.  ``ops`` provides m, offs, sigma,
    proj, dinv and xstar_t.  Returns dict(b, w, iters, status, relres[, history])."""
    op = ops
    m = op.m
    Y = np.asarray(Y, dtype=float).reshape(m, -1)
    k = Y.shape[1]
    n = int(op.offs[-1])
    if maxit is None:
        maxit = m - n + 1
    w = np.zeros((m, k))
    g = -op.proj(Y)
    Dg = op.dinv(g)
    c = np.sum(g * Dg, axis=0)
    u = Dg.copy()
    c1 = c.copy()
    active = c1 > 0
    iters = np.zeros(k, dtype=int)
    status = np.array([STATUS_CONVERGED if not a else STATUS_NOT_CONVERGED for a in active], dtype=object)
    relres = np.where(c1 > 0, 1.0, 0.0)
    cbest = c.copy()
    itbest = np.zeros(k, dtype=int)
    hist = {"w": [w.copy()], "c": [c.copy()]} if record else None
    for it in range(1, maxit + 1):
        if not active.any():
            break
        Su = op.sigma(u)
        dd = np.sum(u * Su, axis=0)
        bad = active & (~np.isfinite(dd) | (dd <= 0))
        for j in np.where(bad)[0]:
            status[j] = STATUS_BREAKDOWN
        active &= ~bad
        lam = np.where(active, c / np.where(active, dd, 1.0), 0.0)
        w = w - lam * u
        g = g - lam * op.proj(Su)
        Dg = op.dinv(g)
        c_new = np.where(active, np.sum(g * Dg, axis=0), c)
        iters = iters + active
        rr = np.sqrt(np.maximum(c_new, 0.0) / np.where(c1 > 0, c1, 1.0))
        relres = np.where(active, rr, relres)
        bad_c = active & (~np.isfinite(c_new) | (c_new < 0))
        for j in np.where(bad_c)[0]:
            status[j] = STATUS_BREAKDOWN
        active &= ~bad_c
        conv = active & (rr <= tol)
        for j in np.where(conv)[0]:
            status[j] = STATUS_CONVERGED
        active &= ~conv
        better = active & (c_new < cbest)
        cbest = np.where(better, c_new, cbest)
        itbest = np.where(better, it, itbest)
        stag = active & (it - itbest >= stag_window)
        for j in np.where(stag)[0]:
            status[j] = STATUS_STAGNATED
        active &= ~stag
        mu = np.where(active, c_new / np.where(c > 0, c, 1.0), 0.0)
        u = np.where(active, Dg + mu * u, u)
        c = np.where(active, c_new, c)
        if record:
            hist["w"].append(w.copy())
            hist["c"].append(c_new.copy())
    b = op.xstar_t(Y - op.sigma(w))
    out = dict(b=b, w=w, iters=iters, status=list(status), relres=relres)
    if record:
        out["history"] = hist
    return out


def sur_pcg_aug3(X_blocks, Omega, Y, iters, delta=None, ops=None):
    """Algorithm glmpcg3 (the alternative PCG-Aug) in the SUR form, for a
    fixed number of steps and without stop tests (its iterates are compared
    with those of Algorithm glmpcg2, which it equals in exact arithmetic).
    It carries s_i (s_1 = r_1, s_{i+1} = r_{i+1} + mu_i s_i) in place of u_i
    and v_i: d_i = s_i^T Pi Sigma Pi s_i, w_{i+1} = w_i - lambda_i Pi s_i,
    r_{i+1} = r_i - lambda_i (Sigma Pi + X X*^T) s_i.  Start w_1 = 0, z_1 = 0.
    Returns dict(b, w, history: list of w iterates and of c)."""
    op = ops if ops is not None else SurOps(X_blocks, Omega, delta)
    m = op.m
    Y = np.asarray(Y, dtype=float).reshape(m, -1)
    k = Y.shape[1]
    w = np.zeros((m, k))
    r = op.sigma(w) - Y                                       # step 2 (z_1 = 0)
    Pr = op.proj(r)
    c = np.sum(Pr * op.dinv(Pr), axis=0)
    s = r.copy()                                              # step 3
    ws, cs = [w.copy()], [c.copy()]
    for _ in range(iters):
        Pis = op.pi(s)
        SPis = op.sigma(Pis)
        dd = np.sum(Pis * SPis, axis=0)                       # step 5
        lam = c / dd
        w = w - lam * Pis                                     # step 6
        r = r - lam * (SPis + op.xmul(op.xstar_t(s)))         # step 7
        Pr = op.proj(r)
        c_new = np.sum(Pr * op.dinv(Pr), axis=0)              # step 8
        mu = c_new / c
        s = r + mu * s                                        # step 12
        c = c_new
        ws.append(w.copy()); cs.append(c.copy())
    b = op.xstar_t(Y - op.sigma(w))
    return dict(b=b, w=w, history={"w": ws, "c": cs})


def pcg_ne(X_blocks, Omega, Y, tol=1e-13, maxit=None, record=False):
    """PCG-NE, the comparator of the Monte-Carlo study and of the SUR and VAR
    experiments: the conjugate gradient method (Algorithm pcg with K = I, no
    preconditioner) on the normal equations (X^T Sigma^-1 X) beta =
    X^T Sigma^-1 y, with Sigma^-1 = Omega^-1 (x) I_M applied as U Omega^-1 and
    X, X^T block by block.  One CG per column of Y, x_1 = 0; a column stops
    when ||h - A beta|| <= tol ||h|| (h = X^T Sigma^-1 y) or at maxit
    (default n, the number of distinct eigenvalues at most).  Omega must be
    positive definite.  Returns dict(b, iters, status, relres[, history])."""
    op = SurOps(X_blocks, Omega)
    Oinv = np.linalg.inv(op.Omega)
    G, M = op.G, op.M
    n = int(op.offs[-1])
    Y = np.asarray(Y, dtype=float).reshape(G * M, -1)
    k = Y.shape[1]
    if maxit is None:
        maxit = n

    def sigma_inv(u):
        U = u.reshape(G, M * u.shape[1])
        return (Oinv.T @ U).reshape(G * M, u.shape[1])

    def apply_a(v):
        return op.xt(sigma_inv(op.xmul(v)))

    h = op.xt(sigma_inv(Y))
    beta = np.zeros((n, k))
    f = apply_a(beta) - h                          # f = G x - h of Algorithm pcg
    p = f.copy()
    c = np.sum(f * f, axis=0)
    c1 = c.copy()
    active = c1 > 0
    iters = np.zeros(k, dtype=int)
    status = np.array([STATUS_CONVERGED if not a else STATUS_NOT_CONVERGED for a in active], dtype=object)
    relres = np.where(c1 > 0, 1.0, 0.0)
    hist = [beta.copy()] if record else None
    for _ in range(maxit):
        if not active.any():
            break
        Ap = apply_a(p)
        dd = np.sum(p * Ap, axis=0)
        lam = np.where(active, c / np.where(active & (dd != 0), dd, 1.0), 0.0)
        beta = beta - lam * p
        f = f - lam * Ap
        c_new = np.sum(f * f, axis=0)
        iters = iters + active
        rr = np.sqrt(c_new / np.where(c1 > 0, c1, 1.0))
        relres = np.where(active, rr, relres)
        conv = active & (rr <= tol)
        for j in np.where(conv)[0]:
            status[j] = STATUS_CONVERGED
        active &= ~conv
        mu = np.where(active, c_new / np.where(c > 0, c, 1.0), 0.0)
        p = np.where(active, f + mu * p, p)
        c = np.where(active, c_new, c)
        if record:
            hist.append(beta.copy())
    out = dict(b=beta, iters=iters, status=list(status), relres=relres)
    if record:
        out["history"] = hist
    return out


def jacobi_delta(Omega):
    """D_0 = diag(Sigma_0): the diagonal preconditioner block of the VAR
    experiments (D = diag(Sigma) = diag(Omega) (x) I_M for the SUR model)."""
    return np.diag(np.asarray(Omega, dtype=float)).copy()


def scaled_identity_delta(Omega):
    """D_0 = alpha I with alpha = max_i Sigma_ii (the other choice of the VAR
    experiments)."""
    Om = np.asarray(Omega, dtype=float)
    return np.full(Om.shape[0], np.max(np.diag(Om)))


def rglm_pcg_aug(X_blocks, Omega, Y, C, d, tol=1e-13, maxit=None, stag_window=25):
    """Algorithm glmpcg2 on the restricted GLM of Sec. 4.1 with D = I.

    eq. (RGLM1setup): Sigma_aug = diag(Omega (x) I_M, 0_kc), X_aug = [(+)X_i; C],
    y_aug = [y; d].  eq. (rglm1m) with D_Z = I, D_C = I:
      X* = X_aug (Z^T Z + C^T C)^-1,   Pi = I - X_aug (Z^T Z + C^T C)^-1 X_aug^T,
    where Z^T Z = (+)_i X_i^T X_i.  Returns dict(b, w, iters, status, relres)."""
    G = len(X_blocks)
    M = X_blocks[0].shape[0]
    n_i = [x.shape[1] for x in X_blocks]
    offs = np.cumsum([0] + n_i)
    n = int(offs[-1])
    kc = C.shape[0]
    m = G * M
    Omega = np.asarray(Omega, dtype=float)
    Y = np.asarray(Y, dtype=float).reshape(m, -1)
    k = Y.shape[1]
    yaug = np.vstack([Y, np.asarray(d, dtype=float).reshape(kc, k)])
    Nmat = C.T @ C
    for i, Xi in enumerate(X_blocks):
        Nmat[offs[i]:offs[i + 1], offs[i]:offs[i + 1]] += Xi.T @ Xi

    def xt(xi):                                               # X_aug^T xi
        top = np.vstack([X_blocks[i].T @ xi[i * M:(i + 1) * M] for i in range(G)])
        return top + C.T @ xi[m:]

    def xmul(v):                                              # X_aug v
        out = np.empty((m + kc, v.shape[1]))
        for i in range(G):
            out[i * M:(i + 1) * M] = X_blocks[i] @ v[offs[i]:offs[i + 1]]
        out[m:] = C @ v
        return out

    def xstar_t(xi):
        return np.linalg.solve(Nmat, xt(xi))

    def pi(xi):
        return xi - xmul(xstar_t(xi))

    def sigma(u):
        kk = u.shape[1]
        S = (Omega.T @ u[:m].reshape(G, M * kk)).reshape(m, kk)
        return np.vstack([S, np.zeros((kc, kk))])

    if maxit is None:
        maxit = m + kc - n + 1
    w = np.zeros((m + kc, k))
    r = sigma(w) - yaug
    Pr = pi(r)
    c = np.sum(Pr * Pr, axis=0)
    u = Pr.copy()
    v = xstar_t(r)
    c1 = c.copy()
    active = c1 > 0
    iters = np.zeros(k, dtype=int)
    status = [STATUS_CONVERGED if not a else STATUS_NOT_CONVERGED for a in active]
    relres = np.where(c1 > 0, 1.0, 0.0)
    cbest = c.copy()
    itbest = np.zeros(k, dtype=int)
    for it in range(1, maxit + 1):
        if not active.any():
            break
        Su = sigma(u)
        dd = np.sum(u * Su, axis=0)
        bad = active & (~np.isfinite(dd) | (dd <= 0))
        for j in np.where(bad)[0]:
            status[j] = STATUS_BREAKDOWN
        active &= ~bad
        lam = np.where(active, c / np.where(active, dd, 1.0), 0.0)
        w = w - lam * u
        r = r - lam * (Su + xmul(v))
        Pr = pi(r)
        c_new = np.where(active, np.sum(Pr * Pr, axis=0), c)
        iters = iters + active
        rr = np.sqrt(np.maximum(c_new, 0.0) / np.where(c1 > 0, c1, 1.0))
        relres = np.where(active, rr, relres)
        conv = active & (rr <= tol)
        for j in np.where(conv)[0]:
            status[j] = STATUS_CONVERGED
        active &= ~conv
        better = active & (c_new < cbest)
        cbest = np.where(better, c_new, cbest)
        itbest = np.where(better, it, itbest)
        stag = active & (it - itbest >= stag_window)
        for j in np.where(stag)[0]:
            status[j] = STATUS_STAGNATED
        active &= ~stag
        mu = np.where(active, c_new / np.where(c > 0, c, 1.0), 0.0)
        v = xstar_t(r) + mu * v
        u = np.where(active, Pr + mu * u, u)
        c = np.where(active, c_new, c)
    b = xstar_t(yaug - sigma(w))
    return dict(b=b, w=w, iters=iters, status=status, relres=relres)


# ----------------------------------------------------------------------------
# restricted multivariate GLM (MVRGLM)
# ----------------------------------------------------------------------------

class MvOps:
    """The applies of the restricted multivariate GLM after model reduction
    (Sec. "Multivariate linear models with parameters restrictions"):
    Y = Z0 B + U with rows of U iid (0, Omega0) and restrictions C_i b_i =
    gamma_i on each column b_i of B (no cross-equation restrictions).  With
    Z0 = Q0 R0 the reduced model has Z = I_G (x) R0, Omega = Omega0 (x) I_N;
    eq. (RGLM1setup) adds the k_i restriction rows of each equation with zero
    variance.  Ordered equation by equation (the row permutation under which
    X* and Pi are block diagonal), equation i holds the N + k_i rows
    [R0; C_i], and the updating QRD [R0; C_i] = Qt_i R_i (eq. MvRGLMQRi) gives
      X*  = (+)_i Qt_i R_i^-T,     P = (+)_i (I - Qt_i Qt_i^T),
      Sigma u: rows 0..N-1 of equation h get sum_g omega_gh u_g[0..N-1],
               the restriction rows get 0.
    The preconditioner block is D = D_Z (+) D_C with D_Z = D0 (x) I_N and
    D_C = D0 on the restriction rows of each equation (delta_i on every row
    of equation i), so Pi = P D^-1 and the delta_i cancel in X*."""

    def __init__(self, R0, C_list, Omega0, delta=None):
        self.R0 = np.asarray(R0, dtype=float)
        self.N = self.R0.shape[0]
        self.G = len(C_list)
        self.C = [np.asarray(c, dtype=float).reshape(-1, self.N) for c in C_list]
        self.k_i = [c.shape[0] for c in self.C]
        self.rows = [self.N + ki for ki in self.k_i]
        self.roff = np.cumsum([0] + self.rows)
        self.m = int(self.roff[-1])
        self.offs = self.N * np.arange(self.G + 1)
        self.Xt = [np.vstack([self.R0, c]) for c in self.C]
        self.QR = [np.linalg.qr(x) for x in self.Xt]           # eq. (MvRGLMQRi)
        self.Omega = np.asarray(Omega0, dtype=float)
        self.delta = np.ones(self.G) if delta is None else np.asarray(delta, dtype=float)

    def _blk(self, v, i):
        return v[self.roff[i]:self.roff[i + 1]]

    def sigma(self, u):
        N = self.N
        out = np.zeros_like(u)
        U0 = np.stack([self._blk(u, i)[:N] for i in range(self.G)])      # (G, N, k)
        S0 = np.tensordot(self.Omega.T, U0, axes=1)                      # (G, N, k)
        for h in range(self.G):
            out[self.roff[h]:self.roff[h] + N] = S0[h]
        return out

    def proj(self, xi):
        out = np.empty_like(xi)
        for i, (Qi, _) in enumerate(self.QR):
            b = self._blk(xi, i)
            out[self.roff[i]:self.roff[i + 1]] = b - Qi @ (Qi.T @ b)
        return out

    def dinv(self, xi):
        return xi / np.repeat(self.delta, self.rows)[:, None]

    def pi(self, xi):
        return self.dinv(self.proj(xi))

    def xstar_t(self, xi):
        return np.vstack([np.linalg.solve(Ri, Qi.T @ self._blk(xi, i)) for i, (Qi, Ri) in enumerate(self.QR)])

    def xmul(self, v):
        return np.vstack([self.Xt[i] @ v[self.offs[i]:self.offs[i + 1]] for i in range(self.G)])


def mvrglm_pcg_aug(Z0, Y, Omega0, C_list, gamma_list=None, tol=1e-13, maxit=None, stag_window=25,
                   delta=None, record=False):
    """MVRGLM: the restricted multivariate GLM estimated by model reduction
    (QR of Z0, Y0 = Q0^T Y) and Algorithm glmpcg2, in the reduced form of
    eq. (urwProj) (``pcg_aug_reduced``: the zero-variance restriction rows
    make lambda_i >> 1, where the literal r-recursion is unstable), with the
    block-diagonal applies of ``MvOps``; at most sum_i k_i + 1 steps in exact
    arithmetic (m + k - n + 1 with m = n = G N).  Y: (M, G) or (M, G, k); gamma_i:
    (k_i,) or (k_i, k), zero when not given.  Returns dict(B (N, G, k), b
    (G N, k) = vec(B), iters, status, relres[, history])."""
    Z0 = np.asarray(Z0, dtype=float)
    Y = np.asarray(Y, dtype=float)
    if Y.ndim == 2:
        Y = Y[:, :, None]
    M, G, k = Y.shape
    Q0, R0 = np.linalg.qr(Z0)                                # model reduction
    Y0 = np.tensordot(Q0.T, Y, axes=1)                        # (N, G, k)
    ops = MvOps(R0, C_list, Omega0, delta)
    parts = []
    for i in range(G):
        gi = np.zeros((ops.k_i[i], k))
        if gamma_list is not None and ops.k_i[i] > 0:
            gi = gi + np.asarray(gamma_list[i], dtype=float).reshape(ops.k_i[i], -1)
        parts.append(np.vstack([Y0[:, i, :], gi]))
    yaug = np.vstack(parts)
    if maxit is None:
        # the bound sum k_i + 1 holds in exact arithmetic; rounding costs a
        # few more steps on ill-conditioned restriction systems
        maxit = 2 * (sum(ops.k_i) + 1) + 10
    res = pcg_aug_reduced(ops, yaug, tol=tol, maxit=maxit, stag_window=stag_window, record=record)
    N = ops.N
    res["B"] = res["b"].reshape(G, N, k).transpose(1, 0, 2)
    res["ops"] = ops
    res["yaug"] = yaug
    return res


# ----------------------------------------------------------------------------
# residuals and the adjoint (gradient) of the augmented-system solution
# ----------------------------------------------------------------------------

def augmented_residual(X_blocks, Omega, Y, w, b):
    """Residual of eq. (aug1): (y - Sigma w - X b,  -X^T w), using the SUR
    applies (no dense matrices), for checks at any size."""
    op = SurOps.__new__(SurOps)
    op.X = X_blocks
    op.Omega = np.asarray(Omega, dtype=float)
    op.G = len(X_blocks)
    op.M = X_blocks[0].shape[0]
    op.n_i = [x.shape[1] for x in X_blocks]
    op.offs = np.cumsum([0] + op.n_i)
    m = op.G * op.M
    Y = np.asarray(Y, dtype=float).reshape(m, -1)
    w = np.asarray(w, dtype=float).reshape(m, -1)
    b = np.asarray(b, dtype=float).reshape(int(op.offs[-1]), -1)
    return Y - op.sigma(w) - op.xmul(b), -op.xt(w)


def sur_gls_gradient(X_blocks, Omega, Y, dL_db):
    """Adjoint of the augmented-system solution (dense, tiny sizes).

    With K = [[Sigma, X], [X^T, 0]] symmetric, (w; b) = K^-1 (y; 0) and a loss
    L(b):  (lam; mu) = K^-1 (0; dL/db),  dL/dy = lam,  dL/dK = -(lam; mu)(w; b)^T.
    Sigma = Omega (x) I_M puts omega_ij on the diagonal of block (i, j), so
    dL/domega_ij = -sum_t Lam[t, i] W[t, j]  (Lam, W the M x G matrices with
    vec(Lam) = lam, vec(W) = w).  Returns (dL_dy (m, k), dL_dOmega (G, G),
    unsymmetrised, summed over right-hand sides)."""
    Sigma, X = sur_dense(X_blocks, Omega)
    m, n = X.shape
    G = len(X_blocks)
    M = m // G
    K = augmented_matrix(Sigma, X)
    Y = np.asarray(Y, dtype=float).reshape(m, -1)
    gb = np.asarray(dL_db, dtype=float).reshape(n, -1)
    H = np.vstack([Y, np.zeros((n, Y.shape[1]))])
    x = np.linalg.solve(K, H)
    adj = np.linalg.solve(K, np.vstack([np.zeros((m, gb.shape[1])), gb]))
    lam = adj[:m]
    w = x[:m]
    gO = np.zeros((G, G))
    for c in range(Y.shape[1]):
        Lm = lam[:, c].reshape(G, M).T
        Wm = w[:, c].reshape(G, M).T
        gO -= Lm.T @ Wm
    return lam, gO


def sur_gls_gradient_kron(X_blocks, Omega, Y, dL_db):
    """Adjoint of eq. (aug1) for positive definite Omega, without forming any
    m x m matrix (eq. (GLS) with Sigma^-1 = Omega^-1 (x) I_M):

      A   = X^T Sigma^-1 X,  block (i, j) = (Omega^-1)_ij X_i^T X_j
      b   = A^-1 X^T Sigma^-1 y,        w  = Sigma^-1 (y - X b)
      lam = Sigma^-1 X A^-1 (dL/db),    mu = -A^-1 (dL/db)

    (w; b) and (lam; mu) solve eq. (aug1) with right-hand sides (y; 0) and
    (0; dL/db):  Sigma lam + X mu = 0 and X^T lam = dL/db.  With M x G
    matrices W, Lam (vec(W) = w, vec(Lam) = lam), Sigma^-1 v = vec(V Omega^-1)
    and dL/dOmega = -sum over right-hand sides of Lam^T W (unsymmetrised).
    Returns (b (n, k), w (m, k), lam (m, k), dL_dOmega (G, G))."""
    G = len(X_blocks)
    M = X_blocks[0].shape[0]
    n_i = [x.shape[1] for x in X_blocks]
    n = sum(n_i)
    offs = np.cumsum([0] + n_i)
    blk = np.repeat(np.arange(G), n_i)
    Oi = np.linalg.inv(Omega)
    Xc = np.hstack(X_blocks)                                   # M x n
    A = Oi[np.ix_(blk, blk)] * (Xc.T @ Xc)
    Y = np.asarray(Y, dtype=float).reshape(G * M, -1)
    gb = np.asarray(dL_db, dtype=float).reshape(n, -1)
    k = Y.shape[1]
    b = np.empty((n, k)); w = np.empty((G * M, k)); lam = np.empty((G * M, k))
    gO = np.zeros((G, G))

    def xt(V):        # X^T vec(V), V: M x G
        return np.concatenate([X_blocks[i].T @ V[:, i] for i in range(G)])

    def x_of(c):      # X c as an M x G matrix
        return np.column_stack([X_blocks[i] @ c[offs[i]:offs[i + 1]] for i in range(G)])

    for c in range(k):
        Ym = Y[:, c].reshape(G, M).T
        b[:, c] = np.linalg.solve(A, xt(Ym @ Oi))
        Wm = (Ym - x_of(b[:, c])) @ Oi
        Lm = x_of(np.linalg.solve(A, gb[:, c])) @ Oi
        w[:, c] = Wm.T.reshape(-1)
        lam[:, c] = Lm.T.reshape(-1)
        gO -= Lm.T @ Wm
    return b, w, lam, gO


def sur_gls_refined(X_blocks, Omega, Y, dL_db=None, steps=4):
    """Solutions of eq. (aug1) for right-hand sides (y; 0) and, if dL_db is
    given, (0; dL/db), accurate beyond the normal equations: mixed-precision
    iterative refinement (Wilkinson; Moler, J. ACM 14, 1967).  The iterate x
    is kept in numpy's extended ``longdouble``, the residual h - K x is
    evaluated in it (Sigma w as W Omega^T with M x G matrices, X b and X^T w
    block by block), and each correction solves K dx = residual in float64
    through the Kronecker inverse (positive definite Omega):
      db = A^-1 (X^T Sigma^-1 r1 - r2),  dw = Sigma^-1 (r1 - X db),
      A = X^T Sigma^-1 X.
    Returns dict(b, w[, lam, dOmega], corrections): dOmega = -sum Lam^T W
    (unsymmetrised, summed over right-hand sides, formed in longdouble);
    corrections holds ||db|| / ||b|| per refinement step."""
    LD = np.longdouble
    G = len(X_blocks)
    M = X_blocks[0].shape[0]
    n_i = [x.shape[1] for x in X_blocks]
    offs = np.cumsum([0] + n_i)
    n = int(offs[-1])
    blk = np.repeat(np.arange(G), n_i)
    Oi = np.linalg.inv(Omega)
    Xc = np.hstack(X_blocks)
    cf = np.linalg.cholesky(Oi[np.ix_(blk, blk)] * (Xc.T @ Xc))
    Xl = [x.astype(LD) for x in X_blocks]
    OmT = np.asarray(Omega, dtype=float).T.astype(LD)

    def k_solve(r1, r2):              # float64 solve of K (dw; db) = (r1; r2)
        R1 = r1.reshape(G, M).T @ Oi
        rhs = np.concatenate([X_blocks[i].T @ R1[:, i] for i in range(G)]) - r2
        db = np.linalg.solve(cf.T, np.linalg.solve(cf, rhs))
        Xdb = np.column_stack([X_blocks[i] @ db[offs[i]:offs[i + 1]] for i in range(G)])
        return ((r1.reshape(G, M).T - Xdb) @ Oi).T.reshape(-1), db

    def refine(h1, h2):               # x = K^-1 (h1; h2), extended-precision residuals
        w = np.zeros(G * M, dtype=LD)
        b = np.zeros(n, dtype=LD)
        corr = []
        for _ in range(steps + 1):
            Wm = w.reshape(G, M).T
            SW = Wm @ OmT
            Xb = np.column_stack([Xl[i] @ b[offs[i]:offs[i + 1]] for i in range(G)])
            r1 = h1 - (SW + Xb).T.reshape(-1)
            r2 = h2 - np.concatenate([Xl[i].T @ Wm[:, i] for i in range(G)])
            dw, db = k_solve(r1.astype(float), r2.astype(float))
            w += dw.astype(LD)
            b += db.astype(LD)
            corr.append(float(np.linalg.norm(db) / max(np.linalg.norm(b.astype(float)), 1e-300)))
        return w, b, corr

    Y = np.asarray(Y, dtype=float).reshape(G * M, -1)
    k = Y.shape[1]
    out = dict(b=np.empty((n, k)), w=np.empty((G * M, k)), corrections=[])
    Ws = []
    for c in range(k):
        w, b, corr = refine(Y[:, c].astype(LD), np.zeros(n, dtype=LD))
        out["b"][:, c] = b.astype(float)
        out["w"][:, c] = w.astype(float)
        out["corrections"].append(corr)
        Ws.append(w)
    if dL_db is not None:
        gb = np.asarray(dL_db, dtype=float).reshape(n, -1)
        out["lam"] = np.empty((G * M, k))
        gO = np.zeros((G, G), dtype=LD)
        for c in range(k):
            lam, _, corr = refine(np.zeros(G * M, dtype=LD), gb[:, c].astype(LD))
            out["lam"][:, c] = lam.astype(float)
            out["corrections"].append(corr)
            gO -= lam.reshape(G, M) @ Ws[c].reshape(G, M).T
        out["dOmega"] = gO.astype(float)
    return out

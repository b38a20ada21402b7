"""Batched solves (one persistent launch over many uneven SUR instances)
against the float64 oracle, instance by instance.  Tolerance: relative
||b - b_oracle|| <= 1e-9 per right-hand side, as for single solves."""
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


def run_batch(probs, k, reduce_rows=False):
    from paper_2510_14471_gb300.sur import GlmSurBatch
    bt = GlmSurBatch([(p.X_blocks, p.Omega) for p in probs], reduce_rows=reduce_rows)
    assert bt.setup_status() == 0
    b, iters, relres, status = bt.solve([p.Y for p in probs], k)
    return bt, [x.cpu().numpy() for x in b], iters.cpu().numpy(), relres.cpu().numpy(), status


@pytest.mark.parametrize("k", [1, 4, 8])
def test_small_batch_matches_oracle(k):
    probs = S.batched_uneven_instances(count=24, k=k, Mmax=900)
    bt, b, iters, relres, status = run_batch(probs, k)
    assert all(s in (0, 4) for s in status), status
    for j, p in enumerate(probs):
        ref = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
        assert relcols(b[j], ref) <= TOL_B, (j, relcols(b[j], ref), iters[j], relres[j])
    tile, ms = bt_tile(bt)
    assert tile in (8, 16, 32)


def bt_tile(bt):
    from paper_2510_14471_gb300 import _lib as L
    return L.glm_sur_batch_tile(bt.handle)


def test_batch_singular_and_edge_instances():
    # singular Omega (b = beta_true), a square block (M = n_i), G = 1
    probs = [S.make_problem(G=5, M=300, n_i=[3, 4, 2, 5, 3], k=2, seed=90, omega="lowrank", rank=3),
             S.make_problem(G=3, M=8, n_i=[8, 2, 5], k=2, seed=91, omega="chol"),
             S.make_problem(G=1, M=77, n_i=[6], k=2, seed=92, omega="chol"),
             S.make_problem(G=12, M=1001, n_i=[10] * 12, k=2, seed=93, omega="wishart")]
    bt, b, iters, relres, status = run_batch(probs, 2)
    assert relcols(b[0], probs[0].beta) <= TOL_B
    for j in (1, 2, 3):
        p = probs[j]
        assert relcols(b[j], O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)) <= TOL_B, j


def test_full_batch_workload_every_instance():
    # 2048 instances, G ~ U{2..12}, M ~ U{200..4000}, n_i ~ U{2..10}, k = 8:
    # every right-hand side of every instance against the structured oracle
    probs = S.batched_uneven_instances(count=2048, k=8)
    bt, b, iters, relres, status = run_batch(probs, 8)
    st = np.array(status).reshape(2048, 8)
    assert np.all(np.isin(st, (0, 4))), np.unique(st)
    # columns that stopped at the float64 rounding floor stay near it
    assert np.max(np.concatenate([np.ravel(r) for r in relres])) <= 1e-10
    errs = np.array([relcols(b[j], O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)) for j, p in enumerate(probs)])
    worst = int(np.argmax(errs))
    assert errs[worst] <= TOL_B, (worst, errs[worst])


@pytest.mark.parametrize("k", [1, 8])
def test_row_reduced_batch_matches_oracle(k):
    # Remark rem:reduction per instance (M_j >= 2 n_j reduced to n_j rows,
    # the others kept whole): the estimates of the full models
    probs = S.batched_uneven_instances(count=24, k=k, Mmax=900)
    probs.append(S.make_problem(G=3, M=10, n_i=[4, 2, 3], k=k, seed=94, omega="chol"))   # M < 2n: kept whole
    bt, b, iters, relres, status = run_batch(probs, k, reduce_rows=True)
    assert all(s in (0, 4) for s in status), status
    for j, p in enumerate(probs):
        ref = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
        assert relcols(b[j], ref) <= TOL_B, (j, relcols(b[j], ref), iters[j], relres[j])


def test_row_reduced_batch_singular_omega_and_rank_deficient_fallback():
    from paper_2510_14471_gb300 import _lib as L
    # singular Omega: b = beta_true on the reduced rows too
    probs = [S.make_problem(G=5, M=300, n_i=[3, 4, 2, 5, 3], k=2, seed=95, omega="lowrank", rank=3),
             S.make_problem(G=12, M=1001, n_i=[10] * 12, k=2, seed=96, omega="wishart")]
    bt, b, iters, relres, status = run_batch(probs, 2, reduce_rows=True)
    assert relcols(b[0], probs[0].beta) <= TOL_B
    assert relcols(b[1], O.sur_gls_structured(probs[1].X_blocks, probs[1].Omega, probs[1].Y)) <= TOL_B
    # equal regressors in every equation: W has no full column rank, the batch is kept whole
    q = S.make_problem(G=3, M=400, n_i=[4, 4, 4], k=2, seed=97, omega="chol", equal_X=True)
    bt2, b2, _, _, st2 = run_batch([q], 2, reduce_rows=True)
    assert relcols(b2[0], O.sur_gls_structured(q.X_blocks, q.Omega, q.Y)) <= TOL_B
    tile, _ = L.glm_sur_batch_tile(bt2.handle)
    assert tile in (8, 16, 32)


def test_row_reduced_full_batch_workload_every_instance():
    # the 2048-instance workload on the reduced rows: every right-hand side
    # of every instance against the structured oracle
    probs = S.batched_uneven_instances(count=2048, k=8)
    bt, b, iters, relres, status = run_batch(probs, 8, reduce_rows=True)
    st = np.array(status).reshape(2048, 8)
    assert np.all(np.isin(st, (0, 4))), np.unique(st)
    errs = np.array([relcols(b[j], O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)) for j, p in enumerate(probs)])
    worst = int(np.argmax(errs))
    assert errs[worst] <= TOL_B, (worst, errs[worst])

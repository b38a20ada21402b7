"""The seeded input generators: deterministic, and the workloads have the
dimensions and structure their recipes state (the sizes the GPU tests, the
golden files and the benchmark rely on)."""
import numpy as np

from synth import sur_inputs as S


def test_generators_are_deterministic():
    a, b = S.make_problem(G=3, M=50, n_i=[2, 3, 4], k=2, seed=9, omega="wishart"), \
        S.make_problem(G=3, M=50, n_i=[2, 3, 4], k=2, seed=9, omega="wishart")
    assert np.array_equal(a.Y, b.Y) and np.array_equal(a.Omega, b.Omega)
    assert all(np.array_equal(x, y) for x, y in zip(a.X_blocks, b.X_blocks))


def test_small_and_benchmark_workload_dimensions():
    p = S.small_g3_m200()
    assert (p.G, p.M, p.n_i, p.k) == (3, 200, [5, 4, 6], 1)
    q = S.singular_g64_m20000(k=2, M=120)            # block widths do not depend on M
    assert q.G == 64 and q.n == 1234 and all(8 <= v <= 32 for v in q.n_i)
    assert np.linalg.matrix_rank(q.Omega) == 56   # Omega = A A^T, A 64 x 56


def test_batched_instances_follow_their_ranges():
    probs = S.batched_uneven_instances(count=16, k=8)
    for p in probs:
        assert 2 <= p.G <= 12 and 200 <= p.M <= 4000 and all(2 <= v <= 10 for v in p.n_i)
        assert abs(np.trace(p.Omega) - 1.0) < 1e-12 and p.Y.shape == (p.G * p.M, 8)
        assert np.all(np.linalg.eigvalsh(p.Omega) > 0)


def test_constrained_and_differentiable_workloads():
    c = S.constrained_g32_m50000(k=2, M=60)
    assert c.n == 512 and c.C.shape == (64, 512) and np.allclose(c.d, c.C @ c.beta)
    ev = np.linalg.eigvalsh(c.Omega)
    assert 0.099 < ev.min() and ev.max() < 10.01
    d, L, target = S.differentiable_g128_m40000(M=30)
    assert d.G == 128 and d.n == 1793 and target.shape == (1793, 1)
    assert np.allclose(np.triu(L, 1), 0) and np.allclose(d.Omega, L @ L.T)

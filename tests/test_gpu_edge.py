"""Edge cases of the GPU solver against the oracle: certificates of infeasible
and unbounded problems, a problem with equality constraints only, SOCs of
ragged dimensions (2 .. 40, both lane-group widths),
the largest supported PSD order (32), a rank-deficient A (a duplicated equality
row: the KKT matrix is singular and only the regularisation makes it factorable),
and a single-variable problem."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import cones as C

pytestmark = pytest.mark.gpu

clr = pytest.importorskip("paper_2412_19027_gb300.clr")
from paper_2412_19027_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_19027_gb300 import build
    build.build()
    clr._lib()


def _solve(P, q, A, b, cones, bits=64):
    s = clr.clr_setup(sp.csc_matrix(P), np.asarray(q, float), sp.csc_matrix(A), np.asarray(b, float), cones,
                      clr.clr_default_settings(bits))
    s.solve()
    out = s.solution()
    s.free()
    return out


def _objective(P, q, x):
    P = np.asarray(sp.csc_matrix(P).todense())
    Pf = np.triu(P) + np.triu(P, 1).T
    return 0.5 * x @ Pf @ x + q @ x


@pytest.mark.parametrize("bits", [64, 32])
def test_primal_infeasible_certificate(bits):
    # x >= 1 and x <= 0
    P, q = np.zeros((1, 1)), np.array([1.0])
    A, b = np.array([[-1.0], [1.0]]), np.array([-1.0, 0.0])
    x, s, z, info = _solve(P, q, A, b, [(C.NONNEG, 2, 0.0)], bits)
    ref = oracle.solve(P, q, A, b, [(C.NONNEG, 2, 0.0)])
    assert info["status_name"] == ref.status_name == "PRIMAL_INFEASIBLE"
    assert b @ z == pytest.approx(-1.0, abs=1e-8)
    assert np.abs(A.T @ z).max() < 1e-6 and z.min() > -1e-8


@pytest.mark.parametrize("bits", [64, 32])
def test_dual_infeasible_certificate(bits):
    # min -x1 - x2 s.t. x >= 0 (as -x + s = 0, s >= 0): unbounded
    P, q = np.zeros((2, 2)), np.array([-1.0, -1.0])
    A, b = -np.eye(2), np.zeros(2)
    x, s, z, info = _solve(P, q, A, b, [(C.NONNEG, 2, 0.0)], bits)
    ref = oracle.solve(P, q, A, b, [(C.NONNEG, 2, 0.0)])
    assert info["status_name"] == ref.status_name == "DUAL_INFEASIBLE"
    # certificate: q'x = -1, A x + s = 0 with s in K, P x = 0
    assert q @ x == pytest.approx(-1.0, abs=1e-8)
    assert np.abs(A @ x + s).max() < 1e-6 and s.min() > -1e-8


def test_equality_constraints_only():
    """Zero cone only: min 1/2 x'Px + q'x s.t. Ax = b is one linear KKT system."""
    rng = np.random.default_rng(3)
    n, m = 30, 12
    M = rng.standard_normal((n, n))
    P = M @ M.T / n + np.eye(n)
    q = rng.standard_normal(n)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    x, s, z, info = _solve(np.triu(P), q, A, b, [(C.ZERO, m, 0.0)])
    assert info["status_name"] == "SOLVED"
    K = np.block([[P, A.T], [A, np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.r_[-q, b])
    np.testing.assert_allclose(x, sol[:n], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(z, sol[n:], rtol=1e-6, atol=1e-7)
    assert np.abs(s).max() == 0.0


def test_ragged_soc_dimensions():
    """SOCs of dimensions 2, 3, 5, 8, 9 and 40 in one problem: the 8-lane and the
    32-lane groups (every SOC at most 8 rows vs. not) against the oracle."""
    for dims in ([2, 3, 5, 8, 2, 8], [2, 3, 5, 8, 9, 40]):
        rng = np.random.default_rng(sum(dims))
        n = 25
        cones = [(C.NONNEG, 10, 0.0)] + [(C.SOC, d, 0.0) for d in dims]
        m = 10 + sum(dims)
        A = sp.random(m, n, density=0.3, random_state=rng, data_rvs=rng.standard_normal).tocsc()
        xs = rng.standard_normal(n)
        s0 = np.concatenate([rng.uniform(0.5, 2, 10)] + [np.r_[3.0 + np.sqrt(d), 0.3 * rng.standard_normal(d - 1)]
                                                         for d in dims])
        b = A @ xs + s0
        q = rng.standard_normal(n)
        P = sp.diags(rng.uniform(0.1, 1.0, n))
        x, s, z, info = _solve(P, q, A, b, cones)
        ref = oracle.solve(P, q, A, b, cones)
        assert info["status_name"] == ref.status_name, (dims, info, ref.status_name)
        if ref.status_name == "SOLVED":
            f, fr = _objective(P, q, x), _objective(P, q, ref.x)
            assert abs(f - fr) <= 1e-6 * max(1.0, abs(fr)), (dims, f, fr)


def _psd32_problem():
    rng = np.random.default_rng(21)
    n, k = 12, 32
    d = k * (k + 1) // 2
    iu, ju = np.triu_indices(k)
    order = np.lexsort((iu, ju))
    iu, ju = iu[order], ju[order]
    wgt = np.where(iu == ju, 1.0, np.sqrt(2.0))

    def svec(X):
        return X[iu, ju] * wgt

    rows, b = [], []
    for c in range(2):
        Aij = [svec((lambda G: (G + G.T) / 2)(rng.standard_normal((k, k)))) for _ in range(n)]
        rows.append(np.stack(Aij, axis=1))
        b.append(svec((2.0 if c == 0 else 40.0) * np.eye(k)))
    An = -np.eye(n)[:4]
    A = sp.csc_matrix(np.vstack(rows + [An]))
    b = np.concatenate(b + [np.zeros(4)])
    q = 3.0 * rng.standard_normal(n)
    P = sp.eye(n)
    cones = [(C.PSD, d, 0.0), (C.PSD, d, 0.0), (C.NONNEG, 4, 0.0)]
    return P, q, A, b, cones


def test_largest_psd_order_solved():
    """PSD(32) cones (528 svec rows each), the largest order the kernels take:
    min |x|^2/2 + q'x with two matrix inequalities B_i - sum_j x_j A_ij >= 0, one of
    them active at the optimum, and a few nonneg rows.  Near convergence the
    inactive cone's Z has eigenvalues ~1e-11 against S ~ 38; the solve reaches
    SOLVED with the oracle's objective and iteration count."""
    P, q, A, b, cones = _psd32_problem()
    x, s, z, info = _solve(P, q, A, b, cones)
    ref = oracle.solve(P, q, A, b, cones)
    assert ref.status_name == info["status_name"] == "SOLVED", info
    f, fr = _objective(P, q, x), _objective(P, q, ref.x)
    assert abs(f - fr) <= 1e-6 * max(1.0, abs(fr))
    assert abs(info["iterations"] - ref.iterations) <= 2, (info["iterations"], ref.iterations)


def test_rank_deficient_equalities():
    """A duplicated equality row: A has deficient row rank, the KKT matrix without
    regularisation is singular; the solution is that of the problem without the
    duplicate."""
    prob = W.nonneg_qp(4, n=20, m=40, density=0.3, rank=3)
    A = sp.vstack([prob.A[:1], prob.A[:1], prob.A]).tocsc()
    x0 = np.linalg.lstsq(prob.A.toarray(), prob.b, rcond=None)[0]
    beq = float((prob.A[:1] @ x0)[0])
    b = np.r_[beq, beq, prob.b]
    cones = [(C.ZERO, 2, 0.0)] + list(prob.cones)
    x, s, z, info = _solve(prob.P, prob.q, A, b, cones)
    ref = oracle.solve(prob.P, prob.q, A, b, cones)
    assert info["status_name"] == ref.status_name == "SOLVED"
    f, fr = prob.objective(x), prob.objective(ref.x)
    assert abs(f - fr) <= 1e-6 * max(1.0, abs(fr))


def test_single_variable():
    # min (x - 2)^2 / 2 s.t. 0 <= x <= 1  ->  x = 1
    P, q = np.array([[1.0]]), np.array([-2.0])
    A, b = np.array([[-1.0], [1.0]]), np.array([0.0, 1.0])
    x, s, z, info = _solve(P, q, A, b, [(C.NONNEG, 2, 0.0)])
    assert info["status_name"] == "SOLVED"
    assert x[0] == pytest.approx(1.0, abs=1e-7)
    assert z @ s == pytest.approx(0.0, abs=1e-7)


def test_incremental_solve_matches_clr_solve():
    """clr_solve_begin / clr_solve_iterate / clr_solve_end run the same kernels
    and graphs as clr_solve: the same iterates bit for bit, and the iteration
    counts of the parts add up to the solve's."""
    prob = W.mixed_cone(3, n=80, n_zero=10, n_nonneg=100, n_soc=15, n_exp=5, n_pow=5, nnz_per_col=4)
    st = clr.clr_default_settings(64)
    s = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
    s.solve()
    x1, s1, z1, info1 = s.solution()
    s.solve_begin()
    total, done, calls = 0, False, 0
    while not done:
        done, ran = s.solve_iterate(3)
        total += ran
        calls += 1
        assert calls < 100
    s.solve_end()
    x2, s2, z2, info2 = s.solution()
    s.free()
    assert info1["status_name"] == info2["status_name"] == "SOLVED"
    assert info1["iterations"] == info2["iterations"] == total
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(z1, z2)

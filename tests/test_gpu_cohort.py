"""Cohorts: many independent problems merged into one solver (clr_batch_setup).

Each problem of a cohort must give the result it gives alone -- here bit for
bit: same status, same iteration count, identical x, s, z (every sum of a
problem is formed in an order that does not depend on the rest of the cohort,
and each problem keeps its own equilibration, ordering and supernodes) -- and
the oracle's answer (status, objective to 1e-6 relative).  With a low-precision
factor a cohort that needs the FP64 escalation takes it as a whole; those
results are compared at the acceptance bar.  Problems of
different sizes, cone families and outcomes (solved, infeasible) share one
cohort; the ones that stop early are frozen while the others go on.
"""
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


def _infeasible_lp():
    # x >= 1 and x <= 0 (nonneg rows b - A x >= 0), plus a free second variable
    P = sp.csc_matrix((2, 2))
    A = sp.csc_matrix(np.array([[-1.0, 0.0], [1.0, 0.0], [0.0, 1.0], [0.0, -1.0]]))
    b = np.array([-1.0, 0.0, 3.0, 3.0])
    q = np.array([1.0, 1.0])
    return W.Problem("infeasible_lp", P, q, A, b, [(C.NONNEG, 4, 0.0)])


def _mixed_cohort():
    return [
        W.nonneg_qp(0),
        W.mixed_cone(1, n=60, n_zero=10, n_nonneg=80, n_soc=12, n_exp=8, n_pow=8, nnz_per_col=4),
        W.mixed_cone(2, n=40, n_zero=5, n_nonneg=30, n_soc=15, soc_dim=4, n_exp=0, n_pow=0, nnz_per_col=5),
        W.banded_lp(0, n=150, window=16),
        W.mpc_qp(0, T=10, nx=4, nu=2),
        W.psd_batch(0, n=60, n_psd=4, psd_k=4, n_nonneg=20, nnz_per_col=4),
        W.psd_batch(1, n=60, n_psd=3, psd_k=5, n_nonneg=20, nnz_per_col=4),  # another PSD order
        W.psd_mixed(1, n=40, orders=(2, 3, 6), per_order=2, n_nonneg=10, nnz_per_col=4),
        _infeasible_lp(),
        W.nonneg_qp(3),
        W.mixed_cone(2, n=200, n_zero=50, n_nonneg=300, n_soc=50, n_exp=10, n_pow=10, nnz_per_col=6),
        # SOCs of 50 and 40 rows in the sparse KKT form (two auxiliary rows each)
        W.mixed_cone(5, n=80, n_zero=10, n_nonneg=60, n_soc=2, soc_dim=50, n_exp=2, n_pow=2, nnz_per_col=5),
        W.mixed_cone(6, n=60, n_zero=6, n_nonneg=40, n_soc=3, soc_dim=40, n_exp=0, n_pow=0, nnz_per_col=5),
    ]


def _alone(prob, st):
    s = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
    s.solve()
    out = s.solution()
    s.free()
    return out


@pytest.mark.parametrize("bits", [64, 32])
def test_cohort_matches_alone_and_oracle(bits):
    probs = _mixed_cohort()
    st = clr.clr_default_settings(bits)
    batch = clr.clr_batch_setup([(p.P, p.q, p.A, p.b, p.cones) for p in probs], st)
    assert batch.size() == len(probs)
    batch.solve()
    iters = []
    for i, p in enumerate(probs):
        xb, sb, zb, ib = batch.solution_of(i)
        xa, sa, za, ia = _alone(p, st)
        assert ib["status_name"] == ia["status_name"], (p.name, ib, ia)
        if ib["fp64_from_iter"] < 0 and ia["fp64_from_iter"] < 0:
            assert ib["iterations"] == ia["iterations"], (p.name, ib, ia)
            for u, v in ((xb, xa), (sb, sa), (zb, za)):
                np.testing.assert_array_equal(u, v, err_msg=p.name)
        elif ib["status_name"] == "SOLVED":
            # a low-precision cohort goes on in FP64 as a whole once one of its problems needs it
            f, fa = p.objective(xb), p.objective(xa)
            assert abs(f - fa) <= 1e-6 * max(1.0, abs(fa)), (p.name, f, fa)
        iters.append(ib["iterations"])
        ref = oracle.solve(p.P, p.q, p.A, p.b, p.cones)
        assert ib["status_name"] == ref.status_name, (p.name, ib["status_name"], ref.status_name)
        if ref.status_name == "SOLVED":
            f, fr = p.objective(xb), p.objective(ref.x)
            assert abs(f - fr) <= 1e-6 * max(1.0, abs(fr)), (p.name, f, fr)
    assert len(set(iters)) > 1  # problems stop at different iterations and stay frozen
    batch.free()


def test_cohort_infeasible_member_certificate():
    probs = [W.nonneg_qp(1), _infeasible_lp(), W.mpc_qp(2, T=12, nx=5, nu=3)]
    batch = clr.clr_batch_setup([(p.P, p.q, p.A, p.b, p.cones) for p in probs])
    batch.solve()
    statuses = [batch.info_of(i)["status_name"] for i in range(3)]
    assert statuses == ["SOLVED", "PRIMAL_INFEASIBLE", "SOLVED"], statuses
    _, _, z, _ = batch.solution_of(1)
    p = probs[1]
    # certificate: A'z = 0, b'z = -1, z in K* (nonneg)
    assert abs(p.b @ z + 1.0) < 1e-8
    assert np.abs(p.A.T @ z).max() < 1e-6
    assert z.min() > -1e-8
    batch.free()


def test_cohort_uneven_mpc_fp32():
    """Uneven MPC problems (the serving workload's shapes), FP32 factor: some of
    them need the FP64 escalation late in the solve (the FP32 factor with the
    paper's regularisation no longer refines to 1e-6 there)."""
    rng = np.random.default_rng(5)
    probs = [W.mpc_qp(int(s), T=int(rng.integers(10, 31)), nx=int(rng.integers(4, 9)), nu=int(rng.integers(2, 5)))
             for s in range(12)]
    st = clr.clr_default_settings(32)
    batch = clr.clr_batch_setup([(p.P, p.q, p.A, p.b, p.cones) for p in probs], st)
    batch.solve()
    for i, p in enumerate(probs):
        x, s, z, info = batch.solution_of(i)
        assert info["status_name"] == "SOLVED", (i, info)
        ref = oracle.solve(p.P, p.q, p.A, p.b, p.cones)
        f, fr = p.objective(x), p.objective(ref.x)
        assert abs(f - fr) <= 1e-6 * max(1.0, abs(fr)), (i, f, fr)
    batch.free()


def test_cohort_update_qb_of_one_member():
    probs = [W.mpc_qp(3, T=10, nx=4, nu=2), W.mpc_qp(4, T=14, nx=6, nu=3)]
    batch = clr.clr_batch_setup([(p.P, p.q, p.A, p.b, p.cones) for p in probs])
    batch.solve()
    x1_before = batch.solution_of(1)[0].copy()
    # a new initial state for problem 0 only: the dynamics rows of b change
    p0 = probs[0]
    b_new = p0.b.copy()
    b_new[: p0.meta["nx"]] *= -0.5
    batch.update_qb_of(0, p0.q, b_new)
    batch.solve()
    x0, _, _, i0 = batch.solution_of(0)
    x1, _, _, _ = batch.solution_of(1)
    ref = oracle.solve(p0.P, p0.q, p0.A, b_new, p0.cones)
    assert i0["status_name"] == "SOLVED"
    f, fr = p0.objective(x0), p0.objective(ref.x)
    assert abs(f - fr) <= 1e-6 * max(1.0, abs(fr))
    np.testing.assert_allclose(x1, x1_before, rtol=0, atol=1e-12)
    batch.free()

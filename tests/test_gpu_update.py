"""Parametric updates of P and A (clr_update_PA): after new values on the same
patterns, a solve matches a fresh setup of the new problem and the oracle on it
(status; objective to 1e-6 relative), for one problem and inside a cohort,
where the other problems' results stay bit-identical."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle

pytestmark = pytest.mark.gpu

clr = pytest.importorskip("paper_2412_19027_gb300.clr")
from paper_2412_19027_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_19027_gb300 import build
    build.build()
    clr._lib()


def _objective(P, q, x):
    P = sp.csc_matrix(P).toarray()
    Pf = np.triu(P) + np.triu(P, 1).T
    return 0.5 * x @ Pf @ x + q @ x


def _same_pattern(M0, M1):
    M0, M1 = sp.csc_matrix(M0), sp.csc_matrix(M1)
    M0.sort_indices()
    M1.sort_indices()
    return np.array_equal(M0.indptr, M1.indptr) and np.array_equal(M0.indices, M1.indices)


def _check_against(P, q, A, b, cones, x, info, bits):
    P = sp.csc_matrix(sp.triu(sp.csc_matrix(P)))
    ref = oracle.solve(P, q, A, b, cones)
    fresh = clr.clr_setup(P, q, A, b, cones, clr.clr_default_settings(bits))
    fresh.solve()
    xf, _, _, inf_f = fresh.solution()
    fresh.free()
    assert info["status_name"] == inf_f["status_name"] == ref.status_name == "SOLVED", (info, inf_f)
    f, ff, fr = _objective(P, q, x), _objective(P, q, xf), _objective(P, q, ref.x)
    assert abs(f - fr) <= 1e-6 * max(1.0, abs(fr)), (f, fr)
    assert abs(ff - fr) <= 1e-6 * max(1.0, abs(fr)), (ff, fr)
    assert abs(info["iterations"] - ref.iterations) <= 2


@pytest.mark.parametrize("bits", [64, 32])
def test_update_PA_mpc_dynamics(bits):
    """MPC re-solve with new dynamics (A), cost weights (P) and initial state (b)."""
    p0 = W.mpc_qp(11, T=12, nx=6, nu=3)
    p1 = W.mpc_qp(12, T=12, nx=6, nu=3)
    assert _same_pattern(p0.A, p1.A)
    P1 = sp.csc_matrix(p0.P * 1.7)
    s = clr.clr_setup(p0.P, p0.q, p0.A, p0.b, p0.cones, clr.clr_default_settings(bits))
    s.solve()
    assert s.solution()[3]["status_name"] == "SOLVED"
    s.update_PA(P=P1, A=p1.A)
    s.update_qb(p1.q, p1.b)
    s.solve()
    x, sl, z, info = s.solution()
    s.free()
    _check_against(P1, p1.q, p1.A, p1.b, p1.cones, x, info, bits)


@pytest.mark.parametrize("which", ["P", "A"])
def test_update_P_or_A_alone(which):
    prob = W.nonneg_qp(5)
    rng = np.random.default_rng(7)
    P1, A1 = sp.csc_matrix(prob.P), sp.csc_matrix(prob.A)
    if which == "P":
        M = rng.standard_normal((prob.n, 3))
        P1 = sp.csc_matrix(prob.P.toarray() + M @ M.T * 0.5)  # dense pattern, as before
        assert _same_pattern(sp.triu(P1), sp.triu(prob.P))
    else:
        A1 = A1.copy()
        A1.data = A1.data * (1.0 + 0.2 * rng.standard_normal(A1.nnz))
    s = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones)
    s.solve()
    s.update_PA(P=P1 if which == "P" else None, A=A1 if which == "A" else None)
    s.solve()
    x, sl, z, info = s.solution()
    s.free()
    _check_against(P1, prob.q, A1, prob.b, prob.cones, x, info, 64)


def test_update_PA_in_a_cohort():
    probs = [W.nonneg_qp(s, n=30, m=60) for s in (1, 2, 3)]
    b = clr.clr_batch_setup([(p.P, p.q, p.A, p.b, p.cones) for p in probs])
    b.solve()
    before = [b.solution_of(i) for i in range(3)]
    A1 = sp.csc_matrix(probs[1].A).copy()
    A1.data = A1.data * 0.8
    P1 = sp.csc_matrix(probs[1].P * 1.3)
    b.update_PA_of(1, P=P1, A=A1)
    b.solve()
    after = [b.solution_of(i) for i in range(3)]
    b.free()
    for i in (0, 2):
        for u, v in zip(before[i][:3], after[i][:3]):
            assert np.array_equal(u, v)
    p = probs[1]
    _check_against(P1, p.q, A1, p.b, p.cones, after[1][0], after[1][3], 64)

"""The paper's benchmark classes (Sec. 5.1 portfolio and Huber QPs, Sec. 5.3
entropy maximisation) as generated in workloads.py: the conic forms are pinned
to the original problems solved by an independent method (scipy's SLSQP /
L-BFGS-B on the problem as the paper states it), through the oracle."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle
from paper_2412_19027_gb300 import workloads as W


def _conic_objective(prob, x):
    P = prob.P.toarray()
    Pf = np.triu(P) + np.triu(P, 1).T
    return 0.5 * x @ Pf @ x + prob.q @ x


@pytest.mark.parametrize("seed", [0, 1])
def test_portfolio_matches_direct_qp(seed):
    prob = W.portfolio_qp(seed, n=30)
    r = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones)
    assert r["status_name"] == "SOLVED"
    n, F, d, mu, g = prob.meta["n"], prob.meta["F"].toarray(), prob.meta["d"], prob.meta["mu"], prob.meta["gamma"]
    Sigma = F @ F.T + np.diag(d)
    x = r["x"][:n]
    # the conic objective is the negated portfolio objective at x
    assert _conic_objective(prob, r["x"]) == pytest.approx(-(mu @ x - g * x @ Sigma @ x), rel=1e-7, abs=1e-9)
    f = lambda v: -(mu @ v - g * v @ Sigma @ v)
    jac = lambda v: -(mu - 2 * g * Sigma @ v)
    ref = minimize(f, np.full(n, 1.0 / n), jac=jac, method="SLSQP", bounds=[(0, None)] * n,
                   constraints=[{"type": "eq", "fun": lambda v: v.sum() - 1.0, "jac": lambda v: np.ones(n)}],
                   options={"ftol": 1e-14, "maxiter": 1000})
    assert ref.success
    assert f(x) == pytest.approx(ref.fun, rel=1e-6, abs=1e-8)
    assert abs(x.sum() - 1.0) < 1e-7 and x.min() > -1e-7


@pytest.mark.parametrize("seed", [0, 1])
def test_huber_matches_direct_minimisation(seed):
    prob = W.huber_qp(seed, n=12)
    r = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones)
    assert r["status_name"] == "SOLVED"
    A, b, T, n = prob.meta["A"].toarray(), prob.meta["b"], prob.meta["T"], prob.meta["n"]

    def huber(v):
        t = A @ v - b
        return np.where(np.abs(t) <= T, t * t, T * (2 * np.abs(t) - T)).sum()

    def grad(v):
        t = A @ v - b
        return A.T @ np.where(np.abs(t) <= T, 2 * t, 2 * T * np.sign(t))

    x = r["x"][:n]
    assert _conic_objective(prob, r["x"]) == pytest.approx(huber(x), rel=1e-7, abs=1e-9)
    ref = minimize(huber, np.zeros(n), jac=grad, method="L-BFGS-B", options={"ftol": 1e-15, "gtol": 1e-12})
    assert huber(x) == pytest.approx(ref.fun, rel=1e-6)


def test_entropy_matches_direct_maximisation():
    """The oracle's iterate on the exponential-cone form reaches the entropy
    maximum to ~1e-7 (every cone is active at the optimum; see the readings)."""
    prob = W.entropy_max(0, n=10)
    r = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones)
    n, A, b = prob.meta["n"], prob.meta["A"], prob.meta["b"]
    x = r["x"][:n]
    assert r["gap_rel"] < 1e-6 and r["res_primal"] < 1e-6
    ent = lambda v: float(-(v * np.log(np.maximum(v, 1e-300))).sum())
    ref = minimize(lambda v: -ent(v), np.full(n, 1.0 / n), jac=lambda v: np.log(np.maximum(v, 1e-300)) + 1.0,
                   method="SLSQP", bounds=[(1e-12, None)] * n,
                   constraints=[{"type": "eq", "fun": lambda v: v.sum() - 1.0},
                                {"type": "ineq", "fun": lambda v: b - A @ v, "jac": lambda v: -A}],
                   options={"ftol": 1e-12, "maxiter": 2000})
    # SLSQP may end on its line search at the optimum; its point must be feasible
    assert abs(ref.x.sum() - 1.0) < 1e-8 and (A @ ref.x - b).max() < 1e-8
    assert ent(x) == pytest.approx(ent(ref.x), rel=1e-6)
    assert -r["obj_primal"] == pytest.approx(ent(ref.x), rel=1e-6)

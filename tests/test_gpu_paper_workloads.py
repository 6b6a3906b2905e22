"""The paper's benchmark classes (Sec. 5.1 portfolio and Huber QPs, Sec. 5.3
entropy maximisation) on the GPU against the oracle: status, objective to 1e-6
relative, iterations within 2; FP64 and FP32 factors."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

clr = pytest.importorskip("paper_2412_19027_gb300.clr")
from paper_2412_19027_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_19027_gb300 import build
    build.build()
    clr._lib()


def _objective(prob, x):
    P = prob.P.toarray()
    Pf = np.triu(P) + np.triu(P, 1).T
    return 0.5 * x @ Pf @ x + prob.q @ x


def _gpu(prob, bits):
    s = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, clr.clr_default_settings(bits))
    s.solve()
    out = s.solution()
    s.free()
    return out


@pytest.mark.parametrize("bits", [64, 32])
@pytest.mark.parametrize("make", [lambda: W.portfolio_qp(3, n=80), lambda: W.huber_qp(3, n=40)],
                         ids=["portfolio", "huber"])
def test_paper_qps_against_oracle(make, bits):
    prob = make()
    x, s, z, info = _gpu(prob, bits)
    ref = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones)
    assert info["status_name"] == ref["status_name"] == "SOLVED", info
    f, fr = _objective(prob, x), _objective(prob, ref["x"])
    assert abs(f - fr) <= 1e-6 * max(1.0, abs(fr)), (f, fr)
    assert abs(info["iterations"] - ref["iterations"]) <= 2, (info["iterations"], ref["iterations"])


def test_entropy_accuracy_reached():
    """Every exponential cone is active at the entropy maximum; the oracle ends
    near a relative gap of 1e-7 (see the readings), and the GPU solve must reach
    the same maximum to 1e-6."""
    prob = W.entropy_max(2, n=20)
    x, s, z, info = _gpu(prob, 64)
    ref = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones)
    assert np.all(np.isfinite(x)) and info["gap_rel"] < 1e-5, info
    n = prob.meta["n"]
    xe, xr = x[:n], ref["x"][:n]
    ent = lambda v: float(-(v * np.log(np.maximum(v, 1e-300))).sum())
    assert ent(xe) == pytest.approx(ent(xr), rel=1e-6)
    assert abs(xe.sum() - 1.0) < 1e-6


@pytest.mark.parametrize("bits", [64, 32])
@pytest.mark.parametrize("n", [20, 60])
def test_entropy_solved_at_the_papers_tolerance(n, bits):
    """Entropy maximisation at the tolerance the paper runs its benchmark classes at
    (eps_feas = eps_inf = 1e-6): SOLVED on both sides, objective to 1e-6 relative,
    iterations within 2 (4 with the FP32 factor)."""
    prob = W.entropy_max(2, n=n)
    st = clr.clr_default_settings(bits, eps_feas=1e-6, eps_inf=1e-6)
    s = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
    s.solve()
    x, sl, z, info = s.solution()
    s.free()
    ref = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones, settings=dict(eps_feas=1e-6, eps_inf=1e-6))
    assert info["status_name"] == ref["status_name"] == "SOLVED", (info, ref["status_name"])
    f, fr = _objective(prob, x), _objective(prob, ref["x"])
    assert abs(f - fr) <= 1e-6 * max(1.0, abs(fr)), (f, fr)
    assert abs(info["iterations"] - ref["iterations"]) <= (2 if bits == 64 else 4), (info["iterations"],
                                                                                      ref["iterations"])


@pytest.mark.xfail(reason="entropy maximisation: every cone active at the optimum; the 1e-8 gap may not be reached",
                   strict=False)
def test_entropy_solved():
    prob = W.entropy_max(2, n=20)
    x, s, z, info = _gpu(prob, 64)
    assert info["status_name"] == "SOLVED", info

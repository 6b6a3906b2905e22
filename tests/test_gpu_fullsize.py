"""Full-size workloads on the GPU, in the configuration the benchmark times.

The mixed-cone QP (KKT order 8 600) is compared with a stored solve of the
oracle (tests/golden/mixed_cone_c1_seed0.json, written by the committed script
beside it: about a minute of the dense oracle).  The dense oracle cannot run at
the other sizes (KKT orders 135 000 and 600 000), so those solves are checked
against what holds at any size:
  * the planted optimum: every problem is built from a chosen complementary
    (x*, s*, z*), so the optimal value is known -- objective to 1e-6 relative;
  * the solver's termination tests at eps_feas = 1e-8 (residuals and gap);
  * the returned s in K and z in K* (cone membership, per family), and
    complementarity s'z small;
  * sampled outputs recomputed one by one by the oracle: the scaling matrix
    H of a random sample of cones at the returned point (Appendix A of the
    paper: NT for SOC/PSD, the BFGS update for exp/pow), against the
    library's step-level entry point on the same cones.
"""
import json
import os

import numpy as np
import pytest

import kkt_checks as KC

from oracle import cones as C

pytestmark = pytest.mark.gpu

clr = pytest.importorskip("paper_2412_19027_gb300.clr")
from paper_2412_19027_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_19027_gb300 import build
    build.build()
    clr._lib()


def _blocks(cones, v):
    out, off = [], 0
    for (t, d, a) in cones:
        out.append((t, d, a, v[off:off + d]))
        off += d
    return out


def _check_cones(cones, s, z, tol):
    for (t, d, a, sv), (_, _, _, zv) in zip(_blocks(cones, s), _blocks(cones, z)):
        if t == C.ZERO:
            assert np.abs(sv).max() <= tol
        elif t == C.NONNEG:
            assert sv.min() >= -tol and zv.min() >= -tol
        elif t == C.SOC:
            assert sv[0] - np.linalg.norm(sv[1:]) >= -tol and zv[0] - np.linalg.norm(zv[1:]) >= -tol
        elif t == C.PSD:
            assert np.linalg.eigvalsh(C.smat(sv)).min() >= -tol
            assert np.linalg.eigvalsh(C.smat(zv)).min() >= -tol


def _sampled_scalings(cones, s, z, mu, rng, k=40):
    """H of a random sample of non-zero cones at the final iterate (pushed a
    little into the interior so that every scaling is defined)."""
    idx = [i for i, (t, d, a) in enumerate(cones) if t not in (C.ZERO, C.NONNEG)]
    if not idx:
        return
    pick = sorted(rng.choice(idx, min(k, len(idx)), replace=False))
    blocks_s, blocks_z = _blocks(cones, s), _blocks(cones, z)
    sub, ss, zz = [], [], []
    for i in pick:
        t, d, a, sv = blocks_s[i]
        zv = blocks_z[i][3]
        e = C.central_point(t, d, a)  # in the interior of both K and K*
        sub.append((t, d, a))
        ss.append(sv + 0.1 * e)
        zz.append(zv + 0.1 * e)
    ss, zz = np.concatenate(ss), np.concatenate(zz)
    H = clr.clr_cones_scaling(sub, ss, zz, mu)
    off = 0
    for (t, d, a), Hg in zip(sub, H):
        sv, zv = ss[off:off + d], zz[off:off + d]
        off += d
        if t in (C.EXP, C.POW):
            Href = C.bfgs_scaling(t, sv, zv, mu, a)
        else:
            Href = C.nt_scaling(t, sv, zv)["H"]
        np.testing.assert_allclose(Hg, Href, rtol=1e-8, atol=1e-10 * np.abs(Href).max())


def _solve_full(prob, bits, **kw):
    st = clr.clr_default_settings(bits, ir_stop_ratio=5.0, **kw)
    s = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
    s.solve()
    x, sl, z, info = s.solution()
    hist = s.history()
    s.free()
    # iteration, mu, pcost, dcost, res_p, res_d, gap, alpha_a, sigma, alpha_c, ir steps, tau
    assert info["status_name"] == "SOLVED", "%s\n%s" % (
        {k: v for k, v in info.items()}, np.array2string(hist[-6:], precision=3, max_line_width=200))
    f_star = prob.objective(prob.x_star)
    f = prob.objective(x)
    assert abs(f - f_star) <= 1e-6 * max(1.0, abs(f_star)), (f, f_star)
    # the termination tests of the solver at eps_feas = 1e-8
    scale_p = max(1.0, np.abs(prob.b).max() + np.abs(x).max() + np.abs(sl).max())
    scale_d = max(1.0, np.abs(prob.q).max() + np.abs(x).max() + np.abs(z).max())
    assert info["res_primal"] <= 1e-8 * scale_p and info["res_dual"] <= 1e-8 * scale_d, info
    # the same test recomputed on the host in FP64 from the returned point
    ok, d = KC.termination(prob.P, prob.q, prob.A, prob.b, x, sl, z, 1e-8 * (1 + 1e-6))
    assert ok, d
    _check_cones(prob.cones, sl, z, 1e-7 * max(1.0, np.abs(sl).max(), np.abs(z).max()))
    assert abs(sl @ z) <= 1e-6 * max(1.0, abs(f_star))
    return x, sl, z, info


@pytest.mark.parametrize("bits", [64, 32])
def test_mixed_cone_n2000_m6600(bits):
    prob = W.mixed_cone(0)
    x, s, z, info = _solve_full(prob, bits)
    _sampled_scalings(prob.cones, s, z, info["mu"] + 1e-3, np.random.default_rng(0))


GOLDEN_C1 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mixed_cone_c1_seed0.json")


@pytest.mark.parametrize("bits", [64, 32])
def test_mixed_cone_n2000_m6600_matches_oracle_golden(bits):
    """The benchmark's mixed-cone QP, FP64 factor and FP32 factor + FP64
    refinement, against the oracle's stored solve: status, iterations within 2,
    objective to 1e-6 relative, the termination test at 1e-8 recomputed on the
    host from the returned point, and the primal optimum x entry by entry.  x is
    unique (P is positive definite); the tolerance 1e-6 max(1, |x|_inf) is
    empirical (two answers at eps_feas = 1e-8 agree to ~1e-8 here).  The dual z is
    not unique (more active rows than variables): it is checked for validity --
    dual residual and gap in the termination test, z in K*."""
    g = json.load(open(GOLDEN_C1))
    prob = W.mixed_cone(0)
    st = clr.clr_default_settings(bits, ir_stop_ratio=5.0)
    s_ = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
    s_.solve()
    x, sl, z, info = s_.solution()
    s_.free()
    assert info["status_name"] == g["status"] == "SOLVED", info
    assert abs(info["iterations"] - g["iterations"]) <= 2, (info["iterations"], g["iterations"])
    f = prob.objective(x)
    assert abs(f - g["objective"]) <= 1e-6 * max(1.0, abs(g["objective"])), (f, g["objective"])
    ok, d = KC.termination(prob.P, prob.q, prob.A, prob.b, x, sl, z, 1e-8 * (1 + 1e-6))
    assert ok, d
    xg = np.array(g["x"])
    assert np.abs(x - xg).max() <= 1e-6 * max(1.0, np.abs(xg).max()), np.abs(x - xg).max()
    sg = prob.b - prob.A @ xg
    assert np.abs(sl - sg).max() <= 1e-6 * max(1.0, np.abs(sg).max()) + d["res_primal"]
    _check_cones(prob.cones, sl, z, 1e-7 * max(1.0, np.abs(sl).max(), np.abs(z).max()))


def test_banded_lp_n200000_m400000_fp32():
    prob = W.banded_lp(0)
    _solve_full(prob, 32)


@pytest.mark.parametrize("bits", [32, 64])
def test_psd_batch_2000x10_n20000(bits):
    """The PSD batch (2000 PSD(10) cones of complementary rank 5 + 5, 5000 nonneg
    rows): SOLVED at eps_feas = 1e-8 against the planted optimum, in FP32 (with
    the FP64 escalation) and in FP64.  Near mu ~ 1e-9 the PSD blocks of H reach
    condition numbers ~1e19: Delta s uses H in factored form, and a breakdown of
    the unpivoted FP64 factor is redone with a larger static regularisation."""
    prob = W.psd_batch(0)
    x, sl, z, info = _solve_full(prob, bits)
    _sampled_scalings(prob.cones, sl, z, info["mu"] + 1e-3, np.random.default_rng(1))


@pytest.mark.parametrize("bits", [32, 64])
def test_big_front_schedules_agree(bits):
    """The dataflow big-front kernel (one launch per level) and the per-panel
    launches run the same arithmetic per tile: the same iterations and the same
    optimum to rounding."""
    prob = W.mixed_cone(0)
    out = {}
    for sched in (0, 1):
        x, s, z, info = _solve_full(prob, bits, big_front_schedule=sched)
        out[sched] = (x, info)
    (x0, i0), (x1, i1) = out[0], out[1]
    assert i0["iterations"] == i1["iterations"], (i0, i1)
    f0, f1 = prob.objective(x0), prob.objective(x1)
    assert abs(f0 - f1) <= 1e-9 * max(1.0, abs(f0))

"""Serving loop (clr_server_*): continuous batching of independent solves.

Requests that arrive while others are on the GPU join later cohorts; every
result must be the one the problem gets alone, bit for bit (same status and
iteration count, identical x, s, z), and the oracle's (objective to 1e-6).
With a low-precision factor a cohort that needs the FP64 escalation takes it
as a whole, so such results are compared at the acceptance bar instead.
"""
import time

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


def _mpc(seed):
    rng = np.random.default_rng(1000 + seed)
    return W.mpc_qp(seed, T=int(rng.integers(10, 41)), nx=int(rng.integers(4, 13)), nu=int(rng.integers(2, 5)))


def _alone(p, st):
    s = clr.clr_setup(p.P, p.q, p.A, p.b, p.cones, st)
    s.solve()
    out = s.solution()
    s.free()
    return out


@pytest.mark.parametrize("bits", [64, 32])
def test_server_results_equal_alone(bits):
    st = clr.clr_default_settings(bits)
    probs = [_mpc(i) for i in range(40)]
    reqs = [clr.Request(p.P, p.q, p.A, p.b, p.cones) for p in probs]
    sv = clr.Server(device_bytes=2 << 30, max_cohort=16, max_active=3, settings=st)
    tickets = []
    for i, r in enumerate(reqs):
        tickets.append(sv.submit(r))
        if i % 10 == 9:
            time.sleep(0.01)  # later requests arrive while earlier cohorts run
    results = [sv.wait(t, 120.0) for t in tickets]
    stats = sv.stats()
    sv.close()
    assert stats["completed"] == len(probs) and stats["failed"] == 0, stats
    assert stats["cohorts"] >= 2 and stats["max_cohort_seen"] >= 2, stats
    for i, (p, res) in enumerate(zip(probs, results)):
        assert res is not None, i
        x, s, z, info = res
        xa, sa, za, ia = _alone(p, st)
        assert info["status_name"] == ia["status_name"] == "SOLVED", (i, info, ia)
        if info["fp64_from_iter"] < 0 and ia["fp64_from_iter"] < 0:
            assert info["iterations"] == ia["iterations"], (i, info, ia)
            for u, v in ((x, xa), (s, sa), (z, za)):
                np.testing.assert_array_equal(u, v, err_msg=str(i))
        else:
            # a low-precision cohort goes on in FP64 as a whole once one of its problems needs it
            f, fa = p.objective(x), p.objective(xa)
            assert abs(f - fa) <= 1e-6 * max(1.0, abs(fa)), (i, f, fa)
        assert info["solve_s"] > 0 and info["setup_s"] >= 0
        if i < 4:
            ref = oracle.solve(p.P, p.q, p.A, p.b, p.cones)
            f, fr = p.objective(x), p.objective(ref.x)
            assert abs(f - fr) <= 1e-6 * max(1.0, abs(fr)), (i, f, fr)


def test_server_reports_input_errors_per_ticket():
    sv = clr.Server(device_bytes=1 << 30, max_cohort=8, max_active=2)
    good = _mpc(3)
    bad = W.Problem("bad", sp.csc_matrix((2, 2)), np.ones(2), sp.csc_matrix(np.eye(2)), np.ones(2),
                    [(C.NONNEG, 3, 0.0)])  # cone dims do not add up to m
    tg = sv.submit(clr.Request(good.P, good.q, good.A, good.b, good.cones))
    with pytest.raises(clr.ClrError) as e:
        tb = sv.submit(clr.Request(bad.P, bad.q, bad.A, bad.b, bad.cones))
        sv.wait(tb, 60.0)
    assert e.value.code == -2  # CLR_E_DIM
    res = sv.wait(tg, 60.0)
    assert res is not None and res[3]["status_name"] == "SOLVED"
    sv.close()

"""Autotuner of the factorization's blocking parameters (clr_autotune): the
choice is a valid setting, is no slower than the defaults on the problems it
was timed on, comes back from the cache file, and solves to the same answer."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

clr = pytest.importorskip("paper_2412_19027_gb300.clr")
from paper_2412_19027_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_19027_gb300 import build
    build.build()
    clr._lib()


def test_autotune_mpc_cohort(tmp_path):
    rng = np.random.default_rng(9)
    probs = [W.mpc_qp(int(s), T=int(rng.integers(10, 31)), nx=int(rng.integers(4, 9)), nu=int(rng.integers(2, 5)))
             for s in range(16)]
    args = [(p.P, p.q, p.A, p.b, p.cones) for p in probs]
    cache = str(tmp_path / "tune.txt")
    st = clr.clr_default_settings(64)
    r = clr.clr_autotune(args, st, iters=3, cache_path=cache)
    assert r["from_cache"] == 0 and r["candidates"] > 0
    assert r["small_front_max"] in (0, 64, 96, 128, 160)
    assert r["amalgamation"] in (0, 1, 2) and r["big_front_schedule"] in (0, 1)
    assert 0 < r["ms_per_iter"] <= r["base_ms_per_iter"]
    r2 = clr.clr_autotune(args, st, iters=3, cache_path=cache)
    assert r2["from_cache"] == 1
    for k in ("small_front_max", "amalgamation", "big_front_schedule"):
        assert r2[k] == r[k]
    tuned = clr.clr_default_settings(64, small_front_max=r["small_front_max"], amalgamation=r["amalgamation"],
                                     big_front_schedule=r["big_front_schedule"])
    a = clr.clr_batch_setup(args, st)
    b = clr.clr_batch_setup(args, tuned)
    a.solve()
    b.solve()
    for i, p in enumerate(probs):
        xa, _, _, ia = a.solution_of(i)
        xb, _, _, ib = b.solution_of(i)
        assert ia["status_name"] == ib["status_name"] == "SOLVED"
        fa, fb = p.objective(xa), p.objective(xb)
        assert abs(fa - fb) <= 1e-7 * max(1.0, abs(fa))
    a.free()
    b.free()

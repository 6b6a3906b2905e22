"""GPU parity tests: the CUDA path (through the C ABI) against the FP64 oracle.

Step level: cone scaling H, step lengths, combined-step d_s, the sparse
LDL^T (same elimination order as the oracle's unpivoted LDL^T).  Solve
level: status, objective (1e-6 relative), residuals and iteration counts
(+-2) on seeded problems of every cone family, plus full-size workloads
against their planted optimum.

Tolerances: step-level FP64 results agree with the oracle to 1e-9 relative
(both evaluate the same closed forms in FP64; differences come from
summation order and from iterative inner solves such as the exp/pow shadow
Newton and the PSD Jacobi SVD).  Solve level follows the acceptance bar:
objective 1e-6 relative, residuals <= 1e-8 (the solver's own termination
test), iterations within 2.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import cones as C
from oracle.linsys import ldl_factor

import kkt_checks as KC

pytestmark = pytest.mark.gpu

clr = pytest.importorskip("paper_2412_19027_gb300.clr")
from paper_2412_19027_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_19027_gb300 import build
    build.build()
    clr._lib()


def _rand_cone_points(rng, cones):
    s, z = [], []
    for (t, d, a) in cones:
        if t == C.ZERO:
            s.append(np.zeros(d))
            z.append(rng.standard_normal(d))
        elif t == C.NONNEG:
            s.append(rng.uniform(0.1, 3.0, d))
            z.append(rng.uniform(0.1, 3.0, d))
        elif t == C.SOC:
            for v in (s, z):
                u = rng.standard_normal(d - 1)
                v.append(np.r_[np.linalg.norm(u) + rng.uniform(0.1, 2.0), u])
        elif t == C.PSD:
            k = C.psd_order(d)
            for v in (s, z):
                M = rng.standard_normal((k, k))
                v.append(C.svec(M @ M.T + 0.2 * np.eye(k)))
        elif t == C.EXP:
            y, x = rng.uniform(0.3, 2.0), rng.uniform(-2.0, 1.0)
            s.append(np.array([x, y, y * math.exp(x / y) + rng.uniform(0.2, 2.0)]))
            u, v_ = -rng.uniform(0.3, 2.0), rng.uniform(-2.0, 2.0)
            z.append(np.array([u, v_, -u * math.exp(v_ / u) / math.e + rng.uniform(0.2, 2.0)]))
        else:
            x, y = rng.uniform(0.3, 2.0, 2)
            s.append(np.array([x, y, rng.uniform(-0.9, 0.9) * x ** a * y ** (1 - a)]))
            u, v_ = rng.uniform(0.3, 2.0, 2)
            z.append(np.array([u, v_, rng.uniform(-0.9, 0.9) * (u / a) ** a * (v_ / (1 - a)) ** (1 - a)]))
    return np.concatenate(s), np.concatenate(z)


MIXED_CONES = ([(C.NONNEG, 7, 0.0), (C.SOC, 5, 0.0), (C.EXP, 3, 0.0), (C.ZERO, 2, 0.0), (C.POW, 3, 0.3),
                (C.SOC, 3, 0.0), (C.SOC, 40, 0.0), (C.POW, 3, 0.7), (C.NONNEG, 3, 0.0), (C.EXP, 3, 0.0)])
PSD_CONES = [(C.PSD, 55, 0.0)] * 3 + [(C.NONNEG, 4, 0.0)]


PSD32_CONES = [(C.PSD, 528, 0.0)] * 2 + [(C.NONNEG, 3, 0.0)]


PSD_MIXED_CONES = ([(C.PSD, 3, 0.0), (C.PSD, 55, 0.0), (C.NONNEG, 2, 0.0), (C.PSD, 6, 0.0), (C.PSD, 528, 0.0),
                    (C.PSD, 1, 0.0), (C.PSD, 21, 0.0)])


# PSD orders at the edges of the scaling kernel's classes (1-4, 5-8, 9-16 a lane per
# column, 17-32 a block per cone), interleaved, and cones of different orders sharing a
# warp (16 with 11, 9 with 12)
PSD_CLASS_CONES = ([(C.PSD, 136, 0.0), (C.PSD, 66, 0.0), (C.NONNEG, 2, 0.0), (C.PSD, 1, 0.0), (C.PSD, 10, 0.0),
                    (C.PSD, 15, 0.0), (C.PSD, 36, 0.0), (C.PSD, 45, 0.0), (C.PSD, 153, 0.0), (C.PSD, 28, 0.0)]
                   + [(C.PSD, 78, 0.0)] * 3)


@pytest.mark.parametrize("cones", [MIXED_CONES, PSD_CONES, [(C.PSD, 6, 0.0)] * 4, PSD32_CONES, PSD_MIXED_CONES,
                                   PSD_CLASS_CONES],
                         ids=["mixed", "psd10", "psd3", "psd32", "psd_mixed_orders", "psd_class_edges"])
def test_cone_scaling_matches_oracle(cones):
    rng = np.random.default_rng(0)
    s, z = _rand_cone_points(rng, cones)
    mu = 0.37
    H = clr.clr_cones_scaling(cones, s, z, mu)
    off = 0
    for (t, d, a), Hg in zip(cones, H):
        sl = slice(off, off + d)
        if t == C.ZERO:
            ref = np.zeros((d, d))
        elif t in (C.NONNEG, C.SOC, C.PSD):
            ref = C.nt_scaling(t, s[sl], z[sl])["H"]
        else:
            ref = C.bfgs_scaling(t, s[sl], z[sl], mu, a)
        np.testing.assert_allclose(Hg, ref, rtol=1e-9, atol=1e-11 * max(1.0, np.abs(ref).max()))
        off += d


@pytest.mark.parametrize("cones", [MIXED_CONES, PSD_CONES, PSD32_CONES, PSD_CLASS_CONES],
                         ids=["mixed", "psd10", "psd32", "psd_class_edges"])
def test_step_length_matches_oracle(cones):
    rng = np.random.default_rng(1)
    for trial in range(5):
        s, z = _rand_cone_points(rng, cones)
        ds, dz = rng.standard_normal(len(s)) * 2, rng.standard_normal(len(z)) * 2
        zero_rows = np.concatenate([np.full(d, t == C.ZERO) for (t, d, a) in cones])
        ds[zero_rows] = 0.0
        got = clr.clr_cones_step_length(cones, s, z, ds, dz, 1.0)
        # oracle: symmetric cones exact, then 0.8-backtracking on exp/pow from there
        amax, off = 1.0, 0
        for (t, d, a) in cones:
            sl = slice(off, off + d)
            if t in (C.NONNEG, C.SOC, C.PSD):
                amax = min(amax, C.step_length_symmetric(t, s[sl], ds[sl]), C.step_length_symmetric(t, z[sl], dz[sl]))
            off += d
        alpha = amax
        while True:
            ok, off = True, 0
            for (t, d, a) in cones:
                sl = slice(off, off + d)
                if t in (C.EXP, C.POW):
                    if not (C.in_int_primal(t, s[sl] + alpha * ds[sl], a) and C.in_int_dual(t, z[sl] + alpha * dz[sl], a)):
                        ok = False
                off += d
            if ok or alpha < 1e-10:
                break
            alpha *= 0.8
        assert got == pytest.approx(alpha, rel=1e-9)


@pytest.mark.parametrize("cones", [MIXED_CONES, PSD_CONES, PSD32_CONES, PSD_CLASS_CONES],
                         ids=["mixed", "psd10", "psd32", "psd_class_edges"])
def test_combined_ds_matches_oracle(cones):
    rng = np.random.default_rng(2)
    s, z = _rand_cone_points(rng, cones)
    dsa, dza = rng.standard_normal(len(s)), rng.standard_normal(len(z))
    smu = 0.05
    got = clr.clr_cones_combined_ds(cones, s, z, dsa, dza, smu)
    off = 0
    for (t, d, a) in cones:
        sl = slice(off, off + d)
        if t == C.ZERO:
            ref = np.zeros(d)
        elif t in (C.NONNEG, C.SOC, C.PSD):
            sc = C.nt_scaling(t, s[sl], z[sl])
            lam = C.lam_vec(t, sc["lam"], d)
            eta = C.jordan_prod(t, sc["WinvT"] @ dsa[sl], sc["W"] @ dza[sl])
            v = C.jordan_prod(t, lam, lam) + eta - smu * C.identity(t, d)
            ref = sc["W"].T @ C.jordan_div(t, sc["lam"], v)
        else:
            ref = s[sl] + smu * C.barrier_grad(t, z[sl], a) + C.third_order_correction(t, z[sl], dza[sl], dsa[sl], a)
        np.testing.assert_allclose(got[sl], ref, rtol=1e-9, atol=1e-10 * max(1.0, np.abs(ref).max()))
        off += d


def _quasidefinite(rng, n, m, density=0.3):
    P = sp.random(n, n, density=density, random_state=int(rng.integers(1 << 30)))
    P = (P @ P.T + 0.5 * sp.eye(n)).toarray()
    A = sp.random(m, n, density=density, random_state=int(rng.integers(1 << 30))).toarray()
    H = np.diag(rng.uniform(0.5, 2.0, m))
    return np.block([[P, A.T], [A, -H]])


@pytest.mark.parametrize("bits,n,m", [(64, 40, 70), (64, 150, 260), (32, 40, 70)])
def test_ldl_matches_oracle_in_same_order(bits, n, m):
    """Element-wise parity of the pivots D and the solution with the oracle's
    unpivoted LDL^T taken in the library's own elimination order."""
    rng = np.random.default_rng(n)
    K = _quasidefinite(rng, n, m)
    N = n + m
    signs = np.r_[np.ones(n), -np.ones(m)]
    rhs = rng.standard_normal(N)
    order = rng.permutation(N)
    x, D, hits = clr.clr_ldl_solve(K, signs, rhs, order=order, factor_bits=bits)
    assert hits == 0
    # the library postorders the elimination tree of `order`; pivots do not depend on
    # the order of independent columns, so compare with the oracle in the same `order`
    Kp = K[np.ix_(order, order)]
    L, Dref, _ = ldl_factor(Kp, signs[order], 1e-13, 2e-7)
    Dref_caller = np.empty(N)
    Dref_caller[order] = Dref
    tol = 1e-9 if bits == 64 else 2e-3
    np.testing.assert_allclose(D, Dref_caller, rtol=tol)
    xref = np.linalg.solve(K, rhs)
    np.testing.assert_allclose(x, xref, rtol=tol, atol=tol * np.abs(xref).max())


def test_ldl_amd_order_solves():
    rng = np.random.default_rng(5)
    K = _quasidefinite(rng, 120, 300, density=0.05)
    signs = np.r_[np.ones(120), -np.ones(300)]
    rhs = rng.standard_normal(420)
    x, D, hits = clr.clr_ldl_solve(K, signs, rhs)
    np.testing.assert_allclose(K @ x, rhs, atol=1e-9)
    assert np.all(D * signs > 0)


def _cone_membership(cones, s, z, tol):
    off = 0
    for (t, d, a) in cones:
        sv, zv = s[off:off + d], z[off:off + d]
        off += d
        if t == C.ZERO:
            assert np.abs(sv).max() <= tol
        elif t == C.NONNEG:
            assert sv.min() >= -tol and zv.min() >= -tol
        elif t == C.SOC:
            assert sv[0] - np.linalg.norm(sv[1:]) >= -tol and zv[0] - np.linalg.norm(zv[1:]) >= -tol
        elif t == C.PSD:
            assert np.linalg.eigvalsh(C.smat(sv)).min() >= -tol
            assert np.linalg.eigvalsh(C.smat(zv)).min() >= -tol
        else:  # exp / pow: the closed cones, checked on a point pushed inward by tol
            e = C.central_point(t, d, a)
            assert C.in_int_primal(t, sv + tol * e, a) and C.in_int_dual(t, zv + tol * e, a)


def _compare_solve(prob, factor_bits=64, iters_tol=2, obj_rtol=1e-6):
    """GPU solve against oracle.solve on the same problem:
    * status SOLVED on both sides, iterations within iters_tol, objective within
      obj_rtol relative;
    * the termination test of the paper at eps_feas = 1e-8 (primal and dual
      residuals, gap) recomputed on the host in FP64 from the returned x, s, z --
      for the GPU's answer and for the oracle's;
    * s in K and z in K* (to 1e-9 of the iterate's size) and s'z small;
    * entry by entry, where the optimum is unique and nondegenerate (zero and
      nonneg cones; kkt_checks.distance_bound): |x_gpu - x_oracle| and
      |z_gpu - z_oracle| within the sum of the two answers' a-posteriori
      distance bounds (x2 for rounding), and s through s = b - A x."""
    st = clr.clr_default_settings(factor_bits)
    solver = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
    solver.solve()
    x, s, z, info = solver.solution()
    solver.free()
    ref = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones)
    assert ref.status == 1
    assert info["status_name"] == "SOLVED", info
    f, fr = prob.objective(x), prob.objective(ref.x)
    assert abs(f - fr) <= obj_rtol * max(1.0, abs(fr)), (f, fr)
    assert abs(info["iterations"] - ref.iterations) <= iters_tol, (info["iterations"], ref.iterations)
    for (xx, ss, zz), who in (((x, s, z), "gpu"), ((ref.x, ref.s, ref.z), "oracle")):
        ok, d = KC.termination(prob.P, prob.q, prob.A, prob.b, xx, ss, zz, 1e-8 * (1 + 1e-6))
        assert ok, (who, d)
        size = max(1.0, np.abs(ss).max(), np.abs(zz).max())
        _cone_membership(prob.cones, ss, zz, 1e-9 * size)
        assert abs(ss @ zz) <= 1e-7 * d["scale_g"], (who, ss @ zz)
    bg = KC.distance_bound(prob.P, prob.q, prob.A, prob.b, prob.cones, x, s, z)
    bo = KC.distance_bound(prob.P, prob.q, prob.A, prob.b, prob.cones, ref.x, ref.s, ref.z)
    if bg is not None and bo is not None:
        slack = 1e-12 * (1.0 + np.abs(ref.x).max() + np.abs(ref.z).max())
        ex, ez = 2.0 * (bg[0] + bo[0]) + slack, 2.0 * (bg[1] + bo[1]) + slack
        assert np.all(np.abs(x - ref.x) <= ex), np.max(np.abs(x - ref.x) - ex)
        assert np.all(np.abs(z - ref.z) <= ez), np.max(np.abs(z - ref.z) - ez)
        As = sp.csc_matrix(prob.A)
        rs = np.abs(prob.A @ x + s - prob.b) + np.abs(prob.A @ ref.x + ref.s - prob.b)
        assert np.all(np.abs(s - ref.s) <= abs(As) @ ex + rs + slack)
    return info, ref


SOLVE_CASES = [
    ("qp_nonneg_n50_m100", lambda: W.nonneg_qp(0)),
    ("qp_nonneg_seed3", lambda: W.nonneg_qp(3)),
    ("mixed_small", lambda: W.mixed_cone(1, n=60, n_zero=10, n_nonneg=80, n_soc=12, n_exp=8, n_pow=8,
                                         nnz_per_col=4)),
    ("mixed_medium", lambda: W.mixed_cone(2, n=200, n_zero=50, n_nonneg=300, n_soc=50, n_exp=10, n_pow=10,
                                          nnz_per_col=6)),
    ("soc_only", lambda: W.mixed_cone(2, n=40, n_zero=5, n_nonneg=30, n_soc=15, soc_dim=4, n_exp=0, n_pow=0,
                                      nnz_per_col=5)),
    ("psd_small", lambda: W.psd_batch(0, n=60, n_psd=4, psd_k=4, n_nonneg=20, nnz_per_col=4)),
    ("psd10_small", lambda: W.psd_batch(1, n=200, n_psd=6, psd_k=10, n_nonneg=40, nnz_per_col=4)),
    ("banded_small", lambda: W.banded_lp(0, n=150, window=16)),
    ("mpc_small", lambda: W.mpc_qp(0, T=10, nx=4, nu=2)),
    ("unique_lp", lambda: W.unique_qp(0, rank=0)),
    ("unique_qp", lambda: W.unique_qp(1, rank=5)),
    ("unique_qp_large", lambda: W.unique_qp(2, n=120, n_eq=20, n_inactive=200, rank=10)),
]


@pytest.mark.parametrize("name,make", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
def test_solve_matches_oracle_fp64(name, make):
    _compare_solve(make(), 64)


FP32_CASES = SOLVE_CASES[:4] + SOLVE_CASES[7:8] + SOLVE_CASES[9:]


@pytest.mark.parametrize("name,make", FP32_CASES, ids=[c[0] for c in FP32_CASES])
def test_solve_matches_oracle_fp32_factor(name, make):
    """FP32 factorization + FP64 refinement reaches the FP64 oracle's answer."""
    _compare_solve(make(), 32, iters_tol=4)


@pytest.mark.parametrize("bits", [64, 32])
def test_ldl_big_fronts_with_update_rows(bits):
    """Natural order on [P A^T; A -H] with dense P (180) and dense H (160): the
    first front has 180 pivots and 160 update rows, the root 160 pivots; both
    exceed one CTA's shared memory and take the blocked big-front path."""
    rng = np.random.default_rng(11)
    n, m = 180, 160
    M = rng.standard_normal((n, n))
    P = M @ M.T / n + np.eye(n)
    B = rng.standard_normal((m, m))
    H = B @ B.T / m + np.eye(m)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.2)
    K = np.block([[P, A.T], [A, -H]])
    N = n + m
    signs = np.r_[np.ones(n), -np.ones(m)]
    rhs = rng.standard_normal(N)
    x, D, hits = clr.clr_ldl_solve(K, signs, rhs, order=np.arange(N), factor_bits=bits)
    assert hits == 0
    L, Dref, _ = ldl_factor(K, signs, 1e-13, 2e-7)
    tol = 1e-10 if bits == 64 else 1e-4
    np.testing.assert_allclose(D, Dref, rtol=tol)
    xref = np.linalg.solve(K, rhs)
    np.testing.assert_allclose(x, xref, rtol=tol, atol=tol * np.abs(xref).max())


@pytest.mark.parametrize("n,m", [(180, 160), (300, 260), (700, 500)])
def test_ldl_big_fronts_tensor_core_updates(n, m):
    """FP32 dataflow factorization whose trailing and E updates run on the
    tensor cores (big_front_schedule 3: TF32 high and low parts, FP32
    accumulation in tensor memory, operand tiles staged by TMA) against the same
    schedule with CUDA-core products (2) and against the oracle's LDL^T: fronts
    of 3 to 11 panels of 64 columns, ragged last pivot and update blocks.
    Schedule 3 puts every level on the tensor cores (1 chooses per level)."""
    rng = np.random.default_rng(n + m)
    M = rng.standard_normal((n, n))
    P = M @ M.T / n + np.eye(n)
    B = rng.standard_normal((m, m))
    H = B @ B.T / m + np.eye(m)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.2)
    K = np.block([[P, A.T], [A, -H]])
    N = n + m
    signs = np.r_[np.ones(n), -np.ones(m)]
    rhs = rng.standard_normal(N)
    order = np.arange(N)
    x1, D1, h1 = clr.clr_ldl_solve(K, signs, rhs, order=order, factor_bits=32, big_front_schedule=3)
    x2, D2, h2 = clr.clr_ldl_solve(K, signs, rhs, order=order, factor_bits=32, big_front_schedule=2)
    assert h1 == 0 and h2 == 0
    L, Dref, _ = ldl_factor(K, signs, 1e-13, 2e-7)
    np.testing.assert_allclose(D1, Dref, rtol=1e-4)
    np.testing.assert_allclose(D2, Dref, rtol=1e-4)
    # both are FP32 factors of the same matrix in the same order: their pivot
    # errors are of the same size (the split products are exact to ~2^-21)
    e1 = np.max(np.abs(D1 - Dref) / np.abs(Dref))
    e2 = np.max(np.abs(D2 - Dref) / np.abs(Dref))
    assert e1 <= 8 * e2 + 1e-6, (e1, e2)
    xref = np.linalg.solve(K, rhs)
    for x in (x1, x2):
        np.testing.assert_allclose(x, xref, rtol=1e-4, atol=1e-4 * np.abs(xref).max())


def test_ldl_big_fronts_bf16_products_refine_to_fp64_accuracy():
    """factor_bits 16: the big-front updates run on the tensor cores with BF16
    operands and FP32 accumulation.  The factor is accurate to a few 1e-3, so the
    pivots match the FP64 factor to 5e-2 and FP64 refinement with it reaches the
    FP64 solution (what the IPM does with it)."""
    rng = np.random.default_rng(12)
    n, m = 300, 260  # fronts of 300 pivots with 260 update rows and a 260-pivot root: several 128-row tiles
    M = rng.standard_normal((n, n))
    P = M @ M.T / n + np.eye(n)
    B = rng.standard_normal((m, m))
    H = B @ B.T / m + np.eye(m)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.2)
    K = np.block([[P, A.T], [A, -H]])
    N = n + m
    signs = np.r_[np.ones(n), -np.ones(m)]
    rhs = rng.standard_normal(N)
    order = np.arange(N)
    x, D, hits = clr.clr_ldl_solve(K, signs, rhs, order=order, factor_bits=16, dyn_reg_eps=1e-6, dyn_reg_delta=1e-4)
    assert hits == 0
    L, Dref, _ = ldl_factor(K, signs, 1e-13, 2e-7)
    np.testing.assert_allclose(D, Dref, rtol=5e-2)
    xref = np.linalg.solve(K, rhs)
    assert np.abs(x - xref).max() < 0.1 * np.abs(xref).max()
    for _ in range(12):  # refinement with the 16-bit-product factor
        dx, _, _ = clr.clr_ldl_solve(K, signs, rhs - K @ x, order=order, factor_bits=16, dyn_reg_eps=1e-6,
                                     dyn_reg_delta=1e-4)
        x = x + dx
    np.testing.assert_allclose(x, xref, rtol=1e-9, atol=1e-9 * np.abs(xref).max())


def test_solve_with_bf16_products_mixed_cone_full_size():
    """The full mixed-cone QP (root front of ~2050 rows, on the tensor cores)
    with 16-bit products and FP64 refinement reaches the planted optimum."""
    prob = W.mixed_cone(0)
    st = clr.clr_default_settings(16, ir_stop_ratio=5.0)
    s = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
    s.solve()
    x, sl, z, info = s.solution()
    s.free()
    assert info["status_name"] == "SOLVED", info
    f_star = prob.objective(prob.x_star)
    assert abs(prob.objective(x) - f_star) <= 1e-6 * max(1.0, abs(f_star))


@pytest.mark.parametrize("family,count", [("nonneg", 5000), ("soc", 700), ("psd", 40)])
def test_cone_stress_inputs_and_timing(family, count):
    """The cone-roofline inputs (small counts of the bench's stress shapes):
    scalings of a sample match the oracle, and the timing entry point runs
    the same kernels and reports the rows and packed H entries it covers."""
    cones, s, z, ds, dz = W.cone_stress(3, family, count)
    pick = [0, count // 2, count - 1] if family != "nonneg" else [0]
    offs = np.cumsum([0] + [d for (_, d, _) in cones])
    sub = [cones[i] for i in pick]
    ss = np.concatenate([s[offs[i]:offs[i + 1]] for i in pick])
    zz = np.concatenate([z[offs[i]:offs[i + 1]] for i in pick])
    H = clr.clr_cones_scaling(sub, ss, zz, 1.0)
    off = 0
    for (t, d, a), Hg in zip(sub, H):
        ref = C.nt_scaling(t, ss[off:off + d], zz[off:off + d])["H"]
        np.testing.assert_allclose(Hg, ref, rtol=1e-9, atol=1e-11 * max(1.0, np.abs(ref).max()))
        off += d
    t = clr.clr_cones_time(cones, s, z, ds, dz, 1.0, reps=3)
    assert t["rows"] == len(s)
    dim = cones[0][1]
    packed = {"nonneg": len(s), "soc": count * dim * (dim + 1) // 2, "psd": count * dim * (dim + 1) // 2}[family]
    assert t["kkt_values"] == packed
    for k in ("scaling_ms", "step_ms", "combined_ds_ms"):
        assert 0.0 < t[k] < 1e3, t


@pytest.mark.parametrize("soc_dim,n_soc,n_exp,bits", [(100, 3, 0, 64), (1000, 1, 0, 64), (100, 3, 4, 64),
                                                     (100, 3, 0, 32)])
def test_large_soc_sparse_form_matches_oracle(soc_dim, n_soc, n_exp, bits):
    """SOCs of 100 and 1000 rows (Sec. 3.3 names cones of thousands of rows) in the sparse KKT
    form (H = eta^2 (I + u u' - v v'), two auxiliary KKT rows per cone) against the oracle, whose
    KKT matrix holds each cone's
    dense H: status, objective, iterations and the host-recomputed termination test; with
    exp/pow cones too (the unit initial point) and with the FP32 factor."""
    prob = W.mixed_cone(4 + soc_dim, n=200, n_zero=20, n_nonneg=150, n_soc=n_soc, soc_dim=soc_dim, n_exp=n_exp,
                        n_pow=n_exp, nnz_per_col=6)
    _compare_solve(prob, bits, iters_tol=2 if bits == 64 else 4)


def test_large_soc_sparse_and_dense_forms_agree():
    """The same problem with its SOCs of 60 rows in the sparse KKT form (soc_expand_dim 33,
    the default) and as dense H blocks (0): two more KKT rows per cone, the same answer."""
    prob = W.mixed_cone(9, n=150, n_zero=10, n_nonneg=100, n_soc=2, soc_dim=60, n_exp=3, n_pow=3, nnz_per_col=6)
    out = {}
    for dim in (33, 0):
        st = clr.clr_default_settings(64, soc_expand_dim=dim)
        sv = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
        sv.solve()
        x, sl, z, info = sv.solution()
        out[dim] = (x, sl, z, info, sv.symbolic_stats())
        sv.free()
    (xe, se, ze, ie, ste), (xd, sd, zd, idn, std_) = out[33], out[0]
    assert ste["kkt_dim"] == std_["kkt_dim"] + 4 and ste["m"] == std_["m"] + 4
    assert ie["status_name"] == idn["status_name"] == "SOLVED", (ie, idn)
    assert abs(ie["iterations"] - idn["iterations"]) <= 1
    fe, fd = prob.objective(xe), prob.objective(xd)
    assert abs(fe - fd) <= 1e-7 * max(1.0, abs(fd)), (fe, fd)
    scale = max(1.0, np.abs(xd).max())
    np.testing.assert_allclose(xe, xd, atol=1e-6 * scale)  # P positive definite: x is unique
    np.testing.assert_allclose(se, sd, atol=1e-6 * max(1.0, np.abs(sd).max()))
    assert len(ze) == len(zd) == prob.A.shape[0]


def test_psd_mixed_orders_solve_matches_oracle():
    """PSD cones of orders 2 .. 16 in one problem (the future direction of Sec. 6):
    status, objective and iterations as the oracle's."""
    info, ref = _compare_solve(W.psd_mixed(0), 64)
    assert ref.status_name == info["status_name"] == "SOLVED"

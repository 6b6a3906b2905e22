"""Pins for the oracle's KKT solver and IPM (no GPU).

What fixes the expected values: planted optima (problems generated from a
chosen complementary (x*, s*, z*)), a hand-solved LP, vertex enumeration and
scipy's LP solver on tiny LPs, the full 4x4 Newton system solved densely,
exact algebraic identities (gap identity, linear-row contraction),
invariance under equilibration / cone order, the PSD(1) = nonneg special
case, the paper's printed constants, and hand-solved cases of the
equilibration (Ruiz passes, clamps, cone-block rule) and of the initial point.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import oracle
from oracle import cones as C
from oracle import ipm
from oracle.linsys import KKTSolver, ldl_factor
from paper_2412_19027_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _solve(prob, **kw):
    return oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones, settings=kw or None, record=True)


def _kkt_residuals(prob, r):
    Pf = (prob.P + sp.triu(prob.P, 1).T).toarray()
    A = prob.A.toarray()
    rp = A @ r.x + r.s - prob.b
    rd = Pf @ r.x + A.T @ r.z + prob.q
    return np.max(np.abs(rp)), np.max(np.abs(rd))


# ------------------------------------------------------------ constants
def test_paper_constants():
    g = _load("paper_constants.json")
    st = oracle.default_settings(64)
    lo = oracle.default_settings(32)
    assert st["backtrack"] == g["backtrack_ratio"]["value"]
    assert st["step_fraction"] == g["step_fraction"]["value"]
    assert st["nbhd_beta"] == g["neighbourhood_beta"]["value"]
    assert st["ir_max_steps"] == g["ir_max_steps"]["value"]
    assert st["ir_abstol"] == g["ir_abstol"]["value"] and st["ir_reltol"] == g["ir_reltol"]["value"]
    assert st["static_reg"] == g["static_reg_full"]["value"]
    assert lo["static_reg"] == pytest.approx(g["static_reg_mixed"]["value"], rel=g["static_reg_mixed"]["rtol"])
    assert lo["static_reg_dyn"] == pytest.approx(g["static_reg_dyn"]["value"], rel=1e-12)
    assert st["static_reg_dyn"] == pytest.approx(g["static_reg_dyn"]["value"], rel=1e-12)


# ------------------------------------------------------------ dense LDL^T
def _random_quasidefinite(rng, n, m):
    M = rng.standard_normal((n, n))
    P = M @ M.T + 0.1 * np.eye(n)
    B = rng.standard_normal((m, m))
    H = B @ B.T + 0.1 * np.eye(m)
    A = rng.standard_normal((m, n))
    return np.block([[P, A.T], [A, -H]])


def test_ldl_reconstructs_quasidefinite():
    rng = np.random.default_rng(0)
    K = _random_quasidefinite(rng, 12, 9)
    signs = np.r_[np.ones(12), -np.ones(9)]
    L, D, hits = ldl_factor(K, signs, 1e-13, 2e-7)
    assert hits == 0
    assert np.all(D * signs > 0)  # quasi-definite => pivot signs are fixed
    err = np.linalg.norm(L @ np.diag(D) @ L.T - K) / np.linalg.norm(K)
    assert err < 1e-13


def test_ldl_dynamic_regularisation_on_wrong_sign_pivot():
    K = np.array([[-1.0, 0.0], [0.0, -1.0]])
    L, D, hits = ldl_factor(K, np.array([1.0, -1.0]), 1e-13, 2e-7)
    assert hits == 1 and D[0] == 2e-7 and D[1] == -1.0


def test_ir_reaches_tolerance():
    rng = np.random.default_rng(1)
    K = _random_quasidefinite(rng, 20, 15)
    st = oracle.default_settings(64)
    st["static_reg"] = 1e-3  # heavy regularisation: only refinement can fix it
    ks = KKTSolver(K, 20, st)
    b = rng.standard_normal(35)
    x = ks.solve(b)
    assert np.max(np.abs(b - K @ x)) <= 1e-12 + 1e-12 * np.max(np.abs(b))
    assert ks.ir_steps >= 1


# ------------------------------------------------------ reduced vs full Newton
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_reduced_direction_matches_full_newton_system(seed):
    """Eq. linsys_4x4 solved densely by Gaussian elimination with partial
    pivoting vs the oracle's path through Eq. linsys_2x2 and Eq. step-direction."""
    rng = np.random.default_rng(seed)
    n, m = 6, 9
    M = rng.standard_normal((n, 3))
    P = M @ M.T
    A = rng.standard_normal((m, n))
    q, b = rng.standard_normal(n), rng.standard_normal(m)
    B = rng.standard_normal((m, m))
    H = B @ B.T + 0.5 * np.eye(m)
    x = rng.standard_normal(n)
    tau, kappa = rng.uniform(0.5, 2), rng.uniform(0.5, 2)
    d = (rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(), rng.standard_normal(m),
         rng.standard_normal())
    K = np.block([[P, A.T], [A, -H]])
    ks = KKTSolver(K, n, oracle.default_settings(64))
    sol2 = ks.solve(np.r_[-q, b])
    got = ipm.reduced_direction(ks, P, q, A, b, H, x, tau, kappa, sol2[:n], sol2[n:], d)

    xi = x / tau
    N = n + m + 1 + m + 1
    Mfull = np.zeros((N, N))
    rhs = np.zeros(N)
    ix, iz, it, is_, ik = slice(0, n), slice(n, n + m), n + m, slice(n + m + 1, n + 2 * m + 1), N - 1
    # row 1: -(P dx + A^T dz + q dtau) = -d_x
    Mfull[ix, ix] = -P
    Mfull[ix, iz] = -A.T
    Mfull[ix, it] = -q
    rhs[ix] = -d[0]
    # row 2: ds - (-A dx + b dtau) = -d_z
    Mfull[iz, ix] = A
    Mfull[iz, it] = -b
    Mfull[iz, is_] = np.eye(m)
    rhs[iz] = -d[1]
    # row 3: dkappa - (-(q + 2 P xi)^T dx - b^T dz + xi^T P xi dtau) = -d_tau
    Mfull[it, ix] = q + 2 * P @ xi
    Mfull[it, iz] = b
    Mfull[it, it] = -(xi @ P @ xi)
    Mfull[it, ik] = 1.0
    rhs[it] = -d[2]
    # H dz + ds = -d_s ; kappa dtau + tau dkappa = -d_kappa
    Mfull[is_, iz] = H
    Mfull[is_, is_] = np.eye(m)
    rhs[is_] = -d[3]
    Mfull[ik, it] = kappa
    Mfull[ik, ik] = tau
    rhs[ik] = -d[4]
    u = np.linalg.solve(Mfull, rhs)
    ref = (u[ix], u[iz], u[it], u[is_], u[ik])
    for g_, r_ in zip(got, ref):
        np.testing.assert_allclose(g_, r_, rtol=1e-9, atol=1e-10)


# ------------------------------------------------------------ planted optima
def test_hand_solved_lp():
    g = _load("lp_2var_handsolved.json")
    A = np.array(g["A"])
    r = oracle.solve(np.zeros((2, 2)), np.array(g["q"]), A, np.array(g["b"]), [(C.NONNEG, 4, 0.0)])
    assert r.status_name == "SOLVED"
    np.testing.assert_allclose(r.x, g["x"], atol=1e-7)
    np.testing.assert_allclose(r.z, g["z"], atol=1e-7)
    np.testing.assert_allclose(r.s, g["s"], atol=1e-7)
    assert r.obj_primal == pytest.approx(g["objective"], rel=1e-8)


PLANTED = [
    ("qp_nonneg", lambda: W.nonneg_qp(0)),
    ("qp_nonneg_seed3", lambda: W.nonneg_qp(3)),
    ("mixed_small", lambda: W.mixed_cone(1, n=60, n_zero=10, n_nonneg=80, n_soc=12, n_exp=8, n_pow=8,
                                         nnz_per_col=4)),
    ("soc_only", lambda: W.mixed_cone(2, n=40, n_zero=5, n_nonneg=30, n_soc=15, soc_dim=4, n_exp=0,
                                      n_pow=0, nnz_per_col=5)),
    ("psd_small", lambda: W.psd_batch(0, n=60, n_psd=4, psd_k=4, n_nonneg=20, nnz_per_col=4)),
    ("banded_small", lambda: W.banded_lp(0, n=150, window=16)),
]


@pytest.mark.parametrize("name,make", PLANTED, ids=[p[0] for p in PLANTED])
def test_planted_optimum(name, make):
    prob = make()
    r = _solve(prob)
    assert r.status_name == "SOLVED", (name, r.status_name)
    f_star = prob.objective(prob.x_star)
    assert prob.objective(r.x) == pytest.approx(f_star, rel=1e-6, abs=1e-6)
    rp, rd = _kkt_residuals(prob, r)
    assert rp < 1e-6 and rd < 1e-6
    # the returned s and z lie in their cones (Sec. 2.1 definitions), up to 1e-7
    off = 0
    for (t, d, a) in prob.cones:
        sl = slice(off, off + d)
        if t == C.NONNEG:
            assert r.s[sl].min() > -1e-7 and r.z[sl].min() > -1e-7
        elif t == C.SOC:
            for v in (r.s[sl], r.z[sl]):
                assert v[0] - np.linalg.norm(v[1:]) > -1e-7
        elif t == C.PSD:
            for v in (r.s[sl], r.z[sl]):
                assert np.linalg.eigvalsh(C.smat(v)).min() > -1e-7
        off += d
    # sanity range of iteration counts printed by the paper (8-24 on its QPs)
    assert 5 <= r.iterations <= 40


def test_gap_identity_and_linear_row_contraction():
    """g_p - g_d = s'z + r_p'z + r_d'x exactly (Eq. residuals-objectives), and
    rows 1-2 of G are linear so ||G_{1,2}|| contracts by 1 - 0.99 alpha_c (1 - sigma)
    per step (Eq. root_finding_G with Eq. linsys_4x4 and Eq. ds-correction-step)."""
    prob = W.mixed_cone(4, n=50, n_zero=8, n_nonneg=60, n_soc=10, n_exp=6, n_pow=6, nnz_per_col=4)
    r = _solve(prob)
    assert r.status_name == "SOLVED"
    Pf = (prob.P + sp.triu(prob.P, 1).T).toarray()
    A = prob.A.toarray()
    x, s, z = r.x, r.s, r.z
    rp = -A @ x - s + prob.b
    rd = Pf @ x + A.T @ z + prob.q
    gp = 0.5 * x @ Pf @ x + prob.q @ x
    gd = -0.5 * x @ Pf @ x - prob.b @ z
    assert gp - gd == pytest.approx(s @ z + rp @ z + rd @ x, rel=1e-9, abs=1e-10)
    h = r.history
    for k in range(len(h) - 1):
        factor = 1 - 0.99 * h[k]["alpha_c"] * (1 - h[k]["sigma"])
        for key in ("G1", "G2"):
            if h[k][key] > 1e-6:
                assert h[k + 1][key] == pytest.approx(factor * h[k][key], rel=1e-5)


# ------------------------------------------------------------ tiny LPs
def _vertex_enumeration(q, A, b):
    """min q'x s.t. A x <= b by enumerating all n-subsets of active rows."""
    m, n = A.shape
    best = None
    for rows in itertools.combinations(range(m), n):
        As = A[list(rows)]
        if abs(np.linalg.det(As)) < 1e-10:
            continue
        x = np.linalg.solve(As, b[list(rows)])
        if np.all(A @ x <= b + 1e-9):
            f = q @ x
            if best is None or f < best[0]:
                best = (f, x)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_tiny_lp_vs_vertex_enumeration_and_linprog(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 5))
    m = int(rng.integers(n + 1, 9))
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m) + (1.0 if seed % 3 else -0.5)
    q = rng.standard_normal(n)
    lp = linprog(q, A_ub=A, b_ub=b, bounds=[(None, None)] * n, method="highs")
    r = oracle.solve(np.zeros((n, n)), q, A, b, [(C.NONNEG, m, 0.0)])
    if lp.status == 0:
        best = _vertex_enumeration(q, A, b)
        assert r.status_name == "SOLVED"
        assert r.obj_primal == pytest.approx(lp.fun, rel=1e-6, abs=1e-6)
        if best is not None:
            assert best[0] == pytest.approx(lp.fun, rel=1e-7, abs=1e-7)
    elif lp.status == 2:
        assert r.status_name == "PRIMAL_INFEASIBLE"
        z = r.z
        assert np.all(z >= -1e-9) and b @ z == pytest.approx(-1.0)
        assert np.max(np.abs(A.T @ z)) < 1e-6
    elif lp.status == 3:
        assert r.status_name == "DUAL_INFEASIBLE"
        x = r.x
        assert q @ x == pytest.approx(-1.0) and np.all(-A @ x >= -1e-6)


def test_infeasible_and_unbounded_certificates():
    # x >= 1 and x <= 0: primal infeasible
    r = oracle.solve(np.zeros((1, 1)), np.array([1.0]), np.array([[-1.0], [1.0]]), np.array([-1.0, 0.0]),
                     [(C.NONNEG, 2, 0.0)])
    assert r.status_name == "PRIMAL_INFEASIBLE"
    assert np.all(r.z >= 0) and r.z @ np.array([-1.0, 0.0]) == pytest.approx(-1.0)
    # min -x s.t. x >= 0: unbounded
    r = oracle.solve(np.zeros((1, 1)), np.array([-1.0]), np.array([[-1.0]]), np.array([0.0]), [(C.NONNEG, 1, 0.0)])
    assert r.status_name == "DUAL_INFEASIBLE"
    assert r.x[0] > 0 and -r.x[0] == pytest.approx(-1.0)


# ------------------------------------------------------------ invariances
def test_equilibration_does_not_change_the_optimum():
    prob = W.mixed_cone(5, n=40, n_zero=6, n_nonneg=40, n_soc=8, n_exp=5, n_pow=5, nnz_per_col=4)
    r1 = _solve(prob)
    r0 = _solve(prob, equilibrate=False)
    assert r1.status_name == r0.status_name == "SOLVED"
    np.testing.assert_allclose(r1.x, r0.x, atol=2e-5)
    assert r1.obj_primal == pytest.approx(r0.obj_primal, rel=1e-7)


def test_cone_order_does_not_change_the_solution():
    prob = W.mixed_cone(6, n=30, n_zero=4, n_nonneg=20, n_soc=6, n_exp=4, n_pow=4, nnz_per_col=4)
    # reverse the cone blocks and the rows with them
    offs = np.cumsum([0] + [d for (_, d, _) in prob.cones])
    order = list(range(len(prob.cones)))[::-1]
    rows = np.concatenate([np.arange(offs[i], offs[i + 1]) for i in order])
    cones2 = [prob.cones[i] for i in order]
    r1 = _solve(prob)
    r2 = oracle.solve(prob.P, prob.q, prob.A.toarray()[rows], prob.b[rows], cones2)
    np.testing.assert_allclose(r2.x, r1.x, atol=1e-9)
    np.testing.assert_allclose(r2.z, r1.z[rows], atol=1e-9)


def test_psd_order_one_equals_nonneg():
    """A PSD cone of order 1 is a nonnegative entry: its NT scaling, lambda,
    step length and corrector equal the nonneg ones entry by entry, and a whole
    problem posed with PSD(1) cones has the same optimum.  (The initial shift
    differs: the merged nonneg cone shifts by one global amount, each PSD(1)
    cone by its own, so the iterates are not identical.)"""
    rng = np.random.default_rng(17)
    for _ in range(20):
        s, z = rng.uniform(0.05, 3.0, 1), rng.uniform(0.05, 3.0, 1)
        ds, dz = rng.standard_normal(1), rng.standard_normal(1)
        a = C.nt_scaling(C.NONNEG, s, z)
        b_ = C.nt_scaling(C.PSD, s, z)
        np.testing.assert_allclose(b_["H"], a["H"], rtol=1e-13)
        np.testing.assert_allclose(b_["lam"], a["lam"], rtol=1e-13)
        assert C.step_length_symmetric(C.PSD, s, ds) == pytest.approx(C.step_length_symmetric(C.NONNEG, s, ds), rel=1e-13)
        for sc, t in ((a, C.NONNEG), (b_, C.PSD)):
            lam = C.lam_vec(t, sc["lam"], 1)
            eta = C.jordan_prod(t, sc["WinvT"] @ ds, sc["W"] @ dz)
            v = C.jordan_prod(t, lam, lam) + eta - 0.3 * C.identity(t, 1)
            sc["ds"] = sc["W"].T @ C.jordan_div(t, sc["lam"], v)
        np.testing.assert_allclose(b_["ds"], a["ds"], rtol=1e-12)
    prob = W.nonneg_qp(7, n=20, m=40, density=0.2, rank=3)
    r_nn = _solve(prob)
    r_psd = oracle.solve(prob.P, prob.q, prob.A, prob.b, [(C.PSD, 1, 0.0)] * 40, record=True)
    assert r_nn.status_name == r_psd.status_name == "SOLVED"
    assert prob.objective(r_psd.x) == pytest.approx(prob.objective(r_nn.x), rel=1e-7)
    assert abs(r_nn.iterations - r_psd.iterations) <= 2


def test_validation_rejects_bad_input():
    with pytest.raises(ipm.ProblemError):
        oracle.solve(np.array([[1.0, 0], [1.0, 1.0]]), np.zeros(2), np.eye(2), np.ones(2), [(C.NONNEG, 2, 0.0)])
    with pytest.raises(ipm.ProblemError):
        oracle.solve(np.eye(2), np.array([np.nan, 0]), np.eye(2), np.ones(2), [(C.NONNEG, 2, 0.0)])
    with pytest.raises(ipm.ProblemError):
        oracle.solve(np.eye(2), np.zeros(2), np.eye(2), np.ones(2), [(C.NONNEG, 3, 0.0)])
    with pytest.raises(ipm.ProblemError):
        oracle.solve(np.eye(1), np.zeros(1), np.ones((3, 1)), np.ones(3), [(C.POW, 3, 1.5)])


def test_psd_cones_of_mixed_orders_reach_the_planted_optimum():
    """PSD cones of orders 2 .. 16 in one problem (interleaved with each other):
    the oracle reaches the planted optimum (every PSD cone handled by its own order)."""
    prob = W.psd_mixed(0)
    r = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones)
    assert r["status_name"] == "SOLVED"
    f, fs = prob.objective(r["x"]), prob.objective(prob.x_star)
    assert abs(f - fs) <= 1e-6 * max(1.0, abs(fs))


@pytest.mark.parametrize("seed,rank", [(0, 0), (1, 5), (2, 3)])
def test_unique_qp_solution_within_posterior_bound(seed, rank):
    """On a QP with a unique nondegenerate optimum (planted), the oracle's answer
    passes the host-recomputed termination test at 1e-8, and its distance to the
    planted (x*, z*) is within the first-order a-posteriori bound that the GPU
    parity tests use to compare two answers entry by entry."""
    from paper_2412_19027_gb300 import workloads as W
    import kkt_checks as KC
    p = W.unique_qp(seed, rank=rank)
    r = oracle.solve(p.P, p.q, p.A, p.b, p.cones)
    assert r.status_name == "SOLVED"
    ok, d = KC.termination(p.P, p.q, p.A, p.b, r.x, r.s, r.z)
    assert ok, d
    bnd = KC.distance_bound(p.P, p.q, p.A, p.b, p.cones, r.x, r.s, r.z)
    assert bnd is not None
    e_x, e_z = bnd
    slack = 1e-12 * (1.0 + np.abs(p.x_star).max())
    assert np.all(np.abs(r.x - p.x_star) <= 2.0 * e_x + slack), np.max(np.abs(r.x - p.x_star) - e_x)
    assert np.all(np.abs(r.z - p.z_star) <= 2.0 * e_z + slack)
    # the bound is informative: far below the size of the solution
    assert e_x.max() < 1e-5 * max(1.0, np.abs(p.x_star).max())


# ---------------------------------------------------------------- equilibration and initial point
# Both are readings of silent passages (Alg. 1 steps 1-2 name them without a method);
# these pins hold the oracle to the reading as stated, on cases solved by hand.

def test_ruiz_equilibration_hand_case():
    """A = diag(4, 1/4), P = 0, q = (1, 1): the first pass scales by 1/sqrt of the
    column and row infinity norms, D = E = (1/2, 2), after which E A D = I and every
    later pass keeps it; the cost scale is 1 / max(mean col norm of P^, ||D q||) = 1/2."""
    st = ipm.default_settings()
    A = np.diag([4.0, 0.25])
    D, E, c = ipm.equilibrate(np.zeros((2, 2)), A, np.ones(2), [(C.NONNEG, 2, 0.0, 0)], st)
    np.testing.assert_allclose(D, [0.5, 2.0], rtol=1e-15)
    np.testing.assert_allclose(E, [0.5, 2.0], rtol=1e-15)
    assert c == pytest.approx(0.5, rel=1e-15)


def test_ruiz_equilibration_tiny_norm_and_clamp():
    """A = [1e-12, 1e12] (one row), P = 0: a column of norm < 1e-8 is left alone;
    1/sqrt(1e12) = 1e-6 is clamped to scale_min = 1e-4 for the other column and the
    row, and the accumulated factors stay clamped at 1e-4 in every later pass;
    ||D q|| = 1 gives c = 1."""
    st = ipm.default_settings()
    A = np.array([[1e-12, 1e12]])
    D, E, c = ipm.equilibrate(np.zeros((2, 2)), A, np.ones(2), [(C.NONNEG, 1, 0.0, 0)], st)
    np.testing.assert_allclose(D, [1.0, 1e-4], rtol=1e-15)
    np.testing.assert_allclose(E, [1e-4], rtol=1e-15)
    assert c == 1.0


def test_ruiz_equilibration_cone_rows_share_one_factor():
    """A = diag(4, 1, 1/4) as one SOC(3): after one pass D = (1/2, 1, 2) (the columns'
    own norms) while all three rows take the factor of the cone's largest row norm,
    E = (1/2, 1/2, 1/2), so the scaled rows still form a second-order cone; as three
    nonnegative rows they would take (1/2, 1, 2)."""
    st = dict(ipm.default_settings(), ruiz_passes=1)
    A = np.diag([4.0, 1.0, 0.25])
    D, E, _ = ipm.equilibrate(np.zeros((3, 3)), A, np.zeros(3), [(C.SOC, 3, 0.0, 0)], st)
    np.testing.assert_allclose(D, [0.5, 1.0, 2.0], rtol=1e-15)
    np.testing.assert_allclose(E, [0.5, 0.5, 0.5], rtol=1e-15)
    _, E2, _ = ipm.equilibrate(np.zeros((3, 3)), A, np.zeros(3), [(C.NONNEG, 3, 0.0, 0)], st)
    np.testing.assert_allclose(E2, [0.5, 1.0, 2.0], rtol=1e-15)


def test_initial_point_hand_solved_lp():
    """min x s.t. x <= 1, -x <= 1 (equilibration off).  With H = I the two solves
    give, by hand: [0; b] -> x = 0, z = (-1, -1), s = -z = (1, 1); [-q; 0] -> z =
    (-1/2, 1/2).  The shift into the cone leaves s (least entry 1) and moves z by
    1 - (-1/2): z = (1, 2).  max_iter = 0 returns that point."""
    r = oracle.solve(np.zeros((1, 1)), np.array([1.0]), np.array([[1.0], [-1.0]]), np.array([1.0, 1.0]),
                     [(C.NONNEG, 2, 0.0)], settings=dict(max_iter=0, equilibrate=0))
    np.testing.assert_allclose(r.x, [0.0], atol=1e-10)
    np.testing.assert_allclose(r.s, [1.0, 1.0], rtol=1e-10)
    np.testing.assert_allclose(r.z, [1.0, 2.0], rtol=1e-10)


def test_initial_point_hand_solved_soc():
    """min x s.t. (2 - x, 3, 4) in SOC(3), i.e. A = (1, 0, 0)', b = (2, 3, 4), q = 1
    (equilibration off).  [0; b] -> x = 2, s = (0, 3, 4), whose least Jordan
    eigenvalue is 0 - 5 = -5, so s + 6 e = (6, 3, 4); [-q; 0] -> z = (-1, 0, 0),
    shifted by 1 - (-1) = 2: z = (1, 0, 0)."""
    r = oracle.solve(np.zeros((1, 1)), np.array([1.0]), np.array([[1.0], [0.0], [0.0]]),
                     np.array([2.0, 3.0, 4.0]), [(C.SOC, 3, 0.0)], settings=dict(max_iter=0, equilibrate=0))
    np.testing.assert_allclose(r.x, [2.0], rtol=1e-10)
    np.testing.assert_allclose(r.s, [6.0, 3.0, 4.0], rtol=1e-10)
    np.testing.assert_allclose(r.z, [1.0, 0.0, 0.0], atol=1e-10)

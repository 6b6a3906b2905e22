"""Pins for the oracle's cone library (no GPU).

Each check is fixed by mathematics or by the paper, not by the oracle itself:
barrier identities of logarithmically homogeneous barriers, finite
differences, the defining equations of the NT and BFGS scalings, step lengths
against bisection on the cone definitions, Jordan-algebra identities, and
special cases that reduce to a simpler cone.
"""
import math

import numpy as np
import pytest

from oracle import cones as C

RNG = np.random.default_rng(1234)


def _exp_dual_pt(rng):
    u = -rng.uniform(0.3, 2.0)
    v = rng.uniform(-2.0, 2.0)
    return np.array([u, v, -u * math.exp(v / u) / math.e + rng.uniform(0.2, 2.0)])


def _exp_primal_pt(rng):
    y = rng.uniform(0.3, 2.0)
    x = rng.uniform(-2.0, 1.0)
    return np.array([x, y, y * math.exp(x / y) + rng.uniform(0.2, 2.0)])


def _pow_dual_pt(rng, a):
    u, v = rng.uniform(0.3, 2.0, 2)
    return np.array([u, v, rng.uniform(-0.95, 0.95) * (u / a) ** a * (v / (1 - a)) ** (1 - a)])


def _pow_primal_pt(rng, a):
    x, y = rng.uniform(0.3, 2.0, 2)
    return np.array([x, y, rng.uniform(-0.95, 0.95) * x ** a * y ** (1 - a)])


def _soc_pt(rng, d):
    u = rng.standard_normal(d - 1)
    return np.r_[np.linalg.norm(u) + rng.uniform(0.1, 2.0), u]


def _psd_pt(rng, k):
    M = rng.standard_normal((k, k))
    return C.svec(M @ M.T + 0.3 * np.eye(k))


NONSYM = [(C.EXP, 0.0), (C.POW, 0.3), (C.POW, 0.5), (C.POW, 0.8)]


def _dual_pt(t, a, rng):
    return _exp_dual_pt(rng) if t == C.EXP else _pow_dual_pt(rng, a)


def _primal_pt(t, a, rng):
    return _exp_primal_pt(rng) if t == C.EXP else _pow_primal_pt(rng, a)


# ---------------------------------------------------------------- barriers
@pytest.mark.parametrize("t,a", NONSYM)
def test_barrier_log_homogeneity(t, a):
    """<grad f(z), z> = -nu, Hess f(z) z = -grad f(z), f(tz) = f(z) - nu log t,
    grad^3 f(z)[z] = -2 Hess f(z) (nu = 3; Sec. 2.2 barrier list)."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        z = _dual_pt(t, a, rng)
        g = C.barrier_grad(t, z, a)
        Hm = C.barrier_hess(t, z, a)
        T = C.barrier_third(t, z, a)
        assert g @ z == pytest.approx(-3.0, rel=1e-12)
        np.testing.assert_allclose(Hm @ z, -g, rtol=1e-10, atol=1e-12)
        for sc in (0.5, 3.0):
            assert C.barrier(t, sc * z, a) == pytest.approx(C.barrier(t, z, a) - 3 * math.log(sc), abs=1e-10)
        np.testing.assert_allclose(np.einsum("ijk,k->ij", T, z), -2 * Hm, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("t,a", NONSYM)
def test_barrier_derivatives_finite_differences(t, a):
    """grad, Hessian and third derivative against central differences of the
    printed barrier f (Sec. 2.2, items 4-5)."""
    rng = np.random.default_rng(11)
    h = 1e-5
    for _ in range(10):
        z = _dual_pt(t, a, rng)
        g = C.barrier_grad(t, z, a)
        Hm = C.barrier_hess(t, z, a)
        T = C.barrier_third(t, z, a)
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            fd_g = (C.barrier(t, z + e, a) - C.barrier(t, z - e, a)) / (2 * h)
            assert fd_g == pytest.approx(g[i], rel=1e-6, abs=1e-7)
            fd_H = (C.barrier_grad(t, z + e, a) - C.barrier_grad(t, z - e, a)) / (2 * h)
            np.testing.assert_allclose(fd_H, Hm[:, i], rtol=1e-6, atol=1e-6)
            fd_T = (C.barrier_hess(t, z + e, a) - C.barrier_hess(t, z - e, a)) / (2 * h)
            np.testing.assert_allclose(fd_T, T[:, :, i], rtol=1e-5, atol=1e-5)


def test_barrier_pow_matches_printed_formula_at_a_point():
    """f for the dual power cone at (1, 1, 0.5), alpha = 1/2, evaluated by hand:
    -log(4 * 1 * 1 - 1/4) - 1/2 log 1 - 1/2 log 1 = -log(3.75)."""
    assert C.barrier(C.POW, np.array([1.0, 1.0, 0.5]), 0.5) == pytest.approx(-math.log(3.75), rel=1e-14)


def test_barrier_exp_matches_printed_formula_at_a_point():
    """f for the dual exponential cone at (-1, 0, 1): psi = 0 + 1 - (-1) log(1/1) = 1,
    so f = -log 1 - log 1 - log 1 = 0."""
    assert C.barrier(C.EXP, np.array([-1.0, 0.0, 1.0])) == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("t,a", NONSYM)
def test_central_point_is_fixed_point(t, a):
    u = C.central_point(t, 3, a)
    np.testing.assert_allclose(-C.barrier_grad(t, u, a), u, rtol=1e-12, atol=1e-14)
    assert C.in_int_primal(t, u, a) and C.in_int_dual(t, u, a)


def test_exp_central_point_norm():
    """The exp central point u = -grad f(u) has <u, u> = <u, -grad f(u)> = nu = 3."""
    u = C.central_point(C.EXP, 3)
    assert u @ u == pytest.approx(3.0, rel=1e-12)


@pytest.mark.parametrize("t,a", NONSYM)
def test_dual_shadow_inverts_gradient(t, a):
    """z_tilde = -grad f*(s) satisfies -grad f(z_tilde) = s, z_tilde in int K*,
    <s, z_tilde> = nu."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        s = _primal_pt(t, a, rng) * rng.uniform(0.01, 100.0)
        zt = C.dual_shadow(t, s, a)
        assert C.in_int_dual(t, zt, a)
        np.testing.assert_allclose(-C.barrier_grad(t, zt, a), s, rtol=1e-9, atol=1e-12)
        assert s @ zt == pytest.approx(3.0, rel=1e-9)


# ------------------------------------------------------------ NT scalings
@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
def test_soc_nt_scaling(d):
    rng = np.random.default_rng(d)
    J = np.diag(np.r_[1.0, -np.ones(d - 1)])
    for _ in range(10):
        s, z = _soc_pt(rng, d), _soc_pt(rng, d)
        sc = C.nt_scaling(C.SOC, s, z)
        W = sc["W"]
        np.testing.assert_allclose(sc["H"] @ z, s, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(W @ z, sc["WinvT"] @ s, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(W.T @ W, sc["H"], rtol=1e-10, atol=1e-10)
        eta2 = C.soc_jnorm(s) / C.soc_jnorm(z)
        np.testing.assert_allclose(W @ J @ W, eta2 * J, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(sc["Winv"] @ W, np.eye(d), atol=1e-10)


def test_nonneg_nt_scaling():
    s, z = RNG.uniform(0.1, 3, 7), RNG.uniform(0.1, 3, 7)
    sc = C.nt_scaling(C.NONNEG, s, z)
    np.testing.assert_allclose(sc["H"] @ z, s)
    np.testing.assert_allclose(sc["lam"] ** 2, s * z)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_psd_nt_scaling(k):
    rng = np.random.default_rng(10 + k)
    for _ in range(5):
        s, z = _psd_pt(rng, k), _psd_pt(rng, k)
        sc = C.nt_scaling(C.PSD, s, z)
        R, Ri, lam = sc["R"], sc["Rinv"], sc["lam"]
        S, Z = C.smat(s), C.smat(z)
        np.testing.assert_allclose(R.T @ Z @ R, np.diag(lam), atol=1e-10)
        np.testing.assert_allclose(Ri @ S @ Ri.T, np.diag(lam), atol=1e-10)
        np.testing.assert_allclose(Ri @ R, np.eye(k), atol=1e-10)
        np.testing.assert_allclose(sc["H"] @ z, s, rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(sc["W"] @ z, sc["WinvT"] @ s, rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(sc["H"], sc["H"].T, atol=1e-10)


@pytest.mark.parametrize("k", [2, 4, 7])
def test_psd_on_diagonal_matrices_is_nonneg(k):
    """Diagonal S, Z, dS, dZ: the PSD cone restricted to diagonal matrices is the
    nonnegative orthant, so its NT scaling, combined-step d_s and step length must
    equal the nonneg closed forms entry by entry (H = s/z, lambda = sqrt(s z),
    d_s = (s z + ds dz - sigma mu)/z, ratio test), whatever order the SVD gives the
    singular values in (R, R^-1 and lambda must be permuted alike)."""
    rng = np.random.default_rng(40 + k)
    dg = lambda v: C.svec(np.diag(v))  # noqa: E731
    for _ in range(5):
        s, z = rng.uniform(0.2, 2.0, k), rng.uniform(0.2, 2.0, k)
        ds, dz = rng.standard_normal(k), rng.standard_normal(k)
        smu = 0.3
        sc = C.nt_scaling(C.PSD, dg(s), dg(z))
        np.testing.assert_allclose(np.sort(sc["lam"]), np.sort(np.sqrt(s * z)), rtol=1e-12)
        np.testing.assert_allclose(sc["H"] @ dg(dz), dg(s / z * dz), rtol=1e-12, atol=1e-13)
        lam = C.lam_vec(C.PSD, sc["lam"], len(dg(s)))
        eta = C.jordan_prod(C.PSD, C.apply_scaling(C.PSD, sc, "WinvT", dg(ds)),
                            C.apply_scaling(C.PSD, sc, "W", dg(dz)))
        v = C.jordan_prod(C.PSD, lam, lam) + eta - smu * C.identity(C.PSD, len(lam))
        d_s = C.apply_scaling(C.PSD, sc, "WT", C.jordan_div(C.PSD, sc["lam"], v))
        np.testing.assert_allclose(d_s, dg((s * z + ds * dz - smu) / z), rtol=1e-11, atol=1e-12)
        a_psd = C.step_length_symmetric(C.PSD, dg(s), dg(ds))
        a_nn = C.step_length_symmetric(C.NONNEG, s, ds)
        assert a_psd == pytest.approx(a_nn, rel=1e-12) or (math.isinf(a_nn) and a_psd > 1e12)


@pytest.mark.parametrize("t,d", [(C.SOC, 2), (C.SOC, 5), (C.PSD, 6), (C.PSD, 15)])
def test_combined_ds_at_equal_s_and_z(t, d):
    """s = z: the NT scaling point is the identity (H = I, W = I, lambda = s), so
    the combined-step d_s with no affine correction reduces to the closed form
    s - sigma mu s^{-1}, the Jordan inverse being J s / (s_0^2 - |s_1|^2) for a SOC
    and S^{-1} for a PSD cone."""
    rng = np.random.default_rng(60 + d)
    smu = 0.4
    for _ in range(4):
        v = _soc_pt(rng, d) if t == C.SOC else _psd_pt(rng, C.psd_order(d))
        sc = C.nt_scaling(t, v, v)
        np.testing.assert_allclose(sc["H"], np.eye(d), atol=1e-12)
        lam = C.lam_vec(t, sc["lam"], d)
        w = C.jordan_prod(t, lam, lam) - smu * C.identity(t, d)
        d_s = C.apply_scaling(t, sc, "WT", C.jordan_div(t, sc["lam"], w))
        if t == C.SOC:
            inv = np.r_[v[0], -v[1:]] / (v[0] ** 2 - v[1:] @ v[1:])
        else:
            inv = C.svec(np.linalg.inv(C.smat(v)))
        np.testing.assert_allclose(d_s, v - smu * inv, rtol=1e-11, atol=1e-12)


def test_svec_is_an_isometry():
    X, Y = C.smat(_psd_pt(RNG, 4)), C.smat(_psd_pt(RNG, 4))
    assert C.svec(X) @ C.svec(Y) == pytest.approx(np.trace(X @ Y), rel=1e-13)
    np.testing.assert_allclose(C.smat(C.svec(X)), X)


# ----------------------------------------------------------- BFGS scaling
@pytest.mark.parametrize("t,a", NONSYM)
def test_bfgs_scaling_secant_equations(t, a):
    """H z = s, H z_tilde = s_tilde, H symmetric positive definite (Appendix A)."""
    rng = np.random.default_rng(5)
    n_bfgs = 0
    for _ in range(30):
        s, z = _primal_pt(t, a, rng), _dual_pt(t, a, rng)
        mu = rng.uniform(0.1, 2.0)
        H = C.bfgs_scaling(t, s, z, mu, a)
        st = -C.barrier_grad(t, z, a)
        zt = C.dual_shadow(t, s, a)
        if 1.0 - 9.0 / ((s @ z) * (st @ zt)) > C.BFGS_DEGENERACY:
            n_bfgs += 1
            np.testing.assert_allclose(H @ z, s, rtol=1e-8, atol=1e-10)
            np.testing.assert_allclose(H @ zt, st, rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose(H, H.T, atol=1e-12)
        assert np.linalg.eigvalsh(H).min() > 0
    assert n_bfgs > 20


def test_bfgs_fallback_on_central_path():
    """On the central path (s = mu s_tilde) BFGS degenerates; H = mu Hess f(z)
    then still satisfies H z = s."""
    u = C.central_point(C.EXP, 3)
    mu = 0.37
    s, z = mu * u, u
    H = C.bfgs_scaling(C.EXP, s, z, mu)
    np.testing.assert_allclose(H @ z, s, rtol=1e-10)


# ------------------------------------------------------------ Jordan algebra
@pytest.mark.parametrize("t,d", [(C.NONNEG, 4), (C.SOC, 5), (C.PSD, 6)])
def test_jordan_identities(t, d):
    rng = np.random.default_rng(2)
    pt = {C.NONNEG: lambda: rng.uniform(0.2, 2, d), C.SOC: lambda: _soc_pt(rng, d),
          C.PSD: lambda: _psd_pt(rng, 3)}[t]
    s, z = pt(), pt()
    e = C.identity(t, d)
    v = rng.standard_normal(d)
    np.testing.assert_allclose(C.jordan_prod(t, e, v), v, atol=1e-13)
    sc = C.nt_scaling(t, s, z)
    lam = C.lam_vec(t, sc["lam"], d)
    x = C.jordan_div(t, sc["lam"], v)
    np.testing.assert_allclose(C.jordan_prod(t, lam, x), v, atol=1e-10)
    # affine invariant of the combined d_s with sigma = 0, eta = 0:
    # W^T (lam \ (lam o lam)) = W^T lam = s
    ds = sc["W"].T @ C.jordan_div(t, sc["lam"], C.jordan_prod(t, lam, lam))
    np.testing.assert_allclose(ds, s, rtol=1e-9, atol=1e-10)


def test_nonneg_corrector_is_mehrotra():
    """For nonneg cones the symmetric d_s reduces to (s z + ds dz - sigma mu)/z."""
    rng = np.random.default_rng(9)
    s, z, ds, dz = rng.uniform(0.1, 2, 6), rng.uniform(0.1, 2, 6), rng.standard_normal(6), rng.standard_normal(6)
    sigma_mu = 0.3
    sc = C.nt_scaling(C.NONNEG, s, z)
    eta = C.jordan_prod(C.NONNEG, sc["WinvT"] @ ds, sc["W"] @ dz)
    v = C.jordan_prod(C.NONNEG, sc["lam"], sc["lam"]) + eta - sigma_mu
    d_s = sc["W"].T @ C.jordan_div(C.NONNEG, sc["lam"], v)
    np.testing.assert_allclose(d_s, (s * z + ds * dz - sigma_mu) / z, rtol=1e-12)


# ------------------------------------------------------------ step lengths
def _bisect_max_step(member, x, dx, hi=1e6):
    lo = 0.0
    if member(x + hi * dx):
        return math.inf
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if member(x + mid * dx):
            lo = mid
        else:
            hi = mid
    return lo


@pytest.mark.parametrize("t,d", [(C.NONNEG, 5), (C.SOC, 2), (C.SOC, 4), (C.SOC, 7), (C.PSD, 6), (C.PSD, 10)])
def test_symmetric_step_length_vs_bisection(t, d):
    rng = np.random.default_rng(d + 100 * t)
    for _ in range(20):
        if t == C.NONNEG:
            x = rng.uniform(0.1, 2, d)
        elif t == C.SOC:
            x = _soc_pt(rng, d)
        else:
            x = _psd_pt(rng, C.psd_order(d))
        dx = rng.standard_normal(d) * rng.uniform(0.1, 5)
        a = C.step_length_symmetric(t, x, dx)
        ref = _bisect_max_step(lambda v: C.in_int_primal(t, v), x, dx)
        if math.isinf(ref):
            assert math.isinf(a) or a > 1e5
        else:
            assert a == pytest.approx(ref, rel=1e-7, abs=1e-9)


def test_pow_half_is_rotated_soc():
    """pow(1/2) membership x^(1/2) y^(1/2) >= |z| <=> x y >= z^2, x, y >= 0, i.e.
    (x + y, x - y, 2z)/sqrt(2)... in SOC.  Compare membership on random points."""
    rng = np.random.default_rng(4)
    for _ in range(500):
        v = rng.standard_normal(3) * 2
        rot = np.array([v[0] + v[1], v[0] - v[1], 2 * v[2]])
        if abs(v[0] * v[1] - v[2] ** 2) < 1e-9 or v[0] == 0 or v[1] == 0:
            continue
        assert C.in_int_primal(C.POW, v, 0.5) == C.in_int_primal(C.SOC, rot)


def test_soc2_is_two_halfspaces():
    """SOC of dimension 2: (t, x) with |x| <= t <=> t + x >= 0 and t - x >= 0."""
    rng = np.random.default_rng(8)
    for _ in range(200):
        v = rng.standard_normal(2)
        assert C.in_int_primal(C.SOC, v) == (v[0] + v[1] > 0 and v[0] - v[1] > 0)


def test_exp_membership_definition():
    """Sec. 2.1: K_exp = {y > 0, y exp(x/y) <= z}; K_exp* = {u < 0, -u exp(v/u) <= e w}."""
    rng = np.random.default_rng(6)
    for _ in range(500):
        x, y, z = rng.standard_normal(3) * 2
        if y > 0 and abs(y * math.exp(min(x / y, 50)) - z) > 1e-9:
            assert C.in_int_primal(C.EXP, np.array([x, y, z])) == (z > y * math.exp(x / y))
        u, v, w = rng.standard_normal(3) * 2
        if u < 0 and w > 0 and abs(-u * math.exp(min(v / u, 50)) - math.e * w) > 1e-9:
            assert C.in_int_dual(C.EXP, np.array([u, v, w])) == (-u * math.exp(v / u) < math.e * w)


def test_shift_to_cone():
    v = np.array([-0.5, 1.0, 2.0])
    np.testing.assert_allclose(C.shift_to_cone(C.NONNEG, v), v + 1.5)
    w = np.array([1.0, 3.0, 4.0])  # t - |x| = -4
    out = C.shift_to_cone(C.SOC, w)
    assert out[0] == pytest.approx(6.0) and C.in_int_primal(C.SOC, out)
    u = np.array([3.0, 0.5])
    np.testing.assert_allclose(C.shift_to_cone(C.NONNEG, u), u)
    np.testing.assert_allclose(C.shift_to_cone(C.ZERO, u), 0.0)


def test_neighbourhood_on_central_path():
    """On the central path <grad f*(s), grad f(z)> = nu/mu, so N(beta) holds
    exactly when beta <= 1 (Sec. 2.2)."""
    u = C.central_point(C.POW, 3, 0.3)
    mu = 0.2
    assert C.neighbourhood_ok(C.POW, mu * u, u, mu, 1e-6, 0.3)
    assert not C.neighbourhood_ok(C.POW, mu * u, u, mu, 1.5, 0.3)


@pytest.mark.parametrize("t,a", NONSYM)
def test_third_order_correction_identity(t, a):
    """grad^3 f(z)[z] = -2 Hess f(z) for a 3-homogeneous barrier, so the
    correction -1/2 grad^3 f(z)[dz, Hess^{-1} ds] equals ds when dz = z
    (Eq. higher-order-correction)."""
    rng = np.random.default_rng(21)
    for _ in range(10):
        z = _dual_pt(t, a, rng)
        ds = rng.standard_normal(3)
        np.testing.assert_allclose(C.third_order_correction(t, z, z, ds, a), ds, rtol=1e-8, atol=1e-10)
        dz = rng.standard_normal(3)
        # bilinear in (dz, ds), symmetric tensor
        e1 = C.third_order_correction(t, z, dz, ds, a)
        e2 = C.third_order_correction(t, z, 2.0 * dz, ds, a)
        np.testing.assert_allclose(e2, 2.0 * e1, rtol=1e-10, atol=1e-12)


def test_failed_shadow_falls_back_and_leaves_the_neighbourhood(monkeypatch):
    """Where z~ = -grad f*(s) cannot be evaluated (a singular Newton system near the
    boundary of the cone), the BFGS scaling is H_a = mu grad^2 f(z) and the trial
    point counts as outside N(beta) -- exercised by making the Newton solve fail."""
    s = np.array([-0.5, 1.0, 2.0])          # interior of the exponential cone
    z = np.array([-1.0, 0.3, 1.5])          # interior of its dual
    assert C.in_int_primal(C.EXP, s) and C.in_int_dual(C.EXP, z)
    mu = 0.7
    H_ok = C.bfgs_scaling(C.EXP, s, z, mu)
    assert C.neighbourhood_ok(C.EXP, s, z, mu, 1e-6)

    def singular(*args, **kwargs):
        raise np.linalg.LinAlgError("Singular matrix")

    monkeypatch.setattr(C, "dual_shadow", singular)
    H_fb = C.bfgs_scaling(C.EXP, s, z, mu)
    np.testing.assert_allclose(H_fb, mu * C.barrier_hess(C.EXP, z), rtol=1e-14)
    assert not np.allclose(H_fb, H_ok)      # the fallback is a different matrix here
    assert C.neighbourhood_ok(C.EXP, s, z, mu, 1e-6) is False


def test_exp_dual_shadow_near_the_boundary():
    """The one-dimensional reduction keeps -grad f(z_tilde) = s as s approaches the
    boundary of the exponential cone (where z_tilde grows like 2 / (y log(z/y) - x))."""
    y, x = 0.05, 0.15
    for rel in (1e-2, 1e-5, 1e-8, 1e-10):
        s = np.array([x, y, y * math.exp(x / y) * (1.0 + rel)])
        u = C.dual_shadow(C.EXP, s)
        assert C.in_int_dual(C.EXP, u)
        np.testing.assert_allclose(-C.barrier_grad(C.EXP, u), s, rtol=1e-9, atol=1e-12)
        gap = y * math.log(s[2] / y) - x
        assert -u[0] == pytest.approx(2.0 / gap, rel=0.05 + 10 * gap)


def test_third_order_correction_dropped_on_singular_hessian(monkeypatch):
    z = np.array([-1.0, 0.3, 1.5])
    dz, ds = np.array([0.1, -0.2, 0.3]), np.array([0.2, 0.1, -0.1])
    eta = C.third_order_correction(C.EXP, z, dz, ds)
    assert np.abs(eta).max() > 0

    def singular(*args, **kwargs):
        raise np.linalg.LinAlgError("Singular matrix")

    monkeypatch.setattr(C.np.linalg, "solve", singular)
    np.testing.assert_array_equal(C.third_order_correction(C.EXP, z, dz, ds), np.zeros(3))


def _near_complementary_psd_pair(rng, k, small):
    """S, Z sharing one orthogonal basis Q, S with k//2 eigenvalues ~small and
    Z with the others ~small (a strictly complementary PSD pair near the end of
    an interior-point solve).  Returns S, Z, Q and Z's eigenvalues."""
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    h = k // 2
    es = np.r_[rng.uniform(0.5, 2.0, k - h), small * rng.uniform(0.5, 2.0, h)]
    ez = np.r_[small * rng.uniform(0.5, 2.0, k - h), rng.uniform(0.5, 2.0, h)]
    return (Q * es) @ Q.T, (Q * ez) @ Q.T, Q, ez


@pytest.mark.parametrize("k", [2, 4, 6])
def test_psd_factored_H_equals_assembled_H(k):
    """H v in factored form, R (R^T V R) R^T, is the assembled svec block of
    nt_scaling times v (both are H = W^T W of Appendix A)."""
    rng = np.random.default_rng(40 + k)
    M1, M2 = rng.standard_normal((k, k)), rng.standard_normal((k, k))
    s, z = C.svec(M1 @ M1.T + 0.3 * np.eye(k)), C.svec(M2 @ M2.T + 0.3 * np.eye(k))
    sc = C.nt_scaling(C.PSD, s, z)
    v = rng.standard_normal(len(s))
    Hv = sc["H"] @ v
    np.testing.assert_allclose(C.psd_apply_H(sc["R"], v), Hv, rtol=1e-12, atol=1e-12 * np.abs(Hv).max())
    # and it maps z to s (H z = s)
    np.testing.assert_allclose(C.psd_apply_H(sc["R"], z), s, rtol=1e-10, atol=1e-12)


def test_psd_factored_H_keeps_the_small_eigenspace_of_S():
    """Near convergence (S, Z of complementary rank, small eigenvalues 1e-9) a
    search direction Delta Z has the scale of Z on each eigen-direction, and the
    exact H Delta Z -- evaluated in 60-digit arithmetic from the same FP64 R --
    has the scale of S: ~1e-9 on the small eigenspace of S.  The factored
    product R (R^T Delta Z R) R^T keeps that block to many digits; the
    assembled svec block (entries up to ~1e9) loses it to cancellation.  This
    is why Delta s of a PSD cone is formed in factored form."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    rng = np.random.default_rng(7)
    k = 6
    S, Z, Q, ez = _near_complementary_psd_pair(rng, k, 1e-9)
    sc = C.nt_scaling(C.PSD, C.svec(S), C.svec(Z))
    R = sc["R"]
    G = rng.standard_normal((k, k))
    dZ = Q @ ((G + G.T) * np.sqrt(np.outer(ez, ez))) @ Q.T  # entries scaled like Z's
    v = C.svec(dZ)
    Rm = mpmath.matrix(R.tolist())
    Qm = mpmath.matrix(Q[:, k - k // 2:].tolist())

    def small_block(Xm):
        # the block on the small eigenspace of S, projected in 60-digit arithmetic
        B = Qm.T * Xm * Qm
        return np.array([[float(B[i, j]) for j in range(B.cols)] for i in range(B.rows)])

    ref = small_block(Rm * (Rm.T * mpmath.matrix(C.smat(v).tolist()) * Rm) * Rm.T)
    err_fact = np.abs(small_block(mpmath.matrix(C.smat(C.psd_apply_H(R, v)).tolist())) - ref).max()
    err_asm = np.abs(small_block(mpmath.matrix(C.smat(sc["H"] @ v).tolist())) - ref).max()
    scale = np.abs(ref).max()
    assert scale < 1e-7  # the exact product is tiny there
    assert err_fact <= 1e-4 * scale, (err_fact, scale)
    assert err_asm > 100 * err_fact, (err_asm, err_fact)


@pytest.mark.parametrize("t,d", [(C.NONNEG, 4), (C.SOC, 5), (C.PSD, 10)])
def test_apply_scaling_matches_the_matrices(t, d):
    """W v, W^{-T} v and W^T v of apply_scaling equal the assembled NT matrices
    times v (PSD in factored form, the others through the matrices)."""
    rng = np.random.default_rng(60 + d)
    if t == C.PSD:
        k = C.psd_order(d)
        M1, M2 = rng.standard_normal((k, k)), rng.standard_normal((k, k))
        s, z = C.svec(M1 @ M1.T + 0.3 * np.eye(k)), C.svec(M2 @ M2.T + 0.3 * np.eye(k))
    elif t == C.SOC:
        s = np.r_[3.0, rng.standard_normal(d - 1)]
        z = np.r_[3.5, rng.standard_normal(d - 1)]
    else:
        s, z = rng.uniform(0.5, 2, d), rng.uniform(0.5, 2, d)
    sc = C.nt_scaling(t, s, z)
    v = rng.standard_normal(d)
    for which, M in (("W", sc["W"]), ("WinvT", sc["WinvT"]), ("WT", sc["W"].T)):
        ref = M @ v
        np.testing.assert_allclose(C.apply_scaling(t, sc, which, v), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # W^{-T} s = W z = lambda
    np.testing.assert_allclose(C.apply_scaling(t, sc, "WinvT", s), C.lam_vec(t, sc["lam"], d), atol=1e-10)
    np.testing.assert_allclose(C.apply_scaling(t, sc, "W", z), C.lam_vec(t, sc["lam"], d), atol=1e-10)

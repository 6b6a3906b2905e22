"""Oracle cone library: plain FP64 NumPy, one cone at a time.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA product path
never imports it and shares no code with it.

Every function follows a passage of the paper (arXiv:2412.19027, "CuClarabel"):

* cone definitions and dual cones ............ Sec. 2.1 "Supported cones"
* barrier functions f of the dual cones ...... Sec. 2.2, barrier list (nonneg, SOC,
  PSD, dual exponential, dual power)
* NT scaling for nonneg / SOC / PSD .......... Appendix A (cvxopt NT scaling), with
  H = W^T W so that H z = s (the KKT's H, Eq. linsys_4x4)
* nonsymmetric (exp / pow) scaling ........... Appendix A: shadow iterates and the
  rank-4 BFGS matrix H, H_a = mu * Hess f(z)
* Jordan product / division, e ............... Eq. ds-correction-step (symmetric)
* Mehrotra and 3rd-order corrections ......... Eq. higher-order-correction
* step lengths ............................... Sec. 2.2 "Find search directions"
  (max alpha with v + alpha*Delta in F; backtracking by 0.8 for exp/pow)
* neighbourhood N(beta) ...................... Sec. 2.2 "Update iterates"

Conventions (readings of the paper where it is silent or garbled):

* f is the barrier of the DUAL cone K*, the central path is s = -mu grad f(z).
  The paper's appendix writes the shadow iterates in the primal-barrier
  convention; here s_tilde = -grad f(z) and z_tilde = -grad f*(s), so that the
  BFGS matrix satisfies H z = s and H z_tilde = s_tilde.
* PSD cones are stored as svec: upper triangle, column by column, off-diagonal
  entries times sqrt(2), so <svec X, svec Y> = trace(X Y).
* SOC has degree 1 (barrier -1/2 log(z0^2 - |z1|^2)), e = (1, 0, ..., 0).
"""
import math

import numpy as np

ZERO, NONNEG, SOC, EXP, POW, PSD = 0, 1, 2, 3, 4, 5
FAMILY_NAMES = {ZERO: "zero", NONNEG: "nonneg", SOC: "soc", EXP: "exp", POW: "pow", PSD: "psd"}
SQRT2 = math.sqrt(2.0)


# --------------------------------------------------------------------------
# svec / smat for PSD cones (Sec. 2.1, PSD cone; storage convention above)
# --------------------------------------------------------------------------
def psd_order(dim):
    """Matrix order k with k(k+1)/2 == dim."""
    k = int(round((math.sqrt(8 * dim + 1) - 1) / 2))
    if k * (k + 1) // 2 != dim:
        raise ValueError("PSD cone dimension %d is not triangular" % dim)
    return k


def svec(X):
    k = X.shape[0]
    out = []
    for j in range(k):
        for i in range(j + 1):
            out.append(X[i, j] if i == j else SQRT2 * X[i, j])
    return np.array(out, dtype=np.float64)


def smat(v):
    k = psd_order(len(v))
    X = np.zeros((k, k))
    idx = 0
    for j in range(k):
        for i in range(j + 1):
            if i == j:
                X[i, i] = v[idx]
            else:
                X[i, j] = X[j, i] = v[idx] / SQRT2
            idx += 1
    return X


# --------------------------------------------------------------------------
# degrees and central points (Sec. 2.2 barrier list)
# --------------------------------------------------------------------------
def degree(ctype, dim):
    if ctype == ZERO:
        return 0
    if ctype == NONNEG:
        return dim
    if ctype == SOC:
        return 1
    if ctype == PSD:
        return psd_order(dim)
    return 3  # EXP, POW


def identity(ctype, dim):
    """The Jordan identity e of a symmetric cone."""
    if ctype == NONNEG:
        return np.ones(dim)
    if ctype == SOC:
        e = np.zeros(dim)
        e[0] = 1.0
        return e
    if ctype == PSD:
        return svec(np.eye(psd_order(dim)))
    raise ValueError("no Jordan identity for cone type %d" % ctype)


def central_point(ctype, dim, alpha=0.0):
    """Point u with u = -grad f(u) (mu = 1 on the central path).

    For the symmetric cones this is e.  For pow it is (sqrt(1+a), sqrt(2-a), 0)
    (checked against the barrier gradient by the tests).  For exp it is found by
    Newton's method on u + grad f(u) = 0, started from (-1, 0.5, 1.2)."""
    if ctype == ZERO:
        return np.zeros(dim)
    if ctype in (NONNEG, SOC, PSD):
        return identity(ctype, dim)
    if ctype == POW:
        return np.array([math.sqrt(1.0 + alpha), math.sqrt(2.0 - alpha), 0.0])
    u = np.array([-1.0, 0.5, 1.2])
    for _ in range(100):
        r = u + barrier_grad(EXP, u)
        J = np.eye(3) + barrier_hess(EXP, u)
        du = np.linalg.solve(J, -r)
        u = u + du
        if np.max(np.abs(du)) < 1e-15:
            break
    return u


# --------------------------------------------------------------------------
# membership (Sec. 2.1 definitions; interior = strict inequalities)
# --------------------------------------------------------------------------
def in_int_primal(ctype, s, alpha=0.0):
    if ctype == ZERO:
        return True
    if ctype == NONNEG:
        return bool(np.all(s > 0))
    if ctype == SOC:
        return bool(s[0] > 0 and s[0] * s[0] - s[1:] @ s[1:] > 0)
    if ctype == PSD:
        return bool(np.linalg.eigvalsh(smat(s)).min() > 0)
    if ctype == EXP:
        x, y, z = s
        return bool(y > 0 and z > 0 and y * math.log(z / y) - x > 0)
    if ctype == POW:
        x, y, z = s
        return bool(x > 0 and y > 0 and x ** alpha * y ** (1 - alpha) - abs(z) > 0)
    raise ValueError(ctype)


def in_int_dual(ctype, z, alpha=0.0):
    if ctype == ZERO:
        return True  # dual of the zero cone is R^n
    if ctype in (NONNEG, SOC, PSD):
        return in_int_primal(ctype, z)
    if ctype == EXP:
        u, v, w = z
        # -u exp(v/u) < e w with u < 0, written in logs: log(-u) + v/u < 1 + log w
        return bool(u < 0 and w > 0 and 1.0 + math.log(w) - math.log(-u) - v / u > 0)
    if ctype == POW:
        u, v, w = z
        return bool(u > 0 and v > 0 and (u / alpha) ** alpha * (v / (1 - alpha)) ** (1 - alpha) - abs(w) > 0)
    raise ValueError(ctype)


# --------------------------------------------------------------------------
# barriers of the dual exp / dual pow cones (Sec. 2.2, items 4 and 5)
#   f(z) = -log(psi(z)) + sum_i g_i(z_i)
# Gradient, Hessian and third derivative follow from the chain rule for
# -log(psi); the separable part contributes on the diagonal only.
# --------------------------------------------------------------------------
def _psi_parts(ctype, z, alpha):
    """psi, grad psi, Hess psi, 3rd-derivative tensor of psi; separable g', g'', g'''."""
    if ctype == EXP:
        r, s, t = z
        psi = s - r - r * math.log(t / (-r))
        g1 = np.array([math.log(-r / t), 1.0, -r / t])
        g2 = np.zeros((3, 3))
        g2[0, 0] = 1.0 / r
        g2[0, 2] = g2[2, 0] = -1.0 / t
        g2[2, 2] = r / (t * t)
        g3 = np.zeros((3, 3, 3))
        g3[0, 0, 0] = -1.0 / (r * r)
        for (i, j, k) in ((0, 2, 2), (2, 0, 2), (2, 2, 0)):
            g3[i, j, k] = 1.0 / (t * t)
        g3[2, 2, 2] = -2.0 * r / (t ** 3)
        # separable: -log(-r) and -log(t)
        sep1 = np.array([-1.0 / r, 0.0, -1.0 / t])
        sep2 = np.array([1.0 / (r * r), 0.0, 1.0 / (t * t)])
        sep3 = np.array([-2.0 / r ** 3, 0.0, -2.0 / t ** 3])
        return psi, g1, g2, g3, sep1, sep2, sep3
    if ctype == POW:
        a = alpha
        u, v, w = z
        phi = (u / a) ** (2 * a) * (v / (1 - a)) ** (2 * (1 - a))
        psi = phi - w * w
        pa, pb = 2 * a, 2 * (1 - a)  # exponents of u and v in phi
        g1 = np.array([pa * phi / u, pb * phi / v, -2.0 * w])
        g2 = np.zeros((3, 3))
        g2[0, 0] = pa * (pa - 1) * phi / (u * u)
        g2[0, 1] = g2[1, 0] = pa * pb * phi / (u * v)
        g2[1, 1] = pb * (pb - 1) * phi / (v * v)
        g2[2, 2] = -2.0
        g3 = np.zeros((3, 3, 3))
        # d^3 phi for phi = C u^pa v^pb: coefficient * phi / (u^i v^j)
        for i in range(3):
            for j in range(3):
                for k in range(3):
                    idx = (i, j, k)
                    if 2 in idx:
                        continue
                    nu_ = idx.count(0)
                    nv_ = idx.count(1)
                    cu = 1.0
                    for q in range(nu_):
                        cu *= (pa - q)
                    cv = 1.0
                    for q in range(nv_):
                        cv *= (pb - q)
                    g3[i, j, k] = cu * cv * phi / (u ** nu_ * v ** nv_)
        sep1 = np.array([-(1 - a) / u, -a / v, 0.0])
        sep2 = np.array([(1 - a) / (u * u), a / (v * v), 0.0])
        sep3 = np.array([-2.0 * (1 - a) / u ** 3, -2.0 * a / v ** 3, 0.0])
        return psi, g1, g2, g3, sep1, sep2, sep3
    raise ValueError(ctype)


def barrier(ctype, z, alpha=0.0):
    if ctype == EXP:
        r, s, t = z
        return -math.log(s - r - r * math.log(t / (-r))) - math.log(-r) - math.log(t)
    if ctype == POW:
        a = alpha
        u, v, w = z
        phi = (u / a) ** (2 * a) * (v / (1 - a)) ** (2 * (1 - a))
        return -math.log(phi - w * w) - (1 - a) * math.log(u) - a * math.log(v)
    raise ValueError(ctype)


def barrier_grad(ctype, z, alpha=0.0):
    psi, g1, _, _, sep1, _, _ = _psi_parts(ctype, z, alpha)
    return -g1 / psi + sep1


def barrier_hess(ctype, z, alpha=0.0):
    psi, g1, g2, _, _, sep2, _ = _psi_parts(ctype, z, alpha)
    return np.outer(g1, g1) / psi ** 2 - g2 / psi + np.diag(sep2)


def barrier_third(ctype, z, alpha=0.0):
    """Full 3x3x3 tensor of third derivatives of f."""
    psi, g1, g2, g3, _, _, sep3 = _psi_parts(ctype, z, alpha)
    T = -g3 / psi
    T += (np.einsum("ij,k->ijk", g2, g1) + np.einsum("ik,j->ijk", g2, g1)
          + np.einsum("jk,i->ijk", g2, g1)) / psi ** 2
    T -= 2.0 * np.einsum("i,j,k->ijk", g1, g1, g1) / psi ** 3
    for i in range(3):
        T[i, i, i] += sep3[i]
    return T


def _exp_dual_shadow(s):
    """z_tilde = (r, v, t) in int K*_exp with -grad f(z_tilde) = s = (x, y, z), for the
    dual barrier f = -log(psi) - log(-r) - log(t), psi = v - r - r log(t / (-r)).

    The three equations reduce to one in rho = -r > 0 (derived from the gradient):
        y: 1/psi = y;   z: (1 + rho y) / t = z;   x: y log(rho z / (1 + rho y)) - 1/rho = x,
    whose left side increases in rho from -inf to y log(z/y) > x (s interior), so the
    root is unique; it is bracketed by doubling and found by bisection on log(rho),
    which stays accurate when s nears the boundary (rho ~ 2 / (y log(z/y) - x))."""
    x, y, z = (float(v) for v in s)
    gap = y * math.log(z / y) - x
    if not (y > 0.0 and z > 0.0 and gap > 0.0):
        raise ValueError("s is not in the interior of the exponential cone")

    def g(rho):
        return y * (math.log(rho * z) - math.log1p(rho * y)) - 1.0 / rho - x

    lo, hi = 1.0, 1.0
    while g(lo) > 0.0:
        lo *= 0.5
    while g(hi) < 0.0:
        hi *= 2.0
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if g(mid) < 0.0:
            lo = mid
        else:
            hi = mid
        if hi <= lo * (1.0 + 1e-15):
            break
    rho = math.sqrt(lo * hi)
    t = (1.0 + rho * y) / z
    v = 1.0 / y - rho - rho * math.log(t / rho)
    return np.array([-rho, v, t])


def dual_shadow(ctype, s, alpha=0.0, tol=1e-28, max_iter=100):
    """z_tilde = -grad f*(s): the point of int K* with -grad f(z_tilde) = s.

    Exponential cone: the one-dimensional reduction of _exp_dual_shadow.  Power
    cone: damped Newton on phi(u) = f(u) + <s, u>, whose minimiser satisfies
    grad f(u) = -s; the step 1/(1 + lambda) (lambda = Newton decrement) keeps
    u inside int K* for a self-concordant f.  Starts at the central point."""
    if ctype == EXP:
        return _exp_dual_shadow(s)
    u = central_point(ctype, 3, alpha)
    for _ in range(max_iter):
        g = barrier_grad(ctype, u, alpha) + s
        Hm = barrier_hess(ctype, u, alpha)
        du = -np.linalg.solve(Hm, g)
        lam2 = -g @ du
        if lam2 < tol:
            u = u + du
            break
        lam = math.sqrt(max(lam2, 0.0))
        step = 1.0 if lam < 0.25 else 1.0 / (1.0 + lam)
        u = u + step * du
    return u


# --------------------------------------------------------------------------
# NT scaling for symmetric cones (Appendix A; W z = W^{-T} s = lambda, H = W^T W)
# --------------------------------------------------------------------------
def soc_jnorm(u):
    return math.sqrt(u[0] * u[0] - u[1:] @ u[1:])


def nt_scaling(ctype, s, z):
    """Returns dict with W (d x d), Winv, WinvT, lam (vector), H = W^T W."""
    d = len(s)
    if ctype == NONNEG:
        w = np.sqrt(s / z)
        W = np.diag(w)
        return dict(W=W, Winv=np.diag(1.0 / w), WinvT=np.diag(1.0 / w),
                    lam=np.sqrt(s * z), H=np.diag(s / z))
    if ctype == SOC:
        ns, nz = soc_jnorm(s), soc_jnorm(z)
        sb, zb = s / ns, z / nz
        J = np.diag(np.r_[1.0, -np.ones(d - 1)])
        gamma = math.sqrt((1.0 + sb @ zb) / 2.0)
        wb = (sb + J @ zb) / (2.0 * gamma)
        eta = math.sqrt(ns / nz)
        Wb = np.zeros((d, d))
        Wb[0, 0] = wb[0]
        Wb[0, 1:] = wb[1:]
        Wb[1:, 0] = wb[1:]
        Wb[1:, 1:] = np.eye(d - 1) + np.outer(wb[1:], wb[1:]) / (1.0 + wb[0])
        W = eta * Wb
        Winv = (J @ Wb @ J) / eta
        H = eta * eta * (2.0 * np.outer(wb, wb) - J)
        return dict(W=W, Winv=Winv, WinvT=Winv.T, lam=W @ z, H=H)
    if ctype == PSD:
        S, Z = smat(s), smat(z)
        Ls = np.linalg.cholesky(S)
        Lz = np.linalg.cholesky(Z)
        U, lam, Vt = np.linalg.svd(Lz.T @ Ls)
        R = Ls @ Vt.T @ np.diag(lam ** -0.5)
        Rinv = np.diag(lam ** -0.5) @ U.T @ Lz.T
        n = d
        W = np.zeros((n, n))
        WinvT = np.zeros((n, n))
        H = np.zeros((n, n))
        M = R @ R.T
        for c in range(n):
            E = np.zeros(n)
            E[c] = 1.0
            X = smat(E)
            W[:, c] = svec(R.T @ X @ R)
            WinvT[:, c] = svec(Rinv @ X @ Rinv.T)
            H[:, c] = svec(M @ X @ M)
        return dict(W=W, Winv=np.linalg.inv(W), WinvT=WinvT, lam=lam, H=H, R=R, Rinv=Rinv)
    raise ValueError(ctype)


def psd_apply_H(R, v):
    """H v for a PSD cone with NT scaling matrix R, in factored form:
    H = W^T W with W(X) = R^T X R (Appendix A), so H v = svec(R (R^T V R) R^T),
    V = smat(v).  Equal to nt_scaling(...)["H"] @ v in exact arithmetic; in
    floating point each factor only carries the square root of H's range.  The
    product is symmetrised by averaging it with its transpose (its rounding is
    not symmetric, and keeping one triangle would mix the large eigen-block's
    rounding into the small one)."""
    Y = R.T @ smat(v) @ R
    X = R @ Y @ R.T
    return svec(0.5 * (X + X.T))


def apply_scaling(ctype, sc, which, v):
    """W v, W^{-T} v or W^T v ('W', 'WinvT', 'WT') for the NT scaling sc of a
    symmetric cone.  PSD cones apply W(X) = R^T X R, W^{-T}(X) = R^{-1} X R^{-T}
    and W^T(X) = R X R^T as congruences with R (Appendix A), symmetrised by
    averaging with the transpose, rather than through the assembled svec
    matrices, whose entries grow like the square root of H's condition number;
    the other cones multiply by the matrices."""
    if ctype == PSD:
        R, Ri = sc["R"], sc["Rinv"]
        V = smat(v)
        if which == "W":
            X = R.T @ V @ R
        elif which == "WinvT":
            X = Ri @ V @ Ri.T
        else:
            X = R @ V @ R.T
        return svec(0.5 * (X + X.T))
    M = {"W": sc["W"], "WinvT": sc["WinvT"], "WT": sc["W"].T}[which]
    return M @ v


# --------------------------------------------------------------------------
# Jordan algebra (Eq. ds-correction-step, symmetric branch)
# --------------------------------------------------------------------------
def jordan_prod(ctype, u, v):
    if ctype == NONNEG:
        return u * v
    if ctype == SOC:
        return np.r_[u @ v, u[0] * v[1:] + v[0] * u[1:]]
    if ctype == PSD:
        U, V = smat(u), smat(v)
        return svec(0.5 * (U @ V + V @ U))
    raise ValueError(ctype)


def jordan_div(ctype, lam, v):
    """x with lam o x = v.  For PSD, lam is the vector of eigenvalues of the
    diagonal matrix Lambda and v, x are svec vectors."""
    if ctype == NONNEG:
        return v / lam
    if ctype == SOC:
        det = lam[0] * lam[0] - lam[1:] @ lam[1:]
        x0 = (lam[0] * v[0] - lam[1:] @ v[1:]) / det
        x1 = (v[1:] - x0 * lam[1:]) / lam[0]
        return np.r_[x0, x1]
    if ctype == PSD:
        V = smat(v)
        k = V.shape[0]
        X = np.zeros((k, k))
        for i in range(k):
            for j in range(k):
                X[i, j] = 2.0 * V[i, j] / (lam[i] + lam[j])
        return svec(X)
    raise ValueError(ctype)


def lam_vec(ctype, lam, dim):
    """lambda as a vector of the cone's coordinates (PSD: svec(diag(lam)))."""
    if ctype == PSD:
        return svec(np.diag(lam))
    return lam


# --------------------------------------------------------------------------
# step lengths (max alpha with x + alpha dx in the cone; Sec. 2.2)
# --------------------------------------------------------------------------
def step_length_symmetric(ctype, x, dx):
    """Largest alpha >= 0 (possibly inf) keeping x + alpha dx in the closed cone."""
    if ctype == ZERO:
        return math.inf
    if ctype == NONNEG:
        neg = dx < 0
        if not np.any(neg):
            return math.inf
        return float(np.min(-x[neg] / dx[neg]))
    if ctype == SOC:
        # q(a) = A a^2 + 2 B a + C, C = J-norm^2 of x > 0; smallest positive root.
        A = dx[0] * dx[0] - dx[1:] @ dx[1:]
        B = x[0] * dx[0] - x[1:] @ dx[1:]
        C = x[0] * x[0] - x[1:] @ x[1:]
        roots = []
        if A == 0.0:
            if B < 0:
                roots.append(-C / (2.0 * B))
        else:
            disc = B * B - A * C
            if disc >= 0:
                sq = math.sqrt(disc)
                roots += [(-B - sq) / A, (-B + sq) / A]
        pos = [r for r in roots if r > 0]
        a_soc = min(pos) if pos else math.inf
        # the t-component must stay nonnegative as well
        if dx[0] < 0:
            a_soc = min(a_soc, -x[0] / dx[0])
        return a_soc
    if ctype == PSD:
        X, dX = smat(x), smat(dx)
        L = np.linalg.cholesky(X)
        Li = np.linalg.inv(L)
        lmin = np.linalg.eigvalsh(Li @ dX @ Li.T).min()
        return math.inf if lmin >= 0 else -1.0 / lmin
    raise ValueError(ctype)


def shift_to_cone(ctype, v):
    """Initialisation shift: if the least Jordan eigenvalue a of v is below
    sqrt(eps), return v + (1 - a) e; zero-cone entries are set to 0."""
    if ctype == ZERO:
        return np.zeros_like(v)
    if ctype == NONNEG:
        a = float(np.min(v))
    elif ctype == SOC:
        a = v[0] - math.sqrt(v[1:] @ v[1:])
    elif ctype == PSD:
        a = float(np.linalg.eigvalsh(smat(v)).min())
    else:
        raise ValueError(ctype)
    if a < math.sqrt(np.finfo(np.float64).eps):
        return v + (1.0 - a) * identity(ctype, len(v))
    return v.copy()


# --------------------------------------------------------------------------
# nonsymmetric scaling (Appendix A): BFGS rank-4 matrix with H z = s, H zt = st
# --------------------------------------------------------------------------
BFGS_DEGENERACY = 1e-6


def bfgs_scaling(ctype, s, z, mu, alpha=0.0):
    """H = S (S^T Z)^{-1} S^T + H_a - H_a Z (Z^T H_a Z)^{-1} Z^T H_a, with
    S = [s, st], Z = [z, zt], st = -grad f(z), zt = -grad f*(s), H_a = mu Hess f(z).
    mu is the global complementarity measure.  When 1 - 9/((s'z)(st'zt)) is below
    BFGS_DEGENERACY (near the central path, where S and Z become rank one), or
    when zt cannot be evaluated (the Newton system of the conjugate barrier is
    singular near the boundary of the cone), the matrix H_a alone is used."""
    st = -barrier_grad(ctype, z, alpha)
    Ha = mu * barrier_hess(ctype, z, alpha)
    try:
        zt = dual_shadow(ctype, s, alpha)
    except (np.linalg.LinAlgError, FloatingPointError, ZeroDivisionError, ValueError):
        return Ha
    sz, stzt = s @ z, st @ zt
    if not (np.all(np.isfinite(zt)) and 1.0 - 9.0 / (sz * stzt) > BFGS_DEGENERACY):
        return Ha
    S = np.column_stack([s, st])
    Z = np.column_stack([z, zt])
    H = S @ np.linalg.solve(S.T @ Z, S.T) + Ha - Ha @ Z @ np.linalg.solve(Z.T @ Ha @ Z, Z.T @ Ha)
    return 0.5 * (H + H.T)


def third_order_correction(ctype, z, dz, ds, alpha=0.0):
    """eta = -1/2 grad^3 f(z)[dz, (grad^2 f(z))^{-1} ds]  (Eq. higher-order-correction).

    Where grad^2 f(z) is singular in floating point (z at the boundary of the dual
    cone to rounding) the term is dropped: eta = 0 for that cone."""
    T = barrier_third(ctype, z, alpha)
    try:
        u = np.linalg.solve(barrier_hess(ctype, z, alpha), ds)
    except np.linalg.LinAlgError:
        return np.zeros(3)
    return -0.5 * np.einsum("ijk,j,k->i", T, dz, u)


def neighbourhood_ok(ctype, s, z, mu, beta, alpha=0.0):
    """nu_i <grad f*(s_i), grad f(z_i)>^{-1} >= beta mu  (Sec. 2.2, N(beta)).

    A trial point at which grad f*(s) cannot be evaluated (the Newton system of
    the conjugate is singular, or a value is not finite) counts as outside the
    neighbourhood, so the step length backs off instead of failing the solve."""
    try:
        zt = dual_shadow(ctype, s, alpha)  # = -grad f*(s)
        st = -barrier_grad(ctype, z, alpha)  # = -grad f(z)
        d = float(zt @ st)
    except (np.linalg.LinAlgError, FloatingPointError, ZeroDivisionError, ValueError):
        return False
    return bool(np.isfinite(d) and d > 0.0 and 3.0 / d >= beta * mu)

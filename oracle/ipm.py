"""Oracle IPM: the homogeneous-embedding predictor-corrector method, plain FP64.

TEST INFRASTRUCTURE ONLY (see oracle/cones.py header).

Follows the paper's Algorithm 1 (primal-dual interior-point method) step by
step, with dense matrices and the dense LDL^T of oracle/linsys.py:

  setup   cone reordering and merging (Sec. 3.5 "Data structures"),
          equilibration (Alg. 1 step 1; method silent -> modified Ruiz reading),
          initial point (Alg. 1 step 2; silent -> reading below)
  loop    residuals / objectives / mu (Eq. residuals-objectives),
          termination and infeasibility tests (Eq. termination-check,
          Eq. infeasibility-check), scaling H (Alg. 1 step 4, Appendix A),
          factor K (step 5, Eq. linsys_2x2), affine direction (step 6,
          Eq. affine-step, Eq. step-direction), affine step length (step 7),
          sigma = (1 - alpha_a)^3 (step 8), combined direction (step 9,
          Eq. ds-correction-step, Eq. higher-order-correction), combined step
          length with the N(beta) check (step 10), v += 0.99 alpha_c Delta_c
          (step 11).

Readings where the paper is silent or garbled (each one is also implemented,
independently, by the CUDA path):
* equilibration: 10 Ruiz passes on [P A^T; A 0] (column infinity norms,
  factor 1/sqrt(norm), norms below 1e-8 leave the column alone, factors and
  accumulated scales clamped to [1e-4, 1e4]; SOC/exp/pow/PSD rows share the
  largest norm of their cone), then cost scaling c = 1/clamp(max(mean_j
  ||P_:j||_inf, ||q||_inf), 1e-4, 1e4) (c = 1 if that max is below 1e-8);
* initial point: all cones symmetric -> two solves with H = I
  ([0; b] gives x and s = -z-part, [-q; 0] gives z), then shift s and z into
  their cones; otherwise x = 0, s = z = central point, zero-cone rows 0;
  tau = kappa = 1;
* the affine right-hand side is d = (G, d_s = s, d_kappa = kappa tau);
* Delta tau uses the first form of Eq. step-direction (the second form drops
  kappa/tau from the denominator);
* eta = (W^{-T} ds_a) o (W dz_a) for symmetric cones;
* exp/pow step length: start from the largest alpha allowed by tau, kappa and
  the symmetric cones (capped at 1), multiply by 0.8 until every exp/pow cone
  is interior (and, for the combined step, inside N(beta) with the trial mu);
* N(beta) is checked on exp/pow cones only; beta = 1e-6;
* H Delta z in Delta s = -d_s - H Delta z is applied per PSD cone as
  W^T (W Delta z) = svec(R (R^T Delta Z R) R^T) (Appendix A, H = W^T W), not
  through the assembled svec block: near convergence that block has entries
  up to ~1/mu and its product loses the small eigen-directions of S; for the
  same reason W, W^{-T} and W^T in the combined-step d_s of a PSD cone are
  congruences with R and R^{-1} (the KKT matrix and its refinement residual
  keep the assembled block);
* dual infeasibility uses q^T x in the first test (printed b^T z);
* infeasibility tests use the unnormalised (homogeneous) iterates.
"""
import math

import numpy as np
import scipy.sparse as sp

from . import cones as C
from .linsys import KKTSolver

SOLVED, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, MAX_ITER, INSUFFICIENT_PROGRESS, NUMERICAL_ERROR = 1, 2, 3, 4, 5, 6
STATUS_NAMES = {0: "UNSOLVED", 1: "SOLVED", 2: "PRIMAL_INFEASIBLE", 3: "DUAL_INFEASIBLE",
                4: "MAX_ITER", 5: "INSUFFICIENT_PROGRESS", 6: "NUMERICAL_ERROR"}

EPS64 = float(np.finfo(np.float64).eps)
EPS32 = float(np.finfo(np.float32).eps)


def default_settings(factor_bits=64):
    """Defaults; the regularisation constants depend on the factor precision
    (Sec. 3.6: delta_s = sqrt(eps_32) ~ 3.45e-4 in mixed precision, 1e-8 in
    full precision).  delta_d = eps^2 is read with eps the FP64 epsilon in both
    modes: with eps_32^2 the term delta_d max|K_ii| reaches ~1e-4 once the
    scaling H grows to ~1e10, and refinement then stalls at T_max (measured
    with this oracle on a mixed-cone problem)."""
    low = factor_bits != 64
    return dict(
        eps_feas=1e-8, eps_inf=1e-8, max_iter=200, factor_bits=factor_bits,
        static_reg=math.sqrt(EPS32) if low else 1e-8,
        static_reg_dyn=EPS64 ** 2,
        dyn_reg_eps=1e-6 if low else 1e-13,
        dyn_reg_delta=1e-4 if low else 2e-7,
        ir_max_steps=10, ir_abstol=1e-12, ir_reltol=1e-12, ir_stop_ratio=0.0,
        equilibrate=True, ruiz_passes=10, scale_min=1e-4, scale_max=1e4,
        step_fraction=0.99, backtrack=0.8, nbhd_beta=1e-6, min_step=1e-10,
    )


class ProblemError(ValueError):
    pass


# --------------------------------------------------------------------------
# setup
# --------------------------------------------------------------------------
def _dense(M, shape):
    if M is None:
        return np.zeros(shape)
    if sp.issparse(M):
        return np.asarray(M.toarray(), dtype=np.float64)
    return np.asarray(M, dtype=np.float64).reshape(shape)


def _validate(Pu, q, A, b, cones):
    n, m = len(q), len(b)
    for name, v in (("P", Pu), ("q", q), ("A", A), ("b", b)):
        if not np.all(np.isfinite(v)):
            raise ProblemError("%s has a NaN or Inf" % name)
    if np.any(np.tril(Pu, -1) != 0):
        raise ProblemError("P must be upper triangular")
    total = 0
    for (t, d, a) in cones:
        if t not in C.FAMILY_NAMES or d < 0:
            raise ProblemError("bad cone")
        if t in (C.EXP, C.POW) and d != 3:
            raise ProblemError("exp/pow cones have dimension 3")
        if t == C.POW and not (0.0 < a < 1.0):
            raise ProblemError("pow exponent must be in (0, 1)")
        if t == C.SOC and d < 1:
            raise ProblemError("SOC dimension must be >= 1")
        if t == C.PSD:
            k = C.psd_order(d)
            if k > 32 or k < 1:
                raise ProblemError("PSD cones of order 1 .. 32 only")
        total += d
    if total != m:
        raise ProblemError("cone dimensions do not add up to m")
    return n, m


def reorder_cones(cones):
    """Stable reorder into zero, nonneg, SOC, exp, pow, PSD; merge all zero
    cones into one and all nonneg cones into one (Sec. 3.3 and 3.5).

    Returns (perm, merged) with new row i = old row perm[i] and merged a list
    of (type, dim, alpha, offset)."""
    offs = np.cumsum([0] + [d for (_, d, _) in cones])
    rank = {C.ZERO: 0, C.NONNEG: 1, C.SOC: 2, C.EXP: 3, C.POW: 4, C.PSD: 5}
    order = sorted(range(len(cones)), key=lambda i: (rank[cones[i][0]], i))
    perm = []
    merged = []
    for fam in (C.ZERO, C.NONNEG):
        rows = []
        for i in order:
            if cones[i][0] == fam:
                rows += list(range(offs[i], offs[i + 1]))
        if rows:
            merged.append([fam, len(rows), 0.0, len(perm)])
            perm += rows
    for i in order:
        t, d, a = cones[i]
        if t in (C.ZERO, C.NONNEG) or d == 0:
            continue
        merged.append([t, d, float(a), len(perm)])
        perm += list(range(offs[i], offs[i + 1]))
    return np.array(perm, dtype=np.int64), [tuple(c) for c in merged]


def _scale_factor(norm, st):
    if norm < 1e-8:
        return 1.0
    return min(max(1.0 / math.sqrt(norm), st["scale_min"]), st["scale_max"])


def equilibrate(P, A, q, cones, st):
    """Modified Ruiz equilibration (reading of Alg. 1 step 1).  Returns D, E, c
    with P_hat = c D P D, q_hat = c D q, A_hat = E A D, b_hat = E b."""
    n, m = P.shape[0], A.shape[0]
    D, E = np.ones(n), np.ones(m)
    if not st["equilibrate"]:
        return D, E, 1.0
    for _ in range(st["ruiz_passes"]):
        Ph = D[:, None] * P * D[None, :]
        Ah = E[:, None] * A * D[None, :]
        colx = np.maximum(np.max(np.abs(Ph), axis=0, initial=0.0), np.max(np.abs(Ah), axis=0, initial=0.0))
        rowz = np.max(np.abs(Ah), axis=1, initial=0.0)
        for (t, d, _, off) in cones:
            if t in (C.SOC, C.EXP, C.POW, C.PSD):
                rowz[off:off + d] = rowz[off:off + d].max()
        dfac = np.array([_scale_factor(v, st) for v in colx])
        efac = np.array([_scale_factor(v, st) for v in rowz])
        D = np.clip(D * dfac, st["scale_min"], st["scale_max"])
        E = np.clip(E * efac, st["scale_min"], st["scale_max"])
    Ph = D[:, None] * P * D[None, :]
    mean_col = float(np.mean(np.max(np.abs(Ph), axis=0))) if n else 0.0
    gamma = max(mean_col, float(np.max(np.abs(D * q), initial=0.0)))
    c = 1.0 if gamma < 1e-8 else 1.0 / min(max(gamma, st["scale_min"]), st["scale_max"])
    return D, E, c


# --------------------------------------------------------------------------
# the IPM
# --------------------------------------------------------------------------
def reduced_direction(ks, Ph, qh, Ah, bh, Hblk, x, tau, kappa, dx2, dz2, d, hmul=None):
    """Search direction from the reduced system (Eq. linsys_2x2) and the
    recovery formulas (Eq. step-direction, first form of Delta tau).

    ks solves K u = r with K = [P A^T; A -H]; (dx2, dz2) solve K u = [-q; b];
    d = (d_x, d_z, d_tau, d_s, d_kappa).  Delta s = -d_s - H Delta z, with
    H Delta z formed by hmul (default: the assembled Hblk times Delta z).
    Returns (Dx, Dz, Dtau, Ds, Dkappa)."""
    d_x, d_z, d_tau, d_s, d_kap = d
    n = len(x)
    sol1 = ks.solve(np.r_[d_x, -(d_z - d_s)])
    dx1, dz1 = sol1[:n], sol1[n:]
    xi = x / tau
    Pxi = Ph @ xi
    qp = qh + 2.0 * Pxi
    num = d_tau - d_kap / tau + qp @ dx1 + bh @ dz1
    den = kappa / tau + xi @ Pxi - qp @ dx2 - bh @ dz2
    Dtau = num / den
    Dx = dx1 + Dtau * dx2
    Dz = dz1 + Dtau * dz2
    Ds = -d_s - (hmul(Dz) if hmul is not None else Hblk @ Dz)
    Dkap = -(d_kap + kappa * Dtau) / tau
    return Dx, Dz, Dtau, Ds, Dkap


class Result(dict):
    __getattr__ = dict.get


def solve(P, q, A, b, cones, settings=None, record=False):
    """Solve min 1/2 x'Px + q'x s.t. Ax + s = b, s in K (Eq. P).

    P: upper triangle (dense or scipy sparse), q (n,), A (m, n), b (m,), cones:
    list of (type, dim, alpha).  Returns a Result with x, s, z in the caller's
    row order, status, iterations and per-iteration history."""
    st = default_settings((settings or {}).get("factor_bits", 64))
    if settings:
        st.update(settings)
    q = np.asarray(q, dtype=np.float64).copy()
    b = np.asarray(b, dtype=np.float64).copy()
    n, m = len(q), len(b)
    Pu = _dense(P, (n, n))
    A0 = _dense(A, (m, n))
    _validate(Pu, q, A0, b, cones)
    Pfull = np.triu(Pu) + np.triu(Pu, 1).T

    perm, K = reorder_cones(cones)
    A0 = A0[perm]
    b = b[perm]
    D, E, c = equilibrate(Pfull, A0, q, K, st)
    Ph = c * D[:, None] * Pfull * D[None, :]
    qh = c * D * q
    Ah = E[:, None] * A0 * D[None, :]
    bh = E * b
    nu = sum(C.degree(t, d) for (t, d, _, _) in K)
    symmetric = all(t in (C.ZERO, C.NONNEG, C.SOC, C.PSD) for (t, _, _, _) in K)

    def unscale(x, s, z):
        return D * x, s / E, E * z / c

    # ---------------- initial point ----------------
    ir_total = 0
    x = np.zeros(n)
    s = np.zeros(m)
    z = np.zeros(m)
    if symmetric:
        Hblk = np.eye(m)
        Kmat = np.block([[Ph, Ah.T], [Ah, -Hblk]])
        ks = KKTSolver(Kmat, n, st)
        sol = ks.solve(np.r_[np.zeros(n), bh])
        x = sol[:n].copy()
        s = -sol[n:]
        sol = ks.solve(np.r_[-qh, np.zeros(m)])
        z = sol[n:].copy()
        ir_total += ks.ir_steps
        for (t, d, _, off) in K:
            s[off:off + d] = C.shift_to_cone(t, s[off:off + d])
            z[off:off + d] = C.shift_to_cone(t, z[off:off + d])
    else:
        for (t, d, a, off) in K:
            s[off:off + d] = C.central_point(t, d, a)
            z[off:off + d] = C.central_point(t, d, a)
    tau, kappa = 1.0, 1.0

    bnorm = float(np.max(np.abs(b), initial=0.0))
    qnorm = float(np.max(np.abs(q), initial=0.0))
    history = []
    status = 0
    info = {}
    it = 0
    try:
        with np.errstate(divide="raise", invalid="raise", over="raise"):
            while True:
                # ---------------- residuals, objectives, mu (step 12 / loop head) -------
                xu, su, zu = unscale(x, s, z)
                xb, sb, zb = xu / tau, su / tau, zu / tau
                Pxb = Pfull @ xb
                r_p = -A0 @ xb - sb + b
                r_d = Pxb + A0.T @ zb + q
                xPx = xb @ Pxb
                g_p = 0.5 * xPx + q @ xb
                g_d = -0.5 * xPx - b @ zb
                mu = (s @ z + kappa * tau) / (nu + 1)
                nrp = float(np.max(np.abs(r_p), initial=0.0))
                nrd = float(np.max(np.abs(r_d), initial=0.0))
                nx = float(np.max(np.abs(xb), initial=0.0))
                ns = float(np.max(np.abs(sb), initial=0.0))
                nz = float(np.max(np.abs(zb), initial=0.0))
                gap = abs(g_p - g_d)
                info = dict(obj_primal=g_p, obj_dual=g_d, res_primal=nrp, res_dual=nrd, gap_abs=gap,
                            gap_rel=gap / max(1.0, min(abs(g_p), abs(g_d))), mu=mu, tau=tau, kappa=kappa)
                if not all(np.isfinite([mu, nrp, nrd, g_p, g_d, tau, kappa])):
                    status = NUMERICAL_ERROR
                    break
                # ---------------- termination (Eq. termination-check) ----------------
                ef = st["eps_feas"]
                if (nrp < ef * max(1.0, bnorm + nx + ns) and nrd < ef * max(1.0, qnorm + nx + nz)
                        and gap < ef * max(1.0, min(abs(g_p), abs(g_d)))):
                    status = SOLVED
                    break
                # ---------------- infeasibility (Eq. infeasibility-check) ------------
                ei = st["eps_inf"]
                btz = b @ zu
                qtx = q @ xu
                nxu = float(np.max(np.abs(xu), initial=0.0))
                nzu = float(np.max(np.abs(zu), initial=0.0))
                nsu = float(np.max(np.abs(su), initial=0.0))
                if btz < -ei and np.max(np.abs(A0.T @ zu), initial=0.0) < -ei * max(1.0, nxu + nzu) * btz:
                    status = PRIMAL_INFEASIBLE
                    break
                if (qtx < -ei and np.max(np.abs(Pfull @ xu), initial=0.0) < -ei * max(1.0, nxu) * qtx
                        and np.max(np.abs(A0 @ xu + su), initial=0.0) < -ei * max(1.0, nxu + nsu) * qtx):
                    status = DUAL_INFEASIBLE
                    break
                if it >= st["max_iter"]:
                    status = MAX_ITER
                    break

                # ---------------- step 4: scaling H per cone -----------------------
                Hblk = np.zeros((m, m))
                scal = {}
                for (t, d, a, off) in K:
                    sl = slice(off, off + d)
                    if t == C.ZERO:
                        continue
                    if t in (C.NONNEG, C.SOC, C.PSD):
                        scal[off] = C.nt_scaling(t, s[sl], z[sl])
                        Hblk[sl, sl] = scal[off]["H"]
                    else:
                        Hblk[sl, sl] = C.bfgs_scaling(t, s[sl], z[sl], mu, a)
                # ---------------- step 5: factor K ---------------------------------
                Kmat = np.block([[Ph, Ah.T], [Ah, -Hblk]])
                ks = KKTSolver(Kmat, n, st)
                sol2 = ks.solve(np.r_[-qh, bh])
                dx2, dz2 = sol2[:n], sol2[n:]
                # residual G (Eq. root_finding_G)
                Px = Ph @ x
                G1 = -(Px + Ah.T @ z + qh * tau)
                G2 = s + Ah @ x - bh * tau
                G3 = kappa + qh @ x + bh @ z + (x @ Px) / tau

                def hmul(v):
                    # H Delta z for Delta s (Eq. step-direction): the assembled blocks,
                    # except that a PSD cone applies H = W^T W in factored form,
                    # R (R^T V R) R^T (Appendix A), which keeps the small
                    # eigen-directions of S accurate once H is ill-conditioned
                    out = Hblk @ v
                    for (t, d, a, off) in K:
                        if t == C.PSD:
                            sl = slice(off, off + d)
                            out[sl] = C.psd_apply_H(scal[off]["R"], v[sl])
                    return out

                def direction(dx_, dz_, dtau_, ds_, dkap_):
                    return reduced_direction(ks, Ph, qh, Ah, bh, Hblk, x, tau, kappa, dx2, dz2,
                                             (dx_, dz_, dtau_, ds_, dkap_), hmul)

                def step_length(Ds, Dz, Dtau, Dkap, neighbourhood):
                    amax = 1.0
                    if Dtau < 0:
                        amax = min(amax, -tau / Dtau)
                    if Dkap < 0:
                        amax = min(amax, -kappa / Dkap)
                    for (t, d, a, off) in K:
                        if t in (C.NONNEG, C.SOC, C.PSD):
                            sl = slice(off, off + d)
                            amax = min(amax, C.step_length_symmetric(t, s[sl], Ds[sl]),
                                       C.step_length_symmetric(t, z[sl], Dz[sl]))
                    nonsym = [(t, d, a, off) for (t, d, a, off) in K if t in (C.EXP, C.POW)]
                    alpha = amax
                    while nonsym:
                        ok = True
                        if neighbourhood:
                            s_t, z_t = s + alpha * Ds, z + alpha * Dz
                            mu_t = (s_t @ z_t + (tau + alpha * Dtau) * (kappa + alpha * Dkap)) / (nu + 1)
                        for (t, d, a, off) in nonsym:
                            sl = slice(off, off + d)
                            sc, zc = s[sl] + alpha * Ds[sl], z[sl] + alpha * Dz[sl]
                            if not (C.in_int_primal(t, sc, a) and C.in_int_dual(t, zc, a)):
                                ok = False
                                break
                            if neighbourhood and not C.neighbourhood_ok(t, sc, zc, mu_t, st["nbhd_beta"], a):
                                ok = False
                                break
                        if ok:
                            break
                        alpha *= st["backtrack"]
                        if alpha < st["min_step"]:
                            alpha = 0.0
                            break
                    return alpha

                # ---------------- step 6: affine direction -------------------------
                ds_a = s.copy()
                Dxa, Dza, Dtaua, Dsa, Dkapa = direction(G1, G2, G3, ds_a, kappa * tau)
                # ---------------- step 7/8: affine step, sigma ----------------------
                alpha_a = step_length(Dsa, Dza, Dtaua, Dkapa, False)
                sigma = (1.0 - alpha_a) ** 3
                # ---------------- step 9: combined direction ----------------------
                ds_c = np.zeros(m)
                for (t, d, a, off) in K:
                    sl = slice(off, off + d)
                    if t == C.ZERO:
                        continue
                    if t in (C.NONNEG, C.SOC, C.PSD):
                        sc = scal[off]
                        lam = C.lam_vec(t, sc["lam"], d)
                        eta = C.jordan_prod(t, C.apply_scaling(t, sc, "WinvT", Dsa[sl]),
                                            C.apply_scaling(t, sc, "W", Dza[sl]))
                        v = C.jordan_prod(t, lam, lam) + eta - sigma * mu * C.identity(t, d)
                        ds_c[sl] = C.apply_scaling(t, sc, "WT", C.jordan_div(t, sc["lam"], v))
                    else:
                        eta = C.third_order_correction(t, z[sl], Dza[sl], Dsa[sl], a)
                        ds_c[sl] = s[sl] + sigma * mu * C.barrier_grad(t, z[sl], a) + eta
                dkap_c = kappa * tau + Dkapa * Dtaua - sigma * mu
                Dx, Dz, Dtau, Ds, Dkap = direction((1 - sigma) * G1, (1 - sigma) * G2, (1 - sigma) * G3, ds_c, dkap_c)
                # ---------------- step 10/11: combined step and update -------------
                alpha_c = step_length(Ds, Dz, Dtau, Dkap, True)
                ir_total += ks.ir_steps
                if record:
                    history.append(dict(iter=it, mu=mu, pcost=g_p, dcost=g_d, res_primal=nrp, res_dual=nrd,
                                        gap=gap, alpha_a=alpha_a, sigma=sigma, alpha_c=alpha_c,
                                        ir_steps=ks.ir_steps, dyn_hits=ks.dyn_hits, tau=tau, kappa=kappa,
                                        G1=float(np.max(np.abs(G1), initial=0.0)),
                                        G2=float(np.max(np.abs(G2), initial=0.0))))
                if alpha_c < st["min_step"]:
                    status = INSUFFICIENT_PROGRESS
                    break
                a = st["step_fraction"] * alpha_c
                x = x + a * Dx
                z = z + a * Dz
                s = s + a * Ds
                tau = tau + a * Dtau
                kappa = kappa + a * Dkap
                it += 1

    except (FloatingPointError, ValueError, ZeroDivisionError, np.linalg.LinAlgError):
        status = NUMERICAL_ERROR  # a non-finite value or a failed factorization

    # ---------------- output (un-scale, un-permute) -------------------------
    xu, su, zu = unscale(x, s, z)
    if status == PRIMAL_INFEASIBLE:
        scale = -(b @ zu)
        xo, so, zo = np.full(n, np.nan), np.full(m, np.nan), zu / scale
    elif status == DUAL_INFEASIBLE:
        scale = -(q @ xu)
        xo, so, zo = xu / scale, su / scale, np.full(m, np.nan)
    else:
        xo, so, zo = xu / tau, su / tau, zu / tau
    s_out = np.empty(m)
    z_out = np.empty(m)
    s_out[perm] = so
    z_out[perm] = zo
    return Result(x=xo, s=s_out, z=z_out, status=status, status_name=STATUS_NAMES[status],
                  iterations=it, ir_steps_total=ir_total, history=history, perm=perm, cones=K,
                  D=D, E=E, c=c, **info)

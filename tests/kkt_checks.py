"""Host-side checks of a returned solution, shared by the oracle and GPU tests.

* ``termination``: the termination test of the paper (Eq. termination-check:
  primal residual, dual residual and duality gap against eps_feas) recomputed
  in FP64 from the returned (x, s, z) of the unscaled problem (Eq. P/D).
* ``distance_bound``: for a problem of zero and nonnegative cones whose
  optimum is nondegenerate, a first-order bound on how far (x, z) lies from
  that optimum.  On the rows B that are active at the point (zero rows, and
  nonneg rows with s_i <= z_i) the KKT conditions read
      P x + A_B' z_B = -q - A_N' z_N + r_d,     A_B x = b_B - s_B + r_p,B,
  and at the optimum the same system holds with r = 0, s_B = 0, z_N = 0.  So
      |(x, z_B) - (x*, z*_B)| <= |M^-1| |(r_d - A_N' z_N, r_p,B - s_B)|,
  M = [P A_B'; A_B 0], entry by entry.  Both sides of the comparison are
  measured at the returned point; None when M is singular (a degenerate or
  non-unique optimum, where only validity is checked).
"""
import numpy as np
import scipy.sparse as sp

ZERO, NONNEG = 0, 1


def _full_P(P):
    P = sp.csc_matrix(P)
    return P + sp.triu(P, 1).T


def termination(P, q, A, b, x, s, z, eps=1e-8):
    """Returns (ok, dict) for the three tests at eps, evaluated on the host."""
    Pf = _full_P(P)
    A = sp.csc_matrix(A)
    rp = A @ x + s - b
    rd = Pf @ x + A.T @ z + q
    xPx = float(x @ (Pf @ x))
    gp = 0.5 * xPx + float(q @ x)
    gd = -0.5 * xPx - float(b @ z)
    inf = lambda v: float(np.max(np.abs(v), initial=0.0))
    d = dict(res_primal=inf(rp), res_dual=inf(rd), gap=abs(gp - gd), pcost=gp, dcost=gd,
             scale_p=max(1.0, inf(b) + inf(x) + inf(s)), scale_d=max(1.0, inf(q) + inf(x) + inf(z)),
             scale_g=max(1.0, min(abs(gp), abs(gd))))
    ok = (d["res_primal"] < eps * d["scale_p"] and d["res_dual"] < eps * d["scale_d"]
          and d["gap"] < eps * d["scale_g"])
    return ok, d


def distance_bound(P, q, A, b, cones, x, s, z, cond_max=1e10):
    """Entry-wise bounds (e_x, e_z) on |x - x*| and |z - z*| (e_z on every row:
    the first-order bound on B, |z_i| itself on N), or None (see module doc)."""
    if any(t not in (ZERO, NONNEG) for (t, _, _) in cones):
        return None
    n, m = len(q), len(b)
    Pf = _full_P(P).toarray()
    Ad = sp.csc_matrix(A).toarray()
    zero = np.concatenate([np.full(d, t == ZERO) for (t, d, _) in cones]) if cones else np.zeros(0, bool)
    B = zero | (s <= z)
    N = ~B
    AB, AN = Ad[B], Ad[N]
    M = np.block([[Pf, AB.T], [AB, np.zeros((AB.shape[0], AB.shape[0]))]])
    if M.shape[0] == 0 or np.linalg.cond(M) > cond_max:
        return None
    rp = Ad @ x + s - b
    rd = Pf @ x + Ad.T @ z + q
    v = np.r_[rd - AN.T @ z[N], rp[B] - s[B]]
    e = np.abs(np.linalg.inv(M)) @ np.abs(v)
    e_z = np.abs(z).copy()
    e_z[B] = e[n:]
    return e[:n], e_z

"""Oracle KKT solver: dense LDL^T + iterative refinement.

TEST INFRASTRUCTURE ONLY (see oracle/cones.py header).

Follows Sec. 3.6 "Solving linear systems" of the paper:
* K = [P A^T; A -H] is quasi-definite once regularised (Eq. linsys_2x2 and the
  remark after it), so an unpivoted LDL^T exists for any symmetric ordering;
* static regularisation delta = delta_s + delta_d * max_i |K_ii|, added with
  the quasi-definite signs (+ on x rows, - on z rows);
* a pivot of the wrong sign, or of magnitude <= eps_dyn, is replaced by
  sign * delta_dyn (dynamic regularisation; eps_dyn and delta_dyn are
  absolute constants, a reading: the paper scales only the static term);
* iterative refinement: x0 = (LDL^T)^{-1} b, then r = b - K x on the
  UNREGULARISED K in FP64, stop when ||r||_inf <= t_abs + t_rel ||b||_inf or
  after T_max refinement steps, else x += (LDL^T)^{-1} r.  An optional stall
  test (setting ir_stop_ratio > 0, off by default, not in the paper) also
  stops once a step has reduced ||r||_inf by less than that factor, provided
  ||r||_inf is already below the acceptance bar 1e-4 max(1, ||b||_inf).

Two factorizations are provided:
* ``ldl_factor``: the unpivoted LDL^T with dynamic regularisation, in the
  order of the matrix it is given.  Unique for a given order, so it serves as
  the element-wise reference for a factorization computed in that order.
* ``KKTSolver`` (used by the oracle IPM): the regularised K is factored by
  LAPACK's symmetric-indefinite LDL^T (Bunch-Kaufman pivoting), which solves
  K_reg u = r backward-stably for any delta.  The quantity the IPM needs is
  the refined solution of K u = r; with delta = 1e-8 on both blocks of an LP
  an unpivoted order can lose every digit of a pivot to cancellation, so the
  oracle does not depend on one.
"""
import numpy as np
import scipy.linalg as sla
from scipy.linalg import solve_triangular


def ldl_factor(Kreg, signs, eps_dyn, delta_dyn):
    """Left-looking column LDL^T of the dense symmetric Kreg (no pivoting).

    Column j: v = Kreg[j:, j] - L[j:, :j] @ (D[:j] * L[j, :j]); d_j = v[0]
    (replaced by signs[j] * delta_dyn when d_j * signs[j] <= eps_dyn);
    L[j+1:, j] = v[1:] / d_j.  Returns (L unit lower, D, number of dynamic
    regularisation hits)."""
    N = Kreg.shape[0]
    L = np.eye(N)
    D = np.zeros(N)
    hits = 0
    for j in range(N):
        v = Kreg[j:, j] - L[j:, :j] @ (D[:j] * L[j, :j])
        d = v[0]
        if d * signs[j] <= eps_dyn:
            d = signs[j] * delta_dyn
            hits += 1
        D[j] = d
        L[j + 1:, j] = v[1:] / d
    return L, D, hits


def ldl_solve(L, D, rhs):
    y = solve_triangular(L, rhs, lower=True, unit_diagonal=True)
    y = y / D
    return solve_triangular(L.T, y, lower=False, unit_diagonal=True)


def regularised(K, n, settings):
    """K + diag(+delta I_n, -delta I_m), delta = delta_s + delta_d max|K_ii|."""
    N = K.shape[0]
    signs = np.r_[np.ones(n), -np.ones(N - n)]
    maxdiag = float(np.max(np.abs(np.diag(K)))) if N else 0.0
    delta = settings["static_reg"] + settings["static_reg_dyn"] * maxdiag
    return K + np.diag(signs * delta), signs, delta


class KKTSolver:
    """Factor once per IPM iteration, solve several right-hand sides."""

    def __init__(self, K, n, settings):
        self.K = K
        self.n = n
        Kreg, signs, self.delta = regularised(K, n, settings)
        self.lu, self.d, self.perm = sla.ldl(Kreg, lower=True)
        self.Lp = self.lu[self.perm]  # unit lower triangular after row permutation
        self.dyn_hits = 0
        self.ir_max = settings["ir_max_steps"]
        self.ir_abs = settings["ir_abstol"]
        self.ir_rel = settings["ir_reltol"]
        self.ir_stop = settings.get("ir_stop_ratio", 0.0)
        self.ir_steps = 0

    def _solve_reg(self, r):
        """u = K_reg^{-1} r from K_reg = Lu d Lu^T with Lu[perm] triangular."""
        y = solve_triangular(self.Lp, r[self.perm], lower=True, unit_diagonal=True)
        # d is block diagonal with 1x1 and 2x2 blocks: solve it as a band matrix
        N = len(r)
        ab = np.zeros((3, N))
        ab[0, 1:] = np.diag(self.d, 1)
        ab[1, :] = np.diag(self.d)
        ab[2, :-1] = np.diag(self.d, -1)
        w = sla.solve_banded((1, 1), ab, y)
        u = np.empty(N)
        u[self.perm] = solve_triangular(self.Lp.T, w, lower=False, unit_diagonal=True)
        return u

    def solve(self, rhs):
        """Refinement on the unregularised K (Sec. 3.6): stop at the tolerance
        or after ir_max steps; a step that makes ||r||_inf larger is undone and
        ends the refinement (the regularised factor is no longer a contraction
        for K there); optionally stop once a step gains less than ir_stop_ratio
        and ||r||_inf is below the acceptance bar 1e-4 max(1, ||rhs||_inf)."""
        x = self._solve_reg(rhs)
        bnorm = float(np.max(np.abs(rhs))) if len(rhs) else 0.0
        prev = np.inf
        last = None
        steps = 0
        while True:
            r = rhs - self.K @ x
            rn = float(np.max(np.abs(r)))
            if last is not None and rn > prev:
                x = x - last
                break
            accept = 1e-4 * max(1.0, bnorm)
            stalled = self.ir_stop > 0 and rn <= accept and not (rn * self.ir_stop < prev)
            if not (rn > self.ir_abs + self.ir_rel * bnorm) or stalled or steps >= self.ir_max:
                break
            prev = rn
            last = self._solve_reg(r)
            x = x + last
            steps += 1
            self.ir_steps += 1
        return x

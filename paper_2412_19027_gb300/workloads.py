"""Seeded synthetic problem generators.

This module builds problem data only.  It holds none of the solver's
arithmetic, so both the CUDA path's tests and the oracle may use it.

Every problem except the MPC family is built from a chosen complementary
optimum (x*, s*, z*): x* ~ N(0, 1); for each nonnegative row, and for each
SOC / exp / pow cone, one half gets s* in the interior and z* = 0, the other
half s* = 0 and z* in the interior of the dual cone; zero-cone rows get
s* = 0 and z* ~ N(0, 1); PSD cones get S* and Z* of complementary rank from
one random orthogonal basis.  Then b = A x* + s* and q = -P x* - A^T z*, so
x*, s*, z* satisfy the KKT conditions of the problem (P)/(D) of the paper.

Cone types: 0 zero, 1 nonneg, 2 SOC, 3 exp, 4 pow, 5 PSD (svec, upper
triangle column-wise, off-diagonals times sqrt(2)).
"""
from dataclasses import dataclass, field
import math

import numpy as np
import scipy.sparse as sp

ZERO, NONNEG, SOC, EXP, POW, PSD = 0, 1, 2, 3, 4, 5


@dataclass
class Problem:
    name: str
    P: sp.csc_matrix          # upper triangle, n x n
    q: np.ndarray
    A: sp.csc_matrix          # m x n
    b: np.ndarray
    cones: list               # [(type, dim, alpha)]
    x_star: np.ndarray = None
    s_star: np.ndarray = None
    z_star: np.ndarray = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return len(self.q)

    @property
    def m(self):
        return len(self.b)

    def objective(self, x):
        Pf = self.P + sp.triu(self.P, 1).T
        return 0.5 * x @ (Pf @ x) + self.q @ x


# ----------------------------------------------------------------------------
# interior points of each cone (definitions of Sec. 2.1 of the paper)
# ----------------------------------------------------------------------------
def _soc_interior(rng, d):
    u = rng.standard_normal(d - 1)
    t = np.linalg.norm(u) * rng.uniform(1.5, 3.0) + rng.uniform(0.5, 2.0)
    return np.r_[t, u]


def _exp_primal_interior(rng):
    y = rng.uniform(0.5, 2.0)
    x = rng.uniform(-2.0, 0.5)
    return np.array([x, y, y * math.exp(x / y) + rng.uniform(0.5, 2.0)])


def _exp_dual_interior(rng):
    u = -rng.uniform(0.5, 2.0)
    v = rng.uniform(-2.0, 2.0)
    return np.array([u, v, -u * math.exp(v / u) / math.e + rng.uniform(0.5, 2.0)])


def _pow_primal_interior(rng, a):
    x, y = rng.uniform(0.5, 2.0, 2)
    return np.array([x, y, rng.uniform(-0.9, 0.9) * x ** a * y ** (1 - a)])


def _pow_dual_interior(rng, a):
    u, v = rng.uniform(0.5, 2.0, 2)
    return np.array([u, v, rng.uniform(-0.9, 0.9) * (u / a) ** a * (v / (1 - a)) ** (1 - a)])


def _svec(X):
    k = X.shape[0]
    r2 = math.sqrt(2.0)
    return np.array([X[i, j] if i == j else r2 * X[i, j] for j in range(k) for i in range(j + 1)])


def _psd_pair(rng, k):
    """S*, Z* (svec) of ranks ceil(k/2) and floor(k/2), S* Z* = 0."""
    Q, R = np.linalg.qr(rng.standard_normal((k, k)))
    Q = Q * np.sign(np.diag(R))[None, :]  # Haar-distributed orthogonal matrix
    r1 = (k + 1) // 2
    Q1, Q2 = Q[:, :r1], Q[:, r1:]
    S = Q1 @ np.diag(rng.uniform(0.5, 2.0, r1)) @ Q1.T
    Z = Q2 @ np.diag(rng.uniform(0.5, 2.0, k - r1)) @ Q2.T
    return _svec(S), _svec(Z)


def complementary_pair(rng, cones):
    """(s*, z*) for a cone list, following the construction in the module doc."""
    m = sum(d for (_, d, _) in cones)
    s = np.zeros(m)
    z = np.zeros(m)
    off = 0
    # nonneg rows and SOC/exp/pow cones: exactly half on each side
    nn_rows = [off_ for off_ in []]
    offs = []
    for (t, d, a) in cones:
        offs.append(off)
        off += d
    nn_rows = np.concatenate([np.arange(o, o + d) for (o, (t, d, _)) in zip(offs, cones) if t == NONNEG] or [np.zeros(0, int)])
    side = np.zeros(len(nn_rows), dtype=bool)
    side[rng.permutation(len(nn_rows))[: len(nn_rows) // 2]] = True
    s[nn_rows[side]] = rng.uniform(0.5, 2.0, int(side.sum()))
    z[nn_rows[~side]] = rng.uniform(0.5, 2.0, int((~side).sum()))
    for fam in (SOC, EXP, POW):
        idx = [i for i, c in enumerate(cones) if c[0] == fam]
        flip = np.zeros(len(idx), dtype=bool)
        flip[rng.permutation(len(idx))[: len(idx) // 2]] = True
        for i, primal_side in zip(idx, flip):
            t, d, a = cones[i]
            o = offs[i]
            if fam == SOC:
                v = _soc_interior(rng, d)
            elif fam == EXP:
                v = _exp_primal_interior(rng) if primal_side else _exp_dual_interior(rng)
            else:
                v = _pow_primal_interior(rng, a) if primal_side else _pow_dual_interior(rng, a)
            if primal_side:
                s[o:o + d] = v
            else:
                z[o:o + d] = v
    for i, (t, d, a) in enumerate(cones):
        o = offs[i]
        if t == ZERO:
            z[o:o + d] = rng.standard_normal(d)
        elif t == PSD:
            k = int(round((math.sqrt(8 * d + 1) - 1) / 2))
            s[o:o + d], z[o:o + d] = _psd_pair(rng, k)
    return s, z


def _sparse_columns(rng, m, n, per_col):
    """A with per_col distinct uniformly random rows per column, N(0,1) values."""
    rows = np.empty(n * per_col, dtype=np.int64)
    for j in range(n):
        rows[j * per_col:(j + 1) * per_col] = np.sort(rng.choice(m, per_col, replace=False))
    cols = np.repeat(np.arange(n), per_col)
    vals = rng.standard_normal(n * per_col)
    return sp.csc_matrix((vals, (rows, cols)), shape=(m, n))


def _finish(name, rng, P_full, A, cones, meta=None):
    n = A.shape[1]
    x = rng.standard_normal(n)
    s, z = complementary_pair(rng, cones)
    P_full = sp.csc_matrix(P_full)
    b = A @ x + s
    q = -(P_full @ x) - A.T @ z
    return Problem(name, sp.csc_matrix(sp.triu(P_full)), np.asarray(q), sp.csc_matrix(A), np.asarray(b),
                   list(cones), x, s, z, meta or {})


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
def nonneg_qp(seed=0, n=50, m=100, density=0.1, rank=5):
    """Nonnegative-cone QP: A m x n with Bernoulli(density) N(0,1) entries,
    P = M M^T with M n x rank N(0,1).  (n=50, m=100 is the small QP case.)"""
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    A = sp.csc_matrix(np.where(mask, rng.standard_normal((m, n)), 0.0))
    M = rng.standard_normal((n, rank))
    return _finish("nonneg_qp_n%d_m%d" % (n, m), rng, M @ M.T, A, [(NONNEG, m, 0.0)])


def unique_qp(seed=0, n=40, n_eq=8, n_inactive=30, rank=5):
    """QP (LP when rank = 0) with a unique, nondegenerate primal-dual optimum:
    n_eq zero rows and n - n_eq active nonneg rows (s* = 0, z* > 0) make a
    square dense Gaussian active block A_B (nonsingular with probability one),
    plus n_inactive inactive nonneg rows (s* > 0, z* = 0).  x* and z* are then
    the only optimum, so two solvers' answers can be compared entry by entry."""
    rng = np.random.default_rng(seed)
    m = n + n_inactive
    A = rng.standard_normal((m, n))
    M = rng.standard_normal((n, rank)) if rank > 0 else np.zeros((n, 1))
    x = rng.standard_normal(n)
    s = np.zeros(m)
    z = np.zeros(m)
    z[:n_eq] = rng.standard_normal(n_eq)
    z[n_eq:n] = rng.uniform(0.5, 2.0, n - n_eq)
    s[n:] = rng.uniform(0.5, 2.0, n_inactive)
    P_full = sp.csc_matrix(M @ M.T)
    b = A @ x + s
    q = -(P_full @ x) - A.T @ z
    cones = [(ZERO, n_eq, 0.0), (NONNEG, m - n_eq, 0.0)]
    return Problem("unique_qp_n%d_m%d" % (n, m), sp.csc_matrix(sp.triu(P_full)), np.asarray(q), sp.csc_matrix(A),
                   np.asarray(b), cones, x, s, z, {"active_rows": n})


def mixed_cone(seed=0, n=2000, n_zero=500, n_nonneg=3000, n_soc=500, soc_dim=5, n_exp=100, n_pow=100,
               pow_alpha=0.3, nnz_per_col=10, p_rank=10):
    """Mixed-cone QP.  Full size: n=2000, m=6600 = 500 zero + 3000 nonneg +
    500 SOC(5) + 100 exp + 100 pow(0.3); A with nnz_per_col N(0,1) entries per
    column at uniform random rows; P = diag(U(0.1, 1)) + F F^T with F
    n x p_rank, N(0,1)/sqrt(p_rank)."""
    rng = np.random.default_rng(seed)
    cones = []
    if n_zero:
        cones.append((ZERO, n_zero, 0.0))
    if n_nonneg:
        cones.append((NONNEG, n_nonneg, 0.0))
    cones += [(SOC, soc_dim, 0.0)] * n_soc + [(EXP, 3, 0.0)] * n_exp + [(POW, 3, pow_alpha)] * n_pow
    m = sum(d for (_, d, _) in cones)
    A = _sparse_columns(rng, m, n, min(nnz_per_col, m))
    F = rng.standard_normal((n, p_rank)) / math.sqrt(p_rank)
    P = np.diag(rng.uniform(0.1, 1.0, n)) + F @ F.T
    return _finish("mixed_cone_n%d_m%d" % (n, m), rng, P, A, cones)


def banded_lp(seed=0, n=200_000, m=None, n_zero=None, window=1024, diag_p=True):
    """Large sparse LP/QP: 8 nnz per column, 6 band rows 2j-2 .. 2j+3 plus 2
    rows uniform in |i - 2j| <= window; P = diag(U(0,1)) with a random half of
    the diagonal set to 0; first quarter of the rows zero cone, rest nonneg."""
    rng = np.random.default_rng(seed)
    m = 2 * n if m is None else m
    n_zero = m // 4 if n_zero is None else n_zero
    rows_l, cols_l = [], []
    j = np.arange(n)
    band = [2 * j + o for o in range(-2, 4)]
    extra = []
    for k in range(2):
        extra.append(2 * j + rng.integers(-window, window + 1, n))
    R = np.stack(band + extra, axis=1)
    R = np.clip(R, 0, m - 1)
    for jj in range(n):
        r = R[jj]
        u = np.unique(r)
        while len(u) < 8:
            u = np.unique(np.r_[u, np.clip(2 * jj + rng.integers(-window, window + 1), 0, m - 1)])
        rows_l.append(u[:8])
    rows = np.concatenate(rows_l)
    cols = np.repeat(j, 8)
    A = sp.csc_matrix((rng.standard_normal(len(rows)), (rows, cols)), shape=(m, n))
    pd = rng.uniform(0.0, 1.0, n) if diag_p else np.zeros(n)
    pd[rng.permutation(n)[: n // 2]] = 0.0
    cones = [(ZERO, n_zero, 0.0), (NONNEG, m - n_zero, 0.0)]
    return _finish("banded_lp_n%d_m%d" % (n, m), rng, sp.diags(pd), A, cones)


def psd_batch(seed=0, n=20_000, n_psd=2000, psd_k=10, n_nonneg=5000, nnz_per_col=6):
    """Batched PSD problem: n_psd PSD(psd_k) cones + n_nonneg nonneg rows,
    A with nnz_per_col N(0,1) entries per column, P = 0."""
    rng = np.random.default_rng(seed)
    d = psd_k * (psd_k + 1) // 2
    cones = [(NONNEG, n_nonneg, 0.0)] + [(PSD, d, 0.0)] * n_psd
    m = n_nonneg + n_psd * d
    A = _sparse_columns(rng, m, n, nnz_per_col)
    return _finish("psd_batch_n%d_m%d" % (n, m), rng, sp.csc_matrix((n, n)), A, cones)


def psd_mixed(seed=0, n=60, orders=(2, 3, 4, 5, 8, 10, 16), per_order=2, n_nonneg=20, nnz_per_col=5):
    """PSD cones of mixed orders (the paper's stated future direction, Sec. 6):
    `per_order` cones of each order in `orders`, interleaved, plus n_nonneg
    nonneg rows; A with nnz_per_col N(0,1) entries per column, P = 0."""
    rng = np.random.default_rng(seed)
    psd = [k for _ in range(per_order) for k in orders]
    cones = [(NONNEG, n_nonneg, 0.0)] + [(PSD, k * (k + 1) // 2, 0.0) for k in psd]
    m = sum(d for (_, d, _) in cones)
    A = _sparse_columns(rng, m, n, min(nnz_per_col, m))
    return _finish("psd_mixed_n%d_m%d" % (n, m), rng, sp.csc_matrix((n, n)), A, cones)


def mpc_qp(seed=0, T=None, nx=None, nu=None, x_bound=5.0, u_bound=1.0, u_soc=1.2, x0_scale=0.5):
    """MPC-shaped QP: states x_1..x_T, inputs u_0..u_{T-1}; x_{t+1} = A_d x_t +
    B_d u_t as zero-cone rows (A_d = G 0.95 / rho(G)); boxes |x| <= 5, |u| <= 1
    as nonneg rows; one SOC ||u_t|| <= 1.2 per step; cost sum x'x + 0.1 u'u.
    Not built from a known optimum."""
    rng = np.random.default_rng(seed)
    T = int(rng.integers(10, 51)) if T is None else T
    nx = int(rng.integers(4, 13)) if nx is None else nx
    nu = int(rng.integers(2, 5)) if nu is None else nu
    G = rng.standard_normal((nx, nx))
    Ad = G * 0.95 / max(abs(np.linalg.eigvals(G)))
    Bd = rng.standard_normal((nx, nu))
    x0 = rng.standard_normal(nx) * x0_scale
    n = T * (nx + nu)
    n_zero = T * nx
    # dynamics rows r = t nx + i: x_{t+1,i} - sum_k A_d[i,k] x_{t,k} - sum_k B_d[i,k] u_{t,k} = (A_d x0)_i if t == 0
    t_i, i_i = np.divmod(np.arange(n_zero), nx)
    r_id, c_id, v_id = np.arange(n_zero), np.arange(n_zero), np.ones(n_zero)
    ta = np.repeat(np.arange(1, T), nx * nx)
    ia = np.tile(np.repeat(np.arange(nx), nx), T - 1)
    ka = np.tile(np.tile(np.arange(nx), nx), T - 1)
    r_a, c_a, v_a = ta * nx + ia, (ta - 1) * nx + ka, -Ad[ia, ka]
    tb = np.repeat(np.arange(T), nx * nu)
    ib = np.tile(np.repeat(np.arange(nx), nu), T)
    kb = np.tile(np.tile(np.arange(nu), nx), T)
    r_b, c_b, v_b = tb * nx + ib, T * nx + tb * nu + kb, -Bd[ib, kb]
    ax0 = np.array([Ad[i] @ x0 for i in range(nx)])
    b_dyn = np.where(t_i == 0, ax0[i_i], 0.0)
    # boxes |v_j| <= ub: rows n_zero + 2j (v_j <= ub) and n_zero + 2j + 1 (-v_j <= ub)
    j = np.arange(n)
    ub = np.where(j < T * nx, x_bound, u_bound)
    r_box, c_box, v_box = n_zero + np.r_[2 * j, 2 * j + 1], np.r_[j, j], np.r_[np.ones(n), -np.ones(n)]
    b_box = np.repeat(ub, 2)
    n_nn = 2 * n
    # one SOC per step: (u_soc, u_t) in SOC(nu + 1)
    ts = np.repeat(np.arange(T), nu)
    ks = np.tile(np.arange(nu), T)
    r0 = n_zero + n_nn
    r_soc, c_soc, v_soc = r0 + ts * (nu + 1) + 1 + ks, T * nx + ts * nu + ks, -np.ones(T * nu)
    b_soc = np.zeros(T * (nu + 1))
    b_soc[:: nu + 1] = u_soc
    rows = np.r_[r_id, r_a, r_b, r_box, r_soc]
    cols = np.r_[c_id, c_a, c_b, c_box, c_soc]
    vals = np.r_[v_id, v_a, v_b, v_box, v_soc]
    b = np.r_[b_dyn, b_box, b_soc]
    m = r0 + T * (nu + 1)
    A = sp.csc_matrix((vals, (rows, cols)), shape=(m, n))
    pd = np.r_[np.full(T * nx, 2.0), np.full(T * nu, 0.2)]
    cones = [(ZERO, n_zero, 0.0), (NONNEG, n_nn, 0.0)] + [(SOC, nu + 1, 0.0)] * T
    return Problem("mpc_T%d_nx%d_nu%d" % (T, nx, nu), sp.csc_matrix(sp.diags(pd)), np.zeros(n), A,
                   np.asarray(b), cones, meta=dict(T=T, nx=nx, nu=nu))


# ----------------------------------------------------------------------------
# the paper's own benchmark classes (Sec. 5.1 quadratic programs, Sec. 5.3
# exponential cone programs), written as conic problems; not built from a known
# optimum (the oracle solves the small instances)

def portfolio_qp(seed=0, n=5000, density=0.5):
    """Portfolio optimisation (Sec. 5.1): maximise mu'x - gamma x' Sigma x s.t.
    1'x = 1, x >= 0, Sigma = F F' + D with rank p = round(0.1 n).  Conic form with
    y = F'x: variables (x, y), minimise gamma (x'Dx + y'y) - mu'x, zero rows
    F'x - y = 0 and 1'x = 1, nonnegative rows -x <= 0.  F n x p with `density`
    N(0, 1) entries, D = diag(U(0, sqrt(p))), mu ~ N(0, 1), gamma = 1."""
    rng = np.random.default_rng(seed)
    p = max(1, int(round(0.1 * n)))
    mask = rng.random((n, p)) < density
    F = sp.csc_matrix(np.where(mask, rng.standard_normal((n, p)), 0.0))
    d = rng.uniform(0.0, math.sqrt(p), n)
    mu = rng.standard_normal(n)
    gamma = 1.0
    P = sp.block_diag([sp.diags(2.0 * gamma * d), sp.identity(p) * (2.0 * gamma)], format="csc")
    q = np.r_[-mu, np.zeros(p)]
    A = sp.vstack([sp.hstack([F.T, -sp.identity(p)]),
                   sp.hstack([sp.csr_matrix(np.ones((1, n))), sp.csr_matrix((1, p))]),
                   sp.hstack([-sp.identity(n), sp.csr_matrix((n, p))])], format="csc")
    b = np.r_[np.zeros(p), 1.0, np.zeros(n)]
    cones = [(ZERO, p + 1, 0.0), (NONNEG, n, 0.0)]
    return Problem("portfolio_n%d_p%d" % (n, p), sp.csc_matrix(sp.triu(P)), q, A, b, cones,
                   meta=dict(n=n, p=p, mu=mu, F=F, d=d, gamma=gamma))


def huber_qp(seed=0, n=5000, density=0.15, T=1.0):
    """Huber fitting (Sec. 5.1): minimise sum_i phi_T(a_i'x - b_i), m = round(1.5 n),
    phi_T(t) = t^2 for |t| <= T, T (2|t| - T) otherwise.  Conic form: variables
    (x, u, r, s), minimise u'u + 2T 1'(r + s) s.t. A x - u - r + s = b (zero
    rows), r, s >= 0; at the optimum u + r - s = Ax - b with u the clipped
    residual.  A m x n with `density` N(0, 1) entries, x_true ~ N(0, 1/n),
    b = A x_true + e with e_i ~ N(0, 1/4), and U(0, 10) on 5 % of the rows."""
    rng = np.random.default_rng(seed)
    m = int(round(1.5 * n))
    mask = rng.random((m, n)) < density
    Ad = sp.csc_matrix(np.where(mask, rng.standard_normal((m, n)), 0.0))
    x_true = rng.standard_normal(n) / math.sqrt(n)
    noise = np.where(rng.random(m) < 0.95, 0.5 * rng.standard_normal(m), rng.uniform(0.0, 10.0, m))
    bd = Ad @ x_true + noise
    I = sp.identity(m, format="csc")
    Z = sp.csc_matrix((m, m))
    P = sp.block_diag([sp.csc_matrix((n, n)), 2.0 * I, Z, Z], format="csc")
    q = np.r_[np.zeros(n + m), 2.0 * T * np.ones(2 * m)]
    A = sp.vstack([sp.hstack([Ad, -I, -I, I]),
                   sp.hstack([sp.csc_matrix((m, n)), Z, -I, Z]),
                   sp.hstack([sp.csc_matrix((m, n)), Z, Z, -I])], format="csc")
    b = np.r_[bd, np.zeros(2 * m)]
    cones = [(ZERO, m, 0.0), (NONNEG, 2 * m, 0.0)]
    return Problem("huber_n%d_m%d" % (n, m), sp.csc_matrix(sp.triu(P)), q, A, b, cones,
                   meta=dict(n=n, m=m, A=Ad, b=bd, T=T))


def entropy_max(seed=0, n=2000):
    """Entropy maximisation (Sec. 5.3): maximise -sum_i x_i log x_i s.t. 1'x = 1,
    A x <= b, m = round(0.5 n), A_ij ~ N(0, n), b = A v / 1'v with v_i ~ U(0, 1)
    (so v / 1'v is feasible).  Conic form: variables (x, t), minimise -1't s.t.
    1'x = 1 (zero row), A x <= b (nonnegative rows), (t_i, x_i, 1) in K_exp for
    each i, i.e. x_i exp(t_i / x_i) <= 1, t_i <= -x_i log x_i."""
    rng = np.random.default_rng(seed)
    m = max(1, int(round(0.5 * n)))
    Ad = rng.standard_normal((m, n)) * math.sqrt(n)
    v = rng.uniform(0.0, 1.0, n)
    bd = Ad @ v / v.sum()
    rows, cols, vals = [], [], []
    for i in range(n):  # exp cone i: rows 3i, 3i + 1, 3i + 2 of the cone block
        rows += [3 * i, 3 * i + 1]
        cols += [n + i, i]
        vals += [-1.0, -1.0]
    E = sp.csc_matrix((vals, (rows, cols)), shape=(3 * n, 2 * n))
    A = sp.vstack([sp.hstack([sp.csr_matrix(np.ones((1, n))), sp.csr_matrix((1, n))]),
                   sp.hstack([sp.csr_matrix(Ad), sp.csr_matrix((m, n))]),
                   E], format="csc")
    be = np.zeros(3 * n)
    be[2::3] = 1.0
    b = np.r_[1.0, bd, be]
    q = np.r_[np.zeros(n), -np.ones(n)]
    cones = [(ZERO, 1, 0.0), (NONNEG, m, 0.0)] + [(EXP, 3, 0.0)] * n
    return Problem("entropy_n%d_m%d" % (n, m), sp.csc_matrix((2 * n, 2 * n)), q, A, b, cones,
                   meta=dict(n=n, m=m, A=Ad, b=bd))


def mpc_stream(seed=0, count=10_000):
    """Seeds and Poisson inter-arrival draws for the MPC serving stream."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(0, 2 ** 31 - 1, count)]


def cone_stress(seed, family, count, soc_dim=5, psd_k=10):
    """Strictly interior s, z and N(0,1) directions ds, dz for `count` cones of
    one family (nonneg: `count` rows; SOC of dimension soc_dim; PSD of order
    psd_k), vectorised for large counts.  Returns (cones, s, z, ds, dz)."""
    rng = np.random.default_rng(seed)
    if family == "nonneg":
        cones = [(NONNEG, count, 0.0)]
        s, z = rng.uniform(0.5, 2.0, count), rng.uniform(0.5, 2.0, count)
        m = count
    elif family == "soc":
        d = soc_dim
        cones = [(SOC, d, 0.0)] * count

        def inner():
            u = rng.standard_normal((count, d - 1))
            t = np.linalg.norm(u, axis=1) * rng.uniform(1.5, 3.0, count) + rng.uniform(0.5, 2.0, count)
            return np.concatenate([t[:, None], u], axis=1).ravel()
        s, z = inner(), inner()
        m = count * d
    elif family == "psd":
        k = psd_k
        dim = k * (k + 1) // 2
        cones = [(PSD, dim, 0.0)] * count
        iu, ju = np.triu_indices(k)  # svec order: upper triangle by columns
        order = np.lexsort((iu, ju))
        iu, ju = iu[order], ju[order]
        wgt = np.where(iu == ju, 1.0, math.sqrt(2.0))

        def inner():
            X = rng.standard_normal((count, k, k))
            M = X @ np.swapaxes(X, 1, 2) / k + 0.5 * np.eye(k)[None]
            return (M[:, iu, ju] * wgt[None, :]).ravel()
        s, z = inner(), inner()
        m = count * dim
    else:
        raise ValueError(family)
    return cones, s, z, rng.standard_normal(m), rng.standard_normal(m)


# Configurations of the measured workloads, by name.
WORKLOADS = {
    "qp_nonneg_n50_m100": lambda seed=0: nonneg_qp(seed),
    "mixed_n2000_m6600": lambda seed=0: mixed_cone(seed),
    "banded_n200000_m400000": lambda seed=0: banded_lp(seed),
    "psd2000x10_n20000": lambda seed=0: psd_batch(seed),
    "mpc": lambda seed=0: mpc_qp(seed),
}

"""Host-side tests of the C-ABI library (no GPU): exported symbols, settings,
input validation, equilibration against the oracle, and the symbolic
factorization against an explicit symbolic elimination."""
import json
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import ipm as OI
from paper_2412_19027_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def clr():
    from paper_2412_19027_gb300 import build
    build.build()
    from paper_2412_19027_gb300 import clr as mod
    mod._lib()
    return mod


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "clr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(clr_[A-Za-z_0-9]+)\s*\(", text)) - {"clr_alloc_fn", "clr_free_fn"})


def test_library_exports_every_declared_symbol(clr):
    lib = clr._lib()
    names = _declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(clr.EXPORTS)


def test_default_settings_follow_the_paper(clr):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    s64, s32 = clr.clr_default_settings(64), clr.clr_default_settings(32)
    assert s64.backtrack == g["backtrack_ratio"]["value"]
    assert s64.step_fraction == g["step_fraction"]["value"]
    assert s64.nbhd_beta == g["neighbourhood_beta"]["value"]
    assert s64.ir_max_steps == g["ir_max_steps"]["value"]
    assert s64.ir_abstol == g["ir_abstol"]["value"] and s64.ir_reltol == g["ir_reltol"]["value"]
    assert s64.static_reg == g["static_reg_full"]["value"]
    assert s32.static_reg == pytest.approx(g["static_reg_mixed"]["value"], rel=g["static_reg_mixed"]["rtol"])
    assert s64.static_reg_dyn == pytest.approx(g["static_reg_dyn"]["value"], rel=1e-12)
    # the same readings as the oracle's defaults
    for bits, s in ((64, s64), (32, s32)):
        o = oracle.default_settings(bits)
        for key in ("eps_feas", "eps_inf", "max_iter", "static_reg", "static_reg_dyn", "dyn_reg_eps",
                    "dyn_reg_delta", "ruiz_passes", "scale_min", "scale_max", "min_step"):
            assert getattr(s, key) == pytest.approx(o[key], rel=1e-15), key
    # 16: the FP32 factor with BF16 products for the large fronts, otherwise the FP32 defaults
    s16 = clr.clr_default_settings(16)
    assert s16.factor_bits == 16 and s16.static_reg == s32.static_reg and s16.dyn_reg_eps == s32.dyn_reg_eps
    for bad in (8, 0, 128):
        with pytest.raises(clr.ClrError):
            clr.clr_default_settings(bad)


def test_validation_errors(clr):
    prob = W.nonneg_qp(0)
    with pytest.raises(clr.ClrError) as e:
        clr.clr_analyze(prob.P, np.r_[prob.q[:-1], np.nan], prob.A, prob.b, prob.cones)
    assert e.value.code == -1
    with pytest.raises(clr.ClrError) as e:
        clr.clr_analyze(prob.P, prob.q, prob.A, prob.b, [(1, 99, 0.0)])
    assert e.value.code == -2
    with pytest.raises(clr.ClrError) as e:
        clr.clr_analyze(prob.P, prob.q, prob.A[:3], prob.b[:3], [(4, 3, 1.5)])
    assert e.value.code == -1


@pytest.mark.parametrize("make", [lambda: W.nonneg_qp(0),
                                  lambda: W.mixed_cone(3, n=50, n_zero=7, n_nonneg=40, n_soc=6, n_exp=4, n_pow=4,
                                                       nnz_per_col=4),
                                  lambda: W.psd_batch(0, n=40, n_psd=3, psd_k=4, n_nonneg=10, nnz_per_col=4)])
def test_equilibration_matches_oracle(clr, make):
    prob = make()
    s = clr.clr_analyze(prob.P, prob.q, prob.A, prob.b, prob.cones)
    D, E, c = s.scaling()
    st = oracle.default_settings(64)
    perm, K = OI.reorder_cones(prob.cones)
    Pu = prob.P.toarray()
    Pf = np.triu(Pu) + np.triu(Pu, 1).T
    Dr, Er, cr = OI.equilibrate(Pf, prob.A.toarray()[perm], prob.q, K, st)
    np.testing.assert_allclose(D, Dr, rtol=1e-13)
    np.testing.assert_allclose(E, Er, rtol=1e-13)
    assert c == pytest.approx(cr, rel=1e-13)
    sym = s.symbolic()
    np.testing.assert_array_equal(sym["row_perm"], perm)


def _kkt_pattern(prob, perm_rows, cones):
    """Lower pattern of K = [P A^T; A -H] with H's block structure (reordered rows)."""
    n, m = prob.n, prob.m
    Pu = sp.csc_matrix(prob.P)
    A = sp.csr_matrix(prob.A)[perm_rows]
    Hp = np.zeros((m, m), dtype=bool)
    for (t, d, a, off) in cones:
        if t in (0, 1):
            for i in range(off, off + d):
                Hp[i, i] = True
        else:
            Hp[off:off + d, off:off + d] = True
    K = np.zeros((n + m, n + m), dtype=bool)
    Pf = (Pu + Pu.T).toarray() != 0
    K[:n, :n] = Pf | np.eye(n, dtype=bool)
    K[n:, :n] = A.toarray() != 0
    K[:n, n:] = K[n:, :n].T
    K[n:, n:] = Hp
    return K


@pytest.mark.parametrize("make", [lambda: W.nonneg_qp(1),
                                  lambda: W.mixed_cone(4, n=40, n_zero=6, n_nonneg=30, n_soc=5, n_exp=3, n_pow=3,
                                                       nnz_per_col=4),
                                  lambda: W.banded_lp(2, n=80, window=8)])
def test_symbolic_factor_covers_fill(clr, make):
    prob = make()
    s = clr.clr_analyze(prob.P, prob.q, prob.A, prob.b, prob.cones)
    sym = s.symbolic()
    stats = s.symbolic_stats()
    N = stats["kkt_dim"]
    perm = sym["perm"]
    assert sorted(perm.tolist()) == list(range(N))
    _, cones = OI.reorder_cones(prob.cones)
    K = _kkt_pattern(prob, sym["row_perm"], cones)
    Kp = K[np.ix_(perm, perm)]
    # explicit symbolic elimination: column j of L = rows reached from j
    L = np.tril(Kp).copy()
    for j in range(N):
        rows = np.nonzero(L[j + 1:, j])[0] + j + 1
        for r in rows:
            L[rows[rows > r], r] = True
    snp, rp, rows = sym["sn_ptr"], sym["row_ptr"], sym["rows"]
    owner = np.empty(N, dtype=np.int64)
    for J in range(len(snp) - 1):
        owner[snp[J]:snp[J + 1]] = J
        fr = rows[rp[J]:rp[J + 1]]
        assert list(fr[: snp[J + 1] - snp[J]]) == list(range(snp[J], snp[J + 1]))  # own columns first
        assert np.all(np.diff(fr) > 0)
    for j in range(N):
        J = owner[j]
        fr = set(rows[rp[J]:rp[J + 1]].tolist())
        need = set(np.nonzero(L[:, j])[0].tolist())
        assert need <= fr, (j, need - fr)
    # every child's update rows lie in its parent's front
    par = sym["sn_parent"]
    for J in range(len(par)):
        if par[J] >= 0:
            c = snp[J + 1] - snp[J]
            upd = set(rows[rp[J] + c:rp[J + 1]].tolist())
            assert upd <= set(rows[rp[par[J]]:rp[par[J] + 1]].tolist())
        else:
            assert rp[J + 1] - rp[J] == snp[J + 1] - snp[J]  # roots have no update rows
    # nnz(L) agrees with the explicit elimination when supernodes add no explicit zeros
    assert stats["l_nnz"] >= int(np.count_nonzero(np.tril(L)))


def test_analysis_of_full_size_mixed_cone_problem(clr):
    """The 2000 dense x columns of the mixed-cone QP (P = diag + rank 10) form one
    root front (plus at most a few columns merged by relaxed amalgamation);
    the constraint rows are eliminated first."""
    prob = W.mixed_cone(0)
    s = clr.clr_analyze(prob.P, prob.q, prob.A, prob.b, prob.cones)
    st = s.symbolic_stats()
    assert st["kkt_dim"] == 8600
    assert 2000 <= st["max_front"] <= 2064
    assert st["n_levels"] <= 8
    assert st["front_pool_entries"] < 10_000_000


def _cohort_members():
    return [W.nonneg_qp(0), W.mpc_qp(1, T=12, nx=5, nu=3),
            W.mixed_cone(1, n=60, n_zero=10, n_nonneg=80, n_soc=12, n_exp=8, n_pow=8, nnz_per_col=4),
            W.psd_batch(0, n=60, n_psd=4, psd_k=4, n_nonneg=20, nnz_per_col=4), W.mpc_qp(2, T=20, nx=8, nu=2)]


def test_cohort_analysis_is_the_union_of_its_members(clr):
    """A merged cohort is block diagonal under the concatenated orders: its
    symbolic factorization is the disjoint union of the members' own (sizes,
    fill and flops add up, the level count is the largest member's)."""
    probs = _cohort_members()
    alone = []
    for p in probs:
        s = clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones)
        alone.append(s.symbolic_stats())
        s.free()
    b = clr.clr_batch_analyze([(p.P, p.q, p.A, p.b, p.cones) for p in probs])
    assert b.size() == len(probs)
    st = b.symbolic_stats()
    for key in ("n", "m", "kkt_dim", "kkt_nnz_lower", "l_nnz", "n_supernodes", "front_pool_entries"):
        assert st[key] == sum(a[key] for a in alone), key
    assert st["factor_flops"] == pytest.approx(sum(a["factor_flops"] for a in alone), rel=1e-12)
    assert st["n_levels"] == max(a["n_levels"] for a in alone)
    assert st["max_front"] == max(a["max_front"] for a in alone)
    b.free()


def test_psd_orders_mixed_and_bounded(clr):
    """PSD cones of different orders are accepted, in one problem and across a
    cohort; an order above 32 is refused (CLR_E_UNSUPPORTED)."""
    p4 = W.psd_batch(0, n=60, n_psd=4, psd_k=4, n_nonneg=20, nnz_per_col=4)
    p5 = W.psd_batch(1, n=60, n_psd=3, psd_k=5, n_nonneg=20, nnz_per_col=4)
    b = clr.clr_batch_analyze([(p.P, p.q, p.A, p.b, p.cones) for p in (p4, p5)])
    assert b.size() == 2
    b.free()
    pm = W.psd_mixed(0)
    s = clr.clr_analyze(pm.P, pm.q, pm.A, pm.b, pm.cones)
    s.free()
    k = 33
    A = sp.csc_matrix(np.ones((k * (k + 1) // 2, 1)))
    with pytest.raises(clr.ClrError) as e:
        clr.clr_analyze(sp.csc_matrix((1, 1)), np.zeros(1), A, np.zeros(A.shape[0]), [(5, A.shape[0], 0.0)])
    assert e.value.code == -3  # CLR_E_UNSUPPORTED


@pytest.mark.parametrize("make", [lambda: W.mixed_cone(0), lambda: W.psd_batch(0, n=2000, n_psd=200, n_nonneg=500),
                                  lambda: W.banded_lp(0, n=4000), lambda: W.mpc_qp(3), lambda: W.nonneg_qp(0)],
                         ids=["mixed_n2000", "psd200x10", "banded_n4000", "mpc", "qp_n50"])
def test_column_counts_match_the_symbolic_factor(clr, make):
    """The column counts that choose the ordering (elimination tree + row
    subtrees, no factor formed) give exactly the nonzeros of the factor that the
    symbolic analysis builds column by column; relaxed amalgamation only adds
    explicit zeros on top."""
    p = make()
    s = clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones)
    st = s.symbolic_stats()
    assert st["l_nnz_counted"] == st["l_nnz_exact"]
    assert st["l_nnz"] >= st["l_nnz_exact"]
    assert st["factor_flops_stored"] >= st["factor_flops"]
    s.free()


def test_cone_rows_first_order_for_sparse_random_A(clr):
    """With P = 0 and a sparse random A over many PSD blocks, AMD takes the
    degree-6 x columns first and fills the constraint block; the cone-rows-first
    candidate leaves only a dense x block and is chosen."""
    p = W.psd_batch(0, n=2000, n_psd=200, n_nonneg=500)
    st = clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones).symbolic_stats()
    assert st["ordering"] == 1
    assert st["max_front"] <= p.n  # the x block, not the constraint block
    assert st["factor_flops"] < 2 * p.n ** 3 / 3.0 * 1.5


def test_blocking_settings_validated_and_applied(clr):
    """small_front_max and amalgamation: range checks, and the amalgamation level
    changes only the supernode partition (same fill, fewer and wider fronts)."""
    p = W.mixed_cone(3, n=300, n_zero=40, n_nonneg=300, n_soc=40, n_exp=10, n_pow=10, nnz_per_col=5)
    for bad in ({"small_front_max": 300}, {"small_front_max": -1}, {"amalgamation": 3},
                {"big_front_schedule": 4}, {"big_front_schedule": -1}):
        with pytest.raises(clr.ClrError):
            clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones, clr.clr_default_settings(64, **bad))
    with pytest.raises(clr.ClrError):  # the FP64 small-front kernel holds at most 160 x 160 in shared memory
        clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones, clr.clr_default_settings(64, small_front_max=200))
    clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones, clr.clr_default_settings(32, small_front_max=200)).free()
    stats = []
    for level in (0, 1, 2):
        s = clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones, clr.clr_default_settings(64, amalgamation=level))
        stats.append(s.symbolic_stats())
        s.free()
    assert len({st["l_nnz_exact"] for st in stats}) == 1
    assert stats[0]["l_nnz"] == stats[0]["l_nnz_exact"]  # no amalgamation: no explicit zeros
    assert stats[0]["n_supernodes"] >= stats[1]["n_supernodes"] >= stats[2]["n_supernodes"]
    assert stats[2]["l_nnz"] >= stats[1]["l_nnz"] >= stats[0]["l_nnz"]


def test_large_soc_sparse_form_layout(clr):
    """SOCs of at least soc_expand_dim rows enter the KKT matrix in sparse form: two
    auxiliary rows each (kkt_dim and m grow by 2 per cone), 3 values per cone row instead
    of a packed d x d block; 0 keeps every SOC dense; a negative value is refused."""
    p = W.mixed_cone(3, n=80, n_zero=10, n_nonneg=40, n_soc=3, soc_dim=50, n_exp=0, n_pow=0, nnz_per_col=5)
    m = p.A.shape[0]
    with pytest.raises(clr.ClrError):
        clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones, clr.clr_default_settings(64, soc_expand_dim=-1))
    stats = {}
    for dim in (0, 33, 51):
        s = clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones, clr.clr_default_settings(64, soc_expand_dim=dim))
        stats[dim] = s.symbolic_stats()
        s.free()
    assert stats[0]["m"] == stats[51]["m"] == m and stats[0]["kkt_dim"] == 80 + m
    assert stats[33]["m"] == m + 6 and stats[33]["kkt_dim"] == 80 + m + 6
    # dense: 3 packed 50 x 50 blocks; sparse: 3 x 50 x 3 values plus 6 auxiliary diagonals
    assert stats[0]["kkt_nnz_lower"] - stats[33]["kkt_nnz_lower"] == 3 * (50 * 51 // 2) - (3 * 50 * 3 + 6)


def test_update_PA_validation(clr):
    """clr_update_PA on a host-analysed solver: values on the setup's patterns are
    accepted (as a matrix of that pattern or as a CSC-ordered array), a changed
    pattern or a wrong count is refused in the binding, NaN by the library."""
    prob = W.nonneg_qp(0)
    s = clr.clr_analyze(prob.P, prob.q, prob.A, prob.b, prob.cones)
    A2 = prob.A.copy()
    A2.data = A2.data * 1.5
    s.update_PA(A=A2)
    s.update_PA(P=sp.triu(prob.P * 2.0))
    s.update_PA(P=None, A=None)
    s.update_PA(A=np.ones(prob.A.nnz))
    with pytest.raises(ValueError):
        s.update_PA(A=np.ones(prob.A.nnz - 1))
    A3 = prob.A.tolil()
    A3[0, :] = 0.0
    A3[0, 0] = 1.0
    A3 = sp.csc_matrix(A3)
    A3.eliminate_zeros()
    with pytest.raises(ValueError):
        s.update_PA(A=A3)
    bad = np.ones(prob.A.nnz)
    bad[3] = np.nan
    with pytest.raises(clr.ClrError) as e:
        s.update_PA(A=bad)
    assert e.value.code == -1
    s.free()


def test_pull_lists_direct_and_sorted_agree(clr):
    """The extend-add source lists of fronts whose children contribute densely are
    placed directly by counting (per block of parent columns); the other fronts'
    by sorting (target, source) pairs.  With pull_lists_direct = 0 every list is
    sorted: the maps, and so the device arithmetic, must be the same
    (maps_digest).  The problems cover fronts with thousands of children
    (entropy, Huber, portfolio), cone blocks (PSD, SOC) and a banded LP."""
    probs = [W.entropy_max(0, n=300), W.huber_qp(0, n=300), W.portfolio_qp(0, n=400),
             W.psd_batch(0, n=1000, n_psd=100, n_nonneg=250), W.banded_lp(0, n=4000, m=8000),
             W.mixed_cone(0, n=400, n_zero=100, n_nonneg=500, n_soc=100, n_exp=20, n_pow=20)]
    for p in probs:
        d = []
        for direct in (1, 0):
            s = clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones, clr.clr_default_settings(64, pull_lists_direct=direct))
            d.append(s.symbolic_stats()["maps_digest"])
            s.free()
        assert d[0] == d[1] and d[0] != 0, p.name
    with pytest.raises(RuntimeError):
        clr.clr_analyze(probs[0].P, probs[0].q, probs[0].A, probs[0].b, probs[0].cones,
                        clr.clr_default_settings(64, pull_lists_direct=2))


def test_threaded_analysis_is_deterministic(clr):
    """A pattern large enough for the threaded host analysis (the two ordering
    candidates on two threads, a front's lists over several threads): repeated
    analyses give the same order and maps, and the sorted lists agree with them."""
    p = W.huber_qp(0, n=1800)
    d = []
    for direct in (1, 1, 0):
        s = clr.clr_analyze(p.P, p.q, p.A, p.b, p.cones, clr.clr_default_settings(64, pull_lists_direct=direct))
        st = s.symbolic_stats()
        assert 2 * st["kkt_nnz_lower"] >= 1 << 20  # the threaded ordering path
        d.append(st["maps_digest"])
        s.free()
    assert d[0] == d[1] == d[2]

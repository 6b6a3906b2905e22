"""The allocation-free dense LDL^T entry point (clr_dense_ldl_solve_noalloc).

Callers such as graph-captured code or real-time control loops cannot
allocate device memory when they solve; this entry point works in a static
device array instead.  The test calls it through the C ABI on device buffers
and compares it with the oracle's unpivoted LDL^T in the same (natural)
order -- pivots D and dynamic-regularisation hits -- and with the solution of
that factorization, on several calls in a row with different matrices (a call
cannot lean on what the previous one left in the shared array): a system of
the largest order, a smaller one, one whose pivot triggers the dynamic
regularisation, and an in-place solve (rhs and x the same buffer).  The upper
triangle of K is filled with NaN: only the lower triangle may be read.
"""
import numpy as np
import pytest

from oracle.linsys import ldl_factor, ldl_solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
clr = pytest.importorskip("paper_2412_19027_gb300.clr")

EPS, DELTA = 1e-13, 2e-7


def _system(rng, n, m):
    M = rng.standard_normal((n, n))
    P = M @ M.T / n + 0.5 * np.eye(n)
    B = rng.standard_normal((m, m))
    H = B @ B.T / m + 0.5 * np.eye(m)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.3)
    return np.block([[P, A.T], [A, -H]]), np.r_[np.ones(n), -np.ones(m)]


def _regularised_system(rng):
    """x-block pivot 3 is zero with no coupling before it: d_3 = 0 <= eps, so the
    rule replaces it by +delta (one hit)."""
    K, signs = _system(rng, 12, 9)
    K[3, :] = 0.0
    K[:, 3] = 0.0
    K[3, 15] = K[15, 3] = 0.7  # coupled to a later row only
    return K, signs


def _call(K, signs, rhs, stream, in_place=False):
    dev = torch.device("cuda:0")
    N = len(rhs)
    Kl = np.tril(K) + np.triu(np.full_like(K, np.nan), 1)  # upper triangle unreadable
    Kd = torch.tensor(Kl, dtype=torch.float64, device=dev).t().contiguous()  # column-major
    sd = torch.tensor(signs, dtype=torch.float64, device=dev)
    bd = torch.tensor(rhs, dtype=torch.float64, device=dev)
    xd = bd if in_place else torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
    Dd = torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
    hd = torch.full((1,), -1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    clr.clr_dense_ldl_solve_noalloc(Kd.data_ptr(), sd.data_ptr(), N, bd.data_ptr(), xd.data_ptr(), Dd.data_ptr(),
                                    EPS, DELTA, hd.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return xd.cpu().numpy(), Dd.cpu().numpy(), int(hd.item())


def test_noalloc_matches_oracle_ldl():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2412_19027_gb300 import build
    build.build()
    rng = np.random.default_rng(2024)
    stream = torch.cuda.Stream()
    cases = [(_system(rng, 70, 58), False),   # N = 128, the maximum
             (_system(rng, 40, 21), False),   # a smaller system after it
             (_regularised_system(rng), False),
             (_system(rng, 30, 30), True)]    # in place: rhs and x one buffer
    for (K, signs), in_place in cases:
        N = K.shape[0]
        rhs = rng.standard_normal(N)
        x, D, hits = _call(K, signs, rhs, stream, in_place)
        L, Dref, hits_ref = ldl_factor(K, signs, EPS, DELTA)
        np.testing.assert_allclose(D, Dref, rtol=1e-9)
        assert hits == hits_ref
        xref = ldl_solve(L, Dref, rhs)
        np.testing.assert_allclose(x, xref, rtol=1e-9, atol=1e-9 * np.abs(xref).max())
        if hits_ref == 0:  # without regularisation the factor is K's own
            np.testing.assert_allclose(K @ x, rhs, atol=1e-8)
    assert hits_ref == 0 and any(ldl_factor(K, s_, EPS, DELTA)[2] == 1 for (K, s_), _ in cases)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    big = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    with pytest.raises(clr.ClrError) as e:
        clr.clr_dense_ldl_solve_noalloc(big.data_ptr(), big.data_ptr(), 129, big.data_ptr(), big.data_ptr())
    assert e.value.code == -3

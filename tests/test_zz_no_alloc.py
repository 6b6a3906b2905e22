"""The allocation-free dense LDL^T entry point (clr_dense_ldl_solve_noalloc).

Callers such as graph-captured code or real-time control loops cannot
allocate device memory when they solve; this entry point works in a static
device array instead.  The test calls it through the C ABI on device buffers
and compares it with the allocating clr_ldl_solve (same natural elimination
order) on two calls in a row, the second on a different matrix, so that a
call cannot lean on what the previous one left in the shared array.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
clr = pytest.importorskip("paper_2412_19027_gb300.clr")


def _system(rng, n, m):
    M = rng.standard_normal((n, n))
    P = M @ M.T / n + 0.5 * np.eye(n)
    B = rng.standard_normal((m, m))
    H = B @ B.T / m + 0.5 * np.eye(m)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.3)
    return np.block([[P, A.T], [A, -H]]), np.r_[np.ones(n), -np.ones(m)]


def test_noalloc_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2412_19027_gb300 import build
    build.build()
    rng = np.random.default_rng(2024)
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    for n, m in ((70, 58), (40, 21)):  # N = 128 (the maximum), then a smaller system
        K, signs = _system(rng, n, m)
        N = n + m
        rhs = rng.standard_normal(N)
        x_ref, D_ref, hits_ref = clr.clr_ldl_solve(K, signs, rhs, order=np.arange(N), factor_bits=64)
        Kd = torch.tensor(K, dtype=torch.float64, device=dev).t().contiguous()  # column-major
        sd = torch.tensor(signs, dtype=torch.float64, device=dev)
        bd = torch.tensor(rhs, dtype=torch.float64, device=dev)
        xd = torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
        Dd = torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
        hd = torch.full((1,), -1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        clr.clr_dense_ldl_solve_noalloc(Kd.data_ptr(), sd.data_ptr(), N, bd.data_ptr(), xd.data_ptr(), Dd.data_ptr(),
                                        1e-13, 2e-7, hd.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        np.testing.assert_allclose(Dd.cpu().numpy(), D_ref, rtol=1e-9)
        np.testing.assert_allclose(xd.cpu().numpy(), x_ref, rtol=1e-9, atol=1e-9 * np.abs(x_ref).max())
        assert int(hd.item()) == hits_ref == 0
        np.testing.assert_allclose(K @ xd.cpu().numpy(), rhs, atol=1e-8)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    big = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    with pytest.raises(clr.ClrError) as e:
        clr.clr_dense_ldl_solve_noalloc(big.data_ptr(), big.data_ptr(), 129, big.data_ptr(), big.data_ptr())
    assert e.value.code == -3

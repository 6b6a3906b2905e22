"""The PSD step-length arithmetic of the CUDA path, compiled for the host (no GPU).

`psd_step.cuh` holds what one thread of the PSD step-length kernel computes for
one side of a cone of order <= 16: the Cholesky factor of S, X = L^{-1} dS L^{-T},
a Householder tridiagonalisation and bisection on Sturm counts for lambda_min
(Sec. 2.2: alpha = -1 / lambda_min, the cone's own ratio test).  The header is
host and device code; this test compiles it with the host compiler and checks
it against the oracle's step length (NumPy's symmetric eigenvalues) on random
cones of every order 1-16, directions that increase S (no restriction), rank-one
directions, a matrix that is not positive definite (no step) and a NaN input.
The GPU tests check the launched kernel itself.
"""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import cones as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2412_19027_gb300", "csrc", "psd_step.cuh")

SHIM = r"""
#include "psd_step.cuh"
extern "C" double step_side(const double* v, const double* dv, int k) {
  if (k <= 4) return clr::psd_step_side<4>(v, dv, k);
  if (k <= 8) return clr::psd_step_side<8>(v, dv, k);
  return clr::psd_step_side<16>(v, dv, k);
}
"""


@pytest.fixture(scope="module")
def step_side(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("psd_step")
    src, lib = d / "shim.cpp", d / "shim.so"
    src.write_text(SHIM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", os.path.dirname(HEADER), str(src), "-o",
                    str(lib)], check=True)
    so = ctypes.CDLL(str(lib))
    so.step_side.restype = ctypes.c_double
    so.step_side.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]

    def call(x, dx, k):
        x = np.ascontiguousarray(x, dtype=np.float64)
        dx = np.ascontiguousarray(dx, dtype=np.float64)
        return so.step_side(x.ctypes.data, dx.ctypes.data, k)
    return call


@pytest.mark.parametrize("k", list(range(1, 17)))
def test_psd_step_side_matches_oracle(step_side, k):
    rng = np.random.default_rng(100 + k)
    d = k * (k + 1) // 2
    for trial in range(60):
        M = rng.standard_normal((k, k))
        x = C.svec(M @ M.T + rng.uniform(1e-3, 1.0) * np.eye(k))
        dx = rng.standard_normal(d) * rng.uniform(0.01, 100.0)
        if trial % 7 == 0:  # increases S: no restriction
            dx = C.svec(np.diag(rng.uniform(0.1, 1.0, k)))
        if trial % 11 == 0:  # rank one, one negative eigenvalue
            v = rng.standard_normal(k)
            dx = C.svec(-np.outer(v, v))
        got, ref = step_side(x, dx, k), C.step_length_symmetric(C.PSD, x, dx)
        if math.isinf(ref) or math.isinf(got):
            assert math.isinf(ref) and math.isinf(got), (trial, got, ref)
        else:
            assert got == pytest.approx(ref, rel=1e-10), trial


@pytest.mark.parametrize("k", [1, 3, 10, 16])
def test_psd_step_side_no_step_cases(step_side, k):
    rng = np.random.default_rng(7 + k)
    d = k * (k + 1) // 2
    M = rng.standard_normal((k, k))
    S = M @ M.T + 0.2 * np.eye(k)
    S[k - 1, k - 1] = -5.0  # not positive definite
    assert step_side(C.svec(S), rng.standard_normal(d), k) == 0.0
    dx = rng.standard_normal(d)
    dx[0] = np.nan
    assert step_side(C.svec(M @ M.T + np.eye(k)), dx, k) == 0.0

"""Oracle: a plain, slow, FP64 CPU implementation of the paper's method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA product path (``paper_2412_19027_gb300``) never imports it and shares no
code, header, table or constant with it; the two meet only through the seeded
problem generators, which hold none of the method's arithmetic.

Modules:
  cones   cone definitions, barriers, NT and BFGS scalings, Jordan algebra,
          corrections, step lengths, neighbourhood (Sec. 2, Appendix A)
  linsys  dense LDL^T with static/dynamic regularisation + iterative
          refinement (Sec. 3.6)
  ipm     Algorithm 1 end to end (setup, loop, output)

Parity pins live in tests/test_oracle_*.py.  Parity unpinned: the exact
iteration path (initial point, equilibration and step heuristics are readings
of a silent paper) is matched GPU-vs-oracle only.
"""
from . import cones, linsys, ipm  # noqa: F401
from .ipm import solve, default_settings, STATUS_NAMES  # noqa: F401

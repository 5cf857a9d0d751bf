"""FP64 CPU oracle of the fictitious-wave CSEM gradient hot path.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline / reference legs of `bench.py` may import or execute anything in
this package.  The CUDA path shares no code with it: the two meet only through
the seeded input generators in `paper_2211_16665_gb300.workloads`, which hold
none of the method's arithmetic.

Modules
  fdtd   -- grid spacings, materials, CFL step, CPML profiles, transform
            weights, point injection / sampling, forward and adjoint runs,
            normalisation, misfit and gradient (paper Secs. 2-3), driving the
            plain-C leap-frog stepper in fdtd_oracle.c.
  basis  -- the regularised least-squares adjoint-source basis (Sec. 3.3):
            the matrix B, the exact push-through solve, a brute-force dense
            solve and the paper's conjugate-gradient (CGNR) iteration.
"""
from . import basis, fdtd  # noqa: F401

"""CPU FP64 oracle for the GKSL -> real linear ODE transformation.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import anything from this package.
It shares no code with the CUDA library (``paper_1912_01491_gb300``) and
never imports it.

Three independent routes to the same numbers (Meyerov et al., Sec. 2):

* ``brute``   -- O1: dense N x N basis matrices, the Lindbladian of
  Eqs. (L0)/(1) applied literally, M_sn = Tr(F_s L(F_n)) (tiny N).
* ``superop`` -- O2: the Lindbladian as an N^2 x N^2 superoperator in the
  matrix-unit basis, projected onto the SU(N) basis; never touches f or d.
* ``Oracle``  -- O3: the paper's formulas, Eqs. (02)-(09), in plain C loops
  (``lb_oracle.c``), with f and d obtained by multiplying sparse basis
  matrices (not by closed-form rules).  Plus classical RK4 (dense, CSR, and
  with the time-dependent Q(t) = Q0 + eps(t) Q1 of the rocked dimer).
"""
from .core import (Oracle, build_library, load_library, lowrank_csr, num_threads, rk4_csr,  # noqa: F401
                   rk4_dense, rk4_dense_td, set_threads)
from . import brute, superop  # noqa: F401

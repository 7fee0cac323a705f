"""GB300-native transformation of GKSL (Lindblad) equations into real linear
ODE systems dv/dt = (Q + R) v + K over the generalized Gell-Mann basis, and
their RK4 integration (Meyerov et al., Sec. 2 and Table 1).

The computation lives in ``liblindblad.so`` (hand-written sm_103a CUDA
behind the C ABI of ``include/lindblad.h``); ``native`` is its ctypes
binding.  Build with ``python -m paper_1912_01491_gb300.build``.
"""
from . import native  # noqa: F401
from .native import (LBError, Basis, Batch, Csr, Propagator, Server, System, pack_bf16, pack_fp32,  # noqa: F401
                     request_bytes, rho_checks, rk4_dense, rk4_workspace, sched_simulate, spectrum,
                     spectrum_density, steady_state)

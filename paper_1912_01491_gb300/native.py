"""ctypes binding of liblindblad.so (include/lindblad.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch supplies device memory (tensors' data_ptr) and streams.
If the shared library is missing this module raises: there is no CPU
fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblindblad.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ETIMEOUT, LB_EUNSUPPORTED, LB_EAGAIN = range(7)
LB_F, LB_D = 0, 1
LB_FP64, LB_FP32, LB_BF16 = 0, 1, 2
LB_SYS_A, LB_SYS_Q, LB_SYS_R, LB_SYS_K = 0, 1, 2, 3
LB_DENSE, LB_CSR = 0, 1
LB_FORM_RK4, LB_FORM_PROPAGATOR = 0, 1
FORMATS = {"dense": LB_DENSE, "csr": LB_CSR}
LB_A_DENSE, LB_A_LOWRANK = 0, 1
PHASES = ("alloc", "h2d", "kernels", "d2h", "free")
PRECISIONS = {"fp64": LB_FP64, "fp32": LB_FP32, "bf16": LB_BF16}
LB_ALG_JOIN, LB_ALG_CLOSED = 0, 1
ALGORITHMS = {"join": LB_ALG_JOIN, "closed": LB_ALG_CLOSED}

_c_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)

LB_REQ_QUEUED, LB_REQ_RUNNING, LB_REQ_ASSEMBLED, LB_REQ_DONE, LB_REQ_FAILED, LB_REQ_CANCELLED = range(6)
LB_ENGINE_CLUSTER, LB_ENGINE_STREAM = 0, 1


class LbRequest(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("precision", ctypes.c_int), ("correct_every", ctypes.c_int),
                ("dt", ctypes.c_double), ("nsteps", ctypes.c_int64), ("H", ctypes.c_void_p),
                ("a", ctypes.c_void_p), ("v0", ctypes.c_void_p), ("v_out", ctypes.c_void_p),
                ("stream", ctypes.c_void_p)]


class LbKossakowski(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_void_p), ("nP", ctypes.c_int), ("gamma", ctypes.c_void_p),
                ("lp_ptr", ctypes.c_void_p), ("lp_idx", ctypes.c_void_p), ("lp_val", ctypes.c_void_p)]


class LbResult(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("engine", ctypes.c_int),
                ("cluster", ctypes.c_int), ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("gpu_ms", ctypes.c_double)]

_lib = None


class LBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("liblindblad error %d: %s" % (code, msg))
        self.code = code


def load():
    """Load liblindblad.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "liblindblad.so is not built (%s); run `python -m paper_1912_01491_gb300.build` "
            "or __graft_entry__.build() -- there is no CPU fallback" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "lb_last_error": (ctypes.c_char_p, []),
        "lb_version": (ctypes.c_int, []),
        "lb_basis_create": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
        "lb_basis_destroy": (ctypes.c_int, [_vp]),
        "lb_basis_dims": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), _i64p, _i64p]),
        "lb_basis_label": (ctypes.c_int, [_vp, _c_i64, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
        "lb_structure_count": (ctypes.c_int, [_vp, ctypes.c_int, _i64p]),
        "lb_structure_export": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _c_i64, _i64p, _vp]),
        "lb_structure_export_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _c_i64, _i64p, _vp]),
        "lb_join_terms": (ctypes.c_int, [_vp, _i64p]),
        "lb_expand": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "lb_rho": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "lb_assemble_dense": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "lb_assemble_dense_ex": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
        "lb_pack_fp32": (ctypes.c_int, [_c_i64, _vp, _vp, _vp]),
        "lb_pack_bf16": (ctypes.c_int, [_c_i64, _vp, _vp, _vp, _vp]),
        "lb_rk4_workspace_bytes": (ctypes.c_size_t, [_c_i64]),
        "lb_steady_workspace_bytes": (ctypes.c_size_t, [_c_i64, ctypes.c_int]),
        "lb_steady_pc_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, _c_i64, ctypes.c_int]),
        "lb_steady_state_pc": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, _vp, ctypes.c_double, ctypes.c_int,
                                              ctypes.c_int, _vp, _vp, _vp, _vp]),
        "lb_steady_state": (ctypes.c_int, [_c_i64, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp,
                                           ctypes.POINTER(ctypes.c_int), _vp, _vp]),
        "lb_rho_checks_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int]),
        "lb_rho_checks": (ctypes.c_int, [_vp, _vp, _c_i64, ctypes.c_double, _vp, _vp, _vp]),
        "lb_propagator_workspace_bytes": (ctypes.c_size_t, [_c_i64, ctypes.c_int, ctypes.c_int]),
        "lb_propagator_form": (ctypes.c_int, [_c_i64, ctypes.c_int, _vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp,
                                              _vp, _vp]),
        "lb_propagate": (ctypes.c_int, [_c_i64, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int, _vp,
                                        ctypes.c_double, _c_i64, _vp, _c_i64, _vp, _vp]),
        "lb_rk4_dense": (ctypes.c_int, [_c_i64, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp, _vp,
                                        ctypes.c_double, _c_i64, _vp, _c_i64, _vp, _vp]),
        "lb_assemble": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(LbKossakowski), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(_vp)]),
        "lb_system_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), _i64p, _i64p]),
        "lb_system_timings": (ctypes.c_int, [_vp, _dp]),
        "lb_system_get_csr": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "lb_host_release": (ctypes.c_int, []),
        "lb_expand_host": (ctypes.c_int, [_vp, _vp, _vp]),
        "lb_rho_host": (ctypes.c_int, [_vp, _vp, _vp]),
        "lb_system_destroy": (ctypes.c_int, [_vp]),
        "lb_system_get": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
        "lb_spectrum": (ctypes.c_int, [_vp, _c_i64, _vp, _vp]),
        "lb_system_spectrum": (ctypes.c_int, [_vp, _vp]),
        "lb_spectrum_density": (ctypes.c_int, [_vp, _c_i64, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
        "lb_system_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
        "lb_system_load": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.POINTER(_vp)]),
        "lb_integrate_resume": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_double, _c_i64]),
        "lb_integrate": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_double,
                                        ctypes.c_double, _c_i64, _vp]),
        "lb_assemble_lowrank_csr": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp,
                                                   ctypes.POINTER(_vp), _vp]),
        "lb_csr_info": (ctypes.c_int, [_vp, _i64p, _i64p, _i64p]),
        "lb_csr_arrays": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "lb_csr_copy": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
        "lb_csr_destroy": (ctypes.c_int, [_vp]),
        "lb_rk4_csr": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_double, _c_i64, _vp, _vp]),
        "lb_rk4_csr_td": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_double, ctypes.c_double, _vp,
                                         ctypes.c_double, _c_i64, _vp, _vp]),
        "lb_batch_create": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
        "lb_batch_set": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
        "lb_batch_assemble": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
        "lb_batch_set_cluster": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
        "lb_batch_set_precision": (ctypes.c_int, [_vp, ctypes.c_int]),
        "lb_batch_tune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _vp, _vp]),
        "lb_batch_integrate": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, _c_i64, _vp,
                                              ctypes.POINTER(ctypes.c_float)]),
        "lb_batch_set_form": (ctypes.c_int, [_vp, ctypes.c_int]),
        "lb_batch_form_propagator": (ctypes.c_int, [_vp, ctypes.c_double, _vp, ctypes.POINTER(ctypes.c_float)]),
        "lb_batch_system": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _i64p]),
        "lb_batch_copy_system": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
        "lb_batch_destroy": (ctypes.c_int, [_vp]),
        "lb_request_bytes": (_c_i64, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "lb_server_create": (ctypes.c_int, [_c_i64, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_vp)]),
        "lb_server_set_cluster": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
        "lb_submit": (ctypes.c_int, [_vp, ctypes.POINTER(LbRequest), ctypes.POINTER(ctypes.c_uint64)]),
        "lb_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(LbResult)]),
        "lb_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(LbResult)]),
        "lb_server_stats": (ctypes.c_int, [_vp, _dp, _dp, _dp, _i64p]),
        "lb_server_reset_stats": (ctypes.c_int, [_vp]),
        "lb_server_destroy": (ctypes.c_int, [_vp]),
        "lb_sched_simulate": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _c_i64, ctypes.c_int, ctypes.c_double,
                                             _vp, _vp]),
        "lb_launch_count": (ctypes.c_longlong, []),
        "lb_assemble_dense_timed": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp,
                                                   ctypes.POINTER(ctypes.c_float)]),
        "lb_assemble_kernel_count": (ctypes.c_int, []),
        "lb_assemble_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
        "lb_probe_fp64": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names the binding declares (each must be exported by the library)."""
    load()
    return [n for n in dir(_lib) if n.startswith("lb_")]


def launch_count():
    """Kernels launched by liblindblad.so in this process."""
    return int(load().lb_launch_count())


def probe_fp64_tflops():
    """Measured FP64 FMA throughput of the current device (TFLOP/s)."""
    out = ctypes.c_double()
    _check(load().lb_probe_fp64(ctypes.byref(out)))
    return out.value


def _check(rc):
    if rc != LB_OK:
        raise LBError(rc, load().lb_last_error().decode(errors="replace"))


def _ptr(t):
    """Device (or host) address of a torch tensor / numpy array, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _f64(t):
    """float64 view of a complex128 tensor (interleaved re, im)."""
    import torch
    if t.dtype == torch.complex128:
        return torch.view_as_real(t)
    return t


def export_capacity(idx, val):
    """Capacity in triples of caller buffers for a structure export: idx a
    contiguous int32 CUDA tensor of shape (n, 3), val a contiguous float64 CUDA
    tensor; the smaller of the two counts.  Raises ValueError otherwise, before
    anything reaches the library (the C entry point receives one capacity for
    both buffers and cannot check them itself)."""
    import torch
    for name, t, dt in (("idx", idx, torch.int32), ("val", val, torch.float64)):
        if not hasattr(t, "device") or not hasattr(t, "dtype"):
            raise ValueError("%s must be a torch tensor" % name)
        if t.device.type != "cuda":
            raise ValueError("%s must be a CUDA tensor, got %s" % (name, t.device))
        if t.dtype != dt:
            raise ValueError("%s must be %s, got %s" % (name, dt, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if idx.dim() != 2 or idx.shape[1] != 3:
        raise ValueError("idx must have shape (n, 3), got %s" % (tuple(idx.shape),))
    if val.dim() != 1:
        raise ValueError("val must be one-dimensional, got %s" % (tuple(val.shape),))
    return min(int(val.numel()), int(idx.shape[0]))


class Basis:
    """Device index tables of the SU(N) basis (lb_basis_create)."""

    def __init__(self, N, stream=None):
        lib = load()
        h = _vp()
        _check(lib.lb_basis_create(int(N), _stream(stream), ctypes.byref(h)))
        self._h = h
        n = ctypes.c_int()
        M = _c_i64()
        P = _c_i64()
        _check(lib.lb_basis_dims(h, ctypes.byref(n), ctypes.byref(M), ctypes.byref(P)))
        self.N, self.M, self.P = n.value, M.value, P.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().lb_basis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def label(self, i):
        t = ctypes.create_string_buffer(2)
        j = ctypes.c_int()
        k = ctypes.c_int()
        _check(load().lb_basis_label(self._h, int(i), t, ctypes.byref(j), ctypes.byref(k)))
        return t.value.decode(), j.value, k.value

    def structure_count(self, which):
        n = _c_i64()
        _check(load().lb_structure_count(self._h, {"f": LB_F, "d": LB_D}[which], ctypes.byref(n)))
        return n.value

    def structure(self, which, stream=None):
        """Kernel (a): canonical sorted nonzero (idx int32 (n,3), val float64) on the device."""
        import torch
        w = {"f": LB_F, "d": LB_D}[which]
        n = self.structure_count(which)
        idx = torch.empty((max(n, 1), 3), dtype=torch.int32, device="cuda")
        val = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
        got = _c_i64()
        _check(load().lb_structure_export(self._h, w, _ptr(idx), _ptr(val), n, ctypes.byref(got),
                                          _stream(stream)))
        return idx[:n], val[:n]

    def structure_into(self, which, idx, val, stream=None):
        """Kernel (a) into caller-owned device buffers idx (int32, >= 3 nnz
        entries) and val (float64, >= nnz) through the entry point that
        allocates no device memory (N <= 256).  Returns nnz."""
        w = {"f": LB_F, "d": LB_D}[which]
        cap = export_capacity(idx, val)
        got = _c_i64()
        _check(load().lb_structure_export_noalloc(self._h, w, _ptr(idx), _ptr(val), cap,
                                                  ctypes.byref(got), _stream(stream)))
        return got.value

    def assemble_dense_timed(self, a, h=None, A=None, K=None, algorithm="closed", stream=None):
        """Dense assembly into preallocated A (and K); returns {kernel name: ms}."""
        lib = load()
        n = lib.lb_assemble_kernel_count()
        ms = (ctypes.c_float * n)()
        _check(lib.lb_assemble_dense_timed(self._h, _ptr(h), _ptr(a), _ptr(A), None, None, _ptr(K),
                                           ALGORITHMS[algorithm], _stream(stream), ms))
        return {lib.lb_assemble_kernel_name(i).decode(): float(ms[i]) for i in range(n)}

    def join_terms(self):
        W = _c_i64()
        _check(load().lb_join_terms(self._h, ctypes.byref(W)))
        return W.value

    def expand(self, A, stream=None):
        """Eq. (02) for an N x N complex128 device tensor -> M complex128 coefficients."""
        import torch
        assert A.dtype == torch.complex128 and A.is_contiguous() and A.shape == (self.N, self.N)
        coef = torch.empty(self.M, dtype=torch.complex128, device=A.device)
        _check(load().lb_expand(self._h, _ptr(A), _ptr(coef), _stream(stream)))
        return coef

    def rho(self, v, stream=None):
        import torch
        assert v.dtype == torch.float64 and v.is_contiguous() and v.numel() == self.M
        out = torch.empty((self.N, self.N), dtype=torch.complex128, device=v.device)
        _check(load().lb_rho(self._h, _ptr(v), _ptr(out), _stream(stream)))
        return out

    def expand_host(self, A):
        """Eq. (02) from a host N x N complex array (lb_expand_host) -> M complex (numpy)."""
        A = np.ascontiguousarray(A, np.complex128)
        assert A.shape == (self.N, self.N)
        coef = np.zeros(self.M, np.complex128)
        _check(load().lb_expand_host(self._h, _ptr(A), _ptr(coef)))
        return coef

    def rho_host(self, v):
        """Eq. (rho) from a host M-vector (lb_rho_host) -> N x N complex (numpy)."""
        v = np.ascontiguousarray(v, np.float64)
        assert v.shape == (self.M,)
        out = np.zeros((self.N, self.N), np.complex128)
        _check(load().lb_rho_host(self._h, _ptr(v), _ptr(out)))
        return out

    def assemble_dense(self, a, h=None, A=True, Q=False, R=False, K=True, algorithm="closed", stream=None):
        """Dense Q, R, K (Eqs. (07)-(09)).  a: M x M complex128 device tensor.

        A, Q, R, K may be True (allocate), False/None (skip) or a preallocated
        float64 tensor.  Returns dict of the requested outputs."""
        import torch
        M = self.M
        assert a.dtype == torch.complex128 and a.is_contiguous() and a.shape == (M, M)
        if h is not None:
            assert h.dtype == torch.float64 and h.is_contiguous() and h.numel() == M
        out = {}
        for name, want, shape in (("A", A, (M, M)), ("Q", Q, (M, M)), ("R", R, (M, M)), ("K", K, (M,))):
            if want is True:
                out[name] = torch.empty(shape, dtype=torch.float64, device=a.device)
            elif want is not None and want is not False:
                out[name] = want
        _check(load().lb_assemble_dense_ex(self._h, _ptr(h), _ptr(a), _ptr(out.get("A")), _ptr(out.get("Q")),
                                           _ptr(out.get("R")), _ptr(out.get("K")), ALGORITHMS[algorithm],
                                           _stream(stream)))
        return out


def pack_fp32(A, out=None, stream=None):
    import torch
    M = A.shape[0]
    out = torch.empty((M, M), dtype=torch.float32, device=A.device) if out is None else out
    _check(load().lb_pack_fp32(M, _ptr(A), _ptr(out), _stream(stream)))
    return out


def pack_bf16(A, out=None, scale=None, stream=None):
    import torch
    M = A.shape[0]
    out = torch.empty((M, M), dtype=torch.int16, device=A.device) if out is None else out
    scale = torch.empty(M, dtype=torch.float32, device=A.device) if scale is None else scale
    _check(load().lb_pack_bf16(M, _ptr(A), _ptr(out), _ptr(scale), _stream(stream)))
    return out, scale


def rk4_workspace(M, device="cuda"):
    import torch
    n = load().lb_rk4_workspace_bytes(M)
    return torch.empty(n, dtype=torch.uint8, device=device)


def rk4_dense(Ap, K, v, dt, nsteps, precision="fp64", scale=None, A64=None, correct_every=0,
              snap_every=0, work=None, stream=None):
    """Classical RK4 on device; v (float64, M) is updated in place.  Returns snapshots or None."""
    import torch
    M = v.numel()
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    work = rk4_workspace(M, v.device) if work is None else work
    snaps = None
    if snap_every:
        snaps = torch.empty((nsteps // snap_every, M), dtype=torch.float64, device=v.device)
    _check(load().lb_rk4_dense(M, p, _ptr(Ap), _ptr(scale), _ptr(A64), int(correct_every), _ptr(K), _ptr(v),
                               float(dt), int(nsteps), _ptr(snaps), int(snap_every), _ptr(work),
                               _stream(stream)))
    return snaps


def steady_state(A, K, v=None, tol=1e-12, max_iter=2000, restart=0, stream=None, basis=None, H=None, sigma=-1.0):
    """FP64 solve of A v = -K on the device (restarted GMRES, lb_steady_state;
    with basis and H, a device N x N complex128 Hamiltonian, preconditioned
    from H's eigenbasis: lb_steady_state_pc).  Returns (v, true relative
    residual, iterations)."""
    import torch
    M = A.shape[0]
    v = torch.zeros(M, dtype=torch.float64, device=A.device) if v is None else v
    res, it = ctypes.c_double(), ctypes.c_int()
    if H is None:
        work = torch.empty(load().lb_steady_workspace_bytes(M, int(restart)), dtype=torch.uint8, device=A.device)
        _check(load().lb_steady_state(M, _ptr(A), _ptr(K), _ptr(v), float(tol), int(max_iter), int(restart),
                                      ctypes.byref(res), ctypes.byref(it), _ptr(work), _stream(stream)))
    else:
        assert basis is not None and H.dtype == torch.complex128 and H.is_contiguous()
        n = load().lb_steady_pc_workspace_bytes(basis.N, M, int(restart))
        if n == 0:
            raise LBError(LB_EINVAL, "bad preconditioned steady-state arguments")
        work = torch.empty(n + 256, dtype=torch.uint8, device=A.device)
        off = (-work.data_ptr()) % 256
        _check(load().lb_steady_state_pc(basis.handle, _ptr(A), _ptr(K), _ptr(H), float(sigma), _ptr(v), float(tol),
                                         int(max_iter), int(restart), ctypes.byref(res), ctypes.byref(it),
                                         ctypes.c_void_p(work.data_ptr() + off), _stream(stream)))
    return v, res.value, it.value


def rho_checks(basis, V, psd_shift=1e-10, stream=None):
    """(Tr rho - 1, max |rho - rho^dagger|, smallest Cholesky pivot of rho +
    psd_shift 1) for each state (rows of V), computed on the device."""
    import torch
    V = V.reshape(-1, basis.M)
    assert V.dtype == torch.float64 and V.is_contiguous()
    out = np.zeros((V.shape[0], 3))
    work = torch.empty(load().lb_rho_checks_workspace_bytes(basis.N), dtype=torch.uint8, device=V.device)
    _check(load().lb_rho_checks(basis.handle, _ptr(V), V.shape[0], float(psd_shift), _ptr(out), _ptr(work),
                                _stream(stream)))
    return out


def spectrum(A, stream=None):
    """Eigenvalues of the dense FP64 matrix A (device tensor, M x M) as a
    complex128 device tensor of length M (lb_spectrum; Sec. 6, Fig. 5)."""
    import torch
    assert A.dtype == torch.float64 and A.is_contiguous() and A.dim() == 2 and A.shape[0] == A.shape[1]
    w = torch.empty(A.shape[0], dtype=torch.complex128, device=A.device)
    _check(load().lb_spectrum(_ptr(A), A.shape[0], _ptr(w), _stream(stream)))
    return w


def spectrum_density(eig, box, nre=100, nim=100, stream=None):
    """Eigenvalues per unit area on an nre x nim grid over box = (re_lo,
    re_hi, im_lo, im_hi) (lb_spectrum_density): a float64 device tensor
    (nre, nim), the real part along the rows."""
    import torch
    assert eig.dtype == torch.complex128 and eig.is_contiguous()
    b = np.ascontiguousarray(box, np.float64)
    d = torch.empty((nre, nim), dtype=torch.float64, device=eig.device)
    _check(load().lb_spectrum_density(_ptr(eig), eig.numel(), _ptr(b), int(nre), int(nim), _ptr(d), _stream(stream)))
    return d


class Propagator:
    """Propagator form of RK4 for one dense system (lb_propagator_form /
    lb_propagate): D' = (P(hA) - 1)/h and c' for step dt, then steps of
    several states at once.  A64, K: device FP64 tensors.  precision "fp64"
    (D' in FP64) or "fp32" (D' from fl32(A64), kept with D' - A for the FP64
    correction)."""

    def __init__(self, A64, K, dt, precision="fp64", nrhs=1, stream=None):
        import torch
        M = A64.shape[0]
        self.M, self.dt, self.precision, self.nrhs = M, float(dt), precision, int(nrhs)
        p = PRECISIONS[precision]
        n = load().lb_propagator_workspace_bytes(M, self.nrhs, p)
        if n == 0:
            raise LBError(LB_EINVAL, "bad propagator arguments")
        self.work = torch.empty(n, dtype=torch.uint8, device=A64.device)
        self.A64 = A64
        self.cp = torch.empty(M, dtype=torch.float64, device=A64.device)
        if precision == "fp64":
            self.D = torch.empty((M, M), dtype=torch.float64, device=A64.device)
            self.R32 = None
            A32 = None
        else:
            A32 = pack_fp32(A64, stream=stream)
            self.D = torch.empty((M, M), dtype=torch.float32, device=A64.device)
            self.R32 = torch.empty((M, M), dtype=torch.float32, device=A64.device)
        _check(load().lb_propagator_form(M, p, _ptr(A64), _ptr(A32), _ptr(K), self.dt, _ptr(self.D), _ptr(self.R32),
                                         _ptr(self.cp), _ptr(self.work), _stream(stream)))

    def step(self, V, nsteps, correct_every=0, snap_every=0, stream=None):
        """Advance V (float64 device tensor, nrhs x M or M) in place; returns snapshots or None."""
        import torch
        R = 1 if V.dim() == 1 else V.shape[0]
        assert V.dtype == torch.float64 and V.is_contiguous() and V.numel() == R * self.M and R <= self.nrhs
        snaps = None
        if snap_every:
            snaps = torch.empty((nsteps // snap_every, R, self.M), dtype=torch.float64, device=V.device)
        _check(load().lb_propagate(self.M, R, PRECISIONS[self.precision], _ptr(self.D), _ptr(self.R32),
                                   _ptr(self.A64) if correct_every else None, _ptr(self.cp), int(correct_every),
                                   _ptr(V), self.dt, int(nsteps), _ptr(snaps), int(snap_every), _ptr(self.work),
                                   _stream(stream)))
        return snaps


class Csr:
    """Sparse system A = Q + R (CSR) and K on the device (lb_assemble_lowrank_csr).

    h: M float64 device tensor or None; channels: list of (gamma, idx, values)
    with idx an int64 device tensor and values a complex128 device tensor."""

    def __init__(self, basis, h=None, channels=(), stream=None):
        import torch
        lib = load()
        gam = np.array([float(g) for g, _, _ in channels], np.float64)
        ptr = np.zeros(len(channels) + 1, np.int64)
        for p, (_, idx, _) in enumerate(channels):
            ptr[p + 1] = ptr[p] + idx.numel()
        dev = "cuda"
        if channels:
            idx = torch.cat([i.to(torch.int64) for _, i, _ in channels]).contiguous()
            val = torch.cat([v.to(torch.complex128) for _, _, v in channels]).contiguous()
        else:
            idx = torch.zeros(1, dtype=torch.int64, device=dev)
            val = torch.zeros(1, dtype=torch.complex128, device=dev)
        self._keep = (idx, val)
        hdl = _vp()
        _check(lib.lb_assemble_lowrank_csr(basis.handle, _ptr(h), len(channels), _ptr(gam), _ptr(ptr), _ptr(idx),
                                           _ptr(val), ctypes.byref(hdl), _stream(stream)))
        self._h = hdl
        M, nnz, terms = _c_i64(), _c_i64(), _c_i64()
        _check(lib.lb_csr_info(hdl, ctypes.byref(M), ctypes.byref(nnz), ctypes.byref(terms)))
        self.M, self.nnz, self.terms = M.value, nnz.value, terms.value

    def close(self):
        if self._h:
            load().lb_csr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def to_host(self):
        """(rowptr int64, col int32, val float64, K float64) as numpy arrays."""
        rp = np.zeros(self.M + 1, np.int64)
        col = np.zeros(max(self.nnz, 1), np.int32)
        val = np.zeros(max(self.nnz, 1), np.float64)
        K = np.zeros(self.M, np.float64)
        _check(load().lb_csr_copy(self._h, _ptr(rp), _ptr(col), _ptr(val), _ptr(K), None))
        return rp, col[:self.nnz], val[:self.nnz], K

    def rk4_td(self, Q1, v, dt, nsteps, seg_start, seg_eps, period, t0=0.0, work=None, stream=None):
        """FP64 RK4 of dv/dt = (A + eps(t) Q1) v + K, eps periodic and
        piecewise constant (lb_rk4_csr_td); v updated in place."""
        work = rk4_workspace(self.M, v.device) if work is None else work
        ss = np.ascontiguousarray(seg_start, np.float64)
        se = np.ascontiguousarray(seg_eps, np.float64)
        assert len(ss) == len(se)
        _check(load().lb_rk4_csr_td(self._h, Q1._h, len(ss), _ptr(ss), _ptr(se), float(period), float(t0), _ptr(v),
                                    float(dt), int(nsteps), _ptr(work), _stream(stream)))

    def rk4(self, v, dt, nsteps, precision="fp64", correct_every=0, work=None, stream=None):
        """RK4 on the CSR system; v (float64 device tensor) updated in place."""
        work = rk4_workspace(self.M, v.device) if work is None else work
        _check(load().lb_rk4_csr(self._h, PRECISIONS[precision], int(correct_every), _ptr(v), float(dt),
                                 int(nsteps), _ptr(work), _stream(stream)))


class Batch:
    """Batched realizations of mixed N (lb_batch_*).  Inputs are torch tensors
    on the device, kept alive by this object."""

    def __init__(self, Ns):
        Ns = np.ascontiguousarray(np.asarray(Ns, dtype=np.int32))
        h = _vp()
        _check(load().lb_batch_create(len(Ns), _ptr(Ns), ctypes.byref(h)))
        self._h = h
        self.Ns = [int(n) for n in Ns]
        self.Ms = [n * n - 1 for n in self.Ns]
        self._keep = {}

    def close(self):
        if self._h:
            load().lb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set(self, r, a, h, v):
        self._keep[r] = (a, h, v)
        _check(load().lb_batch_set(self._h, int(r), _ptr(a), _ptr(h), _ptr(v)))

    def assemble(self, algorithm="closed", stream=None):
        _check(load().lb_batch_assemble(self._h, ALGORITHMS[algorithm], _stream(stream)))

    def set_cluster(self, r, C):
        _check(load().lb_batch_set_cluster(self._h, int(r), int(C)))

    def set_precision(self, precision):
        """"fp32" (default) or "fp64" for integrate and tune."""
        _check(load().lb_batch_set_precision(self._h, PRECISIONS[precision]))

    def set_form(self, form):
        """"rk4" (default: four stages per step) or "propagator" (one product
        per step with D' = (P(hA) - 1)/h)."""
        _check(load().lb_batch_set_form(self._h, {"rk4": LB_FORM_RK4, "propagator": LB_FORM_PROPAGATOR}[form]))

    def form_propagator(self, dt, stream=None):
        """Form D' and c' for step dt now; returns the device time (ms)."""
        ms = ctypes.c_float()
        _check(load().lb_batch_form_propagator(self._h, float(dt), _stream(stream), ctypes.byref(ms)))
        return ms.value

    def tune(self, width=6, probe_steps=20, dt=1e-3, stream=None):
        choice = np.zeros(len(self.Ns), np.int32)
        _check(load().lb_batch_tune(self._h, int(width), int(probe_steps), float(dt), _stream(stream),
                                    _ptr(choice)))
        return choice

    def integrate(self, dt, nsteps, correct_every=0, stream=None):
        ms = ctypes.c_float()
        _check(load().lb_batch_integrate(self._h, int(correct_every), float(dt), int(nsteps), _stream(stream),
                                         ctypes.byref(ms)))
        return ms.value

    def system(self, r):
        """(A64, K) of realization r as host numpy arrays."""
        M = self.Ms[r]
        A = np.zeros((M, M))
        K = np.zeros(M)
        _check(load().lb_batch_copy_system(self._h, int(r), _ptr(A), _ptr(K), None))
        return A, K


def host_release():
    """Return the spare device memory of the host-buffer interface's pool."""
    _check(load().lb_host_release())


class System:
    """Host-buffer interface: lb_assemble / lb_system_* / lb_integrate.

    a: dense M x M complex Kossakowski matrix (numpy), or None with
    channels = [(gamma, idx, values), ...] (host arrays: basis indices and
    complex values of each l_p) for a = sum_p gamma_p l_p l_p^dagger.
    format: "dense" or "csr" (CSR needs channels)."""

    def __init__(self, basis, a=None, H=None, keep_parts=False, algorithm="closed", channels=None, format="dense"):
        lib = load()
        if isinstance(a, _vp):  # an already created handle (System.load)
            self._h, self.basis, self.M = a, basis, basis.M
            self.format = "dense"
            return
        ks = LbKossakowski()
        keep = []
        if channels is not None:
            gam = np.ascontiguousarray([float(g) for g, _, _ in channels], np.float64)
            ptr = np.zeros(len(channels) + 1, np.int64)
            for p, (_, idx, _) in enumerate(channels):
                ptr[p + 1] = ptr[p] + len(idx)
            idx = np.ascontiguousarray(np.concatenate([np.asarray(i, np.int64) for _, i, _ in channels])
                                       if channels else np.zeros(1, np.int64))
            val = np.ascontiguousarray(np.concatenate([np.asarray(v, np.complex128) for _, _, v in channels])
                                       if channels else np.zeros(1, np.complex128))
            keep += [gam, ptr, idx, val]
            ks.kind, ks.nP = LB_A_LOWRANK, len(channels)
            ks.gamma, ks.lp_ptr, ks.lp_idx, ks.lp_val = _ptr(gam), _ptr(ptr), _ptr(idx), _ptr(val)
        else:
            a = np.ascontiguousarray(a, np.complex128)
            assert a.shape == (basis.M, basis.M)
            keep.append(a)
            ks.kind, ks.a = LB_A_DENSE, _ptr(a)
        Hc = None if H is None else np.ascontiguousarray(H, np.complex128)
        h = _vp()
        _check(lib.lb_assemble(basis.handle, _ptr(Hc), ctypes.byref(ks), FORMATS[format], ALGORITHMS[algorithm],
                               int(bool(keep_parts)), ctypes.byref(h)))
        self._h = h
        self.basis = basis
        self.M = basis.M
        self.format = format

    def close(self):
        if self._h:
            load().lb_system_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        f, M, nnz = ctypes.c_int(), _c_i64(), _c_i64()
        _check(load().lb_system_info(self._h, ctypes.byref(f), ctypes.byref(M), ctypes.byref(nnz)))
        return {"format": {LB_DENSE: "dense", LB_CSR: "csr"}[f.value], "M": M.value, "nnz": nnz.value}

    def timings(self):
        """Phase times (ms) of the lb_assemble call that built the system."""
        ms = (ctypes.c_double * len(PHASES))()
        _check(load().lb_system_timings(self._h, ms))
        return {k: float(ms[i]) for i, k in enumerate(PHASES)}

    def get(self, part):
        p = {"A": LB_SYS_A, "Q": LB_SYS_Q, "R": LB_SYS_R, "K": LB_SYS_K}[part]
        out = np.zeros(self.M if part == "K" else (self.M, self.M))
        _check(load().lb_system_get(self._h, p, _ptr(out)))
        return out

    def spectrum(self):
        """Eigenvalues of A (complex128 numpy array of length M) of a dense
        system (lb_system_spectrum)."""
        out = np.zeros(2 * self.M)
        _check(load().lb_system_spectrum(self._h, _ptr(out)))
        return out[0::2] + 1j * out[1::2]

    def get_csr(self):
        """(rowptr int64, col int32, val float64) of a CSR system."""
        nnz = self.info()["nnz"]
        rp = np.zeros(self.M + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        val = np.zeros(max(nnz, 1), np.float64)
        _check(load().lb_system_get_csr(self._h, _ptr(rp), _ptr(col), _ptr(val)))
        return rp, col[:nnz], val[:nnz]

    def integrate(self, v0, t, dt, precision="fp64", correct_every=0, snap_every=0, out=None):
        """RK4 from host v0; returns the final state (M,) or, with snap_every,
        the (n / snap_every, M) snapshots."""
        v0 = np.ascontiguousarray(v0, np.float64)
        n = int(round(t / dt))
        shape = (n // snap_every, self.M) if snap_every else (self.M,)
        out = np.zeros(shape) if out is None else out
        _check(load().lb_integrate(self._h, PRECISIONS[precision], int(correct_every), _ptr(v0), float(t),
                                   float(dt), int(snap_every), _ptr(out)))
        return out

    def integrate_resume(self, v, dt, nsteps, precision="fp64", correct_every=0):
        """Advance the host state v (float64, M) in place by nsteps RK4 steps."""
        assert isinstance(v, np.ndarray) and v.dtype == np.float64 and v.flags.c_contiguous
        _check(load().lb_integrate_resume(self._h, PRECISIONS[precision], int(correct_every), _ptr(v), float(dt),
                                          int(nsteps)))
        return v

    def save(self, path):
        _check(load().lb_system_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, basis, path):
        h = _vp()
        _check(load().lb_system_load(basis.handle, os.fsencode(path), ctypes.byref(h)))
        return cls(basis, h)


def request_bytes(N, precision="fp32", with_H=True):
    """Server memory one request of dimension N holds from admission to completion."""
    return int(load().lb_request_bytes(int(N), PRECISIONS[precision], int(bool(with_H))))


def sched_simulate(arrival_ms, nbytes, service_ms, budget, slots, bypass_ms):
    """Virtual-time replay of the server's admission policy (host only)."""
    arrival = np.ascontiguousarray(arrival_ms, np.float64)
    nb = np.ascontiguousarray(nbytes, np.int64)
    service = np.ascontiguousarray(service_ms, np.float64)
    n = len(arrival)
    assert len(nb) == n and len(service) == n
    start = np.zeros(n)
    finish = np.zeros(n)
    _check(load().lb_sched_simulate(n, _ptr(arrival), _ptr(nb), _ptr(service), int(budget), int(slots),
                                    float(bypass_ms), _ptr(start), _ptr(finish)))
    return start, finish


def _result(r):
    return {"state": r.state, "status": r.status, "engine": r.engine, "cluster": r.cluster,
            "queue_ms": r.queue_ms, "latency_ms": r.latency_ms, "gpu_ms": r.gpu_ms}


class Server:
    """Serving form (lb_server_*).  Device tensors of a request are kept
    referenced until the library no longer reads them."""

    def __init__(self, budget_bytes, slots=16, bypass_ms=2000.0):
        h = _vp()
        _check(load().lb_server_create(int(budget_bytes), int(slots), float(bypass_ms), ctypes.byref(h)))
        self._h = h
        self._inputs = {}   # id -> (a, H, v0): read until LB_REQ_ASSEMBLED
        self._outputs = {}  # id -> v_out: written until LB_REQ_DONE

    def close(self):
        if self._h:
            load().lb_server_destroy(self._h)
            self._h = None
            self._inputs.clear()
            self._outputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_cluster(self, N, C):
        _check(load().lb_server_set_cluster(self._h, int(N), int(C)))

    def submit(self, a, v0, v_out, dt, nsteps, H=None, precision="fp32", correct_every=0, stream=None):
        """Queue one realization; inputs must be complete in the order of
        `stream` (default: torch's current stream) at this call."""
        M = v0.numel()
        N = int(round((M + 1) ** 0.5))
        st = _stream(stream)
        q = LbRequest(N, PRECISIONS[precision], int(correct_every), float(dt), int(nsteps), _ptr(H), _ptr(a),
                      _ptr(v0), _ptr(v_out), st)
        rid = ctypes.c_uint64()
        _check(load().lb_submit(self._h, ctypes.byref(q), ctypes.byref(rid)))
        self._inputs[rid.value] = (a, H, v0)
        self._outputs[rid.value] = v_out
        return rid.value

    def _settle(self, rid, res):
        if res.state >= LB_REQ_ASSEMBLED:
            self._inputs.pop(rid, None)
        if res.state >= LB_REQ_DONE:
            self._outputs.pop(rid, None)

    def poll(self, rid):
        """Result dict once the request is done, None while it is pending."""
        r = LbResult()
        rc = load().lb_poll(self._h, int(rid), ctypes.byref(r))
        self._settle(rid, r)
        if rc == LB_EAGAIN:
            return None
        _check(rc)
        return _result(r)

    def state(self, rid):
        r = LbResult()
        rc = load().lb_poll(self._h, int(rid), ctypes.byref(r))
        if rc not in (LB_OK, LB_EAGAIN):
            _check(rc)
        self._settle(rid, r)
        return r.state

    def wait(self, rid, timeout_ms=600_000.0):
        r = LbResult()
        rc = load().lb_wait(self._h, int(rid), float(timeout_ms), ctypes.byref(r))
        self._settle(rid, r)
        _check(rc)
        return _result(r)

    def stats(self):
        p50, p99, thr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = _c_i64()
        _check(load().lb_server_stats(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(thr),
                                      ctypes.byref(n)))
        return {"p50_ms": p50.value, "p99_ms": p99.value, "throughput_per_s": thr.value, "completed": n.value}

    def reset_stats(self):
        _check(load().lb_server_reset_stats(self._h))

"""ctypes front end of the C oracle (``lb_oracle.c``).  Test infrastructure.

The shared object is compiled with the system C compiler on first use (or
by ``build_library()``), next to the source, and loaded with ctypes.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build_library(force=False):
    """Compile lb_oracle.c into _liboracle.so (plain -O3, OpenMP, no ISA flags)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def load_library():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build_library()
        lib = ctypes.CDLL(_LIB)
        lib.ora_create.restype = ctypes.c_void_p
        lib.ora_create.argtypes = [ctypes.c_int]
        lib.ora_destroy.argtypes = [ctypes.c_void_p]
        lib.ora_M.restype = _i64
        lib.ora_M.argtypes = [ctypes.c_void_p]
        lib.ora_basis_dense.argtypes = [ctypes.c_void_p, _i64, _dp]
        lib.ora_nnz.restype = _i64
        lib.ora_nnz.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        lib.ora_export.argtypes = [ctypes.c_void_p, ctypes.c_int, _i32p, _dp]
        lib.ora_export_ordered.argtypes = [ctypes.c_void_p, ctypes.c_int, _i32p, _dp]
        lib.ora_expand.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        lib.ora_rho.argtypes = [ctypes.c_void_p, _dp, _dp]
        lib.ora_Q.argtypes = [ctypes.c_void_p, _dp, _dp]
        lib.ora_K.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        lib.ora_K_on_f.argtypes = [ctypes.c_void_p, _dp, _dp]
        lib.ora_join_terms.restype = _i64
        lib.ora_join_terms.argtypes = [ctypes.c_void_p]
        lib.ora_R.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        lib.ora_R_entries.argtypes = [ctypes.c_void_p, _dp, _i64, _i64p, _i64p, _dp, _dp, _dp]
        lib.ora_Q_entries.argtypes = [ctypes.c_void_p, _dp, _i64, _i64p, _i64p, _dp]
        lib.ora_R_rows_needed.restype = _i64
        lib.ora_R_rows_needed.argtypes = [ctypes.c_void_p, _i64, _i64p, _i64p, _i64]
        lib.ora_R_entries_rows.restype = ctypes.c_int
        lib.ora_R_entries_rows.argtypes = [ctypes.c_void_p, _i64, _i64p, _dp, _i64, _i64p, _i64p, _dp, _dp]
        lib.ora_R_lowrank.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _i64p, _i64p,
                                      _dp, _dp, _dp, _u8p]
        lib.ora_lowrank_csr.restype = _i64
        lib.ora_lowrank_csr.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, _dp, _i64p, _i64p, _dp, _dp,
                                        ctypes.POINTER(_i64p), ctypes.POINTER(_i32p), ctypes.POINTER(_dp),
                                        ctypes.POINTER(_dp), _dp]
        lib.ora_free.argtypes = [ctypes.c_void_p]
        lib.ora_rk4_dense.argtypes = [_i64, _dp, _dp, _dp, ctypes.c_double, _i64, _i64, _dp, _dp]
        lib.ora_rk4_csr.argtypes = [_i64, _i64p, _i32p, _dp, _dp, _dp, ctypes.c_double, _i64, _dp]
        lib.ora_rk4_dense_td.argtypes = [_i64, _dp, _dp, _dp, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                         ctypes.c_double, _dp, ctypes.c_double, _i64, _dp]
        lib.ora_num_threads.restype = ctypes.c_int
        lib.ora_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _p(a, typ=_dp):
    return a.ctypes.data_as(typ)


def _c128(x):
    """complex128 C-contiguous array -> float64 view (interleaved re, im)."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    return x, x.view(np.float64)


def num_threads():
    return load_library().ora_num_threads()


def set_threads(n):
    load_library().ora_set_threads(int(n))


class Oracle:
    """O3: the paper's formulas for one Hilbert-space dimension N."""

    def __init__(self, N):
        if N < 2:
            raise ValueError("N must be >= 2")
        self.lib = load_library()
        self.N = int(N)
        self.M = self.N * self.N - 1
        self.P = self.N * (self.N - 1) // 2
        self._ctx = self.lib.ora_create(self.N)
        if not self._ctx:
            raise MemoryError("oracle context")

    def close(self):
        if self._ctx:
            self.lib.ora_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- basis --------------------------------------------------------------
    def basis_matrix(self, i):
        out = np.zeros((self.N, self.N), np.complex128)
        self.lib.ora_basis_dense(self._ctx, int(i), _p(out.view(np.float64)))
        return out

    def label(self, i):
        """(type, j, k) with type in 'SJD'; for D, (D, l, l)."""
        P = self.P
        if i < 2 * P:
            t = "S" if i < P else "J"
            p = i % P
            a = 0
            while p >= self.N - 1 - a:
                p -= self.N - 1 - a
                a += 1
            return t, a, a + 1 + p
        l = i - 2 * P + 1
        return "D", l, l

    # -- structure constants -----------------------------------------------
    def nnz(self, which, ordered=False):
        return int(self.lib.ora_nnz(self._ctx, {"f": 0, "d": 1}[which], int(bool(ordered))))

    def structure(self, which, ordered=False):
        """Nonzero f or d: (idx (n,3) int32, val (n,) float64).

        ordered=False: canonical m <= n <= s, sorted lexicographically."""
        w = {"f": 0, "d": 1}[which]
        n = self.nnz(which, ordered)
        idx = np.zeros((n, 3), np.int32)
        val = np.zeros(n, np.float64)
        if n:
            fn = self.lib.ora_export_ordered if ordered else self.lib.ora_export
            fn(self._ctx, w, _p(idx, _i32p), _p(val))
        return idx, val

    def dense_structure(self, which):
        idx, val = self.structure(which, ordered=True)
        T = np.zeros((self.M,) * 3)
        T[idx[:, 0], idx[:, 1], idx[:, 2]] = val
        return T

    def join_terms(self):
        """W = sum_l |Z-section(l)| |F-section(l)|."""
        return int(self.lib.ora_join_terms(self._ctx))

    # -- Eq. (02), Eq. (rho) ---------------------------------------------------
    def expand(self, A):
        A, Af = _c128(A)
        coef = np.zeros(self.M, np.complex128)
        a0 = np.zeros(1, np.complex128)
        self.lib.ora_expand(self._ctx, _p(Af), _p(coef.view(np.float64)), _p(a0.view(np.float64)))
        return coef, complex(a0[0])

    def rho(self, v):
        v = np.ascontiguousarray(v, np.float64)
        out = np.zeros((self.N, self.N), np.complex128)
        self.lib.ora_rho(self._ctx, _p(v), _p(out.view(np.float64)))
        return out

    # -- Eqs. (07)-(09) ---------------------------------------------------------
    def Q(self, h):
        h = np.ascontiguousarray(np.real(h), np.float64)
        Q = np.zeros((self.M, self.M))
        self.lib.ora_Q(self._ctx, _p(h), _p(Q))
        return Q

    def K(self, a, return_imag=False):
        a, af = _c128(a)
        K = np.zeros(self.M)
        Ki = np.zeros(self.M)
        self.lib.ora_K(self._ctx, _p(af), _p(K), _p(Ki))
        return (K, Ki) if return_imag else K

    def K_on_f(self, ima):
        """Eq. (08) from Im a_jk given only on the pairs (j, k) it reads:
        ima[r] belongs to the r-th row (j, k, s) of structure("f", ordered=True)."""
        ima = np.ascontiguousarray(ima, np.float64)
        if ima.shape != (self.nnz("f", ordered=True),):
            raise ValueError("ima must hold one value per ordered nonzero f")
        K = np.zeros(self.M)
        self.lib.ora_K_on_f(self._ctx, _p(ima), _p(K))
        return K

    def R(self, a, return_imag=False, return_scale=False):
        a, af = _c128(a)
        R = np.zeros((self.M, self.M))
        Ri = np.zeros((self.M, self.M)) if return_imag else None
        S = np.zeros((self.M, self.M)) if return_scale else None
        self.lib.ora_R(self._ctx, _p(af), _p(R),
                       _p(Ri) if Ri is not None else None,
                       _p(S) if S is not None else None)
        out = [R]
        if return_imag:
            out.append(Ri)
        if return_scale:
            out.append(S)
        return out[0] if len(out) == 1 else tuple(out)

    def R_entries(self, a, s_idx, n_idx, with_scale=True):
        """Eq. (09) at selected entries; a is the dense M x M matrix (or any
        object exposing a float64 interleaved buffer of it)."""
        a, af = _c128(a)
        s_idx = np.ascontiguousarray(s_idx, np.int64)
        n_idx = np.ascontiguousarray(n_idx, np.int64)
        cnt = len(s_idx)
        out = np.zeros(cnt)
        im = np.zeros(cnt)
        sc = np.zeros(cnt)
        self.lib.ora_R_entries(self._ctx, _p(af), cnt, _p(s_idx, _i64p), _p(n_idx, _i64p),
                               _p(out), _p(im), _p(sc))
        return (out, im, sc) if with_scale else out

    def rows_needed(self, s_idx):
        """Sorted row indices of a read by R_entries_rows for rows s_idx."""
        s_idx = np.ascontiguousarray(np.unique(s_idx), np.int64)
        n = self.lib.ora_R_rows_needed(self._ctx, len(s_idx), _p(s_idx, _i64p), None, 0)
        out = np.zeros(n, np.int64)
        self.lib.ora_R_rows_needed(self._ctx, len(s_idx), _p(s_idx, _i64p), _p(out, _i64p), n)
        return out

    def R_entries_rows(self, row_ids, rows, s_idx, n_idx):
        """Eq. (09) at (s_idx, n_idx) with a given by the rows row_ids (complex (r, M))."""
        row_ids = np.ascontiguousarray(row_ids, np.int64)
        rows, rf = _c128(rows)
        s_idx = np.ascontiguousarray(s_idx, np.int64)
        n_idx = np.ascontiguousarray(n_idx, np.int64)
        out = np.zeros(len(s_idx))
        sc = np.zeros(len(s_idx))
        rc = self.lib.ora_R_entries_rows(self._ctx, len(row_ids), _p(row_ids, _i64p), _p(rf), len(s_idx),
                                         _p(s_idx, _i64p), _p(n_idx, _i64p), _p(out), _p(sc))
        if rc != 0:
            raise ValueError("a row needed by the requested entries was not supplied")
        return out, sc

    def Q_entries(self, h, s_idx, n_idx):
        h = np.ascontiguousarray(np.real(h), np.float64)
        s_idx = np.ascontiguousarray(s_idx, np.int64)
        n_idx = np.ascontiguousarray(n_idx, np.int64)
        out = np.zeros(len(s_idx))
        self.lib.ora_Q_entries(self._ctx, _p(h), len(s_idx), _p(s_idx, _i64p), _p(n_idx, _i64p), _p(out))
        return out

    def R_lowrank(self, gammas, lps):
        """Eq. (09) for a_jk = sum_p gamma_p l_pj conj(l_pk); lps is a list of
        (idx int64, coef complex128) sparse vectors.  Returns (R dense, mask)."""
        nP = len(gammas)
        ptr = np.zeros(nP + 1, np.int64)
        for p, (idx, _) in enumerate(lps):
            ptr[p + 1] = ptr[p] + len(idx)
        idx = np.ascontiguousarray(np.concatenate([np.asarray(i, np.int64) for i, _ in lps]))
        co = np.concatenate([np.asarray(c, np.complex128) for _, c in lps])
        re = np.ascontiguousarray(co.real)
        im = np.ascontiguousarray(co.imag)
        g = np.ascontiguousarray(gammas, np.float64)
        R = np.zeros((self.M, self.M))
        mask = np.zeros((self.M, self.M), np.uint8)
        self.lib.ora_R_lowrank(self._ctx, nP, _p(g), _p(ptr, _i64p), _p(idx, _i64p),
                               _p(re), _p(im), _p(R), _p(mask, _u8p))
        return R, mask.astype(bool)


def _channels(lps, gammas):
    ptr = np.zeros(len(gammas) + 1, np.int64)
    for p, (idx, _) in enumerate(lps):
        ptr[p + 1] = ptr[p] + len(idx)
    idx = np.ascontiguousarray(np.concatenate([np.asarray(i, np.int64) for i, _ in lps]))
    co = np.concatenate([np.asarray(c, np.complex128) for _, c in lps])
    return ptr, idx, np.ascontiguousarray(co.real), np.ascontiguousarray(co.imag), \
        np.ascontiguousarray(gammas, np.float64)


def lowrank_csr(o, h, gammas, lps, with_mag=False):
    """Sparse generator A = Q + R (CSR; entries nonzero beyond rounding) and K
    for a Kossakowski matrix sum_p gamma_p l_p l_p^dagger.
    Returns (rowptr, col, val, K) [+ mag, the summed magnitudes of each entry's terms]."""
    lib = o.lib
    ptr, idx, re, im, g = _channels(lps, gammas)
    h = None if h is None else np.ascontiguousarray(np.real(h), np.float64)
    rp, cp, vp, mp = _i64p(), _i32p(), _dp(), _dp()
    K = np.zeros(o.M)
    nnz = lib.ora_lowrank_csr(o._ctx, _p(h) if h is not None else None, len(gammas), _p(g), _p(ptr, _i64p),
                              _p(idx, _i64p), _p(re), _p(im), ctypes.byref(rp), ctypes.byref(cp),
                              ctypes.byref(vp), ctypes.byref(mp), _p(K))
    rowptr = np.ctypeslib.as_array(rp, shape=(o.M + 1,)).copy()
    col = np.ctypeslib.as_array(cp, shape=(max(nnz, 1),))[:nnz].copy()
    val = np.ctypeslib.as_array(vp, shape=(max(nnz, 1),))[:nnz].copy()
    mag = np.ctypeslib.as_array(mp, shape=(max(nnz, 1),))[:nnz].copy()
    for ptr_ in (rp, cp, vp, mp):
        lib.ora_free(ctypes.cast(ptr_, ctypes.c_void_p))
    return (rowptr, col, val, K, mag) if with_mag else (rowptr, col, val, K)


def rk4_dense(A, K, v0, dt, nsteps, snap_every=0):
    """Classical RK4 for dv/dt = A v + K; returns (v_final, snapshots)."""
    lib = load_library()
    A = np.ascontiguousarray(A, np.float64)
    K = np.ascontiguousarray(K, np.float64)
    v0 = np.ascontiguousarray(v0, np.float64)
    M = len(v0)
    nsnap = nsteps // snap_every if snap_every else 0
    snaps = np.zeros((nsnap, M))
    vout = np.zeros(M)
    lib.ora_rk4_dense(M, _p(A), _p(K), _p(v0), float(dt), int(nsteps), int(snap_every),
                      _p(snaps) if nsnap else None, _p(vout))
    return vout, snaps


def rk4_csr(rowptr, col, val, K, v0, dt, nsteps):
    lib = load_library()
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    v0 = np.ascontiguousarray(v0, np.float64)
    K = np.ascontiguousarray(K, np.float64) if K is not None else None
    vout = np.zeros(len(v0))
    lib.ora_rk4_csr(len(v0), _p(rowptr, _i64p), _p(col, _i32p), _p(val),
                    _p(K) if K is not None else None, _p(v0), float(dt), int(nsteps), _p(vout))
    return vout


def rk4_dense_td(A0, Q1, K, v0, dt, nsteps, seg_start, seg_eps, period, t0=0.0):
    """Classical RK4 for dv/dt = (A0 + eps(t) Q1) v + K with eps periodic and
    piecewise constant (eps = seg_eps[k] on [seg_start[k], seg_start[k+1])
    of each period), each stage at its own time (the end stages taken 1e-6 dt
    inside the step)."""
    lib = load_library()
    A0 = np.ascontiguousarray(A0, np.float64)
    Q1 = np.ascontiguousarray(Q1, np.float64)
    K = np.ascontiguousarray(K, np.float64)
    v0 = np.ascontiguousarray(v0, np.float64)
    ss = np.ascontiguousarray(seg_start, np.float64)
    se = np.ascontiguousarray(seg_eps, np.float64)
    vout = np.zeros(len(v0))
    lib.ora_rk4_dense_td(len(v0), _p(A0), _p(Q1), _p(K), len(ss), _p(ss), _p(se), float(period), float(t0),
                         _p(v0), float(dt), int(nsteps), _p(vout))
    return vout

"""Python binding of the GB300 density-matrix engine (C ABI in include/gdm.h).

Argument marshalling only: every step of the solve runs in the CUDA library
`_build/libgdm.so` (built by `paper_1912_13403_gb300.build`).  Importing this package without
the built library raises ImportError; there is no CPU fallback.

Functions keep the C names (`gdm_init`, `gdm_solve_dm`, ...).  `Handle` and the `op_*`
helpers accept numpy arrays (host memory) or CUDA torch tensors (device memory).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgdm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("CUDA library %s is not built; run `python -m paper_1912_13403_gb300.build` "
                      "(or __graft_entry__.build())" % LIB_PATH)

lib = ctypes.CDLL(LIB_PATH)

GDM_OK, GDM_ERR_ARG, GDM_ERR_STATE, GDM_ERR_NOT_SPD, GDM_ERR_NONFINITE, GDM_ERR_NO_GAP, \
    GDM_ERR_NOT_CONVERGED, GDM_ERR_OOM, GDM_ERR_BUDGET, GDM_ERR_TIMEOUT, GDM_ERR_CUDA = range(11)
GDM_MEM_HOST, GDM_MEM_DEVICE = 0, 1
GDM_PREC_FP64, GDM_PREC_MIXED = 0, 1
GDM_PURIFY_TRS4, GDM_PURIFY_TRS2, GDM_PURIFY_CANONICAL = 0, 1, 2
GDM_PHASE_NEWTON_SCHULZ, GDM_PHASE_REFINE, GDM_PHASE_TRANSFORM, GDM_PHASE_PURIFY = range(4)
GDM_BOUNDS_GERSHGORIN, GDM_BOUNDS_LANCZOS = 0, 1
GDM_BATCH_GROUPED, GDM_BATCH_CONCURRENT = 0, 1


class gdm_info(ctypes.Structure):
    _fields_ = [("ns_iters", ctypes.c_int), ("refine_iters", ctypes.c_int),
                ("purif_iters", ctypes.c_int), ("stop_reason", ctypes.c_int),
                ("idem_err", ctypes.c_double), ("z_err", ctypes.c_double),
                ("trace_err", ctypes.c_double), ("trace_err_raw", ctypes.c_double),
                ("energy", ctypes.c_double),
                ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("trace_fix", ctypes.c_double),
                ("kstage_fraction", ctypes.c_double), ("bounds_restart", ctypes.c_int),
                ("metric_cleanup", ctypes.c_int), ("trace_rescaled", ctypes.c_int),
                ("s_idem_err", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gdm_problem(ctypes.Structure):
    _fields_ = [("n_basis", ctypes.c_int64), ("n_occ", ctypes.c_int64),
                ("H", ctypes.c_void_p), ("ldh", ctypes.c_int64),
                ("S", ctypes.c_void_p), ("lds", ctypes.c_int64), ("mem", ctypes.c_int),
                ("P", ctypes.c_void_p), ("ldp", ctypes.c_int64), ("p_mem", ctypes.c_int)]


class gdm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("energy", ctypes.c_double), ("info", gdm_info),
                ("latency_ms", ctypes.c_double)]

    def as_dict(self):
        return dict(status=self.status, energy=self.energy, info=self.info.as_dict(),
                    latency_ms=self.latency_ms)


class gdm_batch_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("concurrency", ctypes.c_int),
                ("precision", ctypes.c_int), ("engine", ctypes.c_int)]


class gdm_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("slots", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_uint64), ("precision", ctypes.c_int)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)


def _decl(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    globals()[name] = f
    return f


_decl("gdm_init", _int, [ctypes.POINTER(_vp), _i64, _i64, _int])
_decl("gdm_set_precision", _int, [_vp, _int])
_decl("gdm_set_purification", _int, [_vp, _int])
_decl("gdm_set_bounds", _int, [_vp, _int, _int])
_decl("gdm_set_metric_cleanup", _int, [_vp, _dbl])
_decl("gdm_set_truncation", _int, [_vp, _dbl])
_decl("gdm_set_slices", _int, [_vp, _int, _int, _int, _int])
_decl("gdm_set_tolerance", _int, [_vp, _dbl, _dbl])
_decl("gdm_set_max_iter", _int, [_vp, _int, _int])
_decl("gdm_set_trace_correction", _int, [_vp, _int])
_decl("gdm_set_profiling", _int, [_vp, _int])
_decl("gdm_get_profile", _int, [_vp, _int, ctypes.POINTER(_i64), _dp, _dp, _int])
_decl("gdm_get_profile_ex", _int, [_vp, _int, ctypes.POINTER(_i64), _dp, _dp, _dp, _int])
_decl("gdm_launch_count", _i64, [])
_decl("gdm_set_stream", _int, [_vp, _vp])
_decl("gdm_set_overlap", _int, [_vp, _vp, _i64, _int])
_decl("gdm_set_hamiltonian", _int, [_vp, _vp, _i64, _int])
_decl("gdm_solve_dm", _int, [_vp, _vp, _i64, _int, _dp, ctypes.POINTER(gdm_info)])
_decl("gdm_get_edm", _int, [_vp, _vp, _i64, _int])
_decl("gdm_extrapolate_dm", _int, [_vp, _vp, _i64, _int, _vp, _i64, _int])
_decl("gdm_get_history", _int, [_vp, _int, _dp, _dp, _dp, ctypes.POINTER(_int)])
_decl("gdm_reinit", _int, [_vp])
_decl("gdm_finalize", _int, [_vp])
_decl("gdm_status_string", ctypes.c_char_p, [_int])
_decl("gdm_last_error", ctypes.c_char_p, [_vp])
_decl("gdm_batch_release", None, [])
_decl("gdm_solve_batch", _int, [ctypes.POINTER(gdm_problem), _int, ctypes.POINTER(gdm_result),
                                ctypes.POINTER(gdm_batch_config)])
_decl("gdm_server_create", _int, [ctypes.POINTER(_vp), ctypes.POINTER(gdm_server_config)])
_decl("gdm_submit", _int, [_vp, ctypes.POINTER(gdm_problem), ctypes.POINTER(ctypes.c_uint64)])
_decl("gdm_wait", _int, [_vp, ctypes.c_uint64, _dbl, ctypes.POINTER(gdm_result)])
_decl("gdm_poll", _int, [_vp, ctypes.c_uint64, ctypes.POINTER(_int), ctypes.POINTER(gdm_result)])
_decl("gdm_server_destroy", _int, [_vp])
_decl("gdm_op_product", _int, [_vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64, _i64, _int, _int,
                               _int, _int, _vp])
_decl("gdm_op_product_noalloc", _int, [_vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64, _i64, _int,
                                       _int, _int, _int, _vp])
_decl("gdm_op_gershgorin", _int, [_vp, _i64, _i64, _dp, _vp])
_decl("gdm_op_trs4_step", _int, [_vp, _i64, _i64, _dbl, _int, _int, _dp,
                                 ctypes.POINTER(_int), _vp])


class GdmError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = gdm_status_string(status).decode()
        super().__init__("%s%s" % (name, (": " + msg) if msg else ""))


def status_name(st: int) -> str:
    return gdm_status_string(st).decode()


# ------------------------------------------------------------------------------------------
# marshalling helpers
# ------------------------------------------------------------------------------------------

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _buf(x):
    """(pointer, leading dimension, mem kind) of a 2-D row-major float64 buffer."""
    if _is_torch(x):
        if x.dtype.itemsize != 8 or not x.is_floating_point():
            raise TypeError("float64 tensor expected")
        if x.dim() != 2 or x.stride(1) != 1:
            raise ValueError("2-D row-major tensor expected")
        return x.data_ptr(), x.stride(0), (GDM_MEM_DEVICE if x.is_cuda else GDM_MEM_HOST)
    if not isinstance(x, np.ndarray) or x.dtype != np.float64 or x.ndim != 2 or \
            x.strides[1] != 8:
        raise TypeError("2-D row-major float64 numpy array expected")
    return x.ctypes.data, x.strides[0] // 8, GDM_MEM_HOST


def _shape(x):
    return tuple(int(d) for d in x.shape)


def _square(x, n, what):
    """(pointer, leading dimension, mem kind) of an n x n float64 buffer; ValueError for any
    other shape (the library reads or writes n rows of n elements at the given pointer)."""
    if _shape(x) != (n, n):
        raise ValueError("%s must be %d x %d, got %s" % (what, n, n, _shape(x)))
    return _buf(x)


def _device_operands(**mats):
    """Shapes first (so that a mismatch is reported the same way everywhere), then the
    device: every operand of a gdm_op_* call is a CUDA float64 tensor of one device."""
    dev = None
    for name, x in mats.items():
        if not (_is_torch(x) and x.is_cuda):
            raise ValueError("%s must be a CUDA tensor (device pointers only)" % name)
        if dev is None:
            dev = x.device
        elif x.device != dev:
            raise ValueError("%s is on %s, the other operands on %s" % (name, x.device, dev))


def _product_shapes(A, Bt, C, symmetric):
    if len(_shape(A)) != 2 or len(_shape(Bt)) != 2 or len(_shape(C)) != 2:
        raise ValueError("A, Bt and C must be 2-D")
    m, k = _shape(A)
    n, kb = _shape(Bt)
    if kb != k:
        raise ValueError("Bt has %d columns, A has %d (contraction length)" % (kb, k))
    if _shape(C) != (m, n):
        raise ValueError("C must be %d x %d, got %s" % (m, n, _shape(C)))
    if symmetric and m != n:
        raise ValueError("a symmetric product needs m == n")
    return m, n, k


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Handle:
    """One solver handle (gdm_init ... gdm_finalize)."""

    def __init__(self, n_basis: int, n_occ: int, device: int = 0):
        self._h = _vp()
        st = gdm_init(ctypes.byref(self._h), int(n_basis), int(n_occ), int(device))
        if st != GDM_OK:
            raise GdmError(st, "gdm_init(n=%d, n_occ=%d)" % (n_basis, n_occ))
        self.n, self.n_occ = int(n_basis), int(n_occ)

    def _check(self, st, allow=()):
        if st != GDM_OK and st not in allow:
            raise GdmError(st, gdm_last_error(self._h).decode())
        return st

    def set_precision(self, prec):
        return self._check(gdm_set_precision(self._h, prec))

    def set_truncation(self, threshold):
        """Threshold filtering of the purification (0 turns it off)."""
        return self._check(gdm_set_truncation(self._h, float(threshold)))

    def set_bounds(self, method, lanczos_steps=0):
        """Spectral bounds of H~ for the initial guess: GDM_BOUNDS_LANCZOS (default) or
        GDM_BOUNDS_GERSHGORIN; lanczos_steps 0 keeps the current count."""
        return self._check(gdm_set_bounds(self._h, method, int(lanczos_steps)))

    def set_purification(self, method):
        """GDM_PURIFY_TRS4 (default), GDM_PURIFY_TRS2 or GDM_PURIFY_CANONICAL."""
        return self._check(gdm_set_purification(self._h, method))

    def set_slices(self, phase, nslice, max_order, slice_bits=0):
        return self._check(gdm_set_slices(self._h, phase, nslice, max_order, slice_bits))

    def set_tolerance(self, idem_tol, trace_tol):
        return self._check(gdm_set_tolerance(self._h, idem_tol, trace_tol))

    def set_metric_cleanup(self, threshold):
        """S-metric clean-up when |Tr(PS) - n_occ| > threshold (0: always, < 0: never)."""
        return self._check(gdm_set_metric_cleanup(self._h, float(threshold)))

    def set_trace_correction(self, enable):
        return self._check(gdm_set_trace_correction(self._h, int(bool(enable))))

    def set_profiling(self, enable):
        return self._check(gdm_set_profiling(self._h, int(bool(enable))))

    def profile(self, kind=0, reset=False, algorithmic=False):
        """(launches, device ms, tensor-pipe flops[, algorithmic flops]) of the product launches
        since the last reset; kind 0 = sliced tensor-core products, 1 = FP64 products, 2 + p =
        sliced products of phase p.  Algorithmic flops count n^3 per symmetric and 2 n^3 per
        full product."""
        l = _i64(0)
        ms = ctypes.c_double(0)
        fl = ctypes.c_double(0)
        al = ctypes.c_double(0)
        self._check(gdm_get_profile_ex(self._h, kind, ctypes.byref(l), ctypes.byref(ms),
                                       ctypes.byref(fl), ctypes.byref(al), int(bool(reset))))
        if algorithmic:
            return l.value, ms.value, fl.value, al.value
        return l.value, ms.value, fl.value

    def set_max_iter(self, ns_max, purif_max):
        return self._check(gdm_set_max_iter(self._h, ns_max, purif_max))

    def set_stream(self, stream):
        return self._check(gdm_set_stream(self._h, _stream_ptr(stream)))

    def set_overlap(self, S):
        p, ld, mem = _square(S, self.n, "S")
        return self._check(gdm_set_overlap(self._h, p, ld, mem))

    def set_hamiltonian(self, H):
        p, ld, mem = _square(H, self.n, "H")
        return self._check(gdm_set_hamiltonian(self._h, p, ld, mem))

    def solve(self, P=None, allow=(GDM_ERR_NOT_CONVERGED,)):
        """Solve into P (numpy or torch float64 n x n; allocated on the host when None).
        Returns (P, energy, info dict, status)."""
        if P is None:
            P = np.empty((self.n, self.n))
        p, ld, mem = _square(P, self.n, "P")
        e = ctypes.c_double(0.0)
        info = gdm_info()
        st = gdm_solve_dm(self._h, p, ld, mem, ctypes.byref(e), ctypes.byref(info))
        self._check(st, allow)
        return P, e.value, info.as_dict(), st

    def edm(self, Q=None):
        """Energy-weighted density matrix P H P of the last solve into Q (numpy or torch float64
        n x n; allocated on the host when None).  Returns Q."""
        if Q is None:
            Q = np.empty((self.n, self.n))
        q, ld, mem = _square(Q, self.n, "Q")
        self._check(gdm_get_edm(self._h, q, ld, mem))
        return Q

    def extrapolate(self, S_new, P=None):
        """New geometry: S_new becomes the overlap (its Z is computed and cached) and the last
        solve's density matrix is extrapolated to it in Loewdin form.  Returns P (numpy or torch
        float64 n x n; allocated on the host when None)."""
        if P is None:
            P = np.empty((self.n, self.n))
        s, lds, ms = _square(S_new, self.n, "S_new")
        p, ldp, mp = _square(P, self.n, "P")
        self._check(gdm_extrapolate_dm(self._h, s, lds, ms, p, ldp, mp))
        return P

    def history(self, max_rows=1000):
        """Purification history of the last solve: list of (idem, trace, gamma, branch)."""
        idem = (ctypes.c_double * max_rows)()
        tr = (ctypes.c_double * max_rows)()
        gm = (ctypes.c_double * max_rows)()
        br = (ctypes.c_int * max_rows)()
        m = min(gdm_get_history(self._h, max_rows, idem, tr, gm, br), max_rows)
        return [(idem[i], tr[i], gm[i], br[i]) for i in range(m)]

    def reinit(self):
        return self._check(gdm_reinit(self._h))

    def close(self):
        if self._h:
            gdm_finalize(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _problem(H, S, n_occ, P=None):
    n = _shape(H)[0] if len(_shape(H)) == 2 else -1
    ph, ldh, mem = _square(H, n, "H")
    ps, lds, mem2 = _square(S, n, "S")
    if mem != mem2:
        raise ValueError("H and S must live in the same memory")
    p = gdm_problem(H.shape[0], int(n_occ), ph, ldh, ps, lds, mem, None, 0, GDM_MEM_HOST)
    if P is not None:
        pp, ldp, pmem = _square(P, n, "P")
        p.P, p.ldp, p.p_mem = pp, ldp, pmem
    return p


def solve_batch(items, concurrency=4, precision=GDM_PREC_MIXED, device=0,
                engine=GDM_BATCH_GROUPED):
    """Solve a list of (H, S, n_occ, P) tuples as one batch (gdm_solve_batch): by default in
    lockstep with grouped products (GDM_BATCH_GROUPED), or as concurrent solves
    (GDM_BATCH_CONCURRENT).  P may be None.  Returns (status, list of result dicts)."""
    arr = (gdm_problem * len(items))(*[_problem(*it) for it in items])
    res = (gdm_result * len(items))()
    cfg = gdm_batch_config(device, concurrency, precision, engine)
    st = gdm_solve_batch(arr, len(items), res, ctypes.byref(cfg))
    return st, [r.as_dict() for r in res]


def batch_release():
    """Free the grouped batch engine's cached device memory (gdm_batch_release)."""
    gdm_batch_release()


class Server:
    """Request server (gdm_server_*): submit() copies H and S, wait()/poll() return results."""

    def __init__(self, slots=4, hbm_budget_bytes=0, precision=GDM_PREC_MIXED, device=0):
        self._s = _vp()
        cfg = gdm_server_config(device, slots, hbm_budget_bytes, precision)
        st = gdm_server_create(ctypes.byref(self._s), ctypes.byref(cfg))
        if st != GDM_OK:
            raise GdmError(st, "gdm_server_create")
        self._keep = {}

    def submit(self, H, S, n_occ, P=None):
        p = _problem(H, S, n_occ, P)
        t = ctypes.c_uint64(0)
        st = gdm_submit(self._s, ctypes.byref(p), ctypes.byref(t))
        if st != GDM_OK:
            raise GdmError(st, "gdm_submit")
        self._keep[t.value] = P  # the output buffer must outlive the request
        return t.value

    def wait(self, ticket, timeout_s=-1.0):
        r = gdm_result()
        st = gdm_wait(self._s, ticket, timeout_s, ctypes.byref(r))
        if st != GDM_OK:
            raise GdmError(st, "gdm_wait")
        self._keep.pop(ticket, None)
        return r.as_dict()

    def poll(self, ticket):
        d = _int(0)
        r = gdm_result()
        st = gdm_poll(self._s, ticket, ctypes.byref(d), ctypes.byref(r))
        if st != GDM_OK:
            raise GdmError(st, "gdm_poll")
        if d.value:
            self._keep.pop(ticket, None)
            return r.as_dict()
        return None

    def close(self):
        if self._s:
            gdm_server_destroy(self._s)
            self._s = _vp()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def op_product(A, Bt, C, nslice=3, max_order=3, symmetric=False, stream=None, slice_bits=0):
    """C = A @ Bt.T on the device (torch CUDA float64 tensors of one device; C is m x n for
    A m x k and Bt n x k, checked here because the library trusts the sizes it is given)."""
    m, n, k = _product_shapes(A, Bt, C, symmetric)
    _device_operands(A=A, Bt=Bt, C=C)
    pa, lda, _ = _buf(A)
    pb, ldb, _ = _buf(Bt)
    pc, ldc, _ = _buf(C)
    st = gdm_op_product(pa, lda, pb, ldb, pc, ldc, m, n, k,
                        nslice, max_order, slice_bits, int(bool(symmetric)),
                        _stream_ptr(stream))
    if st != GDM_OK:
        raise GdmError(st, "gdm_op_product")
    return C


def op_product_noalloc(A, Bt, C, nslice=3, max_order=3, symmetric=False, stream=None,
                       slice_bits=0):
    """C = A @ Bt.T like op_product, with the library's fixed scratch array instead of device
    allocations (m, n, k <= 1024).  Shapes and device are checked as in op_product."""
    m, n, k = _product_shapes(A, Bt, C, symmetric)
    _device_operands(A=A, Bt=Bt, C=C)
    pa, lda, _ = _buf(A)
    pb, ldb, _ = _buf(Bt)
    pc, ldc, _ = _buf(C)
    st = gdm_op_product_noalloc(pa, lda, pb, ldb, pc, ldc, m, n, k,
                                nslice, max_order, slice_bits, int(bool(symmetric)),
                                _stream_ptr(stream))
    if st != GDM_OK:
        raise GdmError(st, "gdm_op_product_noalloc")
    return C


def op_gershgorin(A, stream=None):
    """Gershgorin bounds (lo, hi) of the square CUDA float64 tensor A."""
    n = _shape(A)[0] if len(_shape(A)) == 2 else -1
    _square(A, n, "A")
    _device_operands(A=A)
    pa, lda, _ = _buf(A)
    out = (ctypes.c_double * 2)()
    st = gdm_op_gershgorin(pa, lda, n, out, _stream_ptr(stream))
    if st != GDM_OK:
        raise GdmError(st, "gdm_op_gershgorin")
    return out[0], out[1]


def op_trs4_step(X, n_occ, nslice=0, max_order=0, stream=None):
    """One TRS4 step in place on the square CUDA float64 tensor X; returns (gamma, branch)."""
    n = _shape(X)[0] if len(_shape(X)) == 2 else -1
    _square(X, n, "X")
    _device_operands(X=X)
    px, ld, _ = _buf(X)
    g = ctypes.c_double(0.0)
    br = ctypes.c_int(-1)
    st = gdm_op_trs4_step(px, ld, n, float(n_occ), nslice, max_order, ctypes.byref(g),
                          ctypes.byref(br), _stream_ptr(stream))
    if st != GDM_OK:
        raise GdmError(st, "gdm_op_trs4_step")
    return g.value, br.value

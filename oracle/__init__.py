"""CPU FP64 oracle - TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference legs of `bench.py` may
import this package.  The GPU product path (`paper_1912_13403_gb300`) never imports it and shares
no code with it.

Two parts:
  * `jacobi.c` (built into `_build/liboracle.so` with gcc + OpenMP): the plain definition of the
    result - Jacobi eigenpairs of S and of H~ = S^{-1/2} H S^{-1/2}, then P = C_occ C_occ^T
    (Sec. 1 Eqs. evp, density_matrix; Sec. 2.2.2 Eq. ntpoly_lowdin) and, on request, the
    energy-weighted density matrix C_occ diag(eps) C_occ^T (Sec. 2.6, Eq. energy_density_matrix);
    `extrapolate_dm` takes a density matrix to a new overlap in Loewdin form (Sec. 2.7).
  * `steps.py` (numpy float64): the individual steps of the purification route written out in
    the paper's order (Eq. ntpoly_scale_hamiltonian initial guess, Eq. ntpoly_purification with
    the trace-resetting map the paper cites, Loewdin orthogonalisation), plus the closed forms
    the synthetic inputs allow.

Parity status: every function here is pinned by `tests/test_oracle_*.py` against closed forms,
library eigensolvers on special cases, invariants or brute force; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "jacobi.c")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "ERR_ARG", 3: "NOT_SPD", 5: "NO_GAP", 6: "NOT_CONVERGED", 7: "OOM"}


def build(force: bool = False) -> str:
    """Compile jacobi.c with gcc (-O2 -fopenmp); returns the path of the shared object."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_jacobi_eigh.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_double,
                                               ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            lib.oracle_jacobi_eigh.restype = ctypes.c_int
            lib.oracle_inv_sqrt.argtypes = [ctypes.c_int64, dp, dp, dp, dp]
            lib.oracle_inv_sqrt.restype = ctypes.c_int
            lib.oracle_density_matrix.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, dp, dp,
                                                  dp, dp, dp, dp, dp]
            lib.oracle_density_matrix.restype = ctypes.c_int
            lib.oracle_density_matrix_edm.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, dp, dp,
                                                      dp, dp, dp, dp, dp, dp]
            lib.oracle_density_matrix_edm.restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    """OpenMP threads the C oracle runs with."""
    return int(_load().oracle_num_threads())


def jacobi_eigh(A, tol: float = 1e-15, max_sweeps: int = 60):
    """Eigenpairs of a symmetric matrix by two-sided cyclic Jacobi.
    Returns (evals ascending, V with eigenvectors in columns, sweeps, status string)."""
    A = _f64(A).copy()
    n = A.shape[0]
    w = np.empty(n)
    V = np.empty((n, n))
    sw = ctypes.c_int(0)
    st = _load().oracle_jacobi_eigh(n, _ptr(A), _ptr(w), _ptr(V), tol, max_sweeps,
                                    ctypes.byref(sw))
    return w, V, int(sw.value), STATUS.get(st, str(st))


def inv_sqrt(S):
    """Loewdin factor Z = S^{-1/2} (Eq. ntpoly_lowdin) via Jacobi.  Returns (Z, status)."""
    S = _f64(S)
    n = S.shape[0]
    Z = np.empty((n, n))
    smin = ctypes.c_double(0)
    smax = ctypes.c_double(0)
    st = _load().oracle_inv_sqrt(n, _ptr(S), _ptr(Z), ctypes.byref(smin), ctypes.byref(smax))
    return Z, STATUS.get(st, str(st))


def density_matrix(H, S, n_occ: int, edm: bool = False):
    """Zero-temperature density matrix (Eq. density_matrix, f_l in {0,1}) of (H, S); with
    edm=True also the energy-weighted density matrix q_ij = sum_l f_l eps_l c_il c_jl
    (Eq. energy_density_matrix) as "Q".

    Returns dict(P, energy, trace_ps, idem, gap, evals, status[, Q])."""
    H = _f64(H)
    S = _f64(S)
    n = H.shape[0]
    P = np.empty((n, n))
    Q = np.empty((n, n)) if edm else None
    w = np.empty(n)
    e, t, d, g = (ctypes.c_double(0) for _ in range(4))
    st = _load().oracle_density_matrix_edm(n, int(n_occ), _ptr(H), _ptr(S), _ptr(P),
                                           ctypes.byref(e), ctypes.byref(t), ctypes.byref(d),
                                           ctypes.byref(g), _ptr(w),
                                           _ptr(Q) if edm else None)
    out = dict(P=P, energy=e.value, trace_ps=t.value, idem=d.value, gap=g.value, evals=w,
               status=STATUS.get(st, str(st)))
    if edm:
        out["Q"] = Q
    return out


def extrapolate_dm(P0, S0, S1):
    """Density-matrix extrapolation to a new geometry in Loewdin form (Sec. 2.7, the Loewdin
    counterpart of Eq. cholesky_extrapolation): P0 is taken to the orthogonal basis of S0 and
    from there to the basis of S1,  P1 = S1^{-1/2} S0^{1/2} P0 S0^{1/2} S1^{-1/2},
    with both square roots from Jacobi eigenpairs.  Returns (P1, status)."""
    S0 = _f64(S0)
    S1 = _f64(S1)
    P0 = _f64(P0)
    w0, U0, _, st0 = jacobi_eigh(S0)
    w1, U1, _, st1 = jacobi_eigh(S1)
    if st0 != "OK" or st1 != "OK":
        return None, st0 if st0 != "OK" else st1
    if w0.min() <= 0.0 or w1.min() <= 0.0:
        return None, "NOT_SPD"
    s0_half = (U0 * np.sqrt(w0)[None, :]) @ U0.T
    s1_mhalf = (U1 * (1.0 / np.sqrt(w1))[None, :]) @ U1.T
    T = s1_mhalf @ s0_half
    P1 = T @ P0 @ T.T
    return 0.5 * (P1 + P1.T), "OK"


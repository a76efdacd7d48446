"""The density matrix by its plain definition with a library eigensolver - TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference legs of `bench.py` may
import this module.  It shares no code with the GPU path.

The same steps as the Jacobi oracle (`jacobi.c`), in the same order, with LAPACK's symmetric
eigensolver (numpy.linalg.eigh, a library primitive) in place of the hand-written Jacobi
rotations, so that the definition can be evaluated at the full workload sizes (n = 4096 in a few
seconds on a many-core host, where cyclic Jacobi takes many minutes):

  1. symmetrise H and S                                        (the inputs' reading)
  2. S = U diag(s) U^T; s_min <= 0 is NOT_SPD                 (Sec. 2.2.2, Eq. ntpoly_lowdin)
  3. Z = U diag(s^{-1/2}) U^T, the Loewdin factor
  4. H~ = Z H Z, symmetrised
  5. H~ = V diag(lam) V^T, lam ascending                       (Sec. 1, Eq. evp in the
                                                                 orthogonal basis)
  6. lam_{N+1} - lam_N at or below 1e-12 of the spectral width is NO_GAP: rounding
     noise, so the occupied subspace is not unique (the Jacobi oracle's rule)
  7. C_occ = Z V[:, :N],  P = C_occ C_occ^T                    (Sec. 1, Eq. density_matrix,
                                                                 f_l = 1 for the N lowest;
     symmetrised, since the library's product need not round the two triangles alike)
  8. E = sum_{l<=N} lam_l, Tr(P S), ||P S P - P||_F            (the outputs)
With edm=True also Q = C_occ diag(lam_occ) C_occ^T            (Sec. 2.6, Eq. energy_density_matrix).

Pinned in tests/test_oracle.py by the same closed forms, golden 2x2 values, diagonal case,
brute-force minimum and invariants as the Jacobi oracle, and against the Jacobi oracle itself.
"""
from __future__ import annotations

import ctypes
import glob
import os

import numpy as np


def _sym(a):
    return 0.5 * (a + a.T)


def density_matrix_eigh(H, S, n_occ: int, edm: bool = False):
    """Zero-temperature density matrix of (H, S) with n_occ occupied states.
    Returns dict(P, energy, trace_ps, idem, gap, evals, status[, Q]) like oracle.density_matrix."""
    H = _sym(np.asarray(H, dtype=np.float64))
    S = _sym(np.asarray(S, dtype=np.float64))
    n = H.shape[0]
    N = int(n_occ)
    out = dict(P=None, energy=float("nan"), trace_ps=float("nan"), idem=float("nan"),
               gap=float("nan"), evals=None, status="OK")
    if H.shape != (n, n) or S.shape != (n, n) or not 0 <= N <= n:
        out["status"] = "ERR_ARG"
        return out
    s, U = np.linalg.eigh(S)
    if s[0] <= 0.0:
        out["status"] = "NOT_SPD"
        return out
    Z = (U * (1.0 / np.sqrt(s))[None, :]) @ U.T
    Ht = _sym(Z @ H @ Z)
    lam, V = np.linalg.eigh(Ht)
    out["evals"] = lam
    if 0 < N < n:
        out["gap"] = float(lam[N] - lam[N - 1])
        if not out["gap"] > 1e-12 * (abs(lam[-1] - lam[0]) + 1e-300):
            out["status"] = "NO_GAP"
            return out
    C = Z @ V[:, :N]
    P = _sym(C @ C.T)
    PS = P @ S
    out.update(P=P, energy=float(np.sum(lam[:N])), trace_ps=float(np.trace(PS)),
               idem=float(np.linalg.norm(PS @ P - P)))
    if edm:
        out["Q"] = _sym((C * lam[:N][None, :]) @ C.T)
    return out


def blas_threads() -> int:
    """Threads of the BLAS/LAPACK library numpy uses (OpenBLAS's own count when it can be
    queried, else the host's core count)."""
    import numpy.linalg as la
    here = os.path.dirname(la.__file__)
    pats = [os.path.join(here, "..", "..", "numpy.libs", "*openblas*"),
            os.path.join(here, "..", "..", "scipy_openblas64", "lib", "*openblas*"),
            os.path.join(here, "..", ".dylibs", "*openblas*")]
    for pat in pats:
        for path in glob.glob(pat):
            try:
                lib = ctypes.CDLL(path)
            except OSError:
                continue
            for name in ("scipy_openblas_get_num_threads64_", "openblas_get_num_threads64_",
                         "openblas_get_num_threads"):
                fn = getattr(lib, name, None)
                if fn is not None:
                    fn.restype = ctypes.c_int
                    v = int(fn())
                    if v > 0:
                        return v
    return os.cpu_count() or 1

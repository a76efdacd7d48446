"""Seeded synthetic (H, S) pairs shaped like the paper's KS-DFT / DFTB workloads.

The paper states the problem as the generalised eigenproblem H C = S C eps (Sec. 1, Eq. evp) and
the density matrix as p_ij = sum_l f_l c_il c_jl (Sec. 1, Eq. density_matrix). Its benchmark
matrices (Sec. 4, Tables 2-4) are not available, so these generators stand in for them.

Every input with a known answer is built from factors:  S = U_s diag(w_s) U_s^T and
H = S^{1/2} Q diag(lam) Q^T S^{1/2}.  Then the generalised eigenpairs are (lam, S^{-1/2} Q) exactly
(H S^{-1/2} Q = S^{1/2} Q diag(lam) = S (S^{-1/2} Q) diag(lam)), which is what the closed-form
checks on the oracle side use.  This module only *builds* inputs: it never forms S^{-1/2}, never
purifies, never forms a density matrix.

All random draws come from numpy's PCG64 (`default_rng(seed)`), so a seed fixes the input.
Dense algebra for the construction (QR, eigh, products) runs in numpy float64, or - for the
n >= 4096 cases, when `device` names a CUDA device - in torch float64 on that device; the random
draws are identical either way.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """One density-matrix problem.

    H, S: dense symmetric float64 (n, n), C-contiguous.  n_occ: number of occupied states
    (f_l in {0, 1}).  factors: construction data for closed forms or None:
      "Q"   (n, n) orthogonal, columns = eigenvectors of the orthogonalised Hamiltonian,
      "lam" (n,) ascending generalised eigenvalues (lam[:n_occ] occupied),
      "S_U", "S_w": S = S_U diag(S_w) S_U^T.
    meta: a small dict describing the recipe (config name, seed, n, gap, cond(S), ...).
    """
    H: np.ndarray
    S: np.ndarray
    n_occ: int
    factors: Optional[dict]
    meta: dict

    @property
    def n(self) -> int:
        return int(self.H.shape[0])


# --------------------------------------------------------------------------------------------
# dense helpers (construction only)
# --------------------------------------------------------------------------------------------

class _Np:
    """numpy float64 backend."""

    @staticmethod
    def asarray(a):
        return np.ascontiguousarray(a, dtype=np.float64)

    @staticmethod
    def qr(a):
        return np.linalg.qr(a)

    @staticmethod
    def eigh(a):
        return np.linalg.eigh(a)

    @staticmethod
    def to_numpy(a):
        return np.ascontiguousarray(a)


class _Torch:
    """torch float64 backend on a CUDA device (construction of large inputs only)."""

    def __init__(self, device):
        import torch  # local import: the CPU path never needs torch
        self.torch = torch
        self.device = device

    def asarray(self, a):
        return self.torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=self.device)

    def qr(self, a):
        return self.torch.linalg.qr(a)

    def eigh(self, a):
        return self.torch.linalg.eigh(a)

    @staticmethod
    def to_numpy(a):
        return np.ascontiguousarray(a.cpu().numpy())


def _backend(device):
    if device is None or str(device) == "cpu":
        return _Np()
    return _Torch(device)


def _sym(a):
    return (a + a.T) * 0.5


def haar_orthogonal(rng: np.random.Generator, n: int, device=None):
    """Haar-distributed orthogonal matrix: QR of a Gaussian with the sign of diag(R) fixed."""
    be = _backend(device)
    g = be.asarray(rng.standard_normal((n, n)))
    q, r = be.qr(g)
    if isinstance(be, _Np):
        d = np.sign(np.diag(r))
        d[d == 0] = 1.0
        return q * d[None, :]
    t = be.torch
    d = t.sign(t.diagonal(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def _assemble(be, Q, lam, S_U, S_w):
    """H = S^{1/2} Q diag(lam) Q^T S^{1/2} and S = S_U diag(S_w) S_U^T, both symmetrised."""
    if isinstance(be, _Np):
        shalf = (S_U * np.sqrt(S_w)[None, :]) @ S_U.T
        S = (S_U * S_w[None, :]) @ S_U.T
        M = shalf @ Q
        H = (M * lam[None, :]) @ M.T
    else:
        t = be.torch
        S_w_t = t.as_tensor(S_w, device=be.device)
        lam_t = t.as_tensor(lam, device=be.device)
        shalf = (S_U * t.sqrt(S_w_t)[None, :]) @ S_U.T
        S = (S_U * S_w_t[None, :]) @ S_U.T
        M = shalf @ Q
        H = (M * lam_t[None, :]) @ M.T
    return _sym(H), _sym(S)


def _pinned_spectrum(rng, n, n_occ, occ_lo, gap, vir_hi, center=0.0):
    """Ascending spectrum: n_occ values U[occ_lo, center-gap/2] with the largest pinned to
    center-gap/2, n-n_occ values U[center+gap/2, vir_hi] with the smallest pinned to
    center+gap/2, so lam[n_occ] - lam[n_occ-1] == gap exactly (up to one rounding)."""
    lo_top = center - 0.5 * gap
    hi_bot = center + 0.5 * gap
    occ = np.sort(rng.uniform(occ_lo, lo_top, n_occ))
    vir = np.sort(rng.uniform(hi_bot, vir_hi, n - n_occ))
    if n_occ > 0:
        occ[-1] = lo_top
    if n - n_occ > 0:
        vir[0] = hi_bot
    return np.concatenate([occ, vir])


# --------------------------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------------------------

def make_config0(seed: int = 0, n: int = 256, n_occ: int = 64, device=None) -> Problem:
    """Plain single solve: n=256, n_occ=64.

    Q Haar; S = I + 0.1 (G + G^T) / (2 sqrt n), G Gaussian, redrawn while cond(S) > 10;
    occupied lam ~ U[-2, -0.5], virtual lam ~ U[0.5, 3] (gap >= 1); H = S^{1/2} Q diag(lam) Q^T S^{1/2}.
    """
    rng = np.random.default_rng(seed)
    be = _backend(device)
    Q = haar_orthogonal(rng, n, device)
    while True:
        G = rng.standard_normal((n, n))
        S0 = np.eye(n) + 0.1 * (G + G.T) / (2.0 * math.sqrt(n))
        S_w, S_U = be.eigh(be.asarray(S0))
        w = be.to_numpy(S_w)
        if w.min() > 0 and w.max() / w.min() <= 10.0:
            break
    occ = np.sort(rng.uniform(-2.0, -0.5, n_occ))
    vir = np.sort(rng.uniform(0.5, 3.0, n - n_occ))
    lam = np.concatenate([occ, vir])
    H, S = _assemble(be, Q, lam, S_U, w)
    return _finish(be, H, S, n_occ, Q, lam, S_U, w,
                   dict(config="config0", seed=seed, n=n, n_occ=n_occ,
                        gap=float(lam[n_occ] - lam[n_occ - 1]) if 0 < n_occ < n else None,
                        cond_S=float(w.max() / w.min())))


def make_spectrum_problem(seed: int, n: int, n_occ: int, cond_S: float, gap: float,
                          occ_lo: float = -3.0, vir_hi: float = 10.0, device=None,
                          config: str = "spectrum") -> Problem:
    """S = Q_s diag(sigma) Q_s^T with sigma log-spaced over [1/cond_S, 1] scaled to mean 1;
    H = S^{1/2} Q diag(lam) Q^T S^{1/2} with a pinned gap (see _pinned_spectrum)."""
    rng = np.random.default_rng(seed)
    be = _backend(device)
    Q = haar_orthogonal(rng, n, device)
    Qs = haar_orthogonal(rng, n, device)
    sig = np.logspace(-math.log10(cond_S), 0.0, n)
    sig = sig * (n / sig.sum())
    lam = _pinned_spectrum(rng, n, n_occ, occ_lo, gap, vir_hi)
    H, S = _assemble(be, Q, lam, Qs, sig)
    return _finish(be, H, S, n_occ, Q, lam, Qs, sig,
                   dict(config=config, seed=seed, n=n, n_occ=n_occ, gap=gap, cond_S=cond_S,
                        occ_lo=occ_lo, vir_hi=vir_hi))


def make_config1(seed: int = 1, n: int = 4096, n_occ: int = 1024, device=None) -> Problem:
    """All-electron-like dense insulator: n=4096, n_occ=1024, cond(S)=1e3 (log-spaced spectrum,
    Haar eigenvectors, mean eigenvalue 1), occupied U[-3, -0.1], virtual U[0.1, 10], gap 0.2."""
    return make_spectrum_problem(seed, n, n_occ, cond_S=1e3, gap=0.2, occ_lo=-3.0, vir_hi=10.0,
                                 device=device, config="config1")


def make_config2(seed: int = 2, n: int = 8192, n_occ: int = 2048, s_amp: float = 0.3,
                 device=None) -> Problem:
    """DFTB-like large system: n=8192, n_occ=2048.

    g Gaussian, symmetrised (g + g^T)/sqrt 2; H_base_ij = g_ij exp(-|i-j|/64).  H_base = V L V^T;
    the occupied part of L is shifted down and the virtual part up by equal amounts so that the
    gap at n_occ is exactly 0.05; that matrix is the orthogonalised Hamiltonian.
    S = I + s_amp * exp(-|i-j|/8) off the diagonal (s_amp = 0.3 gives cond(S) ~ 7.7);
    H = S^{1/2} (V L' V^T) S^{1/2}.
    """
    rng = np.random.default_rng(seed)
    be = _backend(device)
    g = rng.standard_normal((n, n))
    g = (g + g.T) / math.sqrt(2.0)
    idx = np.arange(n)
    dist = np.abs(idx[:, None] - idx[None, :]).astype(np.float64)
    Hb = g * np.exp(-dist / 64.0)
    del g
    L, V = be.eigh(be.asarray(Hb))
    L = be.to_numpy(L).copy()
    shift = 0.5 * (0.05 - (L[n_occ] - L[n_occ - 1]))
    L[:n_occ] -= shift
    L[n_occ:] += shift
    L[n_occ] = L[n_occ - 1] + 0.05
    S0 = np.eye(n) + s_amp * np.exp(-dist / 8.0) * (1.0 - np.eye(n))
    del dist
    S_w, S_U = be.eigh(be.asarray(S0))
    w = be.to_numpy(S_w)
    H, S = _assemble(be, V, L, S_U, w)
    return _finish(be, H, S, n_occ, V, L, S_U, w,
                   dict(config="config2", seed=seed, n=n, n_occ=n_occ, gap=0.05,
                        s_amp=s_amp, cond_S=float(w.max() / w.min())))


def make_banded(seed: int, n: int, n_occ: int, decay: float = 8.0, gap: float = 0.5,
                s_amp: float = 0.3, s_decay: float = 8.0, device=None) -> Problem:
    """Local (sparse-regime) variant of config 2: H_base_ij = g_ij exp(-|i-j|/decay) with the
    gap at n_occ opened to `gap` by shifting the occupied / virtual eigenvalues apart, and
    S = I + s_amp exp(-|i-j|/s_decay) off the diagonal (s_amp = 0 gives S = I, an orthogonal
    basis).  With decay 8 and gap 0.5 the density matrix decays fast enough that most of its
    128 x 128 tiles fall below 1e-5 at n = 2048 and above."""
    rng = np.random.default_rng(seed)
    be = _backend(device)
    g = rng.standard_normal((n, n))
    g = (g + g.T) / math.sqrt(2.0)
    idx = np.arange(n)
    dist = np.abs(idx[:, None] - idx[None, :]).astype(np.float64)
    Hb = g * np.exp(-dist / decay)
    del g
    L, V = be.eigh(be.asarray(Hb))
    L = be.to_numpy(L).copy()
    shift = 0.5 * (gap - (L[n_occ] - L[n_occ - 1]))
    L[:n_occ] -= shift
    L[n_occ:] += shift
    L[n_occ] = L[n_occ - 1] + gap
    S0 = np.eye(n) + s_amp * np.exp(-dist / s_decay) * (1.0 - np.eye(n))
    del dist
    S_w, S_U = be.eigh(be.asarray(S0))
    w = be.to_numpy(S_w)
    if s_amp == 0.0:
        S_U = be.asarray(np.eye(n))
        w = np.ones(n)
    H, S = _assemble(be, V, L, S_U, w)
    return _finish(be, H, S, n_occ, V, L, S_U, w,
                   dict(config="banded", seed=seed, n=n, n_occ=n_occ, decay=decay, gap=gap,
                        s_amp=s_amp, cond_S=float(w.max() / w.min())))


def make_batch_config3(seed: int = 3, count: int = 64, n_lo: int = 512, n_hi: int = 3072,
                       device=None):
    """Batched spin / multi-molecule set: `count` independent problems, n log-uniform in
    [n_lo, n_hi], n_occ = round(n/4), cond(S) log-uniform in [10, 1e3], gap log-uniform in
    [0.05, 0.5]; per-problem seed = seed*1000 + i; spectrum U[-2, -gap/2] / U[gap/2, 3]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        cond = float(math.exp(rng.uniform(math.log(10.0), math.log(1e3))))
        gap = float(math.exp(rng.uniform(math.log(0.05), math.log(0.5))))
        out.append(make_spectrum_problem(seed * 1000 + i, n, int(round(0.25 * n)), cond, gap,
                                         occ_lo=-2.0, vir_hi=3.0, device=device,
                                         config="config3"))
    return out


def make_request_stream(seed: int = 4, count: int = 2000, rate: float = 200.0,
                        n_lo: int = 256, n_hi: int = 8192):
    """Serving stream recipe: Poisson arrivals at `rate` req/s and per-request sizes.

    Returns a list of dicts {arrival_s, n, n_occ, gap, seed}; inputs are built per request with
    make_request_problem (S as in config 0, pinned gap).  Drawing the inputs lazily keeps the
    2000-request stream from holding ~100 GB of host memory.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        gap = float(math.exp(rng.uniform(math.log(0.05), math.log(0.5))))
        reqs.append(dict(arrival_s=t, n=n, n_occ=int(round(0.25 * n)), gap=gap,
                         seed=seed * 100000 + i))
    return reqs


def make_request_problem(req: dict, device=None) -> Problem:
    """One serving request: S as in config 0, H with pinned gap `req['gap']`."""
    rng = np.random.default_rng(req["seed"])
    n, n_occ, gap = req["n"], req["n_occ"], req["gap"]
    be = _backend(device)
    Q = haar_orthogonal(rng, n, device)
    G = rng.standard_normal((n, n))
    S0 = np.eye(n) + 0.1 * (G + G.T) / (2.0 * math.sqrt(n))
    S_w, S_U = be.eigh(be.asarray(S0))
    w = be.to_numpy(S_w)
    lam = _pinned_spectrum(rng, n, n_occ, -2.0, gap, 3.0)
    H, S = _assemble(be, Q, lam, S_U, w)
    return _finish(be, H, S, n_occ, Q, lam, S_U, w,
                   dict(config="config4", seed=req["seed"], n=n, n_occ=n_occ, gap=gap,
                        cond_S=float(w.max() / w.min())))


def make_small_diag(seed: int, n: int, n_occ: int) -> Problem:
    """Diagonal H and S (positive s_ii): the generalised eigenpairs are (h_ii/s_ii, e_i/sqrt s_ii)."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(-2.0, 2.0, n)
    s = rng.uniform(0.5, 2.0, n)
    return Problem(np.diag(h), np.diag(s), n_occ, None,
                   dict(config="diag", seed=seed, n=n, n_occ=n_occ))


def make_random_small(seed: int, n: int, n_occ: int, s_scale: float = 0.2) -> Problem:
    """Unstructured small case: H = sym Gaussian, S = I + s_scale * sym Gaussian / sqrt n
    (redrawn until S is positive definite)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    H = _sym(A)
    while True:
        B = rng.standard_normal((n, n))
        S = np.eye(n) + s_scale * _sym(B) / math.sqrt(n)
        if np.linalg.eigvalsh(S).min() > 0.05:
            break
    return Problem(np.ascontiguousarray(H), np.ascontiguousarray(S), n_occ, None,
                   dict(config="random", seed=seed, n=n, n_occ=n_occ))


def _finish(be, H, S, n_occ, Q, lam, S_U, S_w, meta) -> Problem:
    return Problem(np.ascontiguousarray(be.to_numpy(H)), np.ascontiguousarray(be.to_numpy(S)),
                   int(n_occ),
                   dict(Q=be.to_numpy(Q), lam=np.asarray(lam, dtype=np.float64),
                        S_U=be.to_numpy(S_U), S_w=np.asarray(S_w, dtype=np.float64)),
                   meta)


def make_geometry_step(p: Problem, seed: int, eps: float = 0.02) -> Problem:
    """The next geometry of a constructed problem: S rotated and rescaled a little,
    S' = U' diag(w') U'^T with U' = U_s R (R the orthogonal factor of I + eps G) and
    w' = w_s exp(eps xi), G and xi Gaussian; H' = S'^{1/2} Q diag(lam) Q^T S'^{1/2} keeps the
    orthogonal-basis eigenvectors Q and the spectrum lam of `p`.  (Then the Loewdin-form
    extrapolation of p's density matrix is exactly the density matrix of the new geometry.)"""
    f = p.factors
    if f is None:
        raise ValueError("make_geometry_step needs a problem built from factors")
    rng = np.random.default_rng(seed)
    n = p.n
    G = rng.standard_normal((n, n))
    R, r = np.linalg.qr(np.eye(n) + eps * G)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    R = R * d[None, :]
    S_U = np.asarray(f["S_U"]) @ R
    S_w = np.asarray(f["S_w"]) * np.exp(eps * rng.standard_normal(n))
    Q = np.asarray(f["Q"])
    lam = np.asarray(f["lam"])
    be = _Np()
    H, S = _assemble(be, Q, lam, S_U, S_w)
    meta = dict(p.meta)
    meta.update(config=str(p.meta.get("config", "")) + "+step", step_seed=seed, step_eps=eps,
                cond_S=float(S_w.max() / S_w.min()))
    return _finish(be, H, S, p.n_occ, Q, lam, S_U, S_w, meta)


"""Step-level FP64 definitions of the purification route - TEST INFRASTRUCTURE ONLY.

Each function is the plain numpy statement of one step, in the paper's order:

  1. Loewdin orthogonalisation H~ = S^{-1/2} H S^{-1/2}           (Sec. 2.2.2, Eq. ntpoly_lowdin)
     here with S^{-1/2} from the coupled Newton-Schulz iteration (`newton_schulz_inv_sqrt`), an
     iteration the paper does not name (it names only the Loewdin factor); the Jacobi factor of
     the C oracle is the definition it is checked against.
  2. spectral bounds eps_min, eps_max, "(estimated)" in the paper: Gershgorin discs, which are
     guaranteed outer bounds (`gershgorin_bounds`).
  3. initial guess P_0 = (eps_max I - H~) / (eps_max - eps_min)    (Eq. ntpoly_scale_hamiltonian)
  4. P_{n+1} = f(P_n), f = the 4th-order trace-resetting map the paper selects (Sec. 4, Table 1;
     it cites the method without printing it):  F(X) = X^2 (4X - 3X^2),  G(X) = X^2 (I - X)^2,
     gamma = (N - Tr F) / Tr G,  X <- F + gamma G  for 0 <= gamma <= 6, X <- 2X - X^2 for
     gamma > 6, X <- X^2 for gamma < 0                               (Eq. ntpoly_purification)
  5. back-transform P = S^{-1/2} P~ S^{-1/2}, and the outputs Tr(P S), Tr(P H)
                                                      (Sec. 4 "back-transforming the density matrix")
The paper's Sec. 2.2.2 also names 2nd-order trace resetting, canonical purification and the
generalised hole-particle canonical purification, without formulas; `trs2_step` and
`canonical_step` state the maps of the cited methods that are built, `hole_particle_step` the
hole-particle form that turns out to coincide with the canonical step.  `trs4_filtered_step` and
`trs4_purify_truncated` are the sparse regime the same section describes: every matrix entering
a product is filtered at a threshold (elements below it set to zero).
Closed forms for the synthetic inputs are at the end.  Matrix products are numpy matmul
(a library primitive); there is no blocking, fusion or reordering beyond the formulas.
"""
from __future__ import annotations

import numpy as np


def sym(a):
    return 0.5 * (a + a.T)


# ------------------------------------------------------------------------------------------
# bounds and initial guess
# ------------------------------------------------------------------------------------------

def gershgorin_bounds(A):
    """Outer bounds of the spectrum of symmetric A: min_i (a_ii - r_i), max_i (a_ii + r_i),
    r_i = sum_{j != i} |a_ij|."""
    A = np.asarray(A, dtype=np.float64)
    d = np.diag(A)
    r = np.abs(A).sum(axis=1) - np.abs(d)
    return float((d - r).min()), float((d + r).max())


def initial_guess(Ht, eps_min, eps_max):
    """P_0 = (eps_max I - H~) / (eps_max - eps_min)  (Eq. ntpoly_scale_hamiltonian)."""
    n = Ht.shape[0]
    return (eps_max * np.eye(n) - Ht) / (eps_max - eps_min)


# ------------------------------------------------------------------------------------------
# trace-resetting purification (TRS4)
# ------------------------------------------------------------------------------------------

def trs4_F(X):
    X2 = X @ X
    return X2 @ (4.0 * X - 3.0 * X2)


def trs4_G(X):
    n = X.shape[0]
    Y = np.eye(n) - X
    return (X @ X) @ (Y @ Y)


def trs4_gamma(X, n_occ):
    """gamma = (N - Tr F(X)) / Tr G(X); returns (gamma, Tr F, Tr G)."""
    trF = float(np.trace(trs4_F(X)))
    trG = float(np.trace(trs4_G(X)))
    return (n_occ - trF) / trG if trG != 0.0 else float("inf"), trF, trG


def trs4_step(X, n_occ, gamma_min=0.0, gamma_max=6.0):
    """One TRS4 step.  Returns (X_next, gamma, branch) with branch in {"2X-X2", "X2", "F+gG"}."""
    g, _, _ = trs4_gamma(X, n_occ)
    X2 = X @ X
    if g > gamma_max:
        return sym(2.0 * X - X2), g, "2X-X2"
    if g < gamma_min:
        return sym(X2), g, "X2"
    return sym(trs4_F(X) + g * trs4_G(X)), g, "F+gG"


def trs4_purify(Ht, n_occ, max_iter=200, idem_tol=1e-13, bounds=None):
    """Full TRS4 purification of an orthogonal-basis Hamiltonian.
    Stops when ||X^2 - X||_F <= idem_tol * sqrt(n) (or Tr G underflows).
    Returns (P~, iterations, list of (gamma, branch))."""
    n = Ht.shape[0]
    lo, hi = gershgorin_bounds(Ht) if bounds is None else bounds
    X = initial_guess(Ht, lo, hi)
    hist = []
    for it in range(max_iter):
        err = np.linalg.norm(X @ X - X)
        if err <= idem_tol * np.sqrt(n):
            return X, it, hist
        g, trF, trG = trs4_gamma(X, n_occ)
        if trG <= 1e-300:
            return X, it, hist
        X, g, br = trs4_step(X, n_occ)
        hist.append((g, br))
    return X, max_iter, hist


def mcweeny(X):
    """McWeeny purification 3X^2 - 2X^3 (an idempotency fixer used for the final sweeps)."""
    X2 = X @ X
    return sym(3.0 * X2 - 2.0 * X2 @ X)


# ------------------------------------------------------------------------------------------
# the other purification maps the paper names (Sec. 2.2.2): 2nd-order trace resetting,
# canonical purification, generalised (hole-particle) canonical purification
# ------------------------------------------------------------------------------------------

def trs2_step(X, n_occ):
    """2nd-order trace-resetting step: of X^2 (lowers the trace) and 2X - X^2 (raises it) take the
    one whose trace lands nearer N.  Returns (X_next, branch)."""
    X2 = X @ X
    t1 = float(np.trace(X))
    t2 = float(np.trace(X2))
    if abs(t2 - n_occ) <= abs(2.0 * t1 - t2 - n_occ):
        return sym(X2), "X2"
    return sym(2.0 * X - X2), "2X-X2"


def canonical_initial_guess(Ht, n_occ, eps_min, eps_max):
    """Initial guess of canonical purification: X0 = (lam/n)(mu I - H~) + (N/n) I with
    mu = Tr H~ / n and lam = min(N / (eps_max - mu), (n - N) / (mu - eps_min)), so that
    Tr X0 = N and the spectrum of X0 lies in [0, 1]."""
    n = Ht.shape[0]
    mu = float(np.trace(Ht)) / n
    lam = min(n_occ / (eps_max - mu), (n - n_occ) / (mu - eps_min))
    return (lam / n) * (mu * np.eye(n) - Ht) + (n_occ / n) * np.eye(n)


def canonical_c(X):
    """c = Tr(X^2 - X^3) / Tr(X - X^2), the weight both canonical maps take from X."""
    X2 = X @ X
    X3 = X2 @ X
    return float(np.trace(X2 - X3)) / float(np.trace(X - X2))


def canonical_step(X):
    """Canonical purification step (keeps Tr X): with c = canonical_c(X),
    c >= 1/2: X <- ((1 + c) X^2 - X^3) / c;  c < 1/2: X <- ((1 - 2c) X + (1 + c) X^2 - X^3) / (1 - c).
    Returns (X_next, c)."""
    c = canonical_c(X)
    X2 = X @ X
    X3 = X2 @ X
    if c >= 0.5:
        return sym(((1.0 + c) * X2 - X3) / c), c
    return sym(((1.0 - 2.0 * c) * X + (1.0 + c) * X2 - X3) / (1.0 - c)), c


def hole_particle_step(X):
    """Hole-particle form of a trace-keeping cubic step, with the hole matrix I - X:
    X <- X + beta (X^2 (I - X) - c X (I - X)),  c = Tr(X^2 (I - X)) / Tr(X (I - X)),
    beta = 1 / max(c, 1 - c), the longest step for which the eigenvalue map stays monotone on
    [0, 1].  With this beta it is the canonical step term by term (a pin checks that), which is
    why no separate hole-particle method is built.  Returns (X_next, c, beta)."""
    n = X.shape[0]
    Xh = np.eye(n) - X
    X2 = X @ X
    c = float(np.trace(X2 @ Xh)) / float(np.trace(X @ Xh))
    beta = 1.0 / max(c, 1.0 - c)
    return sym(X + beta * (X2 @ Xh - c * (X @ Xh))), c, beta


def purify(Ht, n_occ, method, max_iter=400, idem_tol=1e-13, bounds=None):
    """Purification of an orthogonal-basis Hamiltonian with `method` in
    {"trs4", "trs2", "canonical"}, from the method's own initial guess, until
    ||X^2 - X||_F <= idem_tol * sqrt(n).  Returns (P~, iterations, traces of the iterates)."""
    n = Ht.shape[0]
    lo, hi = gershgorin_bounds(Ht) if bounds is None else bounds
    if method in ("trs4", "trs2"):
        X = initial_guess(Ht, lo, hi)
    else:
        X = canonical_initial_guess(Ht, n_occ, lo, hi)
    traces = [float(np.trace(X))]
    for it in range(max_iter):
        if np.linalg.norm(X @ X - X) <= idem_tol * np.sqrt(n):
            return X, it, traces
        if method == "trs4":
            X, _, _ = trs4_step(X, n_occ)
        elif method == "trs2":
            X, _ = trs2_step(X, n_occ)
        elif method == "canonical":
            X, _ = canonical_step(X)
        else:
            raise ValueError("unknown purification method %r" % (method,))
        traces.append(float(np.trace(X)))
    return X, max_iter, traces


# ------------------------------------------------------------------------------------------
# truncated (filtered) purification, the sparse regime of Sec. 2.2.2
# ------------------------------------------------------------------------------------------

def filter_small(A, tau):
    """Elements with |a_ij| < tau set to zero (the paper's threshold filtering, Sec. 2.2.2)."""
    return np.where(np.abs(A) >= tau, A, 0.0)


def trs4_filtered_step(X, n_occ, tau):
    """One TRS4 step of the sparse regime: the paper's 4th-order trace-resetting map with every
    matrix that enters a product filtered at tau.  X (already filtered) enters X X; the product
    is filtered, and that filtered matrix is X^2 wherever the map uses it.  With
    F = X^2 (4X - 3X^2) and G = X^2 (I - X)^2 the traces are
    Tr F = 4 <X^2, X> - 3 ||X^2||^2 and Tr G = Tr X^2 - 2 <X^2, X> + ||X^2||^2, and
    gamma = (N - Tr F) / Tr G.  Then
      gamma > 6:  X <- filter(2X - X^2)
      gamma < 0:  X <- X^2 (already filtered)
      otherwise:  F + gamma G = X^2 W with W = gamma I + (4 - 2 gamma) X + (gamma - 3) X^2;
                  W is filtered (it enters the product), X^2 W is formed, symmetrised (the
                  filtered X^2 and W need not commute) and filtered.
    Returns (X_next, dict(X2=filtered X^2, gamma, branch, W=filtered W or None))."""
    n = X.shape[0]
    X2 = filter_small(X @ X, tau)
    t2, t3, t4 = float(np.trace(X2)), float(np.sum(X2 * X)), float(np.sum(X2 * X2))
    trF = 4.0 * t3 - 3.0 * t4
    trG = t2 - 2.0 * t3 + t4
    g = (n_occ - trF) / trG if trG != 0.0 else float("inf")
    info = dict(X2=X2, gamma=g, W=None, trF=trF, trG=trG)
    if g > 6.0:
        info["branch"] = "2X-X2"
        return filter_small(2.0 * X - X2, tau), info
    if g < 0.0:
        info["branch"] = "X2"
        return X2, info
    W = filter_small(g * np.eye(n) + (4.0 - 2.0 * g) * X + (g - 3.0) * X2, tau)
    info.update(branch="F+gG", W=W)
    return filter_small(sym(X2 @ W), tau), info


def trs4_purify_truncated(Ht, n_occ, tau, max_iter=200, bounds=None, idem_tol=1e-13):
    """The filtered TRS4 route from the filtered initial guess (Eq. ntpoly_scale_hamiltonian):
    `trs4_filtered_step` until the idempotency error e = Tr(X - X^2) (X^2 the filtered square)
    has not reached a new low for five steps in a row: filtering leaves a floor of the order of
    the threshold's effect, and steps past it only move X along that floor, so the iterate with
    the smallest |e| is returned.
    The loop also ends at e <= idem_tol N, or when Tr G is exactly zero (gamma undefined: X is
    a projector).  tau = 0 is plain TRS4.  Returns (P~, iterations)."""
    lo, hi = gershgorin_bounds(Ht) if bounds is None else bounds
    X = filter_small(initial_guess(Ht, lo, hi), tau)
    best, best_e = X, np.inf
    rises = 0
    it = 0
    for it in range(max_iter):
        X2 = filter_small(X @ X, tau)
        e = abs(float(np.trace(X) - np.trace(X2)))
        trG = float(np.trace(X2) - 2.0 * np.sum(X2 * X) + np.sum(X2 * X2))
        if e < best_e:
            best, best_e, rises = X, e, 0
        else:
            rises += 1
            if rises >= 5:
                break
        if e <= idem_tol * n_occ or trG == 0.0:
            break
        X, _ = trs4_filtered_step(X, n_occ, tau)
    return best, it


# ------------------------------------------------------------------------------------------
# Loewdin factor by Newton-Schulz
# ------------------------------------------------------------------------------------------

def newton_schulz_inv_sqrt(S, tol=1e-14, max_iter=100):
    """Coupled Newton-Schulz iteration for S^{-1/2}:
    c >= lambda_max(S) (Gershgorin), Y_0 = S/c, Z_0 = I;
    T_k = (3I - Z_k Y_k)/2, Y_{k+1} = Y_k T_k, Z_{k+1} = T_k Z_k;  Z = Z_k / sqrt(c).
    Y_k -> (S/c)^{1/2} and Z_k -> (S/c)^{-1/2}; the residual is ||I - Z_k Y_k||_F.
    Stops when the residual is <= tol * sqrt(n) or stops decreasing once below 1e-6 * sqrt(n)
    (the iteration is only neutrally stable past convergence).  Returns (Z, iterations)."""
    n = S.shape[0]
    _, c = gershgorin_bounds(S)
    I = np.eye(n)
    Y = S / c
    Z = I.copy()
    prev = np.inf
    for it in range(max_iter):
        R = I - Z @ Y
        res = np.linalg.norm(R)
        if res <= tol * np.sqrt(n) or (res <= 1e-6 * np.sqrt(n) and res >= prev):
            return sym(Z) / np.sqrt(c), it
        prev = res
        T = I + 0.5 * R
        Y = Y @ T
        Z = T @ Z
    return sym(Z) / np.sqrt(c), max_iter


def inv_sqrt_refine(Z, S):
    """One step of the residual refinement of an approximate S^{-1/2}:
    delta = I - Z S Z,  Z <- Z (I + delta/2 + 3 delta^2 / 8)  (Taylor series of (I - delta)^{-1/2}),
    symmetrised."""
    n = S.shape[0]
    I = np.eye(n)
    d = I - Z @ S @ Z
    return sym(Z @ (I + 0.5 * d + 0.375 * d @ d))


# ------------------------------------------------------------------------------------------
# the whole route (for cross-checks of the route against the definition)
# ------------------------------------------------------------------------------------------

def purification_route(H, S, n_occ):
    """NS Loewdin -> H~ = Z H Z -> TRS4 -> P = Z P~ Z.  Returns dict(P, energy, trace_ps, ...)."""
    H = sym(np.asarray(H, dtype=np.float64))
    S = sym(np.asarray(S, dtype=np.float64))
    Z, ns_it = newton_schulz_inv_sqrt(S)
    Ht = sym(Z @ H @ Z)
    Pt, it, hist = trs4_purify(Ht, n_occ)
    P = sym(Z @ Pt @ Z)
    return dict(P=P, energy=float(np.sum(P * H)), trace_ps=float(np.sum(P * S)),
                ns_iters=ns_it, purif_iters=it, history=hist, Z=Z, Ht=Ht)


# ------------------------------------------------------------------------------------------
# closed forms and invariants
# ------------------------------------------------------------------------------------------

def closed_form_dm(factors, n_occ):
    """For H = S^{1/2} Q diag(lam) Q^T S^{1/2}, S = U diag(w) U^T:
    C = S^{-1/2} Q solves H C = S C diag(lam) with C^T S C = I (Eq. evp), so
    P = S^{-1/2} Q[:, :N] Q[:, :N]^T S^{-1/2} and E = sum lam[:N] (Eq. density_matrix)."""
    U, w, Q, lam = factors["S_U"], factors["S_w"], factors["Q"], factors["lam"]
    Sm12 = (U * (1.0 / np.sqrt(w))[None, :]) @ U.T
    C = Sm12 @ Q[:, :n_occ]
    return sym(C @ C.T), float(np.sum(lam[:n_occ]))


def closed_form_edm(factors, n_occ):
    """Energy-weighted density matrix of the constructed input (Sec. 2.6, Eq.
    energy_density_matrix): C = S^{-1/2} Q, Q_edm = C[:, :N] diag(lam[:N]) C[:, :N]^T."""
    U, w, Q, lam = factors["S_U"], factors["S_w"], factors["Q"], factors["lam"]
    Sm12 = (U * (1.0 / np.sqrt(w))[None, :]) @ U.T
    C = Sm12 @ Q[:, :n_occ]
    return sym((C * lam[:n_occ][None, :]) @ C.T)


def closed_form_inv_sqrt(factors):
    """S^{-1/2} = U diag(w^{-1/2}) U^T from the construction factors of S."""
    U, w = factors["S_U"], factors["S_w"]
    return sym((U * (1.0 / np.sqrt(w))[None, :]) @ U.T)


def invariants(P, H, S, n_occ):
    """Checks of Eq. density_matrix_conditions mapped to the non-orthogonal metric:
    ||P S P - P||_F, |Tr(P S) - N|, ||P - P^T||_F, ||H P S - S P H||_F, Tr(P H)."""
    PS = P @ S
    return dict(idem=float(np.linalg.norm(PS @ P - P)),
                trace_err=float(abs(np.trace(PS) - n_occ)),
                asym=float(np.linalg.norm(P - P.T)),
                commut=float(np.linalg.norm(H @ P @ S - S @ P @ H)),
                energy=float(np.sum(P * H)))

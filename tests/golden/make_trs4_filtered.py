#!/usr/bin/env python3
"""Write trs4_filtered_6x6.json: two threshold-filtered TRS4 steps on a 6 x 6 banded matrix,
computed in exact rational arithmetic (fractions.Fraction), with every intermediate matrix.

The steps follow the paper's purification route (Sec. 2.2.2): the initial guess
X0 = (eps_max I - H~)/(eps_max - eps_min) from Gershgorin bounds (Eq. ntpoly_scale_hamiltonian),
the trace-resetting 4th-order map P_{n+1} = f(P_n) (Eq. ntpoly_purification; Sec. 4, Table 1)
with F = X^2 (4X - 3X^2), G = X^2 (I - X)^2, gamma = (N - Tr F)/Tr G, and NTPoly's sparsity
by threshold filtering (elements below tau set to zero) of every matrix that enters a product.
In the filtered step, X^2 is the filtered product X X; then F + gamma G = X^2 W with
W = gamma I + (4 - 2 gamma) X + (gamma - 3) X^2, W is filtered, the product X^2 W (no longer
symmetric, since filtered X^2 and W do not commute) is symmetrised and then filtered.

The case is chosen so that each filter placement matters: X0, X^2 and W each have an element
below tau, and in the second step one off-diagonal pair of X^2 W straddles tau (the two entries
lie on either side of it while their mean is above it), so filtering before symmetrising would
give a different matrix.  Every value is exact; the JSON holds the nearest doubles.  Nothing here
calls the GPU path or the oracle.

    python tests/golden/make_trs4_filtered.py   # rewrites the JSON beside this file
"""
import json
import os
from fractions import Fraction as Fr

HERE = os.path.dirname(os.path.abspath(__file__))

H_TILDE = [["9/4", "-7/8", "-1/8", "0", "0", "0"],
           ["-7/8", "1/4", "-1", "1/8", "0", "0"],
           ["-1/8", "-1", "1", "1", "7/32", "0"],
           ["0", "1/8", "1", "-1/4", "-3/4", "1/32"],
           ["0", "0", "7/32", "-3/4", "-5/4", "-3/8"],
           ["0", "0", "0", "1/32", "-3/8", "-5/2"]]
N_OCC = 3
TAU = Fr(1, 128)
STEPS = 2


def mat(rows):
    return [[Fr(v) for v in r] for r in rows]


def mul(A, B):
    n = len(A)
    return [[sum(A[i][k] * B[k][j] for k in range(n)) for j in range(n)] for i in range(n)]


def filtered(A):
    return [[a if abs(a) >= TAU else Fr(0) for a in r] for r in A]


def symmetrised(A):
    n = len(A)
    return [[(A[i][j] + A[j][i]) / 2 for j in range(n)] for i in range(n)]


def trace(A):
    return sum(A[i][i] for i in range(len(A)))


def inner(A, B):
    return sum(a * b for ra, rb in zip(A, B) for a, b in zip(ra, rb))


def below(A):
    """Non-zero entries below tau (the ones a filter removes)."""
    return [[i, j] for i, r in enumerate(A) for j, a in enumerate(r) if 0 < abs(a) < TAU]


def margin(*mats):
    """Smallest relative distance of any entry from tau: how far the float64 rounding of the
    oracle is from flipping a filter decision."""
    return min(abs(abs(a) - TAU) / TAU for A in mats for r in A for a in r if a != 0)


def as_float(A):
    return [[float(a) for a in r] for r in A]


def main():
    Ht = mat(H_TILDE)
    n = len(Ht)
    radius = [sum(abs(Ht[i][j]) for j in range(n) if j != i) for i in range(n)]
    lo = min(Ht[i][i] - radius[i] for i in range(n))
    hi = max(Ht[i][i] + radius[i] for i in range(n))
    X0 = [[((hi if i == j else 0) - Ht[i][j]) / (hi - lo) for j in range(n)] for i in range(n)]
    X = filtered(X0)
    out = {"citation": "Sec. 2.2.2 (threshold filtering; trace-resetting purification), "
                       "Eq. ntpoly_scale_hamiltonian, Eq. ntpoly_purification, Sec. 4 Table 1",
           "H_tilde": as_float(Ht), "n_occ": N_OCC, "tau": float(TAU),
           "eps_min": float(lo), "eps_max": float(hi),
           "X0": as_float(X0), "X0_filtered": as_float(X), "X0_below_tau": below(X0),
           "steps": []}
    margins = [margin(X0)]
    for _ in range(STEPS):
        X2 = mul(X, X)
        X2f = filtered(X2)
        t1, t2, t3, t4 = trace(X), trace(X2f), inner(X2f, X), inner(X2f, X2f)
        trF = 4 * t3 - 3 * t4
        trG = t2 - 2 * t3 + t4
        gamma = (N_OCC - trF) / trG
        assert 0 <= gamma <= 6, "this case takes the F + gamma G branch in both steps"
        W = [[(gamma if i == j else 0) + (4 - 2 * gamma) * X[i][j] + (gamma - 3) * X2f[i][j]
              for j in range(n)] for i in range(n)]
        Wf = filtered(W)
        M = mul(X2f, Wf)
        Msym = symmetrised(M)
        Xn = filtered(Msym)
        margins += [margin(X2), margin(W), margin(Msym), margin(M)]
        out["steps"].append({
            "X2": as_float(X2), "X2_filtered": as_float(X2f), "X2_below_tau": below(X2),
            "traces": {"t1": float(t1), "t2": float(t2), "t3": float(t3), "t4": float(t4)},
            "trF": float(trF), "trG": float(trG), "gamma": float(gamma),
            "W": as_float(W), "W_filtered": as_float(Wf), "W_below_tau": below(W),
            "X2W": as_float(M), "X2W_symmetrised": as_float(Msym),
            "X_next": as_float(Xn), "X_next_trace": float(trace(Xn)),
            "straddling_pairs": [[i, j] for i in range(n) for j in range(i + 1, n)
                                 if (abs(M[i][j]) < TAU) != (abs(M[j][i]) < TAU)]})
        X = Xn
    out["min_relative_margin_to_tau"] = float(min(margins))
    path = os.path.join(HERE, "trs4_filtered_6x6.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote %s (min margin to tau %.3g)" % (path, out["min_relative_margin_to_tau"]))


if __name__ == "__main__":
    main()

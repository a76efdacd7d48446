"""Pins for the CPU oracle (runs without a GPU).

The oracle is checked against things other than itself: closed forms of the synthetic inputs,
library eigensolvers on special cases, hand-derived golden values, invariants of the density
matrix (Sec. 2.2.2, Eq. density_matrix_conditions, mapped to the S metric) and brute force over
all occupation choices on tiny inputs.  A few tests plant a mistake in a copy of an oracle step
and check that a pin catches it.
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import steps
from oracle.lapack import density_matrix_eigh
from workloads import (make_config0, make_random_small, make_small_diag, make_spectrum_problem,
                       haar_orthogonal, make_geometry_step, make_banded)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# Both statements of the definition are pinned by the same closed forms, golden values, special
# cases, brute force and invariants: the Jacobi one (plain rotations, C) and the one with LAPACK's
# eigensolver (numpy), which evaluates the definition at the full workload sizes.
DM_IMPLS = {"jacobi": oracle.density_matrix, "lapack": density_matrix_eigh}


@pytest.fixture(params=sorted(DM_IMPLS))
def dm(request):
    return DM_IMPLS[request.param]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------------------------------
# Jacobi eigensolver
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 7, 40, 41])
def test_jacobi_recovers_constructed_spectrum(n):
    rng = np.random.default_rng(100 + n)
    Q = haar_orthogonal(rng, n)
    lam = np.sort(rng.uniform(-5, 5, n))
    A = (Q * lam) @ Q.T
    w, V, sweeps, st = oracle.jacobi_eigh(A)
    assert st == "OK"
    assert np.max(np.abs(w - lam)) <= 1e-12 * max(1.0, np.abs(lam).max())
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-12 * n
    assert np.linalg.norm(A @ V - V * w) <= 1e-11 * np.linalg.norm(A) + 1e-300


def test_jacobi_matches_library_eigvalsh():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((64, 64))
    A = A + A.T
    w, V, _, st = oracle.jacobi_eigh(A)
    assert st == "OK"
    np.testing.assert_allclose(w, np.linalg.eigvalsh(A), rtol=0, atol=1e-12 * np.abs(w).max())


def test_jacobi_repeated_eigenvalues_keep_orthonormal_basis():
    rng = np.random.default_rng(6)
    n = 12
    Q = haar_orthogonal(rng, n)
    lam = np.array([1.0] * 5 + [2.0] * 7)
    w, V, _, st = oracle.jacobi_eigh((Q * lam) @ Q.T)
    assert st == "OK"
    np.testing.assert_allclose(w, lam, atol=1e-13)
    assert np.linalg.norm(V.T @ V - np.eye(n)) < 1e-12


# ------------------------------------------------------------------------------------------
# density matrix: closed forms, special cases, golden values
# ------------------------------------------------------------------------------------------

def test_dm_config0_closed_form(dm):
    p = make_config0()
    r = dm(p.H, p.S, p.n_occ)
    Pc, Ec = steps.closed_form_dm(p.factors, p.n_occ)
    assert r["status"] == "OK"
    assert rel(r["P"], Pc) <= 1e-11
    assert abs(r["energy"] - Ec) <= 1e-10 * abs(Ec)
    assert abs(r["trace_ps"] - p.n_occ) <= 1e-10
    assert r["idem"] <= 1e-10
    np.testing.assert_allclose(r["evals"], p.factors["lam"], atol=1e-11)


@pytest.mark.parametrize("cond,gap", [(10.0, 0.5), (1e3, 0.2), (1e3, 0.05)])
def test_dm_ill_conditioned_overlap_closed_form(cond, gap, dm):
    p = make_spectrum_problem(7, 96, 24, cond_S=cond, gap=gap)
    r = dm(p.H, p.S, p.n_occ)
    Pc, Ec = steps.closed_form_dm(p.factors, p.n_occ)
    assert r["status"] == "OK"
    assert rel(r["P"], Pc) <= 1e-10
    assert abs(r["energy"] - Ec) <= 1e-10 * max(1.0, abs(Ec))
    assert abs(r["gap"] - gap) <= 1e-10


def test_dm_identity_overlap_is_standard_eigenproblem(dm):
    p = make_random_small(11, 50, 17)
    S = np.eye(50)
    r = dm(p.H, S, p.n_occ)
    w, V = np.linalg.eigh(p.H)
    Vo = V[:, :p.n_occ]
    assert rel(r["P"], Vo @ Vo.T) <= 1e-11
    assert abs(r["energy"] - w[:p.n_occ].sum()) <= 1e-11 * abs(w[:p.n_occ].sum())


def test_dm_diagonal_case(dm):
    p = make_small_diag(3, 20, 6)
    h, s = np.diag(p.H), np.diag(p.S)
    order = np.argsort(h / s, kind="stable")[:6]
    P_expect = np.zeros((20, 20))
    P_expect[order, order] = 1.0 / s[order]
    r = dm(p.H, p.S, 6)
    assert np.max(np.abs(r["P"] - P_expect)) <= 1e-13
    assert abs(r["energy"] - np.sort(h / s)[:6].sum()) <= 1e-13


def test_dm_golden_2x2(dm):
    with open(os.path.join(GOLDEN, "dm_2x2.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        r = dm(np.array(c["H"]), np.array(c["S"]), c["n_occ"])
        np.testing.assert_allclose(r["P"], np.array(c["P"]), atol=1e-14, err_msg=c["name"])
        assert abs(r["energy"] - c["energy"]) <= 1e-14, c["name"]
        np.testing.assert_allclose(r["evals"], c["evals"], atol=1e-14, err_msg=c["name"])


# ------------------------------------------------------------------------------------------
# Energy-weighted density matrix (Sec. 2.6, Eq. energy_density_matrix)
# ------------------------------------------------------------------------------------------

def test_edm_golden_2x2(dm):
    with open(os.path.join(GOLDEN, "dm_2x2.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        r = dm(np.array(c["H"]), np.array(c["S"]), c["n_occ"], edm=True)
        np.testing.assert_allclose(r["Q"], np.array(c["Q"]), atol=1e-14, err_msg=c["name"])


def test_edm_config0_closed_form(dm):
    p = make_config0()
    r = dm(p.H, p.S, p.n_occ, edm=True)
    Qc = steps.closed_form_edm(p.factors, p.n_occ)
    assert rel(r["Q"], Qc) <= 1e-11
    # the P computed alongside is unchanged by asking for Q
    assert np.array_equal(r["P"], dm(p.H, p.S, p.n_occ)["P"])


def test_edm_full_occupation_is_sinv_h_sinv(dm):
    # with every state occupied, C C^T = S^{-1} and Q = C diag(eps) C^T = S^{-1} H S^{-1}
    p = make_random_small(77, 24, 5)
    r = dm(p.H, p.S, 24, edm=True)
    Si = np.linalg.inv(p.S)
    assert rel(r["Q"], Si @ p.H @ Si) <= 1e-11


def test_edm_identities_on_unstructured_input(dm):
    # Q = P H P (C^T H C is diagonal), Tr(Q S) = sum of the occupied eigenvalues = Tr(P H),
    # and Q S P = Q (the range of Q lies in the occupied subspace)
    p = make_random_small(78, 40, 13)
    r = dm(p.H, p.S, 13, edm=True)
    Q, P = r["Q"], r["P"]
    assert rel(Q, P @ p.H @ P) <= 1e-11
    assert abs(np.sum(Q * p.S) - np.sum(r["evals"][:13])) <= 1e-11 * np.abs(r["evals"]).sum()
    assert abs(np.sum(Q * p.S) - r["energy"]) <= 1e-11 * abs(r["energy"])
    assert rel(Q @ p.S @ P, Q) <= 1e-11
    assert np.array_equal(Q, Q.T)


def test_edm_zero_occupation_is_zero():
    p = make_random_small(79, 10, 3)
    r = oracle.density_matrix(p.H, p.S, 0, edm=True)
    assert np.all(r["Q"] == 0.0)


def test_edm_pins_catch_plausible_mistakes():
    # each wrong formula below (a dropped factor, a missing occupation, the wrong eigenvalues)
    # fails the closed-form pin that the oracle's Q passes
    p = make_config0()
    Qc = steps.closed_form_edm(p.factors, p.n_occ)
    r = oracle.density_matrix(p.H, p.S, p.n_occ, edm=True)
    P = r["P"]
    Si = np.linalg.inv(p.S)
    lam = p.factors["lam"]
    U, w, Qf = p.factors["S_U"], p.factors["S_w"], p.factors["Q"]
    C = ((U * (1.0 / np.sqrt(w))[None, :]) @ U.T) @ Qf[:, :p.n_occ]
    wrong = {
        "P H": P @ p.H,
        "all states": Si @ p.H @ Si,
        "unoccupied eigenvalues": (C * lam[p.n_occ:2 * p.n_occ][None, :]) @ C.T,
        "S metric dropped": P @ p.S @ p.H @ p.S @ P,
    }
    assert rel(r["Q"], Qc) <= 1e-11
    for name, Qw in wrong.items():
        assert not rel(Qw, Qc) <= 1e-6, name


# ------------------------------------------------------------------------------------------
# Density-matrix extrapolation (Sec. 2.7, Loewdin form)
# ------------------------------------------------------------------------------------------

def test_extrapolation_closed_form_geometry_step():
    # the step keeps the orthogonal-basis eigenvectors, so the extrapolated P0 is exactly the
    # new geometry's density matrix S1^{-1/2} Q_occ Q_occ^T S1^{-1/2}
    p0 = make_spectrum_problem(31, 48, 12, cond_S=50.0, gap=0.3)
    p1 = make_geometry_step(p0, seed=5, eps=0.05)
    P0 = steps.closed_form_dm(p0.factors, p0.n_occ)[0]
    P1, st = oracle.extrapolate_dm(P0, p0.S, p1.S)
    assert st == "OK"
    assert rel(P1, steps.closed_form_dm(p1.factors, p1.n_occ)[0]) <= 1e-11
    assert rel(P1, oracle.density_matrix(p1.H, p1.S, p1.n_occ)["P"]) <= 1e-10


def test_extrapolation_same_overlap_is_identity_and_keeps_invariants():
    p = make_random_small(81, 30, 9)
    P0 = oracle.density_matrix(p.H, p.S, 9)["P"]
    P1, st = oracle.extrapolate_dm(P0, p.S, p.S)
    assert st == "OK" and rel(P1, P0) <= 1e-12
    # a different overlap: P1 is again a projector in the new metric with the same count
    q = make_random_small(82, 30, 9)
    P1, st = oracle.extrapolate_dm(P0, p.S, q.S)
    assert rel(P1 @ q.S @ P1, P1) <= 1e-11
    assert abs(np.sum(P1 * q.S) - 9) <= 1e-11


def test_extrapolation_diagonal_overlaps_by_hand():
    # S0 = I, S1 = diag(s): P1_ij = P0_ij / sqrt(s_i s_j)
    rng = np.random.default_rng(83)
    n = 9
    Q = haar_orthogonal(rng, n)
    P0 = Q[:, :4] @ Q[:, :4].T
    s1 = rng.uniform(0.5, 2.0, n)
    P1, st = oracle.extrapolate_dm(P0, np.eye(n), np.diag(s1))
    assert st == "OK"
    np.testing.assert_allclose(P1, P0 / np.sqrt(np.outer(s1, s1)), atol=1e-13)
    # a plausible mistake (S1^{-1} instead of S1^{-1/2}) breaks idempotency in the S1 metric
    Pw = P0 / np.outer(s1, s1)
    assert not rel(Pw @ np.diag(s1) @ Pw, Pw) <= 1e-6


def test_extrapolation_rejects_indefinite_overlap():
    S1 = np.eye(6)
    S1[2, 2] = -0.5
    P1, st = oracle.extrapolate_dm(np.eye(6) * 0.5, np.eye(6), S1)
    assert P1 is None and st == "NOT_SPD"


def test_dm_full_occupation_is_inverse_overlap(dm):
    p = make_random_small(12, 30, 30)
    r = dm(p.H, p.S, 30)
    assert rel(r["P"], np.linalg.inv(p.S)) <= 1e-12


def test_dm_zero_occupation(dm):
    p = make_random_small(13, 10, 0)
    r = dm(p.H, p.S, 0)
    assert np.all(r["P"] == 0.0) and r["energy"] == 0.0


@pytest.mark.parametrize("n,n_occ", [(4, 2), (6, 2), (7, 3), (8, 4)])
def test_dm_brute_force_minimum(n, n_occ, dm):
    """Among all projectors onto n_occ generalised eigenvectors, the oracle's P has the least
    band energy Tr(P H), and it equals that projector."""
    p = make_random_small(20 + n, n, n_occ)
    w, C = scipy.linalg.eigh(p.H, p.S)  # library routine, C^T S C = I
    best = None
    for sub in itertools.combinations(range(n), n_occ):
        Cs = C[:, list(sub)]
        P = Cs @ Cs.T
        e = float(np.sum(P * p.H))
        if best is None or e < best[0]:
            best = (e, P)
    r = dm(p.H, p.S, n_occ)
    assert abs(r["energy"] - best[0]) <= 1e-12 * max(1.0, abs(best[0]))
    assert np.max(np.abs(r["P"] - best[1])) <= 1e-11


def test_dm_invariants_on_unstructured_input(dm):
    p = make_random_small(31, 60, 25)
    r = dm(p.H, p.S, p.n_occ)
    inv = steps.invariants(r["P"], p.H, p.S, p.n_occ)
    assert inv["idem"] < 1e-11 and inv["trace_err"] < 1e-11
    assert inv["asym"] == 0.0 and inv["commut"] < 1e-10
    assert abs(inv["energy"] - r["energy"]) < 1e-11 * max(1, abs(r["energy"]))


def test_dm_status_no_gap_and_not_spd(dm):
    rng = np.random.default_rng(1)
    Q = haar_orthogonal(rng, 8)
    lam = np.array([-2.0, -1.0, 0.5, 0.5, 1.0, 2.0, 3.0, 4.0])
    H = (Q * lam) @ Q.T
    r = dm(H, np.eye(8), 3)
    assert r["status"] == "NO_GAP"
    S = np.eye(8)
    S[0, 0] = -1.0
    assert dm(H, S, 3)["status"] == "NOT_SPD"


@pytest.mark.parametrize("n,n_occ,seed", [(64, 17, 41), (150, 60, 42), (97, 1, 43), (97, 96, 44)])
def test_lapack_statement_matches_jacobi(n, n_occ, seed):
    """The two statements of the definition agree on unstructured inputs (no closed form),
    including a single occupied and a single virtual state."""
    p = make_random_small(seed, n, n_occ)
    a = oracle.density_matrix(p.H, p.S, n_occ, edm=True)
    b = density_matrix_eigh(p.H, p.S, n_occ, edm=True)
    assert a["status"] == b["status"] == "OK"
    assert rel(b["P"], a["P"]) <= 1e-12
    assert rel(b["Q"], a["Q"]) <= 1e-11
    assert abs(b["energy"] - a["energy"]) <= 1e-12 * max(1.0, abs(a["energy"]))
    np.testing.assert_allclose(b["evals"], a["evals"], atol=1e-12)


def test_lapack_statement_pins_catch_plausible_mistakes():
    """Mistakes in the steps of the LAPACK statement that its pins must catch: the Cholesky-free
    Loewdin factor replaced by S^{-1} (a dropped square root), the occupied columns taken from the
    top of the spectrum (a wrong index), and P = C^T C (a transposed operand)."""
    p = make_spectrum_problem(17, 80, 20, cond_S=50.0, gap=0.3)
    Pc, Ec = steps.closed_form_dm(p.factors, p.n_occ)
    good = density_matrix_eigh(p.H, p.S, p.n_occ)
    assert rel(good["P"], Pc) <= 1e-11

    s, U = np.linalg.eigh(p.S)

    def route(zpow=-0.5, top=False, transpose=False):
        Z = (U * s ** zpow) @ U.T
        lam, V = np.linalg.eigh(steps.sym(Z @ p.H @ Z))
        cols = V[:, -p.n_occ:] if top else V[:, :p.n_occ]
        C = Z @ cols
        return C.T @ C if transpose else C @ C.T
    assert rel(route(), Pc) <= 1e-11
    assert not rel(route(zpow=-1.0), Pc) <= 1e-3
    assert not rel(route(top=True), Pc) <= 1e-3
    with pytest.raises(ValueError):
        rel(route(transpose=True), Pc)          # wrong shape: N x N instead of n x n


def test_inv_sqrt_matches_factors():
    p = make_spectrum_problem(9, 64, 16, cond_S=1e3, gap=0.3)
    Z, st = oracle.inv_sqrt(p.S)
    assert st == "OK"
    assert rel(Z, steps.closed_form_inv_sqrt(p.factors)) <= 1e-11


# ------------------------------------------------------------------------------------------
# step-level definitions of the purification route
# ------------------------------------------------------------------------------------------

def test_gershgorin_bounds_enclose_spectrum_and_are_tight_for_diagonal():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((40, 40))
    A = A + A.T
    lo, hi = steps.gershgorin_bounds(A)
    w = np.linalg.eigvalsh(A)
    assert lo <= w[0] and hi >= w[-1]
    d = rng.uniform(-3, 4, 9)
    assert steps.gershgorin_bounds(np.diag(d)) == (d.min(), d.max())


def test_initial_guess_maps_bounds_to_unit_interval():
    d = np.array([-3.0, -1.0, 0.0, 2.0, 5.0])
    X0 = steps.initial_guess(np.diag(d), d.min(), d.max())
    np.testing.assert_allclose(np.diag(X0), (5.0 - d) / 8.0)
    assert X0[0, 0] == 1.0 and X0[-1, -1] == 0.0


def test_trs4_step_resets_trace_and_fixes_projectors():
    rng = np.random.default_rng(8)
    n, N = 30, 11
    Q = haar_orthogonal(rng, n)
    x = rng.uniform(0.05, 0.95, n)
    X = (Q * x) @ Q.T
    Xn, g, br = steps.trs4_step(X, N)
    if br == "F+gG":
        assert abs(np.trace(Xn) - N) <= 1e-12      # the trace-resetting property of gamma
    # exact projectors are fixed points of every branch
    Pq = Q[:, :N] @ Q[:, :N].T
    Pn, _, _ = steps.trs4_step(Pq, N)
    assert np.linalg.norm(Pn - Pq) <= 1e-12
    # the map acts on eigenvalues only: eigenvectors are kept
    assert np.linalg.norm(Xn @ X - X @ Xn) <= 1e-12


def test_trs4_purify_reaches_eigh_projector():
    p = make_random_small(41, 80, 30)
    Ht = p.H
    Pt, it, hist = steps.trs4_purify(Ht, 30)
    w, V = np.linalg.eigh(Ht)
    assert w[30] - w[29] > 1e-3
    Vo = V[:, :30]
    assert rel(Pt, Vo @ Vo.T) <= 1e-10
    assert it < 100 and all(0.0 <= g <= 6.0 or br != "F+gG" for g, br in hist)


@pytest.mark.parametrize("method", ["trs4", "trs2", "canonical"])
def test_purification_variants_reach_the_projector(method):
    rng = np.random.default_rng(91)
    n, N = 60, 17
    Q = haar_orthogonal(rng, n)
    lam = np.sort(rng.uniform(-3.0, 3.0, n))
    lam[N:] += 0.5
    Ht = (Q * lam) @ Q.T
    X, it, traces = steps.purify(Ht, N, method)
    assert it < 400
    assert np.linalg.norm(X - Q[:, :N] @ Q[:, :N].T) <= 1e-11
    if method == "canonical":
        # canonical purification keeps the electron count at every iteration
        assert max(abs(t - N) for t in traces) <= 1e-11


def test_canonical_initial_guess_has_trace_n_and_unit_interval_spectrum():
    rng = np.random.default_rng(92)
    n, N = 40, 11
    Q = haar_orthogonal(rng, n)
    lam = rng.uniform(-5.0, 2.0, n)
    Ht = (Q * lam) @ Q.T
    lo, hi = steps.gershgorin_bounds(Ht)
    X0 = steps.canonical_initial_guess(Ht, N, lo, hi)
    w = np.linalg.eigvalsh(X0)
    assert abs(np.trace(X0) - N) <= 1e-12
    assert w.min() >= -1e-12 and w.max() <= 1.0 + 1e-12
    # the map is decreasing in the energy: the lowest level gets the largest occupation
    order = np.argsort(lam)
    occ = np.array([Q[:, k] @ X0 @ Q[:, k] for k in order])
    assert np.all(np.diff(occ) <= 1e-12)


def test_canonical_and_trs2_steps_by_hand():
    # X = diag(0.2, 0.9): Tr(X - X^2) = 0.25, Tr(X^2 - X^3) = 0.113, c = 0.452 < 1/2, so
    # x <- ((1 - 2c) x + (1 + c) x^2 - x^3) / (1 - c):  0.2 -> 0.06928 / 0.548, 0.9 -> 0.53352 / 0.548
    X = np.diag([0.2, 0.9])
    Xn, c = steps.canonical_step(X)
    assert abs(c - 0.452) <= 1e-15
    np.testing.assert_allclose(np.diag(Xn), [0.06928 / 0.548, 0.53352 / 0.548], rtol=1e-14)
    # X = diag(0.3, 0.95): c = (0.063 + 0.045125) / (0.21 + 0.0475) = 0.108125 / 0.2575 < 1/2 too;
    # X = diag(0.6, 0.95): Tr(X-X^2) = 0.24 + 0.0475, Tr(X^2-X^3) = 0.144 + 0.045125, c > 1/2:
    # x <- ((1 + c) x^2 - x^3) / c
    X = np.diag([0.6, 0.95])
    c = (0.144 + 0.045125) / (0.24 + 0.0475)
    Xn, c2 = steps.canonical_step(X)
    assert abs(c2 - c) <= 1e-15 and c > 0.5
    np.testing.assert_allclose(np.diag(Xn), [((1 + c) * 0.36 - 0.216) / c,
                                             ((1 + c) * 0.9025 - 0.857375) / c], rtol=1e-14)
    # TRS2 with N = 1 on diag(0.2, 0.9): Tr X^2 = 0.85, Tr(2X - X^2) = 1.35 -> X^2 (|0.15| < |0.35|)
    Xn, br = steps.trs2_step(np.diag([0.2, 0.9]), 1)
    assert br == "X2"
    np.testing.assert_allclose(np.diag(Xn), [0.04, 0.81], rtol=1e-15)
    Xn, br = steps.trs2_step(np.diag([0.2, 0.5]), 1)   # 0.29 vs 1.11: 2X - X^2
    assert br == "2X-X2"
    np.testing.assert_allclose(np.diag(Xn), [0.36, 0.75], rtol=1e-15)


def test_hole_particle_form_coincides_with_canonical():
    rng = np.random.default_rng(93)
    Q = haar_orthogonal(rng, 12)
    for x in (rng.uniform(0.0, 1.0, 12), np.r_[rng.uniform(0.6, 1.0, 9), rng.uniform(0, 0.2, 3)]):
        X = (Q * x) @ Q.T
        Xc, c = steps.canonical_step(X)
        Xh, c2, beta = steps.hole_particle_step(X)
        assert abs(c - c2) <= 1e-14
        assert np.linalg.norm(Xc - Xh) <= 1e-13


# ------------------------------------------------------------------------------------------
# Truncated purification (threshold filtering, Sec. 2.2.2)
# ------------------------------------------------------------------------------------------

def test_filter_small_by_hand():
    A = np.array([[1e-3, -2e-6, 5e-6], [-2e-6, -4e-5, 0.0], [5e-6, 0.0, 1.0]])
    np.testing.assert_array_equal(steps.filter_small(A, 5e-6),
                                  [[1e-3, 0.0, 5e-6], [0.0, -4e-5, 0.0], [5e-6, 0.0, 1.0]])


def test_truncated_trs4_without_threshold_is_the_projector():
    p = make_banded(7, 256, 64, s_amp=0.0)
    X, it = steps.trs4_purify_truncated(p.H, 64, 0.0)
    Q = p.factors["Q"]
    assert rel(X, Q[:, :64] @ Q[:, :64].T) <= 1e-12
    assert it < 60


def test_truncated_trs4_error_grows_with_threshold_and_keeps_count():
    p = make_banded(8, 512, 128, s_amp=0.0)
    Q = p.factors["Q"]
    Pex = Q[:, :128] @ Q[:, :128].T
    errs = []
    for tau in (1e-9, 1e-7, 1e-5):
        X, _ = steps.trs4_purify_truncated(p.H, 128, tau)
        # the gamma step resets the trace exactly; only the filtered part of W moves it
        assert abs(np.trace(X) - 128) <= 1e-7 * 128
        assert np.array_equal(X, X.T)
        errs.append(rel(X, Pex))
    assert errs[0] < errs[1] < errs[2]
    assert errs[0] <= 1e-6 and errs[2] <= 1e-1
    # the filtered iterate is sparse: most entries far from the diagonal are exactly zero
    X, _ = steps.trs4_purify_truncated(p.H, 128, 1e-5)
    idx = np.arange(512)
    far = np.abs(idx[:, None] - idx[None, :]) > 256
    assert np.mean(X[far] == 0.0) > 0.5


def _golden_trs4_filtered():
    with open(os.path.join(GOLDEN, "trs4_filtered_6x6.json")) as f:
        return json.load(f)


def _filtered_steps(d, step):
    """The oracle's initial guess and steps on the golden case, with `step` as the step."""
    Ht = np.array(d["H_tilde"])
    lo, hi = steps.gershgorin_bounds(Ht)
    X = steps.filter_small(steps.initial_guess(Ht, lo, hi), d["tau"])
    out = [(X, None)]
    for _ in d["steps"]:
        X, info = step(X, d["n_occ"], d["tau"])
        out.append((X, info))
    return (lo, hi), out


def test_filtered_trs4_golden_6x6():
    """Two filtered TRS4 steps on a 6 x 6 banded case, against exact rational values
    (tests/golden/make_trs4_filtered.py): X0, X^2 and W each lose an element to the filter, and
    one off-diagonal pair of X^2 W straddles the threshold."""
    d = _golden_trs4_filtered()
    (lo, hi), out = _filtered_steps(d, steps.trs4_filtered_step)
    assert lo == d["eps_min"] and hi == d["eps_max"]
    np.testing.assert_allclose(out[0][0], d["X0_filtered"], rtol=0, atol=1e-15)
    for k, ref in enumerate(d["steps"]):
        X, info = out[k + 1]
        assert info["branch"] == "F+gG"
        np.testing.assert_allclose(info["X2"], ref["X2_filtered"], rtol=0, atol=1e-14)
        assert abs(info["gamma"] - ref["gamma"]) <= 1e-13 * abs(ref["gamma"])
        np.testing.assert_allclose(info["W"], ref["W_filtered"], rtol=0, atol=1e-14)
        np.testing.assert_allclose(X, ref["X_next"], rtol=0, atol=1e-14)
        assert abs(np.trace(X) - ref["X_next_trace"]) <= 1e-14
    # the case exercises every filter placement
    assert d["X0_below_tau"] and all(s["X2_below_tau"] and s["W_below_tau"] for s in d["steps"])
    assert d["steps"][1]["straddling_pairs"]


def test_filtered_trs4_golden_catches_misplaced_filters():
    """Plausible mistakes in where the filter sits, each of which the golden case rejects."""
    d = _golden_trs4_filtered()
    ref = np.array(d["steps"][-1]["X_next"])
    f = steps.filter_small

    def step(X, N, tau, filt_w=True, filt_after_sym=True, filt_x2_in_traces=True):
        X2 = X @ X
        X2f = f(X2, tau)
        T = X2f if filt_x2_in_traces else X2
        t2, t3, t4 = np.trace(T), np.sum(T * X), np.sum(T * T)
        g = (N - (4 * t3 - 3 * t4)) / (t2 - 2 * t3 + t4)
        W = g * np.eye(X.shape[0]) + (4 - 2 * g) * X + (g - 3) * X2f
        if filt_w:
            W = f(W, tau)
        M = X2f @ W
        Xn = f(steps.sym(M), tau) if filt_after_sym else steps.sym(f(M, tau))
        return Xn, {}

    def final(**kw):
        return _filtered_steps(d, lambda X, N, tau: step(X, N, tau, **kw))[1][-1][0]

    assert np.abs(final() - ref).max() <= 1e-14            # the restatement agrees ...
    assert np.abs(final(filt_w=False) - ref).max() > 1e-6  # ... W left unfiltered
    assert np.abs(final(filt_after_sym=False) - ref).max() > 1e-6  # filtered, then symmetrised
    assert np.abs(final(filt_x2_in_traces=False) - ref).max() > 1e-6  # raw X^2 in gamma
    # the initial guess left unfiltered
    Ht = np.array(d["H_tilde"])
    lo, hi = steps.gershgorin_bounds(Ht)
    X = steps.initial_guess(Ht, lo, hi)
    for _ in d["steps"]:
        X, _ = steps.trs4_filtered_step(X, d["n_occ"], d["tau"])
    assert np.abs(X - ref).max() > 1e-6


def test_newton_schulz_and_refinement():
    p = make_spectrum_problem(12, 64, 16, cond_S=1e3, gap=0.3)
    Zc = steps.closed_form_inv_sqrt(p.factors)
    Z, it = steps.newton_schulz_inv_sqrt(p.S)
    assert rel(Z, Zc) <= 1e-9 and it < 60
    Zp = Zc * (1.0 + 1e-4)                        # a commuting perturbation
    e0 = rel(Zp, Zc)
    e1 = rel(steps.inv_sqrt_refine(Zp, p.S), Zc)
    assert e1 <= 10 * e0 ** 2                     # quadratic (in fact cubic) contraction


def test_refinement_remainder_is_the_closed_form_polynomial():
    # For Z commuting with S, delta = Z S Z - I and one refinement step leave
    # delta' = (I + delta) F^2 - I = (5/8) delta^3 - (15/64) delta^4 + (9/64) delta^5 exactly,
    # F = I - delta/2 + 3 delta^2/8 (the engine's handover rule from Newton-Schulz rests on the
    # leading coefficient 5/8).
    p = make_spectrum_problem(13, 48, 12, cond_S=1e2, gap=0.3)
    w, V = np.linalg.eigh(p.S)
    e = np.linspace(-0.02, 0.03, 48)               # Z = S^{-1/2} (I + e), same eigenvectors
    Z = (V * (w ** -0.5 * np.sqrt(1.0 + e))) @ V.T
    I = np.eye(48)
    d = Z @ p.S @ Z - I
    Zr = steps.inv_sqrt_refine(Z, p.S)
    d1 = Zr @ p.S @ Zr - I
    d2 = d @ d
    poly = 0.625 * d2 @ d - (15.0 / 64.0) * d2 @ d2 + (9.0 / 64.0) * d2 @ d2 @ d
    assert np.linalg.norm(d1 - poly) <= 1e-6 * np.linalg.norm(poly)
    assert np.linalg.norm(d1) <= 0.625 * np.linalg.norm(d) ** 3 * 1.01


def test_mcweeny_fixes_projectors_and_moves_eigenvalues_to_0_1():
    rng = np.random.default_rng(9)
    Q = haar_orthogonal(rng, 20)
    x = np.concatenate([np.full(8, 0.9), np.full(12, 0.1)])
    X = (Q * x) @ Q.T
    Y = steps.mcweeny(X)
    wy = np.linalg.eigvalsh(Y)
    assert np.all(wy[:12] < 0.1) and np.all(wy[12:] > 0.9)


def test_purification_route_matches_closed_form():
    p = make_config0(n=128, n_occ=32, seed=5)
    r = steps.purification_route(p.H, p.S, p.n_occ)
    Pc, Ec = steps.closed_form_dm(p.factors, p.n_occ)
    assert rel(r["P"], Pc) <= 1e-10
    assert abs(r["trace_ps"] - p.n_occ) <= 1e-10
    assert abs(r["energy"] - Ec) <= 1e-10 * abs(Ec)


# ------------------------------------------------------------------------------------------
# planted mistakes: each must be caught by one of the pins above
# ------------------------------------------------------------------------------------------

def _route_with(trs4_step=None, inv_sqrt=None):
    p = make_config0(n=64, n_occ=16, seed=6)
    Z = inv_sqrt(p.S) if inv_sqrt else steps.newton_schulz_inv_sqrt(p.S)[0]
    Ht = steps.sym(Z @ p.H @ Z)
    lo, hi = steps.gershgorin_bounds(Ht)
    X = steps.initial_guess(Ht, lo, hi)
    for _ in range(60):
        X, _, _ = (trs4_step or steps.trs4_step)(X, p.n_occ)
    P = Z @ X @ Z
    Pc, _ = steps.closed_form_dm(p.factors, p.n_occ)
    return rel(P, Pc)


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # a planted mistake diverges
def test_planted_mistakes_are_caught():
    assert _route_with() <= 1e-10

    def wrong_sign_G(X, N):           # G = X^2 (I + X)^2 instead of (I - X)^2
        X2 = X @ X
        Y = np.eye(X.shape[0]) + X
        trF = np.trace(X2 @ (4 * X - 3 * X2))
        G = X2 @ Y @ Y
        g = (N - trF) / np.trace(G)
        g = min(max(g, 0.0), 6.0)
        return steps.sym(X2 @ (4 * X - 3 * X2) + g * G), g, "F+gG"
    assert not _route_with(trs4_step=wrong_sign_G) <= 1e-3   # NaN also counts as caught

    def no_sqrt(S):                   # S^{-1} instead of S^{-1/2}
        return np.linalg.inv(S)
    assert not _route_with(inv_sqrt=no_sqrt) <= 1e-3

    def transposed_scale(S):          # a non-symmetric "S^{-1/2}" (row/column mix-up)
        Z = steps.newton_schulz_inv_sqrt(S)[0]
        return Z @ np.diag(np.linspace(0.99, 1.01, S.shape[0]))
    assert not _route_with(inv_sqrt=transposed_scale) <= 1e-4

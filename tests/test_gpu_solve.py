"""GPU parity of the whole solve (C ABI gdm_init ... gdm_solve_dm) against the CPU oracle.

Bars (from the target the engine is built to): relative Frobenius error of P <= 1e-6 against
the FP64 oracle, |Tr(P S) - n_occ| <= 1e-8, band-energy error <= 1e-6 relative; the all-FP64
path is held to 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import steps
from workloads import (make_config0, make_random_small, make_spectrum_problem, make_config2,
                       make_request_problem, make_geometry_step, make_banded)

pytestmark = pytest.mark.gpu

REL_P = 1e-6
TRACE = 1e-8


@pytest.fixture(scope="module")
def g():
    import paper_1912_13403_gb300 as g
    return g


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solve(g, p, prec=None, device_buffers=False):
    h = g.Handle(p.n, p.n_occ)
    try:
        if prec is not None:
            h.set_precision(prec)
        if device_buffers:
            H = torch.from_numpy(p.H).cuda()
            S = torch.from_numpy(p.S).cuda()
            P = torch.empty_like(H)
            h.set_overlap(S)
            h.set_hamiltonian(H)
            P, e, info, st = h.solve(P)
            return P.cpu().numpy(), e, info, st
        h.set_overlap(p.S)
        h.set_hamiltonian(p.H)
        return h.solve()
    finally:
        h.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_config0_matches_oracle(g, prec):
    p = make_config0()
    ref = oracle.density_matrix(p.H, p.S, p.n_occ)
    P, e, info, st = solve(g, p, g.GDM_PREC_FP64 if prec == "fp64" else None)
    assert st == g.GDM_OK, info
    bar = 1e-9 if prec == "fp64" else REL_P
    assert rel(P, ref["P"]) <= bar, info
    assert abs(e - ref["energy"]) <= bar * abs(ref["energy"])
    assert info["trace_err"] <= TRACE
    assert abs(np.sum(P * p.S) - p.n_occ) <= TRACE
    assert np.array_equal(P, P.T)


@pytest.mark.parametrize("n,n_occ", [(130, 33), (200, 150), (383, 96), (64, 1), (65, 64)])
def test_ragged_sizes_match_oracle(g, n, n_occ):
    p = make_random_small(1000 + n, n, n_occ)
    ref = oracle.density_matrix(p.H, p.S, n_occ)
    assert ref["status"] == "OK"
    P, e, info, st = solve(g, p)
    assert st == g.GDM_OK, info
    assert rel(P, ref["P"]) <= REL_P, info
    assert abs(e - ref["energy"]) <= REL_P * max(1.0, abs(ref["energy"]))
    assert info["trace_err"] <= TRACE


def test_ill_conditioned_overlap_closed_form(g):
    p = make_spectrum_problem(21, 512, 128, cond_S=1e3, gap=0.2)
    Pc, Ec = steps.closed_form_dm(p.factors, p.n_occ)
    P, e, info, st = solve(g, p)
    assert st == g.GDM_OK, info
    assert rel(P, Pc) <= REL_P, info
    assert abs(e - Ec) <= REL_P * abs(Ec)
    assert info["trace_err"] <= TRACE


def test_dftb_like_small_gap_closed_form(g):
    p = make_config2(22, n=1024, n_occ=256)
    Pc, Ec = steps.closed_form_dm(p.factors, p.n_occ)
    P, e, info, st = solve(g, p)
    assert st == g.GDM_OK, info
    assert rel(P, Pc) <= REL_P, info
    assert info["trace_err"] <= TRACE


def test_device_buffers_and_fp64_path_agree(g):
    p = make_config0(seed=3, n=192, n_occ=40)
    P1, e1, i1, _ = solve(g, p, device_buffers=True)
    P2, e2, i2, _ = solve(g, p, g.GDM_PREC_FP64)
    assert rel(P1, P2) <= REL_P
    assert abs(e1 - e2) <= REL_P * abs(e2)


def test_z_cache_and_reinit(g):
    p = make_config0(seed=4, n=160, n_occ=30)
    q = make_request_problem(dict(seed=77, n=160, n_occ=30, gap=0.3))
    with g.Handle(p.n, p.n_occ) as h:
        h.set_overlap(p.S)
        h.set_hamiltonian(p.H)
        _, _, i1, _ = h.solve()
        h.set_hamiltonian(2.0 * p.H)           # same geometry: Z is reused
        P2, e2, i2, _ = h.solve()
        assert i1["ns_iters"] > 0 and i2["ns_iters"] == 0
        ref = oracle.density_matrix(2.0 * p.H, p.S, p.n_occ)
        assert rel(P2, ref["P"]) <= REL_P
        h.reinit()                             # new geometry
        with pytest.raises(g.GdmError):
            h.solve()
        h.set_overlap(q.S)
        h.set_hamiltonian(q.H)
        P3, _, i3, _ = h.solve()
        assert i3["ns_iters"] > 0
        assert rel(P3, oracle.density_matrix(q.H, q.S, q.n_occ)["P"]) <= REL_P


def test_error_paths(g):
    n = 64
    with pytest.raises(g.GdmError):
        g.Handle(n, 0)
    with pytest.raises(g.GdmError):
        g.Handle(n, n)
    with g.Handle(n, 10) as h:
        with pytest.raises(g.GdmError) as ei:
            h.solve()
        assert ei.value.status == g.GDM_ERR_STATE
        S = np.eye(n)
        S[3, 3] = -1.0
        h.set_overlap(S)
        h.set_hamiltonian(np.diag(np.arange(n, dtype=np.float64)))
        with pytest.raises(g.GdmError) as ei:
            h.solve()
        assert ei.value.status == g.GDM_ERR_NOT_SPD
        bad = np.eye(n)
        bad[1, 2] = np.nan
        with pytest.raises(g.GdmError) as ei:
            h.set_hamiltonian(bad)
        assert ei.value.status == g.GDM_ERR_NONFINITE
        assert g.gdm_set_slices(h._h, 3, 5, 1, 0) == g.GDM_ERR_ARG
        assert g.gdm_set_slices(h._h, 3, 1, 2, 0) == g.GDM_ERR_ARG
        assert g.gdm_set_slices(h._h, 3, 3, 3, 13) == g.GDM_ERR_ARG


# ------------------------------------------------------------------------------------------
# Energy-weighted density matrix Q = P H P (Sec. 2.6, Eq. energy_density_matrix)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_edm_matches_oracle(g, prec):
    p = make_config0()
    ref = oracle.density_matrix(p.H, p.S, p.n_occ, edm=True)
    with g.Handle(p.n, p.n_occ) as h:
        if prec == "fp64":
            h.set_precision(g.GDM_PREC_FP64)
        h.set_overlap(p.S)
        h.set_hamiltonian(p.H)
        P, e, info, st = h.solve()
        Q = h.edm()
    bar = 1e-9 if prec == "fp64" else REL_P
    assert rel(Q, ref["Q"]) <= bar, info
    assert rel(Q, steps.closed_form_edm(p.factors, p.n_occ)) <= bar
    assert np.array_equal(Q, Q.T)
    # Tr(Q S) is the band energy
    assert abs(np.sum(Q * p.S) - ref["energy"]) <= bar * abs(ref["energy"])


@pytest.mark.parametrize("n,n_occ", [(130, 33), (383, 96)])
def test_edm_ragged_sizes_device_buffers(g, n, n_occ):
    p = make_random_small(2000 + n, n, n_occ)
    ref = oracle.density_matrix(p.H, p.S, n_occ, edm=True)
    with g.Handle(n, n_occ) as h:
        h.set_overlap(torch.from_numpy(p.S).cuda())
        h.set_hamiltonian(torch.from_numpy(p.H).cuda())
        h.solve()
        Qd = torch.full((n, n + 3), float("nan"), dtype=torch.float64, device="cuda")
        h.edm(Qd[:, :n])
        Q = Qd[:, :n].cpu().numpy()
        assert torch.isnan(Qd[:, n:]).all()        # nothing written beyond the n columns
    assert rel(Q, ref["Q"]) <= REL_P


def test_edm_state_errors(g):
    p = make_config0(seed=5, n=128, n_occ=20)
    with g.Handle(p.n, p.n_occ) as h:
        with pytest.raises(g.GdmError) as ei:
            h.edm()
        assert ei.value.status == g.GDM_ERR_STATE
        h.set_overlap(p.S)
        h.set_hamiltonian(p.H)
        h.solve()
        Q1 = h.edm()
        h.set_hamiltonian(1.5 * p.H)           # P no longer belongs to H
        with pytest.raises(g.GdmError) as ei:
            h.edm()
        assert ei.value.status == g.GDM_ERR_STATE
        h.solve()
        Q2 = h.edm()
        ref = oracle.density_matrix(1.5 * p.H, p.S, p.n_occ, edm=True)
        assert rel(Q2, ref["Q"]) <= REL_P
        assert rel(Q2, 1.5 * Q1) <= 10 * REL_P   # scaling H scales Q, P unchanged
        h.reinit()
        with pytest.raises(g.GdmError) as ei:
            h.edm()
        assert ei.value.status == g.GDM_ERR_STATE


# ------------------------------------------------------------------------------------------
# Density-matrix extrapolation to a new geometry (Sec. 2.7, Loewdin form)
# ------------------------------------------------------------------------------------------

# The route's Z satisfies Z^T S Z = I and equals S^{-1/2} up to a rotation U ~ I left by the
# Newton-Schulz rounding (the refinement fixes the metric, not the rotation).  The extrapolation
# P1 = Z1 Z0^{-1} P0 Z0^{-T} Z1^T is exact as a projector in the new metric whatever U is, and
# deviates from the Loewdin formula by U1 U0^T - I: about 2^-23 (the default 2-slice Newton-Schulz
# format) times the growth of the rounding over the iterations, measured at ~1e-4 for cond(S) =
# 100; with a 3-slice Newton-Schulz format (35 bits) the deviation is below the 1e-6 bar.
EXTRAP_DEFAULT = 1e-3


@pytest.mark.parametrize("prec", ["mixed", "mixed_ns3", "fp64"])
def test_extrapolation_matches_closed_form_and_warm_z(g, prec):
    p0 = make_spectrum_problem(41, 384, 96, cond_S=100.0, gap=0.3)
    p1 = make_geometry_step(p0, seed=7, eps=0.03)
    bar = {"fp64": 1e-9, "mixed_ns3": REL_P, "mixed": EXTRAP_DEFAULT}[prec]
    with g.Handle(p0.n, p0.n_occ) as h:
        if prec == "fp64":
            h.set_precision(g.GDM_PREC_FP64)
        if prec == "mixed_ns3":
            h.set_slices(g.GDM_PHASE_NEWTON_SCHULZ, 3, 2, 12)
        h.set_overlap(p0.S)
        h.set_hamiltonian(p0.H)
        P0, _, _, _ = h.solve()
        P1 = h.extrapolate(p1.S)
        # the step keeps the orthogonal-basis projector: P1 is the new geometry's answer
        assert rel(P1, steps.closed_form_dm(p1.factors, p1.n_occ)[0]) <= bar
        ref, st = oracle.extrapolate_dm(P0, p0.S, p1.S)
        assert st == "OK" and rel(P1, ref) <= bar
        # a projector in the new metric with the same count, at any Newton-Schulz format
        assert abs(np.sum(P1 * p1.S) - p1.n_occ) <= 1e-7
        assert rel(P1 @ p1.S @ P1, P1) <= 1e-6
        # the overlap and its Z carry over; the Hamiltonian does not
        with pytest.raises(g.GdmError) as ei:
            h.solve()
        assert ei.value.status == g.GDM_ERR_STATE
        h.set_hamiltonian(p1.H)
        P, e, info, st = h.solve()
        assert info["ns_iters"] == 0
        assert rel(P, steps.closed_form_dm(p1.factors, p1.n_occ)[0]) <= (
            1e-9 if prec == "fp64" else REL_P)


def test_extrapolation_general_overlaps_device_buffers(g):
    p = make_random_small(3001, 200, 50)
    q = make_random_small(3002, 200, 50)
    ref0 = oracle.density_matrix(p.H, p.S, 50)
    with g.Handle(200, 50) as h:
        with pytest.raises(g.GdmError) as ei:
            h.extrapolate(q.S)
        assert ei.value.status == g.GDM_ERR_STATE
        h.set_overlap(torch.from_numpy(p.S).cuda())
        h.set_hamiltonian(torch.from_numpy(p.H).cuda())
        h.solve()
        Pd = torch.empty((200, 200), dtype=torch.float64, device="cuda")
        h.extrapolate(torch.from_numpy(q.S).cuda(), Pd)
        P1 = Pd.cpu().numpy()
    ref, st = oracle.extrapolate_dm(ref0["P"], p.S, q.S)
    assert rel(P1, ref) <= EXTRAP_DEFAULT
    assert rel(P1 @ q.S @ P1, P1) <= 10 * REL_P
    assert abs(np.sum(P1 * q.S) - 50) <= 1e-7


# ------------------------------------------------------------------------------------------
# Purification variants (Sec. 2.2.2): 2nd-order trace resetting and canonical purification
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("method", ["trs2", "canonical"])
@pytest.mark.parametrize("case", ["config0", "ragged", "cond1e3"])
def test_purification_variants_match_oracle(g, method, case):
    code = {"trs2": g.GDM_PURIFY_TRS2, "canonical": g.GDM_PURIFY_CANONICAL}[method]
    if case == "config0":
        p = make_config0()
        ref = oracle.density_matrix(p.H, p.S, p.n_occ)["P"]
    elif case == "ragged":
        p = make_random_small(1383, 383, 96)
        ref = oracle.density_matrix(p.H, p.S, p.n_occ)["P"]
    else:
        p = make_spectrum_problem(22, 512, 128, cond_S=1e3, gap=0.2)
        ref = steps.closed_form_dm(p.factors, p.n_occ)[0]
    with g.Handle(p.n, p.n_occ) as h:
        h.set_purification(code)
        h.set_overlap(p.S)
        h.set_hamiltonian(p.H)
        P, e, info, st = h.solve()
        hist = h.history()
    assert st == g.GDM_OK, info
    assert rel(P, ref) <= REL_P, info
    assert info["trace_err"] <= TRACE
    branches = {b for (_, _, _, b) in hist}
    if method == "trs2":
        assert branches & {0, 1} and not branches & {2, 4}
    else:
        assert 4 in branches and not branches & {0, 1, 2}
        # canonical purification keeps Tr X = n_occ until the McWeeny endgame
        for idem, trace, c, b in hist:
            if b == 4:
                assert abs(trace - p.n_occ) <= 1e-8 * p.n_occ


def test_purification_method_argument_checked(g):
    with g.Handle(64, 10) as h:
        assert g.gdm_set_purification(h._h, 7) == g.GDM_ERR_ARG
        assert g.gdm_set_purification(h._h, g.GDM_PURIFY_CANONICAL) == g.GDM_OK


# ------------------------------------------------------------------------------------------
# Truncated (threshold-filtered) purification, the sparse regime of Sec. 2.2.2
# ------------------------------------------------------------------------------------------

def _trunc_solve(g, p, tau):
    with g.Handle(p.n, p.n_occ) as h:
        h.set_truncation(tau)
        h.set_overlap(p.S)
        h.set_hamiltonian(p.H)
        return h.solve()


def test_truncation_below_every_element_matches_dense(g):
    # a threshold below every element filters nothing and skips no k block; the filtered route
    # computes X^2 W as a full product and symmetrises it (instead of mirroring the upper
    # triangle), so the two agree to the products' rounding
    p = make_banded(11, 512, 128, s_amp=0.0)
    P0, e0, i0, _ = _trunc_solve(g, p, 0.0)
    P1, e1, i1, _ = _trunc_solve(g, p, 1e-300)
    assert i0["kstage_fraction"] == 1.0
    assert i1["kstage_fraction"] == 1.0
    assert rel(P1, P0) <= 1e-8
    # the stopping test can cross its threshold one step apart on rounding-level differences
    assert abs(i0["purif_iters"] - i1["purif_iters"]) <= 1


@pytest.mark.parametrize("tau", [1e-7, 1e-5])
def test_truncated_purification_matches_oracle_route(g, tau):
    # orthogonal basis (S = I, so the route's Z is exactly I and both sides filter the same
    # matrices); local H with 128 x 128 tiles that vanish
    p = make_banded(12, 1024, 256, s_amp=0.0)
    Q = p.factors["Q"]
    P_exact = Q[:, :p.n_occ] @ Q[:, :p.n_occ].T
    # the same fixed number of filtered steps on both sides (before the idempotency floor, where
    # the stopping decision is sensitive to rounding).  The filtered map is discontinuous at the
    # threshold: two evaluations that differ only by the products' rounding keep or drop the
    # elements of X^2 lying within that rounding of tau, and each such flip moves the iterate by
    # ~tau.  Measured on the oracle (symmetric perturbations of X^2 of 1e-11 of its largest
    # element, the sliced products' rounding level, four trials): at tau = 1e-5 no flip in three
    # trials (9th iterate moved by 1e-9), 4 flips in one (moved by 1.7e-5); at tau = 1e-7 8-18
    # flips each (moved by 3e-7 to 4e-7).  The bounds allow a few flips; the whole-solve checks
    # below hold the route to a quarter of its own truncation error.
    K = 9
    bound_k = {1e-7: 2e-6, 1e-5: 5e-5}[tau]
    with g.Handle(p.n, p.n_occ) as h:
        h.set_truncation(tau)
        h.set_max_iter(0, K)
        h.set_overlap(p.S)
        h.set_hamiltonian(p.H)
        PK, _, infoK, stK = h.solve()
        histK = h.history()
    assert stK == g.GDM_ERR_NOT_CONVERGED and infoK["purif_iters"] == K
    # all K steps are the filtered TRS4 map (the engine's McWeeny endgame has not started), so
    # they compare step for step with the oracle's statement of that map; at the iteration cap
    # the engine resets Tr X to N, and so does the comparison
    assert all(b in (0, 1, 2) for (_, _, _, b) in histK[:K]), histK
    # the oracle starts from the spectral bounds the engine used (its estimated ones)
    lo, hi = infoK["eps_min"], infoK["eps_max"]
    XK = steps.filter_small(steps.initial_guess(p.H, lo, hi), tau)
    for _ in range(K):
        XK, _ = steps.trs4_filtered_step(XK, p.n_occ, tau)
    XK = XK * (p.n_occ / np.trace(XK))
    assert rel(PK, XK) <= bound_k, rel(PK, XK)
    # the whole solve: the engine (McWeeny endgame, stall test) and the oracle (the filtered map
    # to its best iterate) both stop on the filtered idempotency floor; the two controllers
    # land within a few percent of the truncation error of each other (measured on the CPU
    # with the engine's controller restated: 4% at tau = 1e-7, 5% at tau = 1e-5)
    P, e, info, st = _trunc_solve(g, p, tau)
    assert st == g.GDM_OK, info
    X, _ = steps.trs4_purify_truncated(p.H, p.n_occ, tau, bounds=(info["eps_min"], info["eps_max"]))
    err_oracle = rel(X, P_exact)
    assert rel(P, X) <= 0.25 * err_oracle, (rel(P, X), err_oracle)
    assert rel(P, P_exact) <= 1.5 * err_oracle + 1e-6
    assert info["trace_err"] <= TRACE
    # the filtered products skipped part of their k blocks (at n = 1024 only a few tiles of the
    # iterates vanish at 1e-7, a quarter of the density matrix's at 1e-5)
    assert info["kstage_fraction"] < {1e-7: 0.99, 1e-5: 0.9}[tau], info["kstage_fraction"]


def test_truncated_purification_nonorthogonal_basis(g):
    p = make_banded(13, 1024, 256, s_amp=0.3)
    P, e, info, st = _trunc_solve(g, p, 1e-7)
    Pc = steps.closed_form_dm(p.factors, p.n_occ)[0]
    assert st == g.GDM_OK, info
    assert rel(P, Pc) <= 1e-3
    assert info["trace_err"] <= TRACE
    with g.Handle(64, 10) as h:
        assert g.gdm_set_truncation(h._h, -1.0) == g.GDM_ERR_ARG


# ------------------------------------------------------------------------------------------
# Spectral bounds of H~ for the initial guess (Eq. ntpoly_scale_hamiltonian, "estimated")
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["dense", "dftb"])
def test_lanczos_bounds_enclose_and_tighten(g, case):
    # the generalised eigenvalues of the construction are H~'s spectrum (up to rounding)
    p = (make_spectrum_problem(51, 1024, 256, cond_S=1e3, gap=0.2) if case == "dense"
         else make_config2(52, n=1024, n_occ=256))
    lam = p.factors["lam"]
    Pc, _ = steps.closed_form_dm(p.factors, p.n_occ)
    out = {}
    for method in (g.GDM_BOUNDS_GERSHGORIN, g.GDM_BOUNDS_LANCZOS):
        with g.Handle(p.n, p.n_occ) as h:
            h.set_bounds(method)
            h.set_overlap(p.S)
            h.set_hamiltonian(p.H)
            P, e, info, st = h.solve()
        assert st == g.GDM_OK, info
        assert rel(P, Pc) <= REL_P, (method, rel(P, Pc))
        assert info["trace_err"] <= TRACE
        assert info["bounds_restart"] == 0
        span = lam[-1] - lam[0]
        assert info["eps_min"] <= lam[0] - 1e-9 * span and info["eps_max"] >= lam[-1] + 1e-9 * span
        out[method] = (info["eps_max"] - info["eps_min"]) / span, info["purif_iters"], rel(P, Pc)
    width_g, it_g, err_g = out[g.GDM_BOUNDS_GERSHGORIN]
    width_l, it_l, err_l = out[g.GDM_BOUNDS_LANCZOS]
    assert width_l <= 1.1 and width_l < width_g, out   # 2% margin each side
    assert it_l <= it_g, out


def test_too_tight_estimate_restarts_from_gershgorin(g):
    # one Lanczos step estimates a single point: the initial guess then lies far outside [0, 1],
    # the purification leaves the trace range, and the solve runs again from Gershgorin's bounds
    p = make_random_small(61, 200, 50)
    ref = oracle.density_matrix(p.H, p.S, p.n_occ)
    with g.Handle(p.n, p.n_occ) as h:
        h.set_bounds(g.GDM_BOUNDS_LANCZOS, 1)
        h.set_overlap(p.S)
        h.set_hamiltonian(p.H)
        P, e, info, st = h.solve()
        assert st == g.GDM_OK, info
        assert info["bounds_restart"] == 1
        assert rel(P, ref["P"]) <= REL_P
        assert g.gdm_set_bounds(h._h, 7, 0) == g.GDM_ERR_ARG
        assert g.gdm_set_bounds(h._h, g.GDM_BOUNDS_LANCZOS, 65) == g.GDM_ERR_ARG


# ------------------------------------------------------------------------------------------
# Electron count in the S metric (Eq. density_matrix_conditions: P S P = P, Tr(P S) = n_occ)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["near_identity_S", "cond1e3"])
def test_count_without_rescale_and_metric_cleanup(g, case):
    # the count that the route leaves: within 1e-8 for a well-conditioned overlap; at
    # cond(S) = 1e3 the 38-bit products resolve Z^T S Z - I to about 1e-8 per unit count here,
    # and the last-resort rescale (on by default) takes what is above 1e-8
    if case == "near_identity_S":
        p = make_request_problem(dict(seed=91, n=1024, n_occ=256, gap=0.2))
    else:
        p = make_spectrum_problem(92, 1024, 256, cond_S=1e3, gap=0.2)
    Pc, Ec = steps.closed_form_dm(p.factors, p.n_occ)
    raw_bar = TRACE if case == "near_identity_S" else 1e-7
    with g.Handle(p.n, p.n_occ) as h:
        h.set_overlap(p.S)
        h.set_hamiltonian(p.H)
        Pd, ed, idf, std = h.solve()                      # defaults
        assert std == g.GDM_OK, idf
        assert idf["metric_cleanup"] == 0 and idf["s_idem_err"] == -1.0
        assert idf["trace_err_raw"] <= raw_bar, idf
        assert idf["trace_rescaled"] == (1 if idf["trace_err_raw"] > TRACE else 0)
        assert idf["trace_err"] <= TRACE
        h.set_trace_correction(False)                     # neither correction
        P0, e0, i0, st0 = h.solve()
        assert st0 == g.GDM_OK, i0
        assert i0["trace_rescaled"] == 0 and i0["trace_err"] == i0["trace_err_raw"]
        assert rel(P0, Pc) <= REL_P
        h.set_metric_cleanup(0.0)                         # the S-metric step forced on
        P1, e1, i1, st1 = h.solve()
    assert st1 in (g.GDM_OK, g.GDM_ERR_NOT_CONVERGED), i1
    assert i1["metric_cleanup"] == 1 and i1["trace_rescaled"] == 0
    assert rel(P1, Pc) <= REL_P
    assert abs(e1 - Ec) <= REL_P * abs(Ec)
    assert np.array_equal(P1, P1.T)
    # the reported ||P S P - P||_F of the matrix it was given, computed with the transform's
    # products: to a few per cent for a well-conditioned overlap; at cond(S) = 1e3 their
    # rounding is of the order of P S P - P itself (which is why the step is opt-in)
    d0 = np.linalg.norm(P0 @ p.S @ P0 - P0)
    tol = 0.1 if case == "near_identity_S" else 1.0
    assert abs(i1["s_idem_err"] - d0) <= tol * d0, (i1["s_idem_err"], d0)
    if case == "near_identity_S":
        # well conditioned: P S P = P several times closer, the count still within 1e-8
        assert np.linalg.norm(P1 @ p.S @ P1 - P1) <= 0.3 * d0
        assert i1["trace_err"] <= TRACE, i1
    with g.Handle(64, 10) as h:
        assert g.gdm_set_metric_cleanup(h._h, float("nan")) == g.GDM_ERR_ARG

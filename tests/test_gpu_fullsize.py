"""GPU parity at the sizes the benchmark runs, through the C ABI.

Below n ~ 1500 every product of a solve fits in one wave of 128 x 128 output tiles (152 SMs), so
the persistent kernel never walks more than one tile per CTA.  These cases run past that: the
stage ring crosses tiles, the two accumulator sets alternate, the epilogue of one tile overlaps
the MMAs of the next, and the tiles of the last partial wave are split along k.

  * whole solves of the dense-insulator recipe at n = 2560 (210 symmetric / 400 full tiles per
    product) and n = 4096 (the benchmark's own input), and of the DFTB-like recipe at n = 3072
    and n = 8192, against the closed form of the construction and, up to n = 4096, against the
    oracle's LAPACK statement of the definition (Sec. 1, Eqs. evp and density_matrix);
  * products at K = 4096 and K = 8192 in each of the route's three slice formats, every element
    against an FP64 product (cuBLAS DGEMM on the device) and sampled rows against numpy on the
    host, with the per-format bounds of test_gpu_kernels.py widened as the contraction grows.

Bars: ||P - P_ref||_F / ||P_ref||_F <= 1e-6, |Tr(P S) - n_occ| <= 1e-8, relative band-energy
error <= 1e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import steps
from oracle.lapack import density_matrix_eigh
from workloads import make_config1, make_config2, make_spectrum_problem, haar_orthogonal

pytestmark = pytest.mark.gpu

REL_P = 1e-6
TRACE = 1e-8


@pytest.fixture(scope="module")
def g():
    import paper_1912_13403_gb300 as g
    return g


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _solve_device(g, p):
    """One solve with device buffers, as the benchmark runs it."""
    H = torch.from_numpy(p.H).cuda()
    S = torch.from_numpy(p.S).cuda()
    P = torch.empty_like(H)
    with g.Handle(p.n, p.n_occ) as h:
        h.set_overlap(S)
        h.set_hamiltonian(H)
        _, e, info, st = h.solve(P)
    return P.cpu().numpy(), e, info, st


def _check_solve(p, P, e, info, st, g, oracle_too):
    assert st == g.GDM_OK, info
    Pc, Ec = steps.closed_form_dm(p.factors, p.n_occ)
    assert rel(P, Pc) <= REL_P, (rel(P, Pc), info)
    assert abs(e - Ec) <= REL_P * abs(Ec), (e, Ec)
    assert info["trace_err"] <= TRACE, info
    assert abs(float(np.sum(P * p.S)) - p.n_occ) <= TRACE
    assert np.array_equal(P, P.T)
    if oracle_too:
        ref = density_matrix_eigh(p.H, p.S, p.n_occ)
        assert ref["status"] == "OK"
        assert rel(P, ref["P"]) <= REL_P, rel(P, ref["P"])
        assert abs(e - ref["energy"]) <= REL_P * abs(ref["energy"])


def test_dense_insulator_past_one_wave(g):
    # config1's recipe (cond(S) = 1e3 log-spaced, gap 0.2) at n = 2560: 20 x 20 tiles
    p = make_spectrum_problem(31, 2560, 640, cond_S=1e3, gap=0.2, config="config1-like")
    _check_solve(p, *_solve_device(g, p), g, oracle_too=True)


def test_dftb_like_past_one_wave(g):
    # config2's recipe (decay 64, 0.05 gap, S = I + 0.3 exp(-|i-j|/8)) at n = 3072: 24 x 24 tiles
    p = make_config2(32, n=3072, n_occ=768)
    _check_solve(p, *_solve_device(g, p), g, oracle_too=True)


def test_benchmark_input_config1(g):
    # the benchmark's own input (n = 4096, seed 1), in the benchmark's launch configuration
    p = make_config1(seed=1, device="cuda")
    _check_solve(p, *_solve_device(g, p), g, oracle_too=True)


def test_benchmark_input_config2(g):
    # n = 8192 against the closed form (the LAPACK statement of the definition takes about a
    # minute of host time at this size; the closed form is exact by construction)
    p = make_config2(seed=1, device="cuda")
    _check_solve(p, *_solve_device(g, p), g, oracle_too=False)


# ------------------------------------------------------------------------------------------
# products at the route's contraction lengths
# ------------------------------------------------------------------------------------------

# bound per format at K <= ~1000 (x ||a_i|| ||b_j||), as in test_gpu_kernels.py; the FP32
# rounding of the higher orders grows like sqrt(K), so the bound is widened by sqrt(K / 1000)
FORMATS = {(2, 1, 12): 6e-5, (3, 3, 12): 2e-9, (4, 3, 9): 1e-10}


def _projector_like(n, seed):
    """X = Q diag(x) Q^T with x in [0, 1], half of it near 0 or 1: a purification iterate."""
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(rng, n, device="cuda")
    x = np.concatenate([rng.uniform(0.0, 0.05, n // 4), rng.uniform(0.95, 1.0, n // 4),
                        rng.uniform(0.0, 1.0, n - n // 2)])
    xt = torch.from_numpy(x).cuda()
    X = (Q * xt[None, :]) @ Q.T
    return 0.5 * (X + X.T)


def _check_elements(C, A, Bt, tol, rows):
    ref = A @ Bt.T                                         # cuBLAS DGEMM
    bound = tol * torch.outer(torch.linalg.norm(A, dim=1), torch.linalg.norm(Bt, dim=1))
    worst = float(((C - ref).abs() / bound).max())
    assert worst <= 1.0, "max err / bound = %.3g (device FP64 reference)" % worst
    An, Bn, Cn = A[rows].cpu().numpy(), Bt.cpu().numpy(), C[rows].cpu().numpy()
    ref_h = An @ Bn.T                                      # numpy on the host
    bound_h = tol * np.outer(np.linalg.norm(An, axis=1), np.linalg.norm(Bn, axis=1))
    worst_h = float((np.abs(Cn - ref_h) / bound_h).max())
    assert worst_h <= 1.0, "max err / bound = %.3g (host FP64 reference)" % worst_h
    return worst


@pytest.mark.parametrize("fmt", list(FORMATS))
@pytest.mark.parametrize("K", [4096, 8192])
def test_symmetric_product_at_route_size(g, fmt, K):
    X = _projector_like(K, seed=K + fmt[0])
    C = torch.full_like(X, float("nan"))
    g.op_product(X, X, C, nslice=fmt[0], max_order=fmt[1], slice_bits=fmt[2], symmetric=True)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(C).all()), "unwritten entries"
    assert bool((C == C.T).all())
    rows = np.random.default_rng(K).choice(K, 48, replace=False)
    _check_elements(C, X, X, FORMATS[fmt] * max(1.0, np.sqrt(K / 1000.0)), rows)


@pytest.mark.parametrize("fmt", list(FORMATS))
@pytest.mark.parametrize("K", [4096, 8192])
def test_general_product_at_route_size(g, fmt, K):
    rng = np.random.default_rng(3 * K + fmt[0])
    A = torch.from_numpy(rng.standard_normal((K, K))).cuda()
    Bt = torch.from_numpy(rng.standard_normal((K, K))).cuda()
    A[5] *= 1e-3                                             # rows of very different scale
    Bt[-2] *= 1e4
    C = torch.full((K, K), float("nan"), dtype=torch.float64, device="cuda")
    g.op_product(A, Bt, C, nslice=fmt[0], max_order=fmt[1], slice_bits=fmt[2])
    torch.cuda.synchronize()
    assert bool(torch.isfinite(C).all()), "unwritten entries"
    rows = np.concatenate([[5], np.random.default_rng(K + 1).choice(K, 47, replace=False)])
    _check_elements(C, A, Bt, FORMATS[fmt] * max(1.0, np.sqrt(K / 1000.0)), rows)

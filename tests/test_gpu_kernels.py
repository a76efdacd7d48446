"""GPU checks of the individual kernels through the C ABI (gdm_op_*), against FP64 references.

Tolerances follow from the slice format: with S slices of 11 bits and slice pairs up to order L
the product error is a small multiple of 2^(-11 (L+1)) * sqrt(K) * ||a_i|| ||b_j||, plus the FP32
rounding of orders >= 2 (weight <= 2^-46).  The bounds below are that estimate with a factor of
about 4-8 of headroom, checked element by element against ||a_i|| ||b_j||.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FORMATS = {  # (nslice, max_order, trailing bits): bound (x ||a_i|| ||b_j||) at K <= ~1000
    (0, 0, 12): 1e-13,
    (1, 0, 12): 6e-3,
    (2, 1, 12): 6e-5,
    (3, 2, 12): 6e-8,
    (3, 3, 12): 2e-9,
    (4, 3, 12): 2e-9,
    (3, 3, 9): 2e-8,
    (4, 3, 9): 1e-10,
}


@pytest.fixture(scope="module")
def g():
    import paper_1912_13403_gb300 as g
    return g


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check_product(C, A, Bt, tol):
    ref = A @ Bt.T
    na = np.linalg.norm(A, axis=1)
    nb = np.linalg.norm(Bt, axis=1)
    bound = tol * np.outer(na, nb) + 1e-300
    err = np.abs(C - ref)
    worst = float((err / bound).max())
    assert worst <= 1.0, "max err / bound = %.3g" % worst


@pytest.mark.parametrize("fmt", list(FORMATS))
@pytest.mark.parametrize("m,n,k", [(256, 256, 256), (200, 130, 300), (384, 129, 1000), (7, 5, 3)])
def test_product_matches_fp64(g, fmt, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((m, k))
    Bt = rng.standard_normal((n, k))
    A[0] *= 1e-3      # rows of very different scale
    Bt[-1] *= 1e4
    C = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    g.op_product(_dev(A), _dev(Bt), C, nslice=fmt[0], max_order=fmt[1], slice_bits=fmt[2])
    torch.cuda.synchronize()
    _check_product(C.cpu().numpy(), A, Bt, FORMATS[fmt])


@pytest.mark.parametrize("fmt", [(3, 3, 12), (2, 1, 12), (4, 3, 9)])
@pytest.mark.parametrize("k", [8200, 8201])
def test_product_wide_rows(g, fmt, k):
    # rows wider than the one-pass slicing kernel holds (8192 columns): the two-pass row / element
    # slicing (even k) and the per-row generic slicing (odd k); the bound grows like sqrt(K)
    rng = np.random.default_rng(k)
    A = rng.standard_normal((130, k))
    Bt = rng.standard_normal((131, k))
    A[3] *= 1e-3
    C = torch.zeros((130, 131), dtype=torch.float64, device="cuda")
    g.op_product(_dev(A), _dev(Bt), C, nslice=fmt[0], max_order=fmt[1], slice_bits=fmt[2])
    torch.cuda.synchronize()
    _check_product(C.cpu().numpy(), A, Bt, 4.0 * FORMATS[fmt])


@pytest.mark.parametrize("fmt", [(0, 0, 12), (3, 3, 12), (2, 1, 12), (4, 3, 9)])
@pytest.mark.parametrize("n", [128, 300, 515])
def test_symmetric_product_is_exactly_symmetric(g, fmt, n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n))
    X = X + X.T
    C = torch.full((n, n), np.nan, dtype=torch.float64, device="cuda")
    Xd = _dev(X)
    g.op_product(Xd, Xd, C, nslice=fmt[0], max_order=fmt[1], symmetric=True, slice_bits=fmt[2])
    Cn = C.cpu().numpy()
    assert np.all(np.isfinite(Cn)), "unwritten entries"
    assert np.array_equal(Cn, Cn.T)
    _check_product(Cn, X, X, FORMATS[fmt])


def test_product_leading_dimensions(g):
    rng = np.random.default_rng(3)
    Abig = rng.standard_normal((150, 400))
    Bbig = rng.standard_normal((170, 400))
    A = _dev(Abig)[:, :333]
    Bt = _dev(Bbig)[:, :333]
    Cbig = torch.zeros((150, 256), dtype=torch.float64, device="cuda")
    C = Cbig[:, :170]
    g.op_product(A, Bt, C, nslice=3, max_order=3)
    _check_product(C.cpu().numpy(), Abig[:, :333], Bbig[:, :333], FORMATS[(3, 3, 12)])
    assert torch.all(Cbig[:, 170:] == 0)


def test_product_slice_integer_exactness(g):
    """Entries that are small integers times a common power of two are represented exactly by
    one slice, so even the 1-slice product is exact when all partial sums stay below 2^24."""
    rng = np.random.default_rng(4)
    k = 512
    A = rng.integers(-40, 41, (256, k)).astype(np.float64)
    Bt = rng.integers(-40, 41, (256, k)).astype(np.float64)
    # row norms ~ 40*sqrt(512/3) ~ 520 -> sigma = 1024, scale 2: entries 2*a exact in 11 bits
    C = torch.zeros((256, 256), dtype=torch.float64, device="cuda")
    g.op_product(_dev(A), _dev(Bt), C, nslice=1, max_order=0)
    assert np.array_equal(C.cpu().numpy(), A @ Bt.T)


def test_symmetric_diagonal_is_exact(g):
    """The diagonal of a symmetric product is recomputed from the FP64 operands in FP32
    double-float arithmetic (~2^-48 relative): for X X with X a projector (rows of the two
    factors identical) it carries none of the accumulators' truncation bias (which was
    ~-8e-11 relative per entry, i.e. ~1e-8 on the trace of this case)."""
    from workloads import haar_orthogonal
    rng = np.random.default_rng(6)
    n, N = 640, 160
    Q = haar_orthogonal(rng, n)
    P = Q[:, :N] @ Q[:, :N].T
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    Pd = _dev(P)
    g.op_product(Pd, Pd, C, nslice=3, max_order=3, symmetric=True)
    d = np.diag(C.cpu().numpy()) - np.einsum("ij,ij->i", P, P)
    assert np.abs(d).max() <= 1e-14 and abs(d.sum()) <= 1e-12


def test_gershgorin_matches_oracle(g):
    from oracle import steps
    rng = np.random.default_rng(5)
    for n in (1, 9, 300):
        A = rng.standard_normal((n, n))
        A = A + A.T
        lo, hi = g.op_gershgorin(_dev(A))
        elo, ehi = steps.gershgorin_bounds(A)
        assert abs(lo - elo) <= 1e-12 * max(1, abs(elo)) and abs(hi - ehi) <= 1e-12 * max(1, abs(ehi))


@pytest.mark.parametrize("fmt,tol", [((0, 0), 1e-12), ((3, 3), 1e-8)])
@pytest.mark.parametrize("n,n_occ,spread", [(200, 60, (0.05, 0.95)), (257, 100, (0.0, 1.0)),
                                            (128, 32, (0.3, 0.35)), (128, 96, (0.9, 1.0))])
def test_trs4_step_matches_oracle(g, fmt, tol, n, n_occ, spread):
    from oracle import steps
    from workloads import haar_orthogonal
    rng = np.random.default_rng(n + n_occ)
    Q = haar_orthogonal(rng, n)
    x = rng.uniform(spread[0], spread[1], n)
    X = steps.sym((Q * x) @ Q.T)
    Xe, ge, bre = steps.trs4_step(X, n_occ)
    Xd = _dev(X)
    gamma, br = g.op_trs4_step(Xd, n_occ, nslice=fmt[0], max_order=fmt[1])
    names = {0: "2X-X2", 1: "X2", 2: "F+gG"}
    assert names[br] == bre
    # gamma = (N - Tr F)/Tr G amplifies product errors by (N + |Tr F|)/|Tr G|
    _, trF, trG = steps.trs4_gamma(X, n_occ)
    amp = (n_occ + abs(trF)) / abs(trG)
    assert abs(gamma - ge) <= max(tol, 1e-13) * amp * max(1.0, abs(ge))
    err = np.linalg.norm(Xd.cpu().numpy() - Xe) / np.linalg.norm(Xe)
    assert err <= tol

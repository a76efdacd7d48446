"""The Python binding checks shapes and devices before a pointer reaches the library.

The C ABI takes plain pointers and sizes and trusts them (it checks leading dimensions, not the
extent of the caller's buffers), so a C with fewer rows than A, or a Bt with fewer columns than A,
would make a kernel write or read outside an allocation.  These checks run on the CPU: a shape
mismatch is reported before the device check, and host tensors or numpy arrays never reach the
device operations.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1912_13403_gb300 as g
    return g


def _z(*shape):
    return torch.zeros(shape, dtype=torch.float64)


@pytest.mark.parametrize("op", ["op_product", "op_product_noalloc"])
@pytest.mark.parametrize("a,b,c,msg", [
    ((8, 5), (6, 5), (7, 6), "C must be 8 x 6"),        # C short of rows
    ((8, 5), (6, 5), (8, 5), "C must be 8 x 6"),        # C short of columns
    ((8, 5), (6, 4), (8, 6), "contraction length"),     # Bt narrower than A
    ((8, 5), (6, 7), (8, 6), "contraction length"),     # Bt wider than A
])
def test_product_shape_mismatch_rejected(g, op, a, b, c, msg):
    with pytest.raises(ValueError, match=msg):
        getattr(g, op)(_z(*a), _z(*b), _z(*c))


@pytest.mark.parametrize("op", ["op_product", "op_product_noalloc"])
def test_product_symmetric_needs_square(g, op):
    with pytest.raises(ValueError, match="m == n"):
        getattr(g, op)(_z(4, 3), _z(5, 3), _z(4, 5), symmetric=True)


@pytest.mark.parametrize("op", ["op_product", "op_product_noalloc"])
def test_product_host_operands_rejected(g, op):
    # matching shapes, but host memory: never passed on as device pointers
    with pytest.raises(ValueError, match="CUDA tensor"):
        getattr(g, op)(_z(4, 3), _z(5, 3), _z(4, 5))
    a = np.zeros((4, 3))
    with pytest.raises(ValueError, match="CUDA tensor"):
        getattr(g, op)(a, np.zeros((5, 3)), np.zeros((4, 5)))


def test_other_device_ops_check_shape_and_device(g):
    with pytest.raises(ValueError, match="must be 3 x 3"):
        g.op_gershgorin(_z(3, 4))
    with pytest.raises(ValueError, match="CUDA tensor"):
        g.op_gershgorin(_z(3, 3))
    with pytest.raises(ValueError, match="must be 3 x 3"):
        g.op_trs4_step(_z(3, 4), 1)
    with pytest.raises(ValueError, match="CUDA tensor"):
        g.op_trs4_step(_z(3, 3), 1)


def test_problem_and_handle_buffers_must_be_n_by_n(g):
    with pytest.raises(ValueError, match="S must be 4 x 4"):
        g._problem(np.zeros((4, 4)), np.zeros((3, 3)), 1)
    with pytest.raises(ValueError, match="P must be 4 x 4"):
        g._problem(np.zeros((4, 4)), np.zeros((4, 4)), 1, np.zeros((4, 3)))
    # a Handle checks before any CUDA call; exercise the check without creating one
    h = g.Handle.__new__(g.Handle)
    h.n = 4
    with pytest.raises(ValueError, match="S must be 4 x 4"):
        h.set_overlap(np.zeros((5, 5)))
    with pytest.raises(ValueError, match="H must be 4 x 4"):
        h.set_hamiltonian(np.zeros((4, 3)))
    with pytest.raises(ValueError, match="P must be 4 x 4"):
        h.solve(np.zeros((3, 4)))

"""The allocation-free product (gdm_op_product_noalloc) against the allocating one.

gdm_op_product_noalloc serves callers that cannot allocate device memory (another component owns
the memory pool, or the caller cannot afford an allocation inside its loop); it keeps its slices
in a fixed array inside the library.  This file runs last so that a failure here leaves every
other test already run; it must pass alone in a fresh process as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

BOUND = {(3, 3, 12): 2e-9, (4, 3, 9): 1e-10, (2, 1, 12): 6e-5}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_no_alloc_matches_allocating_product_on_consecutive_calls():
    import paper_1912_13403_gb300 as g
    rng = np.random.default_rng(2024)
    # two calls in a row of each case, the second case smaller than the first so that any stale
    # slices of the first would show up in the second
    cases = [(700, 600, 900, (3, 3, 12), False), (300, 200, 257, (3, 3, 12), False),
             (512, 512, 512, (4, 3, 9), True), (129, 129, 1000, (2, 1, 12), True)]
    runs = []
    for m, n, k, fmt, sym in cases:
        A = rng.standard_normal((m, k))
        if sym:
            A = A[:, :m] if k >= m else A
            B = A.copy()
        else:
            B = rng.standard_normal((n, k))
        Ad, Bd = _dev(A), _dev(B)
        C_ref = torch.zeros((m, B.shape[0]), dtype=torch.float64, device="cuda")
        g.op_product(Ad, Bd, C_ref, nslice=fmt[0], max_order=fmt[1], slice_bits=fmt[2],
                     symmetric=sym)
        outs = [torch.full_like(C_ref, np.nan) for _ in range(2)]
        runs.append((A, B, Ad, Bd, C_ref, outs, fmt, sym))
    # every output buffer exists before the first call; one call of each case first (the first
    # call on the device looks up the array's address, and each kernel loads on its first launch)
    for A, B, Ad, Bd, C_ref, outs, fmt, sym in runs:
        g.op_product_noalloc(Ad, Bd, outs[0], nslice=fmt[0], max_order=fmt[1],
                             slice_bits=fmt[2], symmetric=sym)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for A, B, Ad, Bd, C_ref, outs, fmt, sym in runs:
        for C in outs:
            C.fill_(np.nan)
            g.op_product_noalloc(Ad, Bd, C, nslice=fmt[0], max_order=fmt[1],
                                 slice_bits=fmt[2], symmetric=sym)
    torch.cuda.synchronize()
    # the defining property: no device memory was taken, neither from the driver nor from
    # torch's caching allocator
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    for A, B, Ad, Bd, C_ref, outs, fmt, sym in runs:
        Rn = C_ref.cpu().numpy()
        bound = BOUND[fmt] * np.outer(np.linalg.norm(A, axis=1), np.linalg.norm(B, axis=1))
        for call, C in enumerate(outs):
            Cn = C.cpu().numpy()
            assert np.all(np.isfinite(Cn)), (A.shape, call)
            assert np.all(np.abs(Cn - Rn) <= bound), (A.shape, call)
            assert np.all(np.abs(Cn - A @ B.T) <= bound), (A.shape, call)


def test_no_alloc_rejects_sizes_beyond_its_array():
    import paper_1912_13403_gb300 as g
    A = torch.zeros((1025, 8), dtype=torch.float64, device="cuda")
    C = torch.zeros((1025, 1025), dtype=torch.float64, device="cuda")
    with pytest.raises(g.GdmError) as ei:
        g.op_product_noalloc(A, A, C)
    assert ei.value.status == g.GDM_ERR_ARG

"""Batched solves (gdm_solve_batch) and the request server (gdm_server_*), on the GPU.

Each problem solved in a batch or in the server's mix must give the same density matrix as
when it is solved alone on its own handle (same kernels, same inputs: bit-for-bit identical is
expected; the check allows 1e-12 relative), and each must meet the oracle bars.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from workloads import make_random_small, make_spectrum_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1912_13403_gb300 as g
    return g


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def alone(g, p):
    with g.Handle(p.n, p.n_occ) as h:
        h.set_overlap(p.S)
        h.set_hamiltonian(p.H)
        P, e, info, st = h.solve()
    return P, e


def problems():
    sizes = [(300, 75), (130, 40), (520, 130), (257, 64), (64, 16), (700, 175), (200, 150)]
    out = []
    for i, (n, N) in enumerate(sizes):
        if i % 2:
            out.append(make_random_small(500 + i, n, N))
        else:
            out.append(make_spectrum_problem(600 + i, n, N, cond_S=100.0, gap=0.3))
    return out


def test_batch_matches_alone_and_oracle(g):
    ps = problems()
    outs = [np.empty((p.n, p.n)) for p in ps]
    st, res = g.solve_batch([(p.H, p.S, p.n_occ, P) for p, P in zip(ps, outs)], concurrency=3)
    assert st == g.GDM_OK
    for p, P, r in zip(ps, outs, res):
        assert r["status"] == g.GDM_OK
        Pa, ea = alone(g, p)
        assert rel(P, Pa) <= 1e-12 and abs(r["energy"] - ea) <= 1e-12 * abs(ea)
        ref = oracle.density_matrix(p.H, p.S, p.n_occ)
        assert rel(P, ref["P"]) <= 1e-6
        assert r["info"]["trace_err"] <= 1e-8


def test_batch_device_buffers(g):
    ps = problems()[:3]
    items = []
    for p in ps:
        items.append((torch.from_numpy(p.H).cuda(), torch.from_numpy(p.S).cuda(), p.n_occ,
                      torch.empty((p.n, p.n), dtype=torch.float64, device="cuda")))
    st, res = g.solve_batch(items, concurrency=2)
    assert st == g.GDM_OK
    for p, it in zip(ps, items):
        Pa, _ = alone(g, p)
        assert rel(it[3].cpu().numpy(), Pa) <= 1e-12


def test_server_mix_matches_alone(g):
    ps = problems()
    outs = [np.empty((p.n, p.n)) for p in ps]
    with g.Server(slots=3) as srv:
        tickets = []
        for p, P in zip(ps, outs):   # requests arrive while earlier ones run
            tickets.append(srv.submit(p.H, p.S, p.n_occ, P))
            time.sleep(0.002)
        res = [srv.wait(t, 60.0) for t in tickets]
    for p, P, r in zip(ps, outs, res):
        assert r["status"] == g.GDM_OK, r
        assert r["latency_ms"] > 0
        Pa, ea = alone(g, p)
        assert rel(P, Pa) <= 1e-12
        assert abs(r["energy"] - ea) <= 1e-12 * abs(ea)


def test_server_poll_timeout_budget_and_shutdown(g):
    big = make_spectrum_problem(700, 1024, 256, cond_S=10.0, gap=0.3)
    small = make_random_small(701, 100, 30)
    # a budget below one handle of this size is refused at submission
    with g.Server(slots=1, hbm_budget_bytes=1 << 20) as srv:
        with pytest.raises(g.GdmError) as ei:
            srv.submit(small.H, small.S, small.n_occ)
        assert ei.value.status == g.GDM_ERR_BUDGET
    with g.Server(slots=1) as srv:
        t1 = srv.submit(big.H, big.S, big.n_occ, np.empty((1024, 1024)))
        t2 = srv.submit(small.H, small.S, small.n_occ, np.empty((100, 100)))
        with pytest.raises(g.GdmError) as ei:   # t2 waits behind t1 on the single slot
            srv.wait(t2, 0.0)
        assert ei.value.status == g.GDM_ERR_TIMEOUT
        r1 = srv.wait(t1, 60.0)
        assert r1["status"] == g.GDM_OK
        r2 = None
        for _ in range(6000):
            r2 = srv.poll(t2)
            if r2 is not None:
                break
            time.sleep(0.01)
        assert r2 is not None and r2["status"] == g.GDM_OK
        with pytest.raises(g.GdmError):          # a ticket is forgotten once collected
            srv.poll(t2)
    # shutting down with queued requests cancels them
    srv = g.Server(slots=1)
    for _ in range(3):
        srv.submit(big.H, big.S, big.n_occ, np.empty((1024, 1024)))
    srv.close()

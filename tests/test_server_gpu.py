"""Serving runtime on the GPU: requests of different meshes, degrees and right-hand-side
counts give the same field run alone and run together (continuous batching), and each field
solves its own system to the FP64 residual bar."""
import numpy as np
import pytest

import synth
from oracle import problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def O():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_04521_gb300 import build
    build.build()
    from paper_1605_04521_gb300 import oras
    return oras


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


REQUESTS = [
    synth.small(n=4, r=2, nsub=8, overlap=1, nrhs=1),
    synth.small(n=3, r=3, nsub=4, overlap=1, nrhs=3),
    synth.small(n=6, r=1, nsub=8, overlap=2, nrhs=2),
    synth.small(n=5, r=2, nsub=4, overlap=1, nrhs=5),
    synth.small(n=4, r=1, nsub=2, overlap=0, head=False, source="plane"),
    # three of the same shape with long tensor-core factorisations that overlap in time
    synth.small(n=8, r=2, nsub=8, overlap=1, nrhs=1),
    synth.small(n=8, r=2, nsub=8, overlap=1, nrhs=2),
    synth.small(n=8, r=2, nsub=8, overlap=1, nrhs=4),
]


def submit(O, srv, w, p):
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    kw = dict(restart=w.restart, factor_bits=w.factor_bits)
    if w.source == "plane":  # explicit right-hand side, computed by the oracle
        return O.oras_submit(srv, xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, rhs=p.B, tol=w.tol, **kw)
    d = np.concatenate([synth.dipole_ring(w.nrhs), np.tile([0.0, 0.0, 1.0], (w.nrhs, 1))], axis=1)
    return O.oras_submit(srv, xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, dipoles=d, tol=w.tol, **kw)


def test_alone_and_in_the_mix(O):
    probs = [problem.from_workload(w, with_oras=False) for w in REQUESTS]
    # alone: one slot, one request at a time
    alone = []
    srv = O.oras_server_create(max_active=1)
    try:
        for w, p in zip(REQUESTS, probs):
            t = submit(O, srv, w, p)
            x, info, rc = O.oras_wait(srv, t)
            assert rc == O.ORAS_OK, O.oras_server_error(srv, t)
            alone.append(np.asarray(x).reshape(p.A.shape[0], -1))
    finally:
        O.oras_server_destroy(srv)
    # the mix: everything submitted at once, three slots
    srv = O.oras_server_create(max_active=4)
    try:
        tickets = [submit(O, srv, w, p) for w, p in zip(REQUESTS, probs)]
        mix = []
        for t, p in zip(tickets, probs):
            x, info, rc = O.oras_wait(srv, t)
            assert rc == O.ORAS_OK, O.oras_server_error(srv, t)
            assert all(i["converged"] for i in info)
            mix.append(np.asarray(x).reshape(p.A.shape[0], -1))
        st = O.oras_server_stats(srv)
        assert st["completed"] == len(REQUESTS) and st["rejected"] == 0
        assert st["peak_active"] >= 2          # requests were on the GPU together
        assert st["hbm_in_use"] == 0 and st["active"] == 0
        recs = [O.oras_ticket_info(srv, t) for t in tickets]
        assert all(r["submit_s"] <= r["planned_s"] <= r["admitted_s"] <= r["done_s"] for r in recs)
    finally:
        O.oras_server_destroy(srv)
    for w, p, xa, xm in zip(REQUESTS, probs, alone, mix):
        for j in range(xa.shape[1]):
            assert rel(xm[:, j], xa[:, j]) <= 1e-6                     # alone == in the mix
            assert np.array_equal(xm[:, j], xa[:, j])                  # (deterministic kernels)
            b = p.B[:, j]
            assert np.linalg.norm(b - p.A @ xm[:, j]) / np.linalg.norm(b) <= 1e-8 * 1.01


def test_budget_queues_instead_of_overcommitting(O):
    """A budget that holds one request at a time: requests wait in the queue, none is rejected,
    and the bytes in use never exceed the budget."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1, nrhs=1)
    p = problem.from_workload(w, with_oras=False)
    xyz, tets = w.mesh()
    h = O.oras_create(xyz, tets, w.r, w.nsub, w.overlap, restart=w.restart)
    fp = O.oras_footprint(h, 1)
    O.oras_destroy(h)
    budget = int(1.5 * (fp + 2 * p.A.shape[0] * 16 + (4 << 20)))
    srv = O.oras_server_create(hbm_budget=budget, max_active=3)
    try:
        tickets = [submit(O, srv, w, p) for _ in range(3)]
        xs = []
        for t in tickets:
            x, info, rc = O.oras_wait(srv, t)
            assert rc == O.ORAS_OK
            xs.append(x)
        st = O.oras_server_stats(srv)
        assert st["peak_active"] == 1 and st["hbm_peak"] <= budget and st["rejected"] == 0
        assert all(np.array_equal(xs[0], x) for x in xs[1:])
    finally:
        O.oras_server_destroy(srv)

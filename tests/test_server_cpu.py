"""Serving runtime, host logic only (no GPU work is admitted): footprint, rejection by the HBM
budget, set-up errors reported through the ticket, ticket bookkeeping."""
import ctypes as C

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def O():
    from paper_1605_04521_gb300 import build
    build.build()
    from paper_1605_04521_gb300 import oras
    return oras


def _mesh(n=2):
    xyz, tets = synth.kuhn_cube(n)
    return xyz, tets, synth.homogeneous_materials(len(tets))


def test_footprint_counts_arena_and_krylov_basis(O):
    xyz, tets, _ = _mesh(3)
    h = O.oras_create(xyz, tets, 2, 4, 1, restart=20)
    try:
        nsub = O.oras_nsub(h)
        npad = sum(O.oras_subdomain_size(h, s)[2] for s in range(nsub))
        n2 = sum(O.oras_subdomain_size(h, s)[2] ** 2 for s in range(nsub))
        N = O.oras_ndof(h)
        f1, f4 = O.oras_footprint(h, 1), O.oras_footprint(h, 4)
        # FP32 factor arena (8 B per complex entry) is part of it
        assert f1 > 8 * n2
        # three more right-hand sides add at least their FP64 basis (21 vectors) and FP32 Z (20)
        assert f4 - f1 >= 3 * N * (21 * 16 + 20 * 8)
        assert npad % 64 == 0
        with pytest.raises(O.OrasError):
            O.oras_footprint(h, 0)
    finally:
        O.oras_destroy(h)


def test_budget_rejection_and_ticket_records(O):
    srv = O.oras_server_create(hbm_budget=1 << 20, max_active=2, planners=1)
    try:
        xyz, tets, eps = _mesh(2)
        t = O.oras_submit(srv, xyz, tets, eps, None, synth.K0, 1, 2, 1, dipoles=[[0.5, 0.5, 0.5, 0, 0, 1]])
        assert t > 0
        x, info, rc = O.oras_wait(srv, t)
        assert rc == O.ORAS_ERR_REJECTED and x is None
        rec = O.oras_ticket_info(srv, t)
        assert rec["status"] == O.ORAS_ERR_REJECTED and rec["footprint"] > (1 << 20)
        assert rec["submit_s"] <= rec["planned_s"] <= rec["done_s"] and rec["admitted_s"] == 0.0
        assert "budget" in O.oras_server_error(srv, t)
        st = O.oras_server_stats(srv)
        assert st["rejected"] == 1 and st["completed"] == 0 and st["active"] == 0 and st["hbm_in_use"] == 0
        with pytest.raises(O.ServerError):  # retired
            O.oras_wait(srv, t)
    finally:
        O.oras_server_destroy(srv)


def test_setup_errors_come_back_through_the_ticket(O):
    srv = O.oras_server_create(hbm_budget=1 << 20, max_active=1, planners=2)
    try:
        xyz, tets, eps = _mesh(2)
        bad = tets.copy()
        bad[3, 2] = len(xyz) + 5
        t1 = O.oras_submit(srv, xyz, bad, eps, None, synth.K0, 1, 2, 1, dipoles=[[0.5, 0.5, 0.5, 0, 0, 1]])
        t2 = O.oras_submit(srv, xyz, tets, eps, None, synth.K0, 1, 2, 1, rhs=np.ones(7, dtype=complex))
        t3 = O.oras_submit(srv, xyz, tets, eps, None, synth.K0, 9, 2, 1, dipoles=[[0.5, 0.5, 0.5, 0, 0, 1]])
        assert t1 < t2 < t3
        assert O.oras_wait(srv, t1)[2] == O.ORAS_ERR_BAD_MESH
        assert O.oras_wait(srv, t2)[2] == O.ORAS_ERR_INVALID_ARG      # 7 rows != N
        assert "rows" in O.oras_server_error(srv, t2)
        assert O.oras_wait(srv, t3)[2] == O.ORAS_ERR_INVALID_ARG      # r = 9
        assert O.oras_server_stats(srv)["completed"] == 3
    finally:
        O.oras_server_destroy(srv)


def test_submit_argument_checks(O):
    srv = O.oras_server_create(hbm_budget=1 << 20, max_active=1, planners=1)
    try:
        xyz, tets, eps = _mesh(1)
        p, keep = O._problem(xyz, tets, eps, None, synth.K0, 1, 1, 0, None)
        o = O._options()
        b = np.ones((10, 1), dtype=np.complex128)
        d = np.zeros(6)
        sub = O.lib.oras_submit
        assert sub(srv, C.byref(p), C.byref(o), None, 0, None, 1, 1e-8) == O.ORAS_ERR_INVALID_ARG  # no rhs
        assert sub(srv, C.byref(p), C.byref(o), O._ptr(b), 10, O._ptr(d), 1, 1e-8) == O.ORAS_ERR_INVALID_ARG  # both
        assert sub(srv, C.byref(p), C.byref(o), None, 0, O._ptr(d), 0, 1e-8) == O.ORAS_ERR_INVALID_ARG   # k = 0
        assert sub(srv, C.byref(p), C.byref(o), None, 0, O._ptr(d), 1, 0.0) == O.ORAS_ERR_INVALID_ARG   # tol
        assert sub(None, C.byref(p), C.byref(o), None, 0, O._ptr(d), 1, 1e-8) == O.ORAS_ERR_INVALID_ARG
        del keep
        with pytest.raises(O.ServerError):
            O.oras_ticket_info(srv, 12345)
    finally:
        O.oras_server_destroy(srv)


def test_destroy_with_requests_in_flight(O):
    srv = O.oras_server_create(hbm_budget=1 << 20, max_active=1, planners=1)
    xyz, tets, eps = _mesh(3)
    for _ in range(5):
        O.oras_submit(srv, xyz, tets, eps, None, synth.K0, 2, 4, 1, dipoles=[[0.5, 0.5, 0.5, 0, 0, 1]])
    O.oras_server_destroy(srv)   # cancels or finishes every ticket, joins the threads

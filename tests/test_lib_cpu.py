"""CPU-only checks of the CUDA library: it loads, exports every symbol of include/oras.h, and
its host integer set-up (DOF numbering, partition, overlap, N_s, D_s) is bit-exact against
the oracle.  No GPU call is made here."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import dd, topology

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def O():
    from paper_1605_04521_gb300 import build
    build.build()
    from paper_1605_04521_gb300 import oras
    return oras


def test_exports_every_declared_symbol(O):
    hdr = open(os.path.join(ROOT, "include", "oras.h")).read()
    declared = sorted(set(re.findall(r"\b(oras_[a-z_0-9]+)\s*\(", hdr)))
    assert len(declared) >= 25
    for name in declared:
        assert hasattr(O.lib, name), name
        assert name in O.EXPORTS, name


@pytest.mark.parametrize("n,r,nsub,delta,kind", [
    (4, 2, 8, 1, "vertex"), (8, 1, 8, 1, "vertex"), (3, 3, 4, 2, "vertex"), (5, 2, 16, 1, "vertex"),
    (4, 2, 8, 2, "face"), (6, 1, 7, 1, "vertex"), (2, 3, 1, 0, "vertex"), (16, 2, 64, 2, "vertex")])
def test_host_setup_bit_exact(O, n, r, nsub, delta, kind):
    xyz, tets = synth.kuhn_cube(n)
    h = O.oras_create(xyz, tets, r, nsub, delta,
                      overlap_kind=O.ORAS_OVERLAP_FACE if kind == "face" else O.ORAS_OVERLAP_VERTEX)
    try:
        topo = topology.build(tets, len(xyz), r)
        dec = dd.decompose(topo, xyz, nsub, delta, kind=kind)
        assert O.oras_ndof(h) == topo.ndof
        assert np.array_equal(O.oras_dofmap(h, len(tets)), topo.dofmap)
        assert np.array_equal(O.oras_partition(h, len(tets)), dec.part)
        for s in range(nsub):
            dofs, pou, tt = O.oras_subdomain(h, s)
            assert np.array_equal(dofs, dec.dofs[s])
            assert np.array_equal(pou, dec.pou[s].astype(np.uint8))
            assert np.array_equal(tt, dec.tets[s])
            _, _, npad = O.oras_subdomain_size(h, s)
            assert npad % 64 == 0 and npad >= len(dofs) > npad - 64
    finally:
        O.oras_destroy(h)


def test_user_partition_and_csr_pattern(O):
    """A caller-given partition is used as is; the CSR pattern equals the oracle's."""
    import scipy.sparse as sp
    xyz, tets = synth.kuhn_cube(3)
    rng = np.random.default_rng(0)
    part = rng.integers(0, 5, size=len(tets)).astype(np.int32)
    part[:5] = np.arange(5)
    h = O.oras_create(xyz, tets, 2, 5, 1, part=part)
    try:
        assert np.array_equal(O.oras_partition(h, len(tets)), part)
        rowptr = np.empty(O.oras_ndof(h) + 1, dtype=np.int64)
        cols = np.empty(O.oras_nnz(h), dtype=np.int32)
        O._check(h, O.lib.oras_global_csr(h, O._ptr(rowptr), O._ptr(cols), None))
        topo = topology.build(tets, len(xyz), 2)
        nl = topo.dofmap.shape[1]
        rows = np.repeat(topo.dofmap, nl, axis=1).ravel()
        cc = np.tile(topo.dofmap, (1, nl)).ravel()
        P = sp.coo_matrix((np.ones(len(rows)), (rows, cc)), shape=(topo.ndof,) * 2).tocsr()
        P.sort_indices()
        assert np.array_equal(rowptr, P.indptr) and np.array_equal(cols, P.indices)
    finally:
        O.oras_destroy(h)


def test_error_codes(O):
    xyz, tets = synth.kuhn_cube(2)
    bad = tets.copy()
    bad[3, 1] = len(xyz) + 7
    with pytest.raises(O.OrasError) as e:
        O.oras_create(xyz, bad, 1, 2, 0)
    assert e.value.code == O.ORAS_ERR_BAD_MESH
    rep = tets.copy()
    rep[0, 1] = rep[0, 0]
    with pytest.raises(O.OrasError) as e:
        O.oras_create(xyz, rep, 1, 2, 0)
    assert e.value.code == O.ORAS_ERR_BAD_MESH
    flat = xyz.copy()
    flat[:, 2] = 0.0
    with pytest.raises(O.OrasError) as e:
        O.oras_create(flat, tets, 1, 2, 0)
    assert e.value.code == O.ORAS_ERR_BAD_MESH
    for kw in (dict(r=4, nsub=2, overlap=0), dict(r=1, nsub=0, overlap=0),
               dict(r=1, nsub=len(tets) + 1, overlap=0), dict(r=1, nsub=2, overlap=-1)):
        with pytest.raises(O.OrasError) as e:
            O.oras_create(xyz, tets, kw["r"], kw["nsub"], kw["overlap"])
        assert e.value.code == O.ORAS_ERR_INVALID_ARG
    with pytest.raises(O.OrasError) as e:
        O.oras_create(xyz, tets, 1, 2, 0, factor_bits=16)
    assert e.value.code == O.ORAS_ERR_INVALID_ARG
    with pytest.raises(O.OrasError) as e:
        O.oras_create(xyz, tets, 1, 2, 0, transmission=2)
    assert e.value.code == O.ORAS_ERR_INVALID_ARG
    # numeric calls before the numeric set-up report a state error without touching a GPU
    h = O.oras_create(xyz, tets, 1, 2, 0)
    try:
        with pytest.raises(O.OrasError) as e:
            O.oras_solve(h, np.ones(O.oras_ndof(h)), 1e-8)
        assert e.value.code == O.ORAS_ERR_STATE
        with pytest.raises(O.OrasError) as e:
            O.oras_matvec(h, np.ones(O.oras_ndof(h)))
        assert e.value.code == O.ORAS_ERR_STATE
        with pytest.raises(O.OrasError) as e:
            O.oras_matvec_c64(h, np.ones(O.oras_ndof(h)))
        assert e.value.code == O.ORAS_ERR_STATE
        with pytest.raises(O.OrasError) as e:
            O.oras_autotune(h)
        assert e.value.code == O.ORAS_ERR_STATE
    finally:
        O.oras_destroy(h)


def test_release_memory_of_a_missing_device_is_an_error(O):
    """Device 9999 does not exist: INVALID_ARG on a GPU machine, CUDA (no device) here."""
    with pytest.raises(O.OrasError) as e:
        O.oras_release_memory(9999)
    assert e.value.code in (O.ORAS_ERR_INVALID_ARG, O.ORAS_ERR_CUDA)


def test_noalloc_rejects_oversized_scratch_on_host(O):
    """The allocation-free apply keeps its local vectors in a fixed 16 MiB device array; a problem
    whose padded subdomain orders times the FP64 entry size exceed it is rejected from the host
    set-up alone (INVALID_ARG with the needed size), before any device work.  The vector pointers
    are never dereferenced on this path."""
    import ctypes as C
    xyz, tets = synth.kuhn_cube(24)
    h = O.oras_create(xyz, tets, 2, 256, 1, factor_bits=64)
    try:
        total = sum(O.oras_subdomain_size(h, s)[2] for s in range(256))
        assert total * 16 > 16 << 20
        dummy = (C.c_double * 4)()
        rc = O.lib.oras_precond_noalloc(h, C.cast(dummy, C.c_void_p), C.cast(dummy, C.c_void_p), 1)
        assert rc == O.ORAS_ERR_INVALID_ARG
        msg = O.lib.oras_last_error(h).decode()
        assert str(total * 16) in msg and "16777216" in msg
    finally:
        O.oras_destroy(h)
    xyz4, tets4 = synth.kuhn_cube(4)
    h = O.oras_create(xyz4, tets4, 2, 8, 1)
    try:  # a problem that fits: the next check is the call order (no oras_factor yet)
        dummy = (C.c_double * 4)()
        rc = O.lib.oras_precond_noalloc(h, C.cast(dummy, C.c_void_p), C.cast(dummy, C.c_void_p), 1)
        assert rc == O.ORAS_ERR_STATE
    finally:
        O.oras_destroy(h)


def test_beta_face_validation(O):
    """beta_face entries of outer faces must be finite and positive (Sec. 2: beta > 0); entries of
    interior faces are ignored."""
    xyz, tets = synth.kuhn_cube(3)
    topo = topology.build(tets, len(xyz), 1)
    beta = np.full((len(tets), 4), 7.5)
    # interior-face entries may hold anything
    inner = np.ones((len(tets), 4), dtype=bool)
    st = np.sort(tets, axis=1)
    for t in range(len(tets)):
        for lf in range(4):
            if topo.face_tets[topo.tet_faces[t, lf], 1] < 0:
                opp = st[t, (3, 2, 1, 0)[lf]]
                inner[t, list(tets[t]).index(opp)] = False
    assert (~inner).sum() == 12 * 9          # 2 triangles on each of the 6 n^2 boundary squares
    beta[inner] = -1.0
    h = O.oras_create(xyz, tets, 1, 4, 1, beta_face=beta)
    O.oras_destroy(h)
    t, q = np.argwhere(~inner)[5]
    bad = beta.copy()
    bad[t, q] = 0.0
    with pytest.raises(O.OrasError) as e:
        O.oras_create(xyz, tets, 1, 4, 1, beta_face=bad)
    assert e.value.code == O.ORAS_ERR_INVALID_ARG


def _wall_kinds(xyz, tets, walls):
    kind = np.zeros((len(tets), 4), dtype=np.uint8)
    for t in range(len(tets)):
        for q in range(4):
            P = xyz[[tets[t][j] for j in range(4) if j != q]]
            for ax, val in walls:
                if np.all(np.abs(P[:, ax] - val) < 1e-12):
                    kind[t, q] = 1
    return kind


@pytest.mark.parametrize("r", [1, 2, 3])
def test_constrained_dofs_bit_exact(O, r):
    """The degrees of freedom the host set-up constrains for metallic faces (the face-local ones
    of each metallic face) equal the oracle's, found by evaluating the tangential traces of the
    basis functions (Sec. 2 eq. metallicbc), for the four side walls of a 3^3 cube and a caller's
    vertex order that is not sorted."""
    from oracle import ports
    xyz, tets = synth.kuhn_cube(3)
    rng = np.random.default_rng(9)
    tets = np.array([rng.permutation(t) for t in tets])
    kind = _wall_kinds(xyz, tets, [(0, 0.0), (0, 1.0), (1, 0.0), (1, 1.0)])
    topo = topology.build(tets, len(xyz), r)
    ref = ports.constrained_dofs(topo, xyz, ports.face_kind_table(tets, kind))
    h = O.oras_create(xyz, tets, r, 4, 1, face_kind=kind)
    try:
        got = O.oras_constrained_dofs(h)
        assert np.array_equal(got.astype(bool), ref)
    finally:
        O.oras_destroy(h)
    h = O.oras_create(xyz, tets, r, 4, 1)
    try:
        assert not O.oras_constrained_dofs(h).any()
    finally:
        O.oras_destroy(h)


def test_face_kind_validation(O):
    """face_kind entries must be 0 or 1, and 1 only on outer faces; beta_face is not read on
    metallic faces."""
    xyz, tets = synth.kuhn_cube(2)
    kind = _wall_kinds(xyz, tets, [(0, 0.0)])
    beta = np.full((len(tets), 4), 3.0)
    beta[kind == 1] = 0.0                      # not read on metallic faces
    h = O.oras_create(xyz, tets, 2, 2, 1, beta_face=beta, face_kind=kind)
    O.oras_destroy(h)
    bad = kind.copy()
    bad[0, 0] = 2
    with pytest.raises(O.OrasError) as e:
        O.oras_create(xyz, tets, 2, 2, 1, face_kind=bad)
    assert e.value.code == O.ORAS_ERR_INVALID_ARG
    topo = topology.build(tets, len(xyz), 1)
    st = np.sort(tets, axis=1)
    t, lf = next((t, lf) for t in range(len(tets)) for lf in range(4)
                 if topo.face_tets[topo.tet_faces[t, lf], 1] >= 0)
    inner = np.zeros_like(kind)
    inner[t, list(tets[t]).index(st[t, (3, 2, 1, 0)[lf]])] = 1
    with pytest.raises(O.OrasError) as e:
        O.oras_create(xyz, tets, 2, 2, 1, face_kind=inner)
    assert e.value.code == O.ORAS_ERR_INVALID_ARG
    assert abs(O.oras_s_error(np.array([1 + 1j, 2.0]), np.array([1 + 1j, 2.0]))) == 0.0
    assert abs(O.oras_s_error(np.array([2.0, 4.0]), np.array([1.0, 2.0])) - 1.0) < 1e-15

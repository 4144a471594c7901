"""Pins of the CPU oracle against facts it does not compute itself.

Each test states the independent fact it checks: closed forms, identities of the
paper, textbook special cases, library routines and brute force on tiny meshes.
"""
import itertools
from math import comb

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import assemble, basis, dd, elements, fgmres, problem, quadrature, topology


def counts_closed_form(n):
    """Kuhn mesh of n^3 cubes: vertices, edges (axis + face diagonals + body diagonals),
    tets; faces from Euler's formula V - E + F - T = 1 for a ball."""
    V = (n + 1) ** 3
    E = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    T = 6 * n ** 3
    F = 1 - V + E + T
    return V, E, F, T


def ndof_closed_form(n, r):
    """First-kind Nedelec: r per edge, r(r-1) per face, r(r-1)(r-2)/2 per tet."""
    _, E, F, T = counts_closed_form(n)
    return r * E + r * (r - 1) * F + r * (r - 1) * (r - 2) // 2 * T


def random_tet(rng):
    while True:
        v = rng.normal(size=(4, 3))
        if abs(np.linalg.det(v[1:] - v[0])) > 0.3:
            return v


# ---------------------------------------------------------------- counts / numbering

@pytest.mark.parametrize("n", [1, 2, 3, 8, 16])
@pytest.mark.parametrize("r", [1, 2, 3])
def test_counts_match_closed_form(n, r):
    xyz, tets = synth.kuhn_cube(n)
    topo = topology.build(tets, len(xyz), r)
    V, E, F, T = counts_closed_form(n)
    assert (len(xyz), topo.ne, topo.nf, topo.nt) == (V, E, F, T)
    assert topo.ndof == ndof_closed_form(n, r)
    assert V - E + F - T == 1
    # boundary faces: 2 triangles per boundary square, 6 n^2 squares
    assert len(topo.boundary_faces()) == 12 * n * n
    # every DOF used, each exactly once per entity
    assert np.array_equal(np.unique(topo.dofmap), np.arange(topo.ndof))


def test_config_sizes():
    """DOF counts of the five workloads (closed form of the counting rule)."""
    assert ndof_closed_form(8, 1) == 4184
    assert ndof_closed_form(16, 2) == 163424
    assert ndof_closed_form(24, 2) == 542736
    assert ndof_closed_form(32, 3) == 3702048
    xyz, tets = synth.kuhn_cube(16)
    assert topology.build(tets, len(xyz), 2).ndof == 163424


def test_numbering_brute_force_tiny():
    """Pure-Python dictionaries on n = 1, 2 reproduce edge/face ids and the DOF map."""
    for n in (1, 2):
        xyz, tets = synth.kuhn_cube(n)
        for r in (1, 2, 3):
            topo = topology.build(tets, len(xyz), r)
            st = [sorted(int(v) for v in t) for t in tets]
            edges = sorted({(t[a], t[b]) for t in st for (a, b) in basis.LOCAL_EDGES})
            faces = sorted({(t[a], t[b], t[c]) for t in st for (a, b, c) in basis.LOCAL_FACES})
            eid = {e: i for i, e in enumerate(edges)}
            fid = {f: i for i, f in enumerate(faces)}
            ned, nfd, nvd = r, r * (r - 1), r * (r - 1) * (r - 2) // 2
            for ti, t in enumerate(st):
                expect = []
                for (a, b) in basis.LOCAL_EDGES:
                    expect += [eid[(t[a], t[b])] * ned + q for q in range(ned)]
                for (a, b, c) in basis.LOCAL_FACES:
                    expect += [len(edges) * ned + fid[(t[a], t[b], t[c])] * nfd + q
                               for q in range(nfd)]
                expect += [len(edges) * ned + len(faces) * nfd + ti * nvd + q for q in range(nvd)]
                assert list(topo.dofmap[ti]) == expect


# ---------------------------------------------------------------- generators

@pytest.mark.parametrize("r", [1, 2, 3])
def test_subset_is_basis_of_generator_span(r):
    """Sec. 3: the generator family spans the first-kind space of dimension r(r+2)(r+3)/2;
    the selected subset is independent and spans the same space."""
    rng = np.random.default_rng(1)
    verts = random_tet(rng)
    x = (rng.dirichlet(np.ones(4), size=60)) @ verts
    lam = basis.barycentrics(verts, x)
    g = basis.barycentric_gradients(verts)
    sub = np.stack([basis.eval_generator(d[3], d[4], d[5], lam, g).ravel()
                    for d in basis.local_dofs(r)], axis=1)
    full = np.stack([basis.eval_generator(i, j, k, lam, g).ravel()
                     for (i, j, k) in basis.all_generators(r)], axis=1)
    dim = r * (r + 2) * (r + 3) // 2
    assert len(basis.all_generators(r)) == 6 * comb(r + 2, 3)
    assert np.linalg.matrix_rank(full) == dim
    assert np.linalg.matrix_rank(sub) == dim
    assert np.linalg.matrix_rank(np.concatenate([sub, full], axis=1)) == dim
    # every vector polynomial of degree r-1 lies in the space (P_{r-1}^3 subset of ND_r)
    mons = [m for m in itertools.product(range(r), repeat=3) if sum(m) <= r - 1]
    for c in range(3):
        for m in mons:
            f = np.zeros((len(x), 3))
            f[:, c] = np.prod(x ** np.array(m), axis=1)
            coef, *_ = np.linalg.lstsq(sub, f.ravel(), rcond=None)
            assert np.linalg.norm(sub @ coef - f.ravel()) < 1e-10 * max(1.0, np.linalg.norm(f))


def test_whitney_duality():
    """Sec. 3: (1/|e|) int_e w^{e'} . t_e = delta_{e e'} for r = 1 (Gauss-Legendre on edges)."""
    rng = np.random.default_rng(2)
    verts = random_tet(rng)
    g = basis.barycentric_gradients(verts)
    s, w = quadrature.line_rule(4)
    D = np.zeros((6, 6))
    for e, (a, b) in enumerate(basis.LOCAL_EDGES):
        x = verts[a][None, :] + s[:, None] * (verts[b] - verts[a])[None, :]
        lam = basis.barycentrics(verts, x)
        for e2, (i, j) in enumerate(basis.LOCAL_EDGES):
            val = basis.eval_generator(i, j, (0, 0, 0, 0), lam, g)
            D[e, e2] = np.sum(w * (val @ (verts[b] - verts[a])))
    assert np.allclose(D, np.eye(6), atol=1e-13)


def test_r1_element_matrices_closed_form():
    """r = 1: int l_p l_q = |T|(1 + delta_pq)/20 and curl w^{ij} = 2 grad l_i x grad l_j."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        verts = random_tet(rng)
        xyz = verts.copy()
        st = np.array([[0, 1, 2, 3]])
        M, K = elements.element_mass_stiffness(xyz, st, 1)
        g = basis.barycentric_gradients(verts)
        vol = abs(np.linalg.det(verts[1:] - verts[0])) / 6
        I2 = lambda p, q: vol * (1 + (p == q)) / 20.0
        for a, (i, j) in enumerate(basis.LOCAL_EDGES):
            for b, (k, l) in enumerate(basis.LOCAL_EDGES):
                m = (I2(i, k) * g[j] @ g[l] - I2(i, l) * g[j] @ g[k]
                     - I2(j, k) * g[i] @ g[l] + I2(j, l) * g[i] @ g[k])
                kk = 4 * vol * np.cross(g[i], g[j]) @ np.cross(g[k], g[l])
                assert abs(M[0, a, b] - m) < 1e-13 * max(1, abs(m))
                assert abs(K[0, a, b] - kk) < 1e-12 * max(1, abs(kk))


@pytest.mark.parametrize("r", [1, 2, 3])
def test_element_matrices_match_exact_monomial_rule(r):
    """The oracle integrates by quadrature of the evaluated basis; the same matrices computed
    without quadrature, by the exact monomial rule int_T lambda^alpha = 6|T| alpha!/(|alpha|+3)!
    over the term expansion of each generator (tests/elem_tables.py), agree to 1e-12."""
    import elem_tables
    rng = np.random.default_rng(10 + r)
    for _ in range(3):
        verts = random_tet(rng)
        st = np.array([[0, 1, 2, 3]])
        M, K = elements.element_mass_stiffness(verts, st, r)
        Me, Ke = elem_tables.element_mass_stiffness(verts, st, r)
        assert np.abs(M - Me).max() < 1e-12 * np.abs(Me).max()
        assert np.abs(K - Ke).max() < 1e-12 * np.abs(Ke).max()
        for lf in range(4):
            S = elements.face_matrices(verts, st, [0], [lf], r)[0]
            Se = elem_tables.face_matrices(verts, st, [0], [lf], r)[0]
            assert np.abs(S - Se).max() < 1e-12 * np.abs(Se).max()


@pytest.mark.parametrize("r", [1, 2, 3])
def test_batched_basis_matches_pointwise_basis(r):
    """The batched evaluation the oracle integrates with (shared barycentric points, per-tet
    gradients) equals the one-tetrahedron evaluation at physical points (barycentrics solved from
    the coordinates), values and curls, and its face quadrature reproduces the tangential mass of
    a face integrated in physical coordinates."""
    rng = np.random.default_rng(20 + r)
    lam_q, _ = quadrature.tet_rule(r + 1)
    for _ in range(3):
        verts = random_tet(rng)
        g = basis.barycentric_gradients(verts)
        vb, cb = basis.eval_basis_batch(r, lam_q, g[None])
        vp, cp = basis.eval_local_basis(r, verts, lam_q @ verts)
        assert np.abs(vb[0] - vp).max() < 1e-12 * max(1.0, np.abs(vp).max())
        assert np.abs(cb[0] - cp).max() < 1e-12 * max(1.0, np.abs(cp).max())
        lam_f, w_f = quadrature.tri_rule(r + 2)
        for lf, fv in enumerate(basis.LOCAL_FACES):
            S = elements.face_matrices(verts, np.array([[0, 1, 2, 3]]), [0], [lf], r)[0]
            pf = verts[list(fv)]
            nrm = np.cross(pf[1] - pf[0], pf[2] - pf[0])
            area = np.linalg.norm(nrm) / 2
            nrm /= np.linalg.norm(nrm)
            vf, _ = basis.eval_local_basis(r, verts, lam_f @ pf)
            tf = np.cross(vf, nrm[None, None, :])
            Sq = 2 * area * np.einsum("p,pai,pbi->ab", w_f, tf, tf)
            assert np.abs(S - Sq).max() < 1e-12 * np.abs(Sq).max()


# ---------------------------------------------------------------- kernel of curl

def _global_real(topo, Mloc):
    nl = Mloc.shape[1]
    rows = np.repeat(topo.dofmap, nl, axis=1).ravel()
    cols = np.tile(topo.dofmap, (1, nl)).ravel()
    return sp.coo_matrix((Mloc.ravel(), (rows, cols)), shape=(topo.ndof, topo.ndof)).tocsr()


def _fit_gradient(topo, xyz, r, grad_fn):
    """Per-tetrahedron least-squares fit of a gradient field in the local basis; returns the
    global coefficient vector and the worst fit residual and cross-element disagreement."""
    rng = np.random.default_rng(7)
    c = np.full(topo.ndof, np.nan)
    worst_fit = worst_agree = 0.0
    for t in range(topo.nt):
        verts = xyz[topo.st[t]]
        lam = rng.dirichlet(np.ones(4), size=40)
        x = lam @ verts
        val, _ = basis.eval_local_basis(r, verts, x)
        gphi = grad_fn(t, lam, basis.barycentric_gradients(verts), x)
        A = val.transpose(0, 2, 1).reshape(-1, val.shape[1])
        coef, *_ = np.linalg.lstsq(A, gphi.ravel(), rcond=None)
        worst_fit = max(worst_fit, np.linalg.norm(A @ coef - gphi.ravel()) /
                        max(1e-300, np.linalg.norm(gphi)))
        dm = topo.dofmap[t]
        seen = ~np.isnan(c[dm])
        if seen.any():
            worst_agree = max(worst_agree, np.abs(c[dm][seen] - coef[seen]).max())
        c[dm] = coef
    return c, worst_fit, worst_agree


@pytest.mark.parametrize("r", [1, 2, 3])
def test_gradients_in_kernel_of_curl_curl(r):
    """Gradients of continuous piecewise-P_r functions (products of global hat functions and a
    global polynomial) lie in V_h with consistent shared coefficients, and K c = 0."""
    xyz, tets = synth.kuhn_cube(2)
    topo = topology.build(tets, len(xyz), r)
    M, K = elements.element_mass_stiffness(xyz, topo.st, r)
    Kg = _global_real(topo, K)
    rng = np.random.default_rng(5)
    # random multiset of r global vertices forming a simplex of the mesh
    picks = []
    for _ in range(4):
        t = topo.st[rng.integers(topo.nt)]
        picks.append(tuple(rng.choice(t, size=r, replace=True)))

    def hat_product_grad(t, lam, g, x):
        verts = list(topo.st[t])
        out = np.zeros((lam.shape[0], 3))
        for pk in picks:
            if not all(v in verts for v in pk):
                continue
            loc = [verts.index(v) for v in pk]
            for i in range(len(loc)):
                others = np.prod([lam[:, loc[j]] for j in range(len(loc)) if j != i], axis=0) \
                    if len(loc) > 1 else np.ones(lam.shape[0])
                out += others[:, None] * g[loc[i]][None, :]
        return out

    coefs = rng.normal(size=3)

    def poly_grad(t, lam, g, x):
        # phi = sum_c coefs_c * x_c^r  -> grad = r x_c^{r-1} e_c
        return r * coefs[None, :] * x ** (r - 1)

    for fn in (hat_product_grad, poly_grad):
        c, fit, agree = _fit_gradient(topo, xyz, r, fn)
        assert fit < 1e-11
        assert agree < 1e-10
        assert np.linalg.norm(Kg @ c) <= 1e-12 * spla.norm(Kg) * np.linalg.norm(c)


@pytest.mark.parametrize("n,r", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2)])
def test_rank_of_curl_curl_and_mass(n, r):
    """rank(K) = N - (dim P_r Lagrange - 1) (kernel = gradients) and M is SPD (basis independent)."""
    xyz, tets = synth.kuhn_cube(n)
    topo = topology.build(tets, len(xyz), r)
    M, K = elements.element_mass_stiffness(xyz, topo.st, r)
    Kd = _global_real(topo, K).toarray()
    Md = _global_real(topo, M).toarray()
    V, E, F, T = counts_closed_form(n)
    dim_lagrange = V + (r - 1) * E + (r - 1) * (r - 2) // 2 * F
    ev = np.linalg.eigvalsh(Kd)
    rank = int((ev > 1e-9 * ev.max()).sum())
    assert rank == topo.ndof - (dim_lagrange - 1)
    assert ev.min() > -1e-10 * ev.max()          # K symmetric positive semi-definite
    assert np.linalg.eigvalsh(Md).min() > 0
    assert np.allclose(Kd, Kd.T, atol=1e-13 * np.abs(Kd).max())


# ---------------------------------------------------------------- solver pins

def _small_problem(n, r, nsub, delta, source="dipole", head=True, k0=synth.K0):
    w = synth.small(n=n, r=r, nsub=nsub, overlap=delta, head=head, source=source, k0=k0)
    return w, problem.from_workload(w)


@pytest.mark.parametrize("n", [2, 4])
def test_fgmres_matches_direct_solve(n):
    """O-T4: ORAS-FGMRES to 1e-12 agrees with a sparse direct solve to 1e-10."""
    _, p = _small_problem(n, 2, 8 if n == 4 else 2, 1)
    xd = spla.spsolve(p.A.tocsc(), p.B[:, 0])
    res = problem.solve(p, tol=1e-12, m=50)[0]
    assert res.converged
    assert np.linalg.norm(res.x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_one_subdomain_is_direct_solve():
    """O-T5: N_sub = 1 => A_1 = A and D_1 = I, so FGMRES converges in one iteration."""
    _, p = _small_problem(3, 2, 1, 0, source="plane", head=False)
    assert np.allclose(dd.local_matrix(p.topo, p.xyz, p.eps_r, p.mu_r, p.k0, p.dec, 0),
                       p.A.toarray(), atol=1e-12 * abs(p.A).max())
    res = problem.solve(p, tol=1e-10, m=10)[0]
    assert res.iterations == 1
    xd = spla.spsolve(p.A.tocsc(), p.B[:, 0])
    assert np.linalg.norm(res.x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_fgmres_dense_identity_preconditioner():
    """Unrestarted GMRES on an n x n system reaches the exact solution within n steps
    (textbook property); compare with numpy.linalg.solve."""
    rng = np.random.default_rng(4)
    n = 40
    A = np.eye(n) * 6 + rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    res = fgmres.fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-13, m=n)
    assert res.iterations <= n
    assert res.converged
    assert np.linalg.norm(res.x - np.linalg.solve(A, b)) < 1e-11 * np.linalg.norm(res.x)


def test_givens_rotation_properties():
    rng = np.random.default_rng(9)
    for _ in range(20):
        a = complex(*rng.normal(size=2))
        b = complex(*rng.normal(size=2))
        c, s = fgmres.givens(a, b)
        assert abs(c * c + abs(s) ** 2 - 1) < 1e-14
        assert abs(-np.conj(s) * a + c * b) < 1e-14
        assert abs(abs(c * a + s * b) - np.hypot(abs(a), abs(b))) < 1e-13


def _hcurl_error(topo, xyz, r, x, Efn, curlfn):
    lam, w = quadrature.tet_rule(r + 3)
    e2 = 0.0
    for t in range(topo.nt):
        verts = xyz[topo.st[t]]
        vol = abs(np.linalg.det(verts[1:] - verts[0])) / 6
        pts = lam @ verts
        val, cur = basis.eval_local_basis(r, verts, pts)
        c = x[topo.dofmap[t]]
        Eh = np.einsum("a,pai->pi", c, val)
        Ch = np.einsum("a,pai->pi", c, cur)
        d0 = Efn(pts) - Eh
        d1 = curlfn(pts) - Ch
        e2 += 6 * vol * np.sum(w * (np.abs(d0) ** 2 + np.abs(d1) ** 2).sum(axis=1))
    return np.sqrt(e2)


@pytest.mark.parametrize("r,ns", [(1, (4, 8)), (2, (2, 4)), (3, (2, 4))])
def test_plane_wave_convergence_order(r, ns):
    """O-T6: exact plane wave with impedance data; the H(curl) error falls like h^r."""
    k0 = synth.k0_for_wavelengths(0.5)
    eps = synth.EPS_GEL
    gamma = k0 * np.sqrt(eps)
    d, pvec = synth.PLANE_D, synth.PLANE_P

    def Efn(x):
        return np.exp(-1j * gamma * (x @ d))[:, None] * pvec[None, :]

    def curlfn(x):
        return (-1j * gamma) * np.exp(-1j * gamma * (x @ d))[:, None] * np.cross(d, pvec)[None, :]

    errs = []
    for n in ns:
        xyz, tets = synth.kuhn_cube(n)
        eps_r, mu_r = synth.homogeneous_materials(len(tets))
        p = problem.build(xyz, tets, eps_r, mu_r, k0, r, [("plane", d, pvec)], with_oras=False)
        x = spla.spsolve(p.A.tocsc(), p.B[:, 0])
        errs.append(_hcurl_error(p.topo, xyz, r, x, Efn, curlfn))
    slope = np.log(errs[0] / errs[1]) / np.log(ns[1] / ns[0])
    assert slope >= r - 0.2, (errs, slope)


def test_degree_two_needs_fewer_unknowns_than_degree_one():
    """Sec. 5.2 / Table 1: the degree-2 elements reach a given accuracy with far fewer unknowns
    than degree 1.  Plane wave at the benchmark's frequency (two wavelengths across the cube):
    degree 2 on 4^3 cubes (2,936 DOFs) has a smaller H(curl) error than degree 1 on 8^3 cubes
    (4,184 DOFs)."""
    k0 = synth.k0_for_wavelengths(2.0)
    gamma = k0 * np.sqrt(synth.EPS_GEL)
    d, pvec = synth.PLANE_D, synth.PLANE_P

    def Efn(x):
        return np.exp(-1j * gamma * (x @ d))[:, None] * pvec[None, :]

    def curlfn(x):
        return (-1j * gamma) * np.exp(-1j * gamma * (x @ d))[:, None] * np.cross(d, pvec)[None, :]

    out = {}
    for r, n in ((1, 8), (2, 4)):
        xyz, tets = synth.kuhn_cube(n)
        eps_r, mu_r = synth.homogeneous_materials(len(tets))
        p = problem.build(xyz, tets, eps_r, mu_r, k0, r, [("plane", d, pvec)], with_oras=False)
        x = spla.spsolve(p.A.tocsc(), p.B[:, 0])
        out[r] = (p.topo.ndof, _hcurl_error(p.topo, xyz, r, x, Efn, curlfn))
    assert out[2][0] < out[1][0] and out[2][1] < 0.9 * out[1][1], out


# ---------------------------------------------------------------- algebra / decomposition

def test_algebraic_identities_config1():
    """O-T7: A = A^T (bilinear form, no conjugation), sum_s R_s^T D_s R_s = I exactly,
    every DOF in at least one N_s, and local matrices complex symmetric."""
    w = synth.config(0)
    p = problem.from_workload(w)
    A = p.A
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    S = np.zeros(p.topo.ndof)
    cover = np.zeros(p.topo.ndof, dtype=int)
    for s, Ns in enumerate(p.dec.dofs):
        np.add.at(S, Ns, p.dec.pou[s])
        np.add.at(cover, Ns, 1)
    assert np.array_equal(S, np.ones(p.topo.ndof))
    assert cover.min() >= 1
    As = dd.local_matrix(p.topo, p.xyz, p.eps_r, p.mu_r, p.k0, p.dec, 3)
    assert np.abs(As - As.T).max() <= 1e-14 * np.abs(As).max()


def test_rcb_gives_octants():
    """RCB of the 4^3-cube mesh into 8 parts gives the 8 octant blocks of 2^3 cubes (x split
    first on the tie: all centroid sums are exact for n = 4)."""
    xyz, tets = synth.kuhn_cube(4)
    topo = topology.build(tets, len(xyz), 1)
    part = dd.rcb(xyz, topo.st, 8)
    cube = np.arange(len(tets)) // 6
    ci, cj, ck = cube % 4, (cube // 4) % 4, cube // 16
    octant = (ci >= 2).astype(int) + 2 * (cj >= 2) + 4 * (ck >= 2)
    # x splits first, then y, then z (depth-first ids): id = 4*(x hi) + 2*(y hi) + (z hi)
    expect = 4 * (ci >= 2) + 2 * (cj >= 2) + (ck >= 2)
    assert np.array_equal(part, expect)
    assert np.all(np.bincount(part) == 48)
    assert len(np.unique(octant)) == 8


def test_overlap_one_layer_closed_form():
    """One vertex layer around the corner octants of the 4^3-cube mesh covers exactly the
    27 cubes [0,3)^3 (origin octant) or [1,4)^3 (far octant): 162 tetrahedra."""
    xyz, tets = synth.kuhn_cube(4)
    topo = topology.build(tets, len(xyz), 2)
    part = dd.rcb(xyz, topo.st, 8)
    ov = dd.overlap_tets(topo.st, len(xyz), part, 8, 1)
    cube = np.arange(len(tets)) // 6
    ci, cj, ck = cube % 4, (cube // 4) % 4, cube // 16
    near = np.nonzero((ci < 3) & (cj < 3) & (ck < 3))[0]
    far = np.nonzero((ci >= 1) & (cj >= 1) & (ck >= 1))[0]
    assert np.array_equal(ov[0], near)
    assert np.array_equal(ov[7], far)


def test_ownership_brute_force_tiny():
    """Owner of each DOF = part of the lowest tet containing its entity (pure-Python loop)."""
    xyz, tets = synth.kuhn_cube(2)
    topo = topology.build(tets, len(xyz), 3)
    dec = dd.decompose(topo, xyz, 4, 1)
    expect = {}
    for t in range(topo.nt):
        for g in topo.dofmap[t]:
            if int(g) not in expect:
                expect[int(g)] = int(dec.part[t])
    assert all(dec.owner[g] == o for g, o in expect.items())


def test_dipole_load_is_point_evaluation():
    """b_a = w_a(x0).z: reproduce with the product-formula basis evaluation at x0."""
    xyz, tets = synth.kuhn_cube(3)
    topo = topology.build(tets, len(xyz), 2)
    x0 = np.array([0.31, 0.52, 0.77])
    b = assemble.dipole_load(topo, xyz, x0, [0, 0, 1.0])
    t, _ = assemble.locate_point(topo, xyz, x0)
    val, _ = basis.eval_local_basis(2, xyz[topo.st[t]], x0[None, :])
    assert np.allclose(b[topo.dofmap[t]], val[0, :, 2], atol=1e-13)
    assert np.count_nonzero(b) <= basis.n_local(2)


def test_quadrature_rules_exactness():
    """Conical-product rules integrate monomials exactly (closed forms of the simplex:
    int lambda^alpha = alpha! / (|alpha| + d)! on the reference simplex of dimension d)."""
    from math import factorial
    lam, w = quadrature.tet_rule(4)
    for alpha in [(0, 0, 0, 0), (1, 2, 0, 3), (2, 2, 2, 1), (0, 0, 7, 0)]:
        exact = np.prod([factorial(a) for a in alpha]) / factorial(sum(alpha) + 3)
        assert abs(np.sum(w * np.prod(lam ** np.array(alpha), axis=1)) - exact) < 1e-15
    lam, w = quadrature.tri_rule(4)
    for alpha in [(0, 0, 0), (3, 2, 2), (0, 7, 0)]:
        exact = np.prod([factorial(a) for a in alpha]) / factorial(sum(alpha) + 2)
        assert abs(np.sum(w * np.prod(lam ** np.array(alpha), axis=1)) - exact) < 1e-15


def test_ras_and_oras_local_rows_agree_inside_the_subdomain():
    """RAS (Dirichlet transmission, A_s = R_s A R_s^T) and ORAS (impedance transmission, element
    sums over Omega_s^delta plus i w~ S on its boundary faces, Sec. 4) differ only through the
    subdomain boundary: the row of a DOF whose every incident tetrahedron lies in Omega_s^delta is
    the same in both, and boundary rows differ."""
    from oracle import dd
    w = synth.small(n=4, r=2, nsub=8, overlap=1)
    P = problem.from_workload(w, with_oras=False)
    dec = dd.decompose(P.topo, P.xyz, w.nsub, w.overlap)
    A = P.A.tocsr()
    nt, nl = P.topo.dofmap.shape
    g_all = P.topo.dofmap.ravel()
    t_all = np.repeat(np.arange(nt), nl)
    for s in (0, 3, 7):
        member = np.zeros(nt, dtype=bool)
        member[dec.tets[s]] = True
        outside = np.zeros(P.topo.ndof, dtype=bool)
        outside[g_all[~member[t_all]]] = True          # DOF touched by a tet outside Omega_s^delta
        Ns = dec.dofs[s]
        inside = ~outside[Ns]
        Ar = dd.restricted_matrix(A, dec, s)
        Ao = dd.local_matrix(P.topo, P.xyz, P.eps_r, P.mu_r, P.k0, dec, s)
        scale = np.abs(Ar).max()
        assert inside.any() and (~inside).any()
        assert np.abs(Ar[inside] - Ao[inside]).max() <= 1e-13 * scale
        assert np.abs(Ar[~inside] - Ao[~inside]).max(axis=1).min() > 1e-6 * scale


@pytest.mark.parametrize("n,r,nsub", [(4, 2, 8), (5, 1, 16)])
def test_oras_converges_faster_than_ras(n, r, nsub):
    """The paper's comparison (Sec. 4-5): impedance transmission (ORAS) needs fewer FGMRES
    iterations than Dirichlet transmission (RAS) with the same subdomains."""
    from oracle import dd, fgmres
    w = synth.small(n=n, r=r, nsub=nsub, overlap=1)
    P = problem.from_workload(w)
    ras = dd.ORAS(P.topo, P.xyz, P.eps_r, P.mu_r, P.k0, P.dec, transmission="dirichlet", A_global=P.A.tocsr())
    b = P.B[:, 0]
    it_o = fgmres.fgmres(lambda v: P.A @ v, P.oras.apply, b, 1e-8, 50, 5000).iterations
    it_r = fgmres.fgmres(lambda v: P.A @ v, ras.apply, b, 1e-8, 50, 5000).iterations
    assert it_o < it_r


def test_oas_is_symmetric_and_oras_is_not():
    """Sec. 4: without the partition of unity, M_OAS = sum_s R_s^T A_s^-1 R_s is symmetric for a
    symmetric problem (here complex symmetric: A = A^T and every A_s = A_s^T); the D_s of ORAS
    break that symmetry.  Dense M from the oracle's apply on the unit vectors."""
    w = synth.small(n=3, r=1, nsub=4, overlap=1)
    P = problem.from_workload(w)
    n = P.topo.ndof
    E = np.eye(n)
    for weights, symmetric in (("none", True), ("pou", False)):
        M = dd.ORAS(P.topo, P.xyz, P.eps_r, P.mu_r, P.k0, P.dec, weights=weights)
        D = np.stack([M.apply(E[:, j]) for j in range(n)], axis=1)
        asym = np.abs(D - D.T).max() / np.abs(D).max()
        assert (asym <= 1e-12) if symmetric else (asym >= 1e-3), (weights, asym)


@pytest.mark.parametrize("n,r,nsub", [(4, 2, 8), (5, 1, 16)])
def test_oras_converges_faster_than_oas(n, r, nsub):
    """Sec. 4: in practice OAS (no partition of unity) converges more slowly than ORAS."""
    w = synth.small(n=n, r=r, nsub=nsub, overlap=1)
    P = problem.from_workload(w)
    oas = dd.ORAS(P.topo, P.xyz, P.eps_r, P.mu_r, P.k0, P.dec, weights="none")
    b = P.B[:, 0]
    it_oras = fgmres.fgmres(lambda v: P.A @ v, P.oras.apply, b, 1e-8, 50, 5000).iterations
    it_oas = fgmres.fgmres(lambda v: P.A @ v, oas.apply, b, 1e-8, 50, 5000).iterations
    assert it_oras < it_oas


# ---------------------------------------------------------------- impedance terms, closed form

def _constant_field_coefficients(topo, xyz, r, c):
    """Coefficient vector of the constant field c (= grad(c . x), in V_h for every r), fitted
    tetrahedron by tetrahedron from point values; the fit must be exact and consistent."""
    u, fit, agree = _fit_gradient(topo, xyz, r, lambda t, lam, g, x: np.broadcast_to(c, x.shape).copy())
    assert fit < 1e-11 and agree < 1e-10
    return u


def _jittered_kuhn(n, seed):
    """Kuhn cube with interior vertices moved (boundary vertices stay on the cube faces, so the
    outer normals stay the axis directions) -- general interior face normals."""
    xyz, tets = synth.kuhn_cube(n)
    rng = np.random.default_rng(seed)
    inner = np.all((xyz > 1e-12) & (xyz < 1 - 1e-12), axis=1)
    xyz = xyz.copy()
    xyz[inner] += rng.uniform(-0.2, 0.2, size=(inner.sum(), 3)) / n
    return xyz, tets


def _face_geometry(xyz, st, t, lf):
    """Area and unit normal of local face lf of tetrahedron t, from the vertex coordinates."""
    pf = xyz[st[t, list(basis.LOCAL_FACES[lf])]]
    nrm = np.cross(pf[1] - pf[0], pf[2] - pf[0])
    area = np.linalg.norm(nrm) / 2
    return area, nrm / np.linalg.norm(nrm)


@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("caller_beta", [False, True])
def test_global_matrix_on_a_constant_field(r, caller_beta):
    """For a constant field E = c (curl E = 0) the weak form of Sec. 2 gives, independently of the
    basis,  u^T A u = -k0^2 sum_T eps_T |T| |c|^2 + i sum_{outer f} beta_f |f| |c x n_f|^2,
    with beta_f the caller's per-face table (looked up through the caller's vertex order) or
    k0 sqrt(Re eps) of the adjacent tetrahedron.  A wrong beta, face, area or normal fails it."""
    xyz, tets = _jittered_kuhn(2, seed=r)
    rng = np.random.default_rng(100 + r)
    tets = np.array([rng.permutation(t) for t in tets])     # caller's vertex order is arbitrary
    topo = topology.build(tets, len(xyz), r)
    eps = rng.uniform(30, 60, len(tets)) - 1j * rng.uniform(5, 25, len(tets))
    mu = np.ones(len(tets), dtype=np.complex128)
    k0 = synth.K0
    beta_face = rng.uniform(4.0, 20.0, size=(len(tets), 4)) if caller_beta else None
    beta_lf = None if beta_face is None else assemble.face_beta_table(tets, beta_face)
    A = assemble.global_matrix(topo, xyz, eps, mu, k0, beta_lf)
    for c in (np.array([1.0, 0.0, 0.0]), np.array([0.3, -1.2, 0.7])):
        u = _constant_field_coefficients(topo, xyz, r, c)
        _, vol, _ = elements.geometry(xyz, topo.st)
        expect = -k0 ** 2 * np.sum(eps * vol) * (c @ c)
        for f in topo.boundary_faces():
            t = topo.face_tets[f, 0]
            lf = int(np.nonzero(topo.tet_faces[t] == f)[0][0])
            area, nrm = _face_geometry(xyz, topo.st, t, lf)
            if caller_beta:   # face lf of the sorted tet is opposite the caller's vertex with that id
                opp = topo.st[t, basis.FACE_OPPOSITE[lf]]
                beta = beta_face[t, list(tets[t]).index(opp)]
            else:
                beta = k0 * np.sqrt(eps[t].real)
            expect += 1j * beta * area * np.sum(np.cross(c, nrm) ** 2)
        got = u @ (A @ u)
        assert abs(got - expect) <= 1e-11 * abs(expect), (got, expect)


@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("delta", [0, 1])
def test_local_matrix_interface_term_on_a_constant_field(r, delta):
    """Impedance transmission of Sec. 4 in closed form: for the constant field c restricted to
    N_s,  u_s^T A_s u_s = -k0^2 sum_{T in Omega_s} eps_T |T| |c|^2
    + i sum_{f outer face of Omega_s} beta_f |f| |c x n_f|^2
    + i sum_{f interface face of Omega_s} w~_f |f| |c x n_f|^2,
    w~_f = k0 sqrt(Re eps) of the tetrahedron of f inside Omega_s^delta (the materials differ
    from tetrahedron to tetrahedron, so the outside one would fail), every face found from the
    geometry alone."""
    xyz, tets = _jittered_kuhn(3, seed=7 + r)
    topo = topology.build(tets, len(xyz), r)
    rng = np.random.default_rng(200 + r)
    eps = rng.uniform(30, 60, len(tets)) - 1j * rng.uniform(5, 25, len(tets))
    mu = np.ones(len(tets), dtype=np.complex128)
    k0 = synth.K0
    dec = dd.decompose(topo, xyz, 4, delta)
    c = np.array([0.4, 1.0, -0.6])
    u = _constant_field_coefficients(topo, xyz, r, c)
    _, vol, _ = elements.geometry(xyz, topo.st)
    for s in range(4):
        As = dd.local_matrix(topo, xyz, eps, mu, k0, dec, s)
        us = u[dec.dofs[s]]
        inside = np.zeros(topo.nt, dtype=bool)
        inside[dec.tets[s]] = True
        expect = -k0 ** 2 * np.sum(eps[inside] * vol[inside]) * (c @ c)
        n_iface = 0
        for t in dec.tets[s]:
            for lf in range(4):
                a, b = topo.face_tets[topo.tet_faces[t, lf]]
                other = b if a == t else a
                if other >= 0 and inside[other]:
                    continue
                area, nrm = _face_geometry(xyz, topo.st, t, lf)
                coef = k0 * np.sqrt(eps[t].real)       # outer face: beta; interface: w~ of t
                expect += 1j * coef * area * np.sum(np.cross(c, nrm) ** 2)
                n_iface += other >= 0
        assert n_iface > 0
        got = us @ (As @ us)
        assert abs(got - expect) <= 1e-11 * abs(expect), (s, got, expect)


def test_face_beta_table_brute_force():
    """beta of the sorted local face lf = the caller's entry of the face opposite the same vertex."""
    rng = np.random.default_rng(5)
    tets = np.array([rng.permutation(10)[:4] for _ in range(20)])
    beta = rng.uniform(1, 2, size=(20, 4))
    tab = assemble.face_beta_table(tets, beta)
    for t in range(20):
        st = sorted(tets[t])
        for lf, fv in enumerate(basis.LOCAL_FACES):
            opp = (set(range(4)) - set(fv)).pop()
            assert tab[t, lf] == beta[t, list(tets[t]).index(st[opp])]

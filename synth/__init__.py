"""Seeded synthetic inputs for the ORAS-FGMRES Maxwell solver.

This module produces the *inputs* of the method only: tetrahedral meshes,
per-tetrahedron material values, wave numbers and source parameters.  It holds
none of the method's arithmetic (no basis functions, integrals, assembly,
decomposition or Krylov steps), so the CPU oracle and the CUDA library can both
consume its arrays without sharing any computation.

The workloads stand in for the imaging-chamber problems of Sec. 5 (meshes and
measured data of the chamber are not available): a unit cube split into
n^3 cubes, each cut into 6 tetrahedra (Kuhn/Freudenthal split), filled with the
lossy matching medium of Sec. 5.1 (eps_r = 44 - 20i) and, for the head-like
configurations, a ball and a small perturbation of different permittivity.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

# Permittivity of the matching gel used in Sec. 5.1 / 5.2.
EPS_GEL = complex(44.0, -20.0)
# Head-like layers of the synthetic configurations.
EPS_BALL = complex(40.0, -15.0)
EPS_PERT = complex(60.0, -25.0)
BALL_CENTRE = (0.5, 0.5, 0.5)
BALL_RADIUS = 0.35
PERT_CENTRE = (0.6, 0.5, 0.5)
PERT_RADIUS = 0.08
RING_RADIUS = 0.45


def k0_for_wavelengths(waves: float, eps: complex = EPS_GEL) -> float:
    """Free-space wave number giving `waves` in-medium wavelengths across the unit cube.

    Re(k0 * sqrt(eps)) * 1 = 2*pi*waves, principal square root.
    """
    s = np.sqrt(complex(eps))
    return 2.0 * math.pi * waves / s.real


K0 = k0_for_wavelengths(2.0)  # 1.84948..., used by every configuration


def kuhn_cube(n: int):
    """Unit cube, n^3 cubes, 6 tetrahedra per cube (Kuhn split).

    Vertex id = i + (n+1)*(j + (n+1)*k), coordinates (i, j, k)/n.
    For each cube with corner c (cube order: i fastest, then j, then k) and each
    permutation pi of (x, y, z) in lexicographic order, the tetrahedron is
    {c, c + e_pi0, c + e_pi0 + e_pi1, c + (1,1,1)}.
    Returns xyz float64[(n+1)^3, 3] and tets int32[6 n^3, 4].
    """
    m = n + 1
    g = np.arange(m, dtype=np.float64) / n
    kk, jj, ii = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)

    def vid(i, j, k):
        return i + m * (j + m * k)

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # cube order with i fastest: iterate k, j, i
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    unit = np.eye(3, dtype=np.int64)
    tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for p, perm in enumerate(itertools.permutations(range(3))):
        c = np.stack([ci, cj, ck], axis=1)
        v1 = c + unit[perm[0]]
        v2 = v1 + unit[perm[1]]
        v3 = c + 1
        for q, v in enumerate((c, v1, v2, v3)):
            tets[:, p, q] = vid(v[:, 0], v[:, 1], v[:, 2])
    return xyz, tets.reshape(-1, 4).astype(np.int32)


def tet_centroids(xyz, tets):
    """Centroid used for material assignment (input generation only)."""
    return xyz[tets].mean(axis=1)


def homogeneous_materials(nt: int, eps: complex = EPS_GEL):
    eps_r = np.full(nt, eps, dtype=np.complex128)
    mu_r = np.ones(nt, dtype=np.complex128)
    return eps_r, mu_r


def head_materials(xyz, tets, pert_radius=PERT_RADIUS, eps_pert=EPS_PERT):
    """Layered head-like medium decided by the tetrahedron centroid (strict '<' radius tests).

    Perturbation overrides the ball, which overrides the background gel.
    """
    c = tet_centroids(xyz, tets)
    d_ball = np.sqrt(((c - np.array(BALL_CENTRE)) ** 2).sum(axis=1))
    d_pert = np.sqrt(((c - np.array(PERT_CENTRE)) ** 2).sum(axis=1))
    eps_r = np.full(len(tets), EPS_GEL, dtype=np.complex128)
    eps_r[d_ball < BALL_RADIUS] = EPS_BALL
    eps_r[d_pert < pert_radius] = eps_pert
    mu_r = np.ones(len(tets), dtype=np.complex128)
    return eps_r, mu_r


def dipole_ring(k: int):
    """k source points on a ring of radius 0.45 around the cube centre, in the plane z = 0.5."""
    th = 2.0 * math.pi * np.arange(k) / k
    return np.stack([0.5 + RING_RADIUS * np.cos(th), 0.5 + RING_RADIUS * np.sin(th),
                     np.full(k, 0.5)], axis=1)


# Plane-wave direction and polarisation of the impedance-data configuration.
PLANE_D = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
PLANE_P = np.array([3.0, 0.0, -1.0]) / math.sqrt(10.0)


@dataclass
class Workload:
    """One synthetic problem: mesh, materials, frequency, discretisation and solver knobs."""
    name: str
    n: int
    r: int
    nsub: int
    overlap: int
    restart: int
    tol: float
    factor_bits: int          # 64 = FP64 local factors, 32 = FP32 local factors
    head: bool
    source: str               # "plane" or "dipole"
    nrhs: int = 1
    k0: float = K0
    pert_radius: float = PERT_RADIUS
    eps_pert: complex = EPS_PERT
    arrival_s: float = 0.0
    extra: dict = field(default_factory=dict)

    def mesh(self):
        return kuhn_cube(self.n)

    def materials(self, xyz, tets):
        if self.head:
            return head_materials(xyz, tets, self.pert_radius, self.eps_pert)
        return homogeneous_materials(len(tets))

    def sources(self):
        if self.source == "plane":
            return [("plane", PLANE_D.copy(), PLANE_P.copy())]
        pts = dipole_ring(self.nrhs)
        return [("dipole", pts[j], np.array([0.0, 0.0, 1.0])) for j in range(self.nrhs)]


def config(idx: int) -> Workload:
    """The five synthetic workloads (index 0..4)."""
    if idx == 0:
        return Workload("cube8_r1_plane_fp64", n=8, r=1, nsub=8, overlap=1, restart=50,
                        tol=1e-8, factor_bits=64, head=False, source="plane")
    if idx == 1:
        return Workload("head16_r2_dipole_fp32", n=16, r=2, nsub=64, overlap=2, restart=100,
                        tol=1e-8, factor_bits=32, head=True, source="dipole", nrhs=1)
    if idx == 2:
        return Workload("head24_r2_32dipoles_fp32", n=24, r=2, nsub=256, overlap=1, restart=100,
                        tol=1e-8, factor_bits=32, head=True, source="dipole", nrhs=32)
    if idx == 4:
        return Workload("head32_r3_dipole_fp32", n=32, r=3, nsub=4096, overlap=0, restart=100,
                        tol=1e-8, factor_bits=32, head=True, source="dipole", nrhs=1)
    raise ValueError("config 3 is the serving stream: use serving_requests()")


def small(n=4, r=2, nsub=8, overlap=1, head=True, source="dipole", nrhs=1,
          factor_bits=32, restart=50, tol=1e-8, k0=K0) -> Workload:
    """Small case the oracle finishes in seconds (parity tests)."""
    return Workload(f"small_n{n}_r{r}_s{nsub}_d{overlap}", n=n, r=r, nsub=nsub, overlap=overlap,
                    restart=restart, tol=tol, factor_bits=factor_bits, head=head,
                    source=source, nrhs=nrhs, k0=k0)


def serving_requests(count=200, seed=160504521):
    """Serving stream: Poisson arrivals (mean 5/s) of seed-drawn solve requests."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for q in range(count):
        t += rng.exponential(0.2)
        n = int(rng.integers(8, 25))
        r = int(rng.choice([1, 2, 3]))
        k = int(rng.choice([1, 8, 32]))
        rad = float(rng.uniform(0.03, 0.12))
        eps = complex(rng.uniform(50.0, 70.0), -rng.uniform(15.0, 30.0))
        nt = 6 * n ** 3
        e = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
        f = 1 - (n + 1) ** 3 + e + nt
        ndof = r * e + r * (r - 1) * f + r * (r - 1) * (r - 2) // 2 * nt
        nsub = 1 << max(0, math.ceil(math.log2(ndof / 2500.0)))
        out.append(Workload(f"req{q}", n=n, r=r, nsub=nsub, overlap=1, restart=50, tol=1e-8,
                            factor_bits=32, head=True, source="dipole", nrhs=k,
                            pert_radius=rad, eps_pert=eps, arrival_s=t))
    return out

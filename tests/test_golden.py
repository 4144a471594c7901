"""Pins taken from the constants the paper prints (tests/golden/sec5_materials.txt).

The paper's chamber meshes and measured coefficients are not available, so what can be
pinned to its printed numbers is (i) the material data the synthetic workloads use and
(ii) the boundary model of Sec. 2: with the e^{i omega t} convention and a non-dissipative
medium (sigma = 0, so gamma equals the wave number omega~ and the impedance coefficient
beta = gamma), an outgoing plane wave at normal incidence satisfies the impedance condition
exactly.  Its impedance data g must then vanish on the face it leaves through, and be
2 i gamma E_T on the face it enters through.  A flipped sign of the i beta term, or beta taken
from the wrong medium, breaks the first property.
"""
from __future__ import annotations

import math
import pathlib

import numpy as np
import pytest

import synth
from oracle import assemble, basis, topology

GOLDEN = pathlib.Path(__file__).parent / "golden" / "sec5_materials.txt"


def load_golden():
    vals = {}
    for line in GOLDEN.read_text().splitlines():
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, val = (s.strip() for s in line.split("=", 1))
        parts = val.split()
        vals[key] = complex(float(parts[0]), float(parts[1])) if len(parts) == 2 else float(parts[0])
    return vals


def test_golden_file_is_consistent():
    g = load_golden()
    assert g["rings"] * g["antennas_per_ring"] == g["antennas"] == 160
    assert g["frequency_hz"] == 1e9
    for key in ("eps_r_gel", "eps_r_ceramic", "eps_r_cylinder"):
        assert isinstance(g[key], complex)
    assert g["eps_r_cylinder"].imag == 0.0 and g["eps_r_ceramic"].imag == 0.0


def test_synthetic_background_is_the_matching_solution():
    g = load_golden()
    assert synth.EPS_GEL == g["eps_r_gel"]
    # the frequency reading: two in-medium wavelengths across the unit cube
    wavelength = 2.0 * math.pi / (synth.K0 * np.sqrt(g["eps_r_gel"])).real
    assert abs(wavelength - 0.5) < 1e-12
    # lossy medium (Im eps < 0 with e^{i omega t}): the plane wave decays along d
    gamma = synth.K0 * np.sqrt(g["eps_r_gel"])
    assert gamma.imag < 0.0


def _dofs_on_plane(topo, xyz, axis, value, r):
    """DOFs whose basis functions have a tangential trace on the plane x_axis = value only
    (edges inside that square face of the cube, and faces lying in it)."""
    other = [a for a in range(3) if a != axis]
    ev = xyz[topo.edges]                                      # [E,2,3]
    on = np.all(np.abs(ev[:, :, axis] - value) < 1e-12, axis=1)
    mid = ev.mean(axis=1)
    inner = np.all((mid[:, other] > 1e-12) & (mid[:, other] < 1 - 1e-12), axis=1)
    ned, nfd = basis.n_edge_dofs(r), basis.n_face_dofs(r)
    out = [e * ned + q for e in np.nonzero(on & inner)[0] for q in range(ned)]
    fv = xyz[topo.faces]                                      # [F,3,3]
    fon = np.all(np.abs(fv[:, :, axis] - value) < 1e-12, axis=1)
    out += [topo.ne * ned + f * nfd + q for f in np.nonzero(fon)[0] for q in range(nfd)]
    return np.array(sorted(out), dtype=np.int64)


def _plane_wave_b(r, eps, k0=1.3):
    xyz, tets = synth.kuhn_cube(3)
    topo = topology.build(tets, len(xyz), r)
    eps_r = np.full(topo.nt, eps, dtype=np.complex128)
    mu_r = np.ones(topo.nt, dtype=np.complex128)
    d = np.array([1.0, 0.0, 0.0])
    p = np.array([0.0, 0.6, 0.8])
    b = assemble.plane_wave_load(topo, xyz, eps_r, mu_r, k0, d, p)
    return topo, xyz, b


@pytest.mark.parametrize("r", [1, 2, 3])
def test_outgoing_plane_wave_satisfies_the_impedance_condition(r):
    g = load_golden()
    topo, xyz, b = _plane_wave_b(r, g["eps_r_cylinder"])
    out = _dofs_on_plane(topo, xyz, 0, 1.0, r)
    inn = _dofs_on_plane(topo, xyz, 0, 0.0, r)
    assert len(out) and len(inn) == len(out)
    scale = np.abs(b).max()
    assert np.abs(b[out]).max() <= 1e-12 * scale
    assert np.abs(b[inn]).max() >= 0.1 * scale


def test_inflow_data_is_twice_the_incoming_trace():
    # On the inflow face x = 0 (normal -x) the phase is 1 and (curl E) x n = i gamma E_T, so
    # g = 2 i gamma p there.  For r = 1 the constant p is represented exactly by its edge
    # circulations c_e = p . (x_b - x_a) (the duality of the degree-1 generators), so on the
    # DOFs of that face the quadrature load must equal 2 i gamma (S c), S the boundary
    # tangential mass matrix of the global system (for real eps and mu the only imaginary
    # part of A is beta S).
    g = load_golden()
    k0 = 1.3
    eps = g["eps_r_cylinder"]
    topo, xyz, b = _plane_wave_b(1, eps, k0)
    nt = topo.nt
    A = assemble.global_matrix(topo, xyz, np.full(nt, eps, dtype=np.complex128),
                               np.ones(nt, dtype=np.complex128), k0)
    gamma = k0 * math.sqrt(eps.real)
    S = A.imag / gamma
    p = np.array([0.0, 0.6, 0.8])
    c = (xyz[topo.edges[:, 1]] - xyz[topo.edges[:, 0]]) @ p
    expect = 2j * gamma * (S @ c)
    inn = _dofs_on_plane(topo, xyz, 0, 0.0, 1)
    assert np.abs(b[inn] - expect[inn]).max() <= 1e-12 * np.abs(expect[inn]).max()
    assert np.abs(expect[inn]).min() > 0.0


def test_flipped_impedance_sign_is_caught(monkeypatch):
    # plant the mistake in the oracle: beta of the wrong sign (an incoming-wave condition)
    g = load_golden()
    monkeypatch.setattr(assemble, "impedance_beta",
                        lambda k0, eps_r, mu_r: -k0 * np.sqrt(np.real(mu_r) * np.real(eps_r)))
    topo, xyz, b = _plane_wave_b(1, g["eps_r_cylinder"])
    out = _dofs_on_plane(topo, xyz, 0, 1.0, 1)
    assert np.abs(b[out]).max() >= 0.1 * np.abs(b).max()

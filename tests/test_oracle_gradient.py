"""Pins of the oracle's discrete gradient term (Eq. 4) and of the total field (Eq. 2) against
the exact derivative of the discrete energy, the continuum field of Eq. 4 and the analytic
180-degree wall of Eqs. 9-10 (Sec. 4.1)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import System, TERM_ALL, TERM_GRAD, TERM_LANDAU

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_total_field_is_minus_energy_gradient():
    # two materials, vacuum holes, anisotropic cells, every term on
    shape = (3, 4, 5)
    nx, ny, nz = shape
    rng = np.random.default_rng(0)
    mat = np.ones((nz, ny, nx), np.uint8); mat[:2] = 2; mat[4, 3, 2] = 0; mat[0, 0, 0] = 0; mat[2, 1, 1] = 0
    m2 = dict(synth.PTO, G12=3e-11, G44=7e-11, G44p=2e-11, r_s=1.3)
    s = System(shape, (1e-9, 1.1e-9, 0.9e-9), mat, {1: synth.BTO, 2: m2}, 300, 45.0,
               E_ext=(1e7, -2e7, 3e7), terms=TERM_ALL, conv="direct")
    P = rng.uniform(-0.3, 0.3, (3, nz, ny, nx)); P[:, mat == 0] = 0
    h = s.fields(P)["total"]
    hmax = np.abs(h).max()
    eps = 1e-6
    for c in range(3):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    if mat[z, y, x] == 0:
                        assert np.all(h[:, z, y, x] == 0)
                        continue
                    Pp = P.copy(); Pp[c, z, y, x] += eps
                    Pm = P.copy(); Pm[c, z, y, x] -= eps
                    fd = -(s.energy(Pp)["total"] - s.energy(Pm)["total"]) / (2 * eps) / s.V
                    assert abs(fd - h[c, z, y, x]) < 1e-7 * hmax


def _grad_system(shape, cell, G):
    nx, ny, nz = shape
    mat = synth.material(a1_form=2, **G)
    return System(shape, cell, np.ones((nz, ny, nx), np.uint8), {1: mat}, 300.0, terms=TERM_GRAD)


@pytest.mark.parametrize("G", [dict(G11=3e-10, G12=0.0, G44=0.0, G44p=0.0),
                               dict(G11=2e-10, G12=-4e-11, G44=3e-11, G44p=1e-11),
                               dict(G11=0.0, G12=5e-11, G44=2e-11, G44p=6e-11)])
def test_interior_field_matches_continuum_eq4(G):
    # quadratic polynomials: central differences are exact, so interior cells reproduce
    # h_x = G11 Px,xx + (G44+G'44)(Px,yy + Px,zz) + (G12+G44-G'44)(Py,xy + Pz,xz) (and cyclic)
    shape, cell = (9, 8, 7), (1e-9, 1.3e-9, 0.7e-9)
    nx, ny, nz = shape
    s = _grad_system(shape, cell, G)
    z, y, x = np.meshgrid(np.arange(nz) * cell[2], np.arange(ny) * cell[1], np.arange(nx) * cell[0],
                          indexing="ij")
    rng = np.random.default_rng(1)
    q = rng.normal(size=(3, 6)) * 1e15      # coefficients of x^2, y^2, z^2, xy, xz, yz per component
    mon = [x * x, y * y, z * z, x * y, x * z, y * z]
    P = np.stack([sum(q[i, k] * mon[k] for k in range(6)) for i in range(3)])
    h = s.fields(P)["grad"]
    G11, G12, Gs, Gd = G["G11"], G["G12"], G["G44"] + G["G44p"], G["G44"] - G["G44p"]
    C = G12 + Gd
    # second derivatives of component i: d_aa = 2 q[i,a], d_xy = q[i,3], d_xz = q[i,4], d_yz = q[i,5]
    dd = lambda i, a, b: 2 * q[i, a] if a == b else q[i, {(0, 1): 3, (0, 2): 4, (1, 2): 5}[tuple(sorted((a, b)))]]
    inner = (slice(2, nz - 2), slice(2, ny - 2), slice(2, nx - 2))
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        want = G11 * dd(i, i, i) + Gs * (dd(i, j, j) + dd(i, k, k)) + C * (dd(j, i, j) + dd(k, i, k))
        got = h[i][inner]
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9 * abs(want) + 1e-6)


def test_face_energy_of_uniform_gradient():
    # linear Px(x) with G11 only: F = 1/2 G11 (dPx/dx)^2 times the volume between first and last centre
    shape, cell = (10, 3, 2), (1e-9, 1e-9, 1e-9)
    s = _grad_system(shape, cell, dict(G11=4e-10, G12=0.0, G44=0.0, G44p=0.0))
    g = 1e7
    P = np.zeros((3, 2, 3, 10)); P[0] = g * np.arange(10) * cell[0]
    F = s.energy(P)["grad"]
    assert F == pytest.approx(0.5 * 4e-10 * g * g * (9 * cell[0]) * (3 * cell[1]) * (2 * cell[2]), rel=1e-12)


def _wall_profile(d_nm, component, G11, G44):
    w = GOLD["wall_180"]
    a1, a11 = w["alpha1"], w["alpha11"]
    L = 24.0   # nm, Neumann ends far from the wall (tanh tail below 1e-7 there)
    n = int(round(L / d_nm))
    mat = synth.wall_material(alpha1=a1, alpha11=a11, G11=G11, G44=G44, G44p=G44)
    s = System((n, 1, 1), (d_nm * 1e-9, 1e-9, 1e-9), np.ones((1, 1, n), np.uint8), {1: mat}, 300.0,
               terms=TERM_LANDAU | TERM_GRAD)
    xc = (np.arange(n) + 0.5) * d_nm - L / 2           # wall centre between the two middle cells
    Pinf = np.sqrt(abs(a1) / (2 * a11))
    P = np.zeros((3, 1, 1, n)); P[component, 0, 0] = Pinf * np.sign(xc)
    Geff = G11 if component == 0 else 2 * G44
    dt = 0.2 / (4 * Geff / (d_nm * 1e-9) ** 2 + 6 * abs(a1))
    P, steps, ok = s.relax(P, dt, 1e-13, Pinf, 2_000_000, check_every=256)
    assert ok
    xi = np.sqrt(Geff / abs(a1)) * 1e9                   # Eq. 9 / Eq. 10 width, nm
    exact = Pinf * np.tanh(xc / xi)
    return np.abs(P[component, 0, 0] - exact).max() / Pinf, Pinf, xi


@pytest.mark.parametrize("component,G11,G44", [(1, 0.0, 1.73e-10), (0, 3.46e-10, 0.0)])
def test_180_wall_matches_tanh_at_second_order(component, G11, G44):
    # Eq. 10 (Py(x), G44 = G'44 as printed in Sec. 4.1) and Eq. 9 (Px(x), G11 only)
    e1, Pinf, xi = _wall_profile(0.4, component, G11, G44)
    e2, _, _ = _wall_profile(0.2, component, G11, G44)
    assert Pinf == pytest.approx(0.70711, abs=1e-5)
    if component == 1:
        assert xi == pytest.approx(1.41006, abs=1e-5)
    assert e2 < 5e-3
    assert 3.5 < e1 / e2 < 4.5

"""Pins of the oracle's electrostatic field (Eqs. 5-6, open boundary P = 0 outside, Sec. 2)."""
import numpy as np
import pytest

import synth
from oracle import System, TERM_ELEC
from oracle import electrostatics as es
from tests.test_oracle_tensor import aharoni_dz

EPS0 = synth.EPS0


def _system(shape, cell, mat, eps_b, conv):
    return System(shape, cell, mat, {1: synth.BTO}, 300.0, eps_b, terms=TERM_ELEC, conv=conv)


@pytest.mark.parametrize("shape,cell", [((4, 4, 2), (1e-9, 1e-9, 1e-9)), ((8, 8, 4), (1e-9, 1.2e-9, 0.8e-9)),
                                        ((5, 3, 7), (1e-9, 1e-9, 2e-9)), ((1, 1, 6), (1e-9, 1e-9, 1e-9)),
                                        ((1, 1, 1), (1e-9, 1e-9, 1e-9))])
def test_fft_convolution_equals_direct_sum(shape, cell):
    nx, ny, nz = shape
    rng = np.random.default_rng(11)
    mat = np.ones((nz, ny, nx), np.uint8)
    if nx * ny * nz > 4:
        mat.flat[rng.choice(nx * ny * nz, 3, replace=False)] = 0
    P = rng.uniform(-0.3, 0.3, (3, nz, ny, nx))
    P[:, mat == 0] = 0
    Ed = _system(shape, cell, mat, 45.0, "direct").electrostatic_field(P)
    Ef = _system(shape, cell, mat, 45.0, "fft").electrostatic_field(P)
    assert np.abs(Ed - Ef).max() <= 1e-13 * np.abs(Ed).max()


def test_single_cell_field_is_self_term():
    # one cube uniformly polarized along z: E = -Pz/(3 eps0 epsB) (cube self-factor 1/3)
    s = _system((1, 1, 1), (1e-9,) * 3, np.ones((1, 1, 1), np.uint8), 45.0, "direct")
    E = s.electrostatic_field(np.array([0, 0, 0.2]).reshape(3, 1, 1, 1))
    assert E[2, 0, 0, 0] == pytest.approx(-0.2 / (3 * EPS0 * 45.0), rel=1e-13)
    assert abs(E[0, 0, 0, 0]) < 1e-6 and abs(E[1, 0, 0, 0]) < 1e-6


def test_uniform_prism_energy_matches_aharoni():
    # F_el = -1/2 int E.P = 1/2 V_tot Pz^2 D_z/(eps0 epsB) for a uniformly polarized prism
    shape, cell = (6, 5, 3), (1e-9, 1.1e-9, 0.9e-9)
    nx, ny, nz = shape
    s = _system(shape, cell, np.ones((nz, ny, nx), np.uint8), 20.0, "fft")
    P = np.zeros((3, nz, ny, nx)); P[2] = 0.3
    F = s.energy(P)["elec"]
    Vt = nx * ny * nz * s.V
    Dz = aharoni_dz(nx * cell[0] / 2, ny * cell[1] / 2, nz * cell[2] / 2)
    assert F == pytest.approx(0.5 * Vt * 0.3 ** 2 * Dz / (EPS0 * 20.0), rel=1e-11)


def test_thin_slab_depolarizing_field():
    # uniformly out-of-plane polarized film: E_z -> -Pz/(eps0 epsB) at the centre, error O(t/L)
    errs = []
    for L in (16, 32, 64):
        shape = (L, L, 2)
        s = _system(shape, (1e-9,) * 3, np.ones((2, L, L), np.uint8), 45.0, "fft")
        P = np.zeros((3, 2, L, L)); P[2] = 0.25
        E = s.electrostatic_field(P)
        ez = E[2, :, L // 2, L // 2].mean()
        errs.append(abs(ez / (-0.25 / (EPS0 * 45.0)) - 1.0))
    assert errs[2] < 0.05
    assert errs[0] / errs[1] > 1.7 and errs[1] / errs[2] > 1.7   # first order in t/L


def test_field_opposes_uniform_polarization_everywhere():
    shape = (6, 6, 6)
    s = _system(shape, (1e-9,) * 3, np.ones((6, 6, 6), np.uint8), 45.0, "fft")
    P = np.zeros((3, 6, 6, 6)); P[0] = 0.1
    E = s.electrostatic_field(P)
    assert np.all(E[0] < 0)


def test_kappa_scales_with_background_permittivity():
    shape = (4, 3, 2)
    rng = np.random.default_rng(5)
    P = rng.uniform(-0.2, 0.2, (3, 2, 3, 4))
    m = np.ones((2, 3, 4), np.uint8)
    E1 = _system(shape, (1e-9,) * 3, m, 1.0, "direct").electrostatic_field(P)
    E45 = _system(shape, (1e-9,) * 3, m, 45.0, "direct").electrostatic_field(P)
    assert np.allclose(E1, 45.0 * E45, rtol=1e-13)
    assert es.kappa(1.0) == pytest.approx(1 / EPS0)

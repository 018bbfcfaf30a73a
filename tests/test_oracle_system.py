"""Pins of the oracle's explicit step (Eq. 1, L = 1): gradient flow of Eq. 2 must lower F."""
import numpy as np
import pytest

import synth
from oracle import System, TERM_ALL, coefficients


@pytest.mark.parametrize("case", ["bto_film", "bilayer_with_vacuum"])
def test_total_energy_decreases_monotonically(case):
    if case == "bto_film":
        shape = (8, 8, 4)
        mat = np.ones((4, 8, 8), np.uint8)
        mats = {1: synth.BTO}
        eps_b, E = 45.0, (0.0, 0.0, 0.0)
        a = abs(coefficients(synth.BTO, 300.0)["a1x"])
    else:
        shape = (6, 5, 6)
        mat = synth.layer_map(shape, [(0, 2, 2), (2, 5, 1)])
        mat[3, 2, 2] = 0
        mats = {1: synth.PTO, 2: synth.STO}
        eps_b, E = 649.0, (0.0, 0.0, 5e7)
        a = abs(coefficients(synth.PTO, 300.0)["a1x"])
    nx, ny, nz = shape
    s = System(shape, (1e-9,) * 3, mat, mats, 300.0, eps_b, E_ext=E, terms=TERM_ALL)
    P = synth.uniform_P(shape, 0.05, 3).astype(np.float64)
    P[:, mat == 0] = 0
    dt = 0.004 / a
    F = [s.energy(P)["total"]]
    for _ in range(60):
        P = s.step(P, dt)
        F.append(s.energy(P)["total"])
    assert np.all(np.diff(F) < 0)
    assert np.all(P[:, mat == 0] == 0)


def test_relaxed_state_has_small_field():
    shape = (6, 6, 3)
    s = System(shape, (1e-9,) * 3, np.ones((3, 6, 6), np.uint8), {1: synth.BTO}, 300.0, 45.0)
    P = synth.uniform_P(shape, 0.01, 9).astype(np.float64)
    a = abs(coefficients(synth.BTO, 300.0)["a1x"])
    P, steps, ok = s.relax(P, 0.004 / a, 1e-9, 0.2649, 200000)
    assert ok
    h = s.fields(P)["total"]
    # per-step change below 1e-9 P0 means |h| dt < 1e-9 P0
    assert np.abs(h).max() * 0.004 / a < 1.01e-9 * 0.2649

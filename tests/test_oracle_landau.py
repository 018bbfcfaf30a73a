"""Pins of the oracle's Landau term (Eq. 3), material coefficients (Table 1) and the homogeneous
equilibria of Eq. 12 (Sec. 4.2), against values the paper prints and closed-form roots."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import System, TERM_LANDAU, coefficients
from oracle import landau

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_table1_pto_alpha1_matches_wall_section():
    g = GOLD["pto_alpha1_300K"]
    assert coefficients(synth.PTO, g["T"])["a1x"] == pytest.approx(g["alpha1"], rel=1e-14)


def test_strain_form_scales_only_z_quadratic():
    c = coefficients(dict(synth.PTO, r_s=1.8), 300.0)
    assert c["a1z"] == pytest.approx(1.8 * c["a1x"]) and c["a1y"] == c["a1x"]


def test_field_is_minus_gradient_of_energy_density():
    rng = np.random.default_rng(7)
    for mat, T in [(synth.BTO, 250.0), (synth.PTO, 300.0), (synth.STO, 300.0),
                   (dict(synth.PTO, r_s=1.6), 300.0)]:
        c = coefficients(mat, T)
        P = rng.uniform(-0.6, 0.6, (3, 50))
        h = landau.field(P, c)
        eps = 1e-6
        for i in range(3):
            d = np.zeros((3, 1)); d[i] = eps
            fd = -(landau.energy_density(P + d, c) - landau.energy_density(P - d, c)) / (2 * eps)
            assert np.allclose(h[i], fd, rtol=1e-7, atol=1e-9 * np.abs(h).max())


# --- homogeneous equilibria of Eq. 12, written in the test from Eq. 3 restricted to the three
# --- symmetric directions: u = (per-component value)^2,  f = n a1 u + b u^2 + c u^3.
def _reduced(c, phase):
    a1, a11, a12, a111, a112, a123 = (c[k] for k in ("a1x", "a11", "a12", "a111", "a112", "a123"))
    if phase == "T":   # (p, 0, 0)
        return 1, a1, a11, a111
    if phase == "O":   # (p, p, 0)
        return 2, 2 * a1, 2 * a11 + a12, 2 * a111 + 2 * a112
    if phase == "R":   # (p, p, p)
        return 3, 3 * a1, 3 * a11 + 3 * a12, 3 * a111 + 6 * a112 + a123
    raise ValueError(phase)


def closed_form_phase(c, phase):
    """(|P|, f) of the stable root of df/du = 0 for a phase, or None."""
    n, A, B, C = _reduced(c, phase)
    roots = np.roots([3 * C, 2 * B, A]) if C != 0 else np.array([-A / (2 * B)])
    best = None
    for u in roots:
        if abs(u.imag) > 1e-12 * abs(u) or u.real <= 0:
            continue
        u = u.real
        if 2 * B + 6 * C * u <= 0:      # radial minimum only
            continue
        f = A * u + B * u * u + C * u ** 3
        if best is None or f < best[1]:
            best = (np.sqrt(n * u), f)
    return best


def _relax_single_cell(mat, T, direction, p):
    s = System((1, 1, 1), (1e-9,) * 3, np.ones((1, 1, 1), np.uint8), {1: mat}, T, terms=TERM_LANDAU)
    P = (np.asarray(direction, float) / np.linalg.norm(direction) * p).reshape(3, 1, 1, 1)
    dt = 0.01 / abs(coefficients(mat, T)["a1x"])
    P, steps, ok = s.relax(P, dt, 1e-15, 1.0, 400000, check_every=64)
    assert ok
    return P.ravel(), s.energy(P)["land"] / s.V


@pytest.mark.parametrize("T,phase,direction", [(300.0, "T", (0, 0, 1)), (250.0, "O", (1, 1, 0)),
                                               (200.0, "R", (1, 1, 1)), (150.0, "R", (-1, 1, -1)),
                                               (350.0, "T", (1, 0, 0))])
def test_single_cell_relaxes_to_analytic_root(T, phase, direction):
    c = coefficients(synth.BTO, T)
    mag, f = closed_form_phase(c, phase)
    P, F = _relax_single_cell(synth.BTO, T, direction, 0.9 * mag)
    assert np.linalg.norm(P) == pytest.approx(mag, rel=1e-12)
    assert F == pytest.approx(f, rel=1e-12)
    d = np.asarray(direction, float)
    assert np.allclose(P / np.linalg.norm(P), d / np.linalg.norm(d), atol=1e-10)


def test_bto_300K_tetragonal_value():
    mag, f = closed_form_phase(coefficients(synth.BTO, 300.0), "T")
    assert mag == pytest.approx(0.2649096, abs=2e-7)


@pytest.mark.parametrize("T", ["300", "250", "150"])
def test_global_minimum_phase_matches_paper(T):
    want = GOLD["bto_global_minimum_phase"][T]
    c = coefficients(synth.BTO, float(T))
    energies = {ph: closed_form_phase(c, ph)[1] for ph in "TOR" if closed_form_phase(c, ph)}
    assert min(energies, key=energies.get) == want
    # and the oracle's own energy density agrees with the closed form at each root
    for ph, f in energies.items():
        n, *_ = _reduced(c, ph)
        mag = closed_form_phase(c, ph)[0]
        v = np.array([1.0] * n + [0.0] * (3 - n)) * mag / np.sqrt(n)
        assert landau.energy_density(v.reshape(3, 1), c)[0] == pytest.approx(f, rel=1e-12)


def _classify(P):
    a = np.sort(np.abs(P), axis=0)[::-1]
    r1, r2 = a[1] / a[0], a[2] / a[0]
    return np.where(r1 < 1e-3, "T", np.where(r2 < 1e-3, "O", "R"))


@pytest.mark.parametrize("T,want", [(50.0, "R"), (350.0, "T")])
def test_random_small_starts_follow_paper_phase_statistics(T, want):
    # Sec. 4.2 / Fig. 2(c): random orientation, magnitudes ~1e-3 C/m^2, Landau only
    n = 300
    rng = np.random.default_rng(int(T))
    d = rng.normal(size=(3, n)); d /= np.linalg.norm(d, axis=0)
    P = (d * rng.uniform(0.5e-3, 1.5e-3, n)).reshape(3, 1, 1, n)
    s = System((n, 1, 1), (1e-9,) * 3, np.ones((1, 1, n), np.uint8), {1: synth.BTO}, T, terms=TERM_LANDAU)
    dt = 0.01 / abs(coefficients(synth.BTO, T)["a1x"])
    P, steps, ok = s.relax(P, dt, 1e-12, 1.0, 200000, check_every=64)
    assert ok
    assert np.all(_classify(P.reshape(3, n)) == want)

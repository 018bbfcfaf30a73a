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


def test_ac_field_enters_at_step_time():
    # one cell, applied field only: dP/dt = E_ext(t) exactly, so Euler sums E_ext(t_i) dt
    s = System((1, 1, 1), (1e-9,) * 3, np.ones((1, 1, 1), np.uint8), {1: synth.BTO}, 300.0, terms=8,
               E_ext=(1e7, 0.0, 0.0), E_ac=(0.0, 0.0, 2e8), freq=1e9, phase=0.3)
    dt, n = 1e-11, 37
    P = s.run(np.zeros((3, 1, 1, 1)), dt, n, t0=2e-10)
    t = 2e-10 + dt * np.arange(n)
    assert P[0, 0, 0, 0] == pytest.approx(n * dt * 1e7, rel=1e-12)
    assert P[2, 0, 0, 0] == pytest.approx(np.sum(2e8 * np.sin(2 * np.pi * 1e9 * t + 0.3)) * dt, rel=1e-12)


@pytest.mark.parametrize("method,order", [("euler", 1), ("heun", 2)])
def test_integrator_convergence_order(method, order):
    # one BaTiO3 cell, Landau term only: halving dt divides the error at a fixed time by 2^order
    from oracle import TERM_LANDAU
    s = System((1, 1, 1), (1e-9,) * 3, np.ones((1, 1, 1), np.uint8), {1: synth.BTO}, 300.0, terms=TERM_LANDAU)
    a = abs(coefficients(synth.BTO, 300.0)["a1x"])
    P0 = np.array([0.02, 0.05, 0.11]).reshape(3, 1, 1, 1)
    t_end = 0.5 / a
    ref = s.run(P0, t_end / 4096, 4096, method="heun")
    err = [np.abs(s.run(P0, t_end / n, n, method=method) - ref).max() for n in (32, 64, 128)]
    r1, r2 = err[0] / err[1], err[1] / err[2]
    assert 0.8 * 2 ** order < r1 < 1.25 * 2 ** order
    assert 0.8 * 2 ** order < r2 < 1.25 * 2 ** order


def _ivp_reference(s, P0, t_end, t0=0.0):
    """the same ODE integrated by scipy's DOP853 to rtol 1e-13 (an independent integrator)"""
    from scipy.integrate import solve_ivp
    shape = P0.shape
    f = lambda t, y: s.fields(y.reshape(shape), t)["total"].ravel()
    r = solve_ivp(f, (t0, t0 + t_end), P0.ravel(), method="DOP853", rtol=1e-13, atol=1e-16)
    assert r.success
    return r.y[:, -1].reshape(shape)


def _cell_system(with_ac):
    from oracle import TERM_LANDAU, TERM_EXT
    kw = dict(E_ac=(0.0, 1e6, 3e6), freq=2e7, phase=0.4) if with_ac else {}
    return System((1, 1, 1), (1e-9,) * 3, np.ones((1, 1, 1), np.uint8), {1: synth.BTO}, 300.0,
                  terms=TERM_LANDAU | (TERM_EXT if with_ac else 0), **kw)


@pytest.mark.parametrize("method,order", [("rk45", 4), ("ab3m2", 3)])
@pytest.mark.parametrize("with_ac", [False, True])
def test_higher_order_integrators_converge_at_their_order(method, order, with_ac):
    # one BaTiO3 cell (Landau, plus a time-dependent applied field): the error at a fixed time
    # against DOP853 falls by 2^order per halving of dt; wrong stage times or weights break it
    s = _cell_system(with_ac)
    a = abs(coefficients(synth.BTO, 300.0)["a1x"])
    P0 = np.array([0.02, 0.05, 0.11]).reshape(3, 1, 1, 1)
    t_end = 0.5 / a
    ref = _ivp_reference(s, P0, t_end, t0=1e-10)
    err = [np.abs(s.run(P0, t_end / n, n, t0=1e-10, method=method) - ref).max() for n in (64, 128, 256)]
    r1, r2 = err[0] / err[1], err[1] / err[2]
    assert 0.75 * 2 ** order < r1 < 1.35 * 2 ** order, (err, r1)
    assert 0.75 * 2 ** order < r2 < 1.35 * 2 ** order, (err, r2)


def test_rkf45_error_estimate_is_fifth_order_and_tracks_the_true_error():
    # one step: |P5 - P4| scales as dt^5, and P5 is closer to the exact solution than P4
    s = _cell_system(True)
    a = abs(coefficients(synth.BTO, 300.0)["a1x"])
    P0 = np.array([0.02, 0.05, 0.11]).reshape(3, 1, 1, 1)
    est, true4 = [], []
    for dt in (0.025 / a, 0.0125 / a, 0.00625 / a):
        P4, P5 = s.rkf45_step(P0, dt, 3e-10)
        ex = _ivp_reference(s, P0, dt, t0=3e-10)
        est.append(np.abs(P5 - P4).max())
        true4.append(np.abs(P4 - ex).max())
        assert np.abs(P5 - ex).max() < 0.5 * true4[-1]
    assert 0.7 * 32 < est[0] / est[1] < 1.4 * 32
    assert 0.7 * 32 < est[1] / est[2] < 1.4 * 32
    # the estimate has the size of the true error of the advancing solution
    assert all(0.3 < e / t < 3.0 for e, t in zip(est, true4))


def test_ab3m2_first_step_is_heun_and_film_order_holds():
    shape = (3, 3, 2)
    s = System(shape, (1e-9,) * 3, np.ones((2, 3, 3), np.uint8), {1: synth.BTO}, 300.0, 45.0)
    a = abs(coefficients(synth.BTO, 300.0)["a1x"])
    P0 = synth.uniform_P(shape, 0.05, 11).astype(np.float64)
    dt = 0.004 / a
    assert np.allclose(s.ab3m2_run(P0, dt, 1), s.heun_step(P0, dt), rtol=1e-13, atol=1e-16)
    # all four terms on a small film (gradient and electrostatic coupling): orders hold as well
    t_end = 0.08 / a
    ref = _ivp_reference(s, P0, t_end)
    for method, order in (("rk45", 4), ("ab3m2", 3)):
        err = [np.abs(s.run(P0, t_end / n, n, method=method) - ref).max() for n in (32, 64)]
        assert 0.6 * 2 ** order < err[0] / err[1] < 1.5 * 2 ** order, (method, err)

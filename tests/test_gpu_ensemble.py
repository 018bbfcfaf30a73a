"""Landau-only ensemble of independent single-cell relaxations (Sec. 4.2, Fig. 2(c)).

A grid of cells with only the Landau term is a set of independent single-cell runs of Eq. 1;
the paper relaxes 1500 random starts (|P| ~ 1e-3 C/m^2, random orientation) per temperature and
counts the phases reached.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import System, TERM_LANDAU, coefficients

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _shape(n):
    return (n // 30, 30, 1)     # any layout: the cells do not interact


def _starts(n, T):
    rng = np.random.default_rng(int(T) + 7)
    d = rng.normal(size=(3, n)); d /= np.linalg.norm(d, axis=0)
    nx, ny, nz = _shape(n)
    return (d * rng.uniform(0.5e-3, 1.5e-3, n)).astype(np.float32).reshape(3, nz, ny, nx)


def _classify(P):
    a = np.sort(np.abs(P.reshape(3, -1)), axis=0)[::-1]
    r1, r2 = a[1] / a[0], a[2] / a[0]
    return np.where(r1 < 1e-2, "T", np.where(r2 < 1e-2, "O", "R"))


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_28800_b300 import tdgl
    c = tdgl.Context(0)
    yield c
    c.close()


def _gpu_ensemble(ctx, T, n):
    from paper_2605_28800_b300 import tdgl
    nx, ny, nz = _shape(n)
    s = tdgl.Sim(ctx, (nx, ny, nz), (1e-9,) * 3)
    s.define_material(1, synth.BTO)
    s.set_material_map(np.ones((nz, ny, nx), np.uint8))
    s.set_temperature(T)
    s.set_terms(tdgl.TERM_LANDAU)
    P = _starts(n, T)
    s.set_P(P)
    dt = 0.01 / abs(coefficients(synth.BTO, T)["a1x"])
    steps, ok = s.relax(dt, 1e-7, 400000, check_every=64)
    assert ok
    return s.get_P(), P, dt


@pytest.mark.parametrize("T,want", [(50.0, "R"), (350.0, "T")])
def test_gpu_ensemble_reproduces_paper_phase_extremes(ctx, T, want):
    # Fig. 2(c): all rhombohedral within 0-100 K, all tetragonal above 300 K (1500 starts)
    P, _, _ = _gpu_ensemble(ctx, T, 1500)
    assert np.all(_classify(P) == want)


@pytest.mark.parametrize("T", [200.0, 250.0, 280.0])
def test_gpu_ensemble_phase_counts_match_oracle(ctx, T):
    n = 600
    Pg, P0, dt = _gpu_ensemble(ctx, T, n)
    nx, ny, nz = _shape(n)
    o = System((nx, ny, nz), (1e-9,) * 3, np.ones((nz, ny, nx), np.uint8), {1: synth.BTO}, T, terms=TERM_LANDAU)
    Po, _, ok = o.relax(P0.astype(np.float64), dt, 1e-9, 1.0, 400000, check_every=64)
    assert ok
    cg, co = _classify(Pg), _classify(Po)
    # same basin for (almost) every start; starts on a separatrix may legitimately differ
    assert np.mean(cg == co) >= 0.99
    for ph in "TOR":
        assert abs(np.sum(cg == ph) - np.sum(co == ph)) <= 0.01 * n

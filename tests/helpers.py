"""Test helpers: build the same problem for the CUDA path (through the C ABI) and the oracle."""
from __future__ import annotations

import numpy as np

import synth


def gpu_sim(ctx, shape, cell, mat, materials, T, eps_b, E=(0.0, 0.0, 0.0), terms=15, P=None, scales=None):
    from paper_2605_28800_b300 import tdgl
    s = tdgl.Sim(ctx, shape, cell)
    for mid, rec in materials.items():
        s.define_material(mid, rec)
    s.set_material_map(np.ascontiguousarray(mat, dtype=np.uint8))
    s.set_temperature(T)
    s.set_eps_b(eps_b)
    s.set_field(E)
    s.set_terms(terms)
    if scales is not None:
        s.set_scales(*scales)
    if P is not None:
        s.set_P(np.ascontiguousarray(P, dtype=np.float32))
    return s


def oracle_sys(shape, cell, mat, materials, T, eps_b, E=(0.0, 0.0, 0.0), terms=15, conv="fft"):
    from oracle import System
    return System(shape, cell, mat, materials, T, eps_b, E_ext=E, terms=terms, conv=conv)


def mixed_case(shape, seed=0, vacuum=3):
    """Two materials in z layers, a few vacuum cells, random P (zero on vacuum)."""
    nx, ny, nz = shape
    mat = np.ones((nz, ny, nx), np.uint8)
    if nz > 1:
        mat[: max(1, nz // 3)] = 2
    rng = np.random.default_rng(seed)
    if vacuum and nx * ny * nz > 4:
        mat.flat[rng.choice(nx * ny * nz, min(vacuum, nx * ny * nz // 4), replace=False)] = 0
    P = synth.uniform_P(shape, 0.2, seed + 100)
    P[:, mat == 0] = 0
    return mat, P


def rel_err(a, b, ref=None):
    ref = np.abs(b).max() if ref is None else ref
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max() / max(ref, 1e-300))

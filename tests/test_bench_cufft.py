"""The cuFFT comparison in bench.py rebuilds the padded 3x3 kernel from impulse responses (the field
of a unit P at a corner cell) using the parities of N; checked here on the CPU: an FFT convolution
with the rebuilt kernel equals the oracle's direct O(N^2) field sum."""
import importlib.util
import os

import numpy as np

from oracle import electrostatics as es, tensor as ten

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_kernel_from_impulse_responses_reproduces_the_direct_field():
    b = _bench()
    n = (5, 4, 3)
    nx, ny, nz = n
    cell, eps_b = (1e-9, 1.1e-9, 0.9e-9), 45.0
    Nf = ten.full(n, cell)
    K = np.zeros((3, 3, nz, ny, nx))
    for j in range(3):
        P = np.zeros((3, nz, ny, nx))
        P[j, 0, 0, 0] = 1.0
        K[:, j] = es.direct(P, Nf, eps_b)
    M = (12, 9, 6)          # any padding >= 2n - 1 per axis, even and odd
    Kh = np.fft.rfftn(b.padded_from_impulses(K, M), axes=(2, 3, 4))
    assert np.abs(Kh.imag).max() <= 1e-12 * np.abs(Kh.real).max()    # real by the parities
    P = np.random.default_rng(0).normal(size=(3, nz, ny, nx))
    Ph = np.fft.rfftn(P, s=(M[2], M[1], M[0]), axes=(1, 2, 3))
    E = np.fft.irfftn(np.einsum("ijzyx,jzyx->izyx", Kh, Ph), s=(M[2], M[1], M[0]), axes=(1, 2, 3))[:, :nz, :ny, :nx]
    Ed = es.direct(P, Nf, eps_b)
    assert np.abs(E - Ed).max() <= 1e-12 * np.abs(Ed).max()

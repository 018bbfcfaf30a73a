"""ORACLE (test infrastructure).  Open-boundary electrostatic field of Eqs. 5-6.

With P uniform inside each cell (Sec. 3) and P = 0 outside the sample (Sec. 2), Eq. 6 averaged
over a cell is the discrete convolution
    E_el(a) = -(1/(eps0 epsB)) sum_b N(r_a - r_b) P(b),
N the cell-pair averaged interaction tensor (tensor.py).  Two evaluations:
* ``direct``: that sum written out, O(N^2), for small grids (the definition);
* ``fft``:    the same linear convolution through numpy's FFT on a grid zero-padded to 2n per
              axis, so that the circular convolution equals the linear one (Sec. 3: FFT-based).
Eq. 5 gives the energy  F_el = -1/2 V sum_a E_el(a) . P(a).
"""
from __future__ import annotations

import numpy as np

from . import tensor as _tensor

EPS0 = 8.8541878128e-12   # F/m, CODATA 2018

# (row i, column j) -> component index in (xx, yy, zz, xy, xz, yz)
_IDX = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]


def kappa(eps_b):
    return 1.0 / (EPS0 * eps_b)


def direct(P, Nfull, eps_b):
    """E (3, nz, ny, nx) by the O(N^2) sum.  Nfull from tensor.full()."""
    _, nz, ny, nx = P.shape
    k = kappa(eps_b)
    E = np.zeros(P.shape)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    src = P.reshape(3, -1)
    zb, yb, xb = zz.ravel(), yy.ravel(), xx.ravel()
    for a in range(nz * ny * nx):
        za, ya, xa = zb[a], yb[a], xb[a]
        iz, iy, ix = za - zb + nz - 1, ya - yb + ny - 1, xa - xb + nx - 1
        Nab = Nfull[:, iz, iy, ix]                          # (6, Ncells)
        for i in range(3):
            s = 0.0
            for j in range(3):
                s += np.dot(Nab[_IDX[i][j]], src[j])
            E[i].flat[a] = -k * s
    return E


def padded_kernel(oct_, M):
    """Tensor on the zero-padded periodic grid of size M = (Mx, My, Mz), Mi >= 2 ni - 1.

    Entry at index (kz, ky, kx) holds N at the offset congruent to it modulo M that lies in
    [-(n-1), n-1]; indices that correspond to no such offset hold zero.
    """
    _, nz, ny, nx = oct_.shape
    Mx, My, Mz = M

    def axis(n, Mi):
        idx = np.arange(Mi)
        off = np.where(idx < n, idx, idx - Mi)
        valid = np.abs(off) <= n - 1
        return np.clip(np.abs(off), 0, n - 1), np.sign(off) + (off == 0), valid

    ax_, sx, vx = axis(nx, Mx)
    ay_, sy, vy = axis(ny, My)
    az_, sz, vz = axis(nz, Mz)
    out = np.zeros((6, Mz, My, Mx))
    valid = vz[:, None, None] & vy[None, :, None] & vx[None, None, :]
    for c in range(6):
        px, py, pz = _tensor.PARITY[c]
        sgn = ((sz if pz < 0 else np.ones(Mz))[:, None, None]
               * (sy if py < 0 else np.ones(My))[None, :, None]
               * (sx if px < 0 else np.ones(Mx))[None, None, :])
        out[c] = np.where(valid, oct_[c][np.ix_(az_, ay_, ax_)] * sgn, 0.0)
    return out


class FFTConvolver:
    """Zero-padded FFT convolution with a fixed tensor (padding 2n per axis)."""

    def __init__(self, n, cell, oct_=None):
        nx, ny, nz = n
        self.n = n
        self.M = (2 * nx, 2 * ny, 2 * nz)
        o = _tensor.octant(n, cell) if oct_ is None else oct_
        K = padded_kernel(o, self.M)
        self.Khat = np.fft.rfftn(K, axes=(1, 2, 3))

    def apply(self, P, eps_b):
        nx, ny, nz = self.n
        Mx, My, Mz = self.M
        Pp = np.zeros((3, Mz, My, Mx))
        Pp[:, :nz, :ny, :nx] = P
        Ph = np.fft.rfftn(Pp, axes=(1, 2, 3))
        Eh = np.empty_like(Ph)
        for i in range(3):
            Eh[i] = sum(self.Khat[_IDX[i][j]] * Ph[j] for j in range(3))
        E = np.fft.irfftn(Eh, s=(Mz, My, Mx), axes=(1, 2, 3))[:, :nz, :ny, :nx]
        return -kappa(eps_b) * E


def energy(E, P, V):
    return -0.5 * V * float(np.sum(E * P))

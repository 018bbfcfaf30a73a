"""ORACLE (test infrastructure).  ctypes front end of tensor.c (FP64 cell-interaction tensor).

The shared library is compiled from tensor.c by ``oracle.build.build()`` (gcc, -fopenmp).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import library_path, build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(
                os.path.join(os.path.dirname(__file__), "tensor.c")):
            build()
        lib = ctypes.CDLL(path)
        d = ctypes.c_double
        p6 = ctypes.POINTER(ctypes.c_double)
        lib.oracle_tensor_newell.argtypes = [d, d, d, d, d, d, p6]
        lib.oracle_tensor_far.argtypes = [d, d, d, d, d, d, ctypes.c_int, p6]
        lib.oracle_tensor_offset.argtypes = [ctypes.c_int] * 3 + [d, d, d, p6]
        lib.oracle_tensor_octant.argtypes = [ctypes.c_int] * 3 + [d, d, d, p6]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def newell(X, Y, Z, cell):
    """Near-field closed form at a metric offset; returns (xx, yy, zz, xy, xz, yz)."""
    out = np.zeros(6)
    _load().oracle_tensor_newell(X, Y, Z, *cell, _ptr(out))
    return out


def far(X, Y, Z, cell, m):
    """Far-field Gauss-Legendre rule (m points per tent half) at a metric offset."""
    out = np.zeros(6)
    _load().oracle_tensor_far(X, Y, Z, *cell, m, _ptr(out))
    return out


def offset(i, j, k, cell):
    """Tensor at an integer cell offset with the built-in near/far switch."""
    out = np.zeros(6)
    _load().oracle_tensor_offset(i, j, k, *cell, _ptr(out))
    return out


def octant(n, cell):
    """Non-negative offsets: array (6, nz, ny, nx) for offsets [0,nx) x [0,ny) x [0,nz)."""
    nx, ny, nz = n
    out = np.zeros((6, nz, ny, nx))
    _load().oracle_tensor_octant(nx, ny, nz, *cell, _ptr(out))
    return out


# parity of each component under a sign flip of (x, y, z): +1 even, -1 odd
PARITY = np.array([[1, 1, 1], [1, 1, 1], [1, 1, 1], [-1, -1, 1], [-1, 1, -1], [1, -1, -1]])


def full(n, cell, oct_=None):
    """All offsets in [-(n-1), n-1]^3: array (6, 2nz-1, 2ny-1, 2nx-1), index = offset + n - 1.

    Negative offsets come from the octant through the reflection symmetries of the tensor
    (diagonal components even in every axis; N_ij odd in i and in j).
    """
    nx, ny, nz = n
    o = octant(n, cell) if oct_ is None else oct_
    ox = np.abs(np.arange(-(nx - 1), nx))
    oy = np.abs(np.arange(-(ny - 1), ny))
    oz = np.abs(np.arange(-(nz - 1), nz))
    sx = np.sign(np.arange(-(nx - 1), nx)) + (np.arange(-(nx - 1), nx) == 0)
    sy = np.sign(np.arange(-(ny - 1), ny)) + (np.arange(-(ny - 1), ny) == 0)
    sz = np.sign(np.arange(-(nz - 1), nz)) + (np.arange(-(nz - 1), nz) == 0)
    out = np.empty((6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1))
    for c in range(6):
        px, py, pz = PARITY[c]
        sgn = ((sz if pz < 0 else np.ones_like(sz))[:, None, None]
               * (sy if py < 0 else np.ones_like(sy))[None, :, None]
               * (sx if px < 0 else np.ones_like(sx))[None, None, :])
        out[c] = o[c][np.ix_(oz, oy, ox)] * sgn
    return out

"""ORACLE (test infrastructure).  Landau free energy density of Eq. 3 and its field.

Eq. 3:  f = a1 (Px^2+Py^2+Pz^2) + a11 (Px^4+Py^4+Pz^4) + a12 (Px^2Py^2 + Py^2Pz^2 + Pz^2Px^2)
          + a111 (Px^6+Py^6+Pz^6) + a112 (Px^4(Py^2+Pz^2) + Py^4(Px^2+Pz^2) + Pz^4(Px^2+Py^2))
          + a123 Px^2 Py^2 Pz^2,
with the z quadratic coefficient r_s*a1 under the strain form of Sec. 4.4 (a1x, a1y, a1z).
The field is h_i = -df/dP_i, differentiated by hand term by term.
"""
from __future__ import annotations

import numpy as np


def energy_density(P, c):
    """f(P) in J/m^3.  P: (3, ...) arrays; c: coefficient dict (scalars or broadcastable arrays)."""
    x2, y2, z2 = P[0] ** 2, P[1] ** 2, P[2] ** 2
    return (c["a1x"] * x2 + c["a1y"] * y2 + c["a1z"] * z2
            + c["a11"] * (x2 ** 2 + y2 ** 2 + z2 ** 2)
            + c["a12"] * (x2 * y2 + y2 * z2 + z2 * x2)
            + c["a111"] * (x2 ** 3 + y2 ** 3 + z2 ** 3)
            + c["a112"] * (x2 ** 2 * (y2 + z2) + y2 ** 2 * (x2 + z2) + z2 ** 2 * (x2 + y2))
            + c["a123"] * x2 * y2 * z2)


def field(P, c):
    """h = -df/dP, shape (3, ...)."""
    h = np.empty_like(P, dtype=np.float64)
    sq = [P[0] ** 2, P[1] ** 2, P[2] ** 2]
    a1 = [c["a1x"], c["a1y"], c["a1z"]]
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        p, pi2, pj2, pk2 = P[i], sq[i], sq[j], sq[k]
        d = (2.0 * a1[i] * p
             + 4.0 * c["a11"] * p * pi2
             + 2.0 * c["a12"] * p * (pj2 + pk2)
             + 6.0 * c["a111"] * p * pi2 ** 2
             + c["a112"] * (4.0 * p * pi2 * (pj2 + pk2) + 2.0 * p * (pj2 ** 2 + pk2 ** 2))
             + 2.0 * c["a123"] * p * pj2 * pk2)
        h[i] = -d
    return h

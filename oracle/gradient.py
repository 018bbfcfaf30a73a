"""ORACLE (test infrastructure).  Discrete gradient (Ginzburg) energy of Eq. 4 and its exact field.

Eq. 4 expands to
    F_grad = 1/2 G11 sum_i P_{i,i}^2 + 1/2 (G44 + G'44) sum_{i != j} P_{i,j}^2
             + G12 sum_{i<j} P_{i,i} P_{j,j} + (G44 - G'44) sum_{i<j} P_{i,j} P_{j,i},
whose continuum field is  h_x = G11 dxx Px + (G44+G'44)(dyy+dzz) Px + (G12+G44-G'44)(dxy Py + dxz Pz).

The paper gives no discrete form and no boundary rule for this term (Sec. 3 only says finite
differences; the open boundary of Sec. 2 concerns electrostatics).  Reading used here:

* square terms live on cell faces: for two adjacent material cells a, b along axis d,
  1/2 G_face V ((P_i(b) - P_i(a))/dx_d)^2 with G_face the mean of the two cells' directional
  coefficient (G11 when i == d, G44 + G'44 otherwise).  Faces to vacuum or to the outside
  carry nothing (natural, Neumann boundary).
* cross terms live on material cells: V [G12 sum_{i<j} D_iP_i D_jP_j + (G44-G'44) sum_{i<j}
  D_jP_i D_iP_j] with D_d the central difference along d, where a neighbour outside the
  material is replaced by the cell itself (mirror ghost).
* the field is the exact -(1/V) dF/dP of this discrete energy.  For the cross terms it is
  (Phi(a+e_d) - Phi(a-e_d)) / (2 dx_d) with Phi the flux multiplying D_d P_i, where a flux
  at a non-material neighbour is replaced by -Phi(a) (the adjoint of the mirror ghost).

Arrays: P (3, nz, ny, nx); mat (nz, ny, nx) with 0 = vacuum; per-cell coefficient arrays.
"""
from __future__ import annotations

import numpy as np


def _ax(d):
    """spatial array axis of direction d (0 = x, 1 = y, 2 = z) for (nz, ny, nx) arrays."""
    return 2 - d


def _sl(ndim, ax, s):
    idx = [slice(None)] * ndim
    idx[ax] = s
    return tuple(idx)


def _neighbour(a, d, s):
    """(value at cell + s*e_d, inside-grid flag); zero where the neighbour is outside."""
    ax = _ax(d)
    out = np.zeros_like(a)
    ok = np.zeros(a.shape, dtype=bool)
    nd = a.ndim
    if a.shape[ax] > 1:
        if s > 0:
            out[_sl(nd, ax, slice(0, -1))] = a[_sl(nd, ax, slice(1, None))]
            ok[_sl(nd, ax, slice(0, -1))] = True
        else:
            out[_sl(nd, ax, slice(1, None))] = a[_sl(nd, ax, slice(0, -1))]
            ok[_sl(nd, ax, slice(1, None))] = True
    return out, ok


def _mat_neighbour(m, d, s):
    v, ok = _neighbour(m.astype(np.int8), d, s)
    return (v > 0) & ok


def central(Q, m, d, h):
    """D_d Q with mirror ghosts (neighbour outside the material -> the cell's own value)."""
    qp, _ = _neighbour(Q, d, +1)
    qm, _ = _neighbour(Q, d, -1)
    mp = _mat_neighbour(m, d, +1)
    mm = _mat_neighbour(m, d, -1)
    qp = np.where(mp, qp, Q)
    qm = np.where(mm, qm, Q)
    return np.where(m, (qp - qm) / (2.0 * h), 0.0)


def adjoint_central(Phi, m, d, h):
    """(Phi(a+e_d) - Phi(a-e_d)) / (2h) with odd ghosts (non-material neighbour -> -Phi(a))."""
    fp, _ = _neighbour(Phi, d, +1)
    fm, _ = _neighbour(Phi, d, -1)
    mp = _mat_neighbour(m, d, +1)
    mm = _mat_neighbour(m, d, -1)
    fp = np.where(mp, fp, -Phi)
    fm = np.where(mm, fm, -Phi)
    return np.where(m, (fp - fm) / (2.0 * h), 0.0)


def field_and_energy(P, mat, coef, cell):
    """Return (h_grad (3, nz, ny, nx), F_grad in J).

    coef: dict of per-cell arrays G11, G12, G44, G44p (zero in vacuum); cell: (dx, dy, dz).
    """
    m = mat > 0
    V = cell[0] * cell[1] * cell[2]
    h = np.zeros(P.shape, dtype=np.float64)
    F = 0.0
    G11, G12 = coef["G11"], coef["G12"]
    G44s = coef["G44"] + coef["G44p"]
    Gd = coef["G44"] - coef["G44p"]
    # square terms on faces
    for d in range(3):
        ax = _ax(d)
        n = P.shape[ax + 1]
        if n < 2:
            continue
        lo = _sl(3, ax, slice(0, n - 1))
        hi = _sl(3, ax, slice(1, n))
        both = m[lo] & m[hi]
        inv = 1.0 / cell[d] ** 2
        for i in range(3):
            Gdir = G11 if i == d else G44s
            Gf = 0.5 * (Gdir[lo] + Gdir[hi])
            diff = P[i][hi] - P[i][lo]
            flux = np.where(both, Gf * diff * inv, 0.0)
            h[i][lo] += flux
            h[i][hi] -= flux
            F += 0.5 * V * float(np.sum(np.where(both, Gf * diff * diff * inv, 0.0)))
    # cross terms on cells
    if np.any(G12 != 0.0) or np.any(Gd != 0.0):
        D = [[central(P[i], m, d, cell[d]) for d in range(3)] for i in range(3)]  # D[i][d] = D_d P_i
        dens = (G12 * (D[0][0] * D[1][1] + D[1][1] * D[2][2] + D[2][2] * D[0][0])
                + Gd * (D[0][1] * D[1][0] + D[1][2] * D[2][1] + D[0][2] * D[2][0]))
        F += V * float(np.sum(np.where(m, dens, 0.0)))
        for i in range(3):
            others = [j for j in range(3) if j != i]
            Phi = G12 * sum(D[j][j] for j in others)
            h[i] += adjoint_central(Phi, m, i, cell[i])
            for j in others:
                h[i] += adjoint_central(Gd * D[j][i], m, j, cell[j])
    h[:, ~m] = 0.0
    return h, F

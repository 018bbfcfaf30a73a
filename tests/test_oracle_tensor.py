"""Pins of the oracle's cell-interaction tensor (Eq. 6 cell-averaged; the demagnetization-tensor
analogy of Sec. 2 and Sec. 3, ref. [40]) against closed forms and mathematical identities."""
import numpy as np
import pytest

from oracle import tensor

CELLS = [(1.0, 1.0, 1.0), (1.0, 2.0, 3.0), (0.5, 0.5, 1.7), (2.0, 1.0, 0.25)]


def aharoni_dz(a, b, c):
    """Volume-averaged demagnetizing factor along z of a 2a x 2b x 2c prism (Aharoni,
    J. Appl. Phys. 83, 3432 (1998)), written from the published closed form."""
    R = np.sqrt(a * a + b * b + c * c)
    ab, bc, ac = np.sqrt(a * a + b * b), np.sqrt(b * b + c * c), np.sqrt(a * a + c * c)
    s = ((b * b - c * c) / (2 * b * c) * np.log((R - a) / (R + a))
         + (a * a - c * c) / (2 * a * c) * np.log((R - b) / (R + b))
         + b / (2 * c) * np.log((ab + a) / (ab - a)) + a / (2 * c) * np.log((ab + b) / (ab - b))
         + c / (2 * a) * np.log((bc - b) / (bc + b)) + c / (2 * b) * np.log((ac - a) / (ac + a))
         + 2 * np.arctan(a * b / (c * R)) + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * R + c / (a * b) * (ac + bc)
         - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c))
    return s / np.pi


def test_aharoni_reference_itself():
    # the closed form used below: cube = 1/3 and the three factors sum to one
    assert aharoni_dz(1, 1, 1) == pytest.approx(1 / 3, abs=1e-14)
    a, b, c = 0.7, 2.0, 3.1
    assert aharoni_dz(a, b, c) + aharoni_dz(b, c, a) + aharoni_dz(c, a, b) == pytest.approx(1, abs=1e-13)


@pytest.mark.parametrize("cell", CELLS)
def test_self_term_trace_is_one(cell):
    N = tensor.offset(0, 0, 0, cell)
    assert N[:3].sum() == pytest.approx(1.0, abs=1e-13)
    assert np.all(np.abs(N[3:]) < 1e-14)
    assert np.all(N[:3] > 0)


def test_cube_self_term_is_one_third():
    N = tensor.offset(0, 0, 0, (1.0, 1.0, 1.0))
    assert np.allclose(N[:3], 1 / 3, atol=1e-14)


@pytest.mark.parametrize("cell", CELLS)
def test_off_site_trace_vanishes(cell):
    # Laplace: the potential of a neighbour cell is harmonic in the target cell
    rng = np.random.default_rng(3)
    for _ in range(40):
        i, j, k = rng.integers(-30, 31, size=3)
        if i == j == k == 0:
            continue
        N = tensor.offset(int(i), int(j), int(k), cell)
        assert abs(N[:3].sum()) < 1e-10 * np.abs(N[:3]).max()


def test_reflection_symmetries():
    cell = (1.0, 2.0, 3.0)
    for (i, j, k) in [(1, 2, 3), (2, 0, 1), (5, 3, 2), (9, 4, 11), (1, 1, 0)]:
        base = tensor.offset(i, j, k, cell)
        for sx, sy, sz in [(-1, 1, 1), (1, -1, 1), (1, 1, -1), (-1, -1, -1)]:
            v = tensor.offset(sx * i, sy * j, sz * k, cell)
            par = np.array([(sx if p[0] < 0 else 1) * (sy if p[1] < 0 else 1) * (sz if p[2] < 0 else 1)
                            for p in tensor.PARITY])
            # rounding of the Newell differences near the switch radius reaches ~2e-12
            assert np.abs(v - par * base).max() < 1e-11 * np.abs(base).max()


def test_newell_and_quadrature_agree_on_overlap_band():
    # two independent evaluations of the same cell-pair average
    cell = (1.0, 1.3, 0.8)
    for off in [(4, 1, 0), (3, 3, 2), (5, 2, 1), (6, 0, 3), (2, 5, 2)]:
        X, Y, Z = (o * c for o, c in zip(off, cell))
        a = tensor.newell(X, Y, Z, cell)
        b = tensor.far(X, Y, Z, cell, 10)
        assert np.abs(a - b).max() < 1e-10 * np.abs(a).max()


@pytest.mark.parametrize("cell,order", [((1.0, 1.0, 1.0), 4), ((1.0, 1.0, 2.0), 2)])
def test_far_field_tends_to_point_dipole(cell, order):
    # the cell-pair average differs from the point dipole by the tent's moments times
    # derivatives of the kernel; the second moments are isotropic for a cube and the kernel
    # is harmonic, so cubes converge at fourth order and other cuboids at second order
    direction = np.array([3.0, 2.0, 1.0]) / np.sqrt(14.0)
    V = cell[0] * cell[1] * cell[2]

    def dev(R):
        r = R * direction
        N = tensor.far(*r, cell, 6)
        D = -(V / (4 * np.pi)) * (3 * np.outer(direction, direction) - np.eye(3)) / R ** 3
        Dv = np.array([D[0, 0], D[1, 1], D[2, 2], D[0, 1], D[0, 2], D[1, 2]])
        return np.abs(N - Dv).max() / np.abs(Dv).max()

    d1, d2 = dev(20.0), dev(40.0)
    assert d2 < 1e-3
    assert 0.85 * 2 ** order < d1 / d2 < 1.15 * 2 ** order


@pytest.mark.parametrize("n,cell", [((3, 4, 5), (1.0, 1.2, 0.8)), ((6, 6, 2), (1.0, 1.0, 1.0)),
                                    ((7, 3, 4), (0.5, 1.0, 2.0))])
def test_prism_average_equals_aharoni(n, cell):
    # sum over all cell pairs of a uniformly polarized prism / cell count = prism demag factor
    nx, ny, nz = n
    Nf = tensor.full(n, cell)
    tot = np.zeros(3)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                tot += Nf[:3, z:z + nz, y:y + ny, x:x + nx].sum(axis=(1, 2, 3))
    tot /= nx * ny * nz
    a, b, c = nx * cell[0] / 2, ny * cell[1] / 2, nz * cell[2] / 2
    expect = np.array([aharoni_dz(b, c, a), aharoni_dz(c, a, b), aharoni_dz(a, b, c)])
    assert np.allclose(tot, expect, rtol=1e-11, atol=1e-13)


def test_full_table_matches_direct_offsets():
    n, cell = (4, 3, 5), (1.0, 1.5, 0.7)
    Nf = tensor.full(n, cell)
    for (i, j, k) in [(-3, 2, -4), (0, -2, 1), (3, -1, 0), (-1, -1, -1)]:
        direct = tensor.offset(i, j, k, cell)
        assert np.abs(Nf[:, k + 4, j + 2, i + 3] - direct).max() < 1e-11 * np.abs(direct).max()

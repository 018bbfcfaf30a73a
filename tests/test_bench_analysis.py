"""Host-side analysis used by the Sec. 4.4 experiment modes of bench.py: loop areas and the
topological charge of planar textures, pinned by closed forms (no GPU)."""
import numpy as np
import pytest

import bench


def neel_texture(n=64, R=20.0, core_down=True, center=(31.5, 31.5)):
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    x -= center[0]
    y -= center[1]
    r = np.hypot(x, y)
    th = np.where(r < R, np.pi * (1.0 - r / R), 0.0)
    ph = np.arctan2(y, x)
    p = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    if not core_down:
        p[2] *= -1.0
    return p


def test_loop_area_of_an_ellipse_and_a_rectangle():
    t = np.linspace(0.0, 2.0 * np.pi, 4001)[:-1]
    # polygon inscribed in the ellipse: area pi a b (1 - O(1/n^2))
    assert bench.loop_area(3.0 * np.cos(t), 2.0 * np.sin(t)) == pytest.approx(6.0 * np.pi, rel=1e-5)
    # orientation does not change the area
    assert bench.loop_area(3.0 * np.cos(t), -2.0 * np.sin(t)) == pytest.approx(6.0 * np.pi, rel=1e-5)
    assert bench.loop_area([0, 4, 4, 0], [0, 0, 1.5, 1.5]) == pytest.approx(6.0)
    # a curve traced back along itself encloses nothing
    assert bench.loop_area([0, 1, 2, 1], [0, 1, 2, 1]) == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("R,center", [(20.0, (31.5, 31.5)), (12.0, (25.0, 37.2)), (25.0, (32.0, 30.0))])
def test_topological_charge_of_skyrmions_is_plus_or_minus_one(R, center):
    # a texture uniform along the border has an integer charge; a Neel skyrmion has |Q| = 1, its
    # sign set by the core direction, and a Bloch rotation of the in-plane part keeps Q
    p = neel_texture(R=R, center=center)
    assert bench.topological_charge(p) == pytest.approx(-1.0, abs=1e-9)
    assert bench.topological_charge(neel_texture(R=R, center=center, core_down=False)) == pytest.approx(1.0, abs=1e-9)
    bloch = np.stack([-p[1], p[0], p[2]])
    assert bench.topological_charge(bloch) == pytest.approx(-1.0, abs=1e-9)
    # amplitudes do not matter (the charge uses unit vectors)
    assert bench.topological_charge(0.7 * p) == pytest.approx(-1.0, abs=1e-9)


def test_topological_charge_of_trivial_textures_is_zero():
    n = 48
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    uniform = np.stack([0 * x, 0 * x, 1 + 0 * x])
    assert bench.topological_charge(uniform) == pytest.approx(0.0, abs=1e-12)
    # a 180-degree wall (P_z changes sign across a line) carries no charge
    th = np.pi * (1 + np.tanh((x - 24) / 3.0)) / 2
    wall = np.stack([np.sin(th), 0 * x, np.cos(th)])
    assert bench.topological_charge(wall) == pytest.approx(0.0, abs=1e-12)
    # two skyrmions of opposite core add to zero, two of the same core to two
    a = neel_texture(n=96, R=14.0, center=(25.0, 47.5))
    b = neel_texture(n=96, R=14.0, center=(70.0, 47.5))
    both = a.copy()
    inside_b = np.hypot(*np.mgrid[0:96, 0:96][::-1] - np.array([70.0, 47.5])[:, None, None]) < 14.0
    both[:, inside_b] = b[:, inside_b]
    assert bench.topological_charge(both) == pytest.approx(-2.0, abs=1e-9)


def test_plane_texture_counts_domains_and_curl():
    n = 40
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    # two stripe domains of +-P_z: two domains, no charge, no curl
    stripes = np.stack([0 * x, 0 * x, np.where(x < 20, 0.7, -0.7)])
    t = bench.plane_texture(stripes)
    assert t["domains"] == 2 and t["frac_up"] == pytest.approx(0.5) and t["mean_curl"] == pytest.approx(0.0)
    # an in-plane vortex P = (-y, x) s has curl 2 s per cell in its interior
    s = 0.01
    vortex = np.stack([-(y - 19.5) * s, (x - 19.5) * s, 0.05 + 0 * x])
    assert bench.plane_texture(vortex)["mean_curl"] == pytest.approx(2 * s, rel=1e-12)

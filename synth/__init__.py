"""Seeded synthetic inputs for the TDGL ferroelectric hot path.

This module is shared by the FP64 oracle side and the CUDA side of every test and of the
benchmark. It holds *inputs only*: the raw Table 1 coefficients as printed in the paper, grid
recipes for the benchmark workloads, seeded initial polarization fields and material maps. It
holds none of the method's arithmetic: it never evaluates a coefficient at a temperature, never
computes a field, an energy or a tensor. Each side does that in its own code.

Material records use SI units and the same field names as ``tdgl_material`` in ``include/tdgl.h``:

    alpha1 = a0 * (T - T0)                              (a1_form = 0, linear)
    alpha1 = coth_A * (coth(coth_Ts/T) - coth(coth_Ts/coth_T1))   (a1_form = 1)
    alpha1 = a0                                         (a1_form = 2, temperature independent)
    alpha11  = a11_0  + a11_T  * (T - a11_Tref)
    alpha111 = a111_0 + a111_T * (T - a111_Tref)
    alpha12, alpha112, alpha123, G11, G12, G44, G44p constant;
    r_s scales the z quadratic coefficient (strain form of Sec. 4.4, r_s = 1 means none).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "material", "BTO", "PTO", "STO", "STO_LITERAL", "wall_material",
    "uniform_P", "layer_map", "cylinder_start", "batch_sizes",
    "CONFIG1", "CONFIG2", "CONFIG4", "EPS0",
]

#: vacuum permittivity, F/m (CODATA 2018); a physical constant, not method arithmetic
EPS0 = 8.8541878128e-12


def material(**kw) -> dict:
    """A material record with every field present (defaults: zero coefficients, r_s = 1)."""
    m = dict(a1_form=0, a0=0.0, T0=0.0, coth_A=0.0, coth_Ts=0.0, coth_T1=1.0,
             a11_0=0.0, a11_T=0.0, a11_Tref=0.0, a12=0.0,
             a111_0=0.0, a111_T=0.0, a111_Tref=0.0, a112=0.0, a123=0.0,
             G11=0.0, G12=0.0, G44=0.0, G44p=0.0, r_s=1.0)
    for k, v in kw.items():
        if k not in m:
            raise KeyError(f"unknown material field {k!r}")
        m[k] = v
    return m


# Table 1, BaTiO3 column [46,47]: alpha1 = 3.34e5 (T - 381); alpha11 = 4.69e6 (T - 393) - 2.02e8;
# alpha12 = 3.23e8; alpha111 = -5.52e7 (T - 393) + 2.76e9; alpha112 = 4.47e9; alpha123 = 4.91e9;
# G11 = 5.1e-10, G12 = -2.0e-11, G44 = G'44 = 2.0e-11 (G110 = 5.1e-10).
BTO = material(a0=3.34e5, T0=381.0, a11_0=-2.02e8, a11_T=4.69e6, a11_Tref=393.0, a12=3.23e8,
               a111_0=2.76e9, a111_T=-5.52e7, a111_Tref=393.0, a112=4.47e9, a123=4.91e9,
               G11=5.1e-10, G12=-2.0e-11, G44=2.0e-11, G44p=2.0e-11)

# Table 1, PbTiO3 column [48]: alpha1 = 3.85e5 (T - 752); alpha11 = -7.3e7; alpha12 = 7.5e8;
# alpha111 = 2.6e8; alpha112 = 6.1e8; alpha123 = -3.7e9; G11 = 1.038e-10, G12 = 0,
# G44 = G'44 = 5.19e-11 (G110 = 1.73e-10).
PTO = material(a0=3.85e5, T0=752.0, a11_0=-7.3e7, a12=7.5e8, a111_0=2.6e8, a112=6.1e8,
               a123=-3.7e9, G11=1.038e-10, G12=0.0, G44=5.19e-11, G44p=5.19e-11)

# Table 1, SrTiO3 column [49]: alpha1 printed as 405[coth(54/T) - coth(54/30)] with unit N m^2 C^-2.
# Read as 4.05e7 (garbled exponent: the literal 405 gives a dielectric constant near 3e7); the
# literal value is kept as STO_LITERAL. alpha11 = 1.7e9, alpha12 = 1.37e9; the sixth-order and
# gradient entries are "-" in the table: sixth order set to 0, gradient taken from PbTiO3.
STO = material(a1_form=1, coth_A=4.05e7, coth_Ts=54.0, coth_T1=30.0, a11_0=1.7e9, a12=1.37e9,
               G11=1.038e-10, G12=0.0, G44=5.19e-11, G44p=5.19e-11)
STO_LITERAL = dict(STO, coth_A=405.0)


def wall_material(alpha1=-1.7402e8, alpha11=1.7402e8, G11=0.0, G44=1.73e-10, G44p=1.73e-10) -> dict:
    """The 180-degree wall test material of Sec. 4.1 (alpha1, alpha11 and G44 = G'44 as printed)."""
    return material(a1_form=2, a0=alpha1, a11_0=alpha11, G11=G11, G44=G44, G44p=G44p)


def uniform_P(shape_xyz, amp, seed, dtype=np.float32) -> np.ndarray:
    """Seeded polarization, uniform in [-amp, amp] C/m^2, shape (3, nz, ny, nx), x fastest.

    Drawn with numpy's Philox bit generator; returned in float32 so that both sides start
    from exactly the same values.
    """
    nx, ny, nz = shape_xyz
    g = np.random.Generator(np.random.Philox(seed))
    return g.uniform(-amp, amp, size=(3, nz, ny, nx)).astype(dtype)


def layer_map(shape_xyz, layers) -> np.ndarray:
    """uint8 material map (nz, ny, nx) from [(z0, z1, id), ...] half-open z ranges; rest vacuum."""
    nx, ny, nz = shape_xyz
    m = np.zeros((nz, ny, nx), np.uint8)
    for z0, z1, mid in layers:
        m[z0:z1] = mid
    return m


def cylinder_start(shape_xyz, radius, p_up, noise, seed, z_range=None) -> np.ndarray:
    """Uniform +p_up along z with a centred reversed cylinder (axis z) plus uniform noise."""
    nx, ny, nz = shape_xyz
    P = uniform_P(shape_xyz, noise, seed, np.float64)
    y, x = np.mgrid[0:ny, 0:nx]
    inside = (x - (nx - 1) / 2.0) ** 2 + (y - (ny - 1) / 2.0) ** 2 <= radius ** 2
    z0, z1 = (0, nz) if z_range is None else z_range
    P[2, z0:z1] += np.where(inside, -p_up, p_up)[None]
    return P.astype(np.float32)


def batch_sizes(n=48, choices=(32, 48, 64, 96), seed=0) -> list:
    """Cube edge lengths for the uneven batched sweep: each choice n/len(choices) times, shuffled."""
    per = n // len(choices)
    sizes = [c for c in choices for _ in range(per)]
    g = np.random.Generator(np.random.Philox(seed))
    g.shuffle(sizes)
    return [int(s) for s in sizes]


#: 32x32x8 BaTiO3 thin film, 1 nm cells, +-0.01 C/m^2 start (seed 1), 300 K, eps_B = 45,
#: isotropic gradient (G11 = G44 + G'44 = G110, no cross coupling), zero field, 200 steps.
CONFIG1 = dict(shape=(32, 32, 8), cell=(1e-9, 1e-9, 1e-9), seed=1, amp=0.01, T=300.0, eps_b=45.0,
               material=dict(BTO, G12=0.0, G44=2.55e-10, G44p=2.55e-10), dt_star=0.004, steps=200)

#: 128^3 BaTiO3 cube, 1 nm cells, +-0.01 start (seed 2), full Table 1 gradient, eps_B = 45,
#: temperatures 450 -> 200 K in 25 K steps, relaxation to max|dP| < 1e-6 P0 per step.
CONFIG2 = dict(shape=(128, 128, 128), cell=(1e-9, 1e-9, 1e-9), seed=2, amp=0.01, eps_b=45.0,
               material=BTO, temperatures=[450.0 - 25.0 * i for i in range(11)], tol=1e-6,
               dt_star=0.004)

#: 256x256x64 bilayer: PbTiO3 on top (z 32..63), SrTiO3 below (z 0..31), eps_B = 649, 300 K,
#: reversed cylinder of radius 20 cells, Ez swept +-200 MV/m in 81 points.
CONFIG4 = dict(shape=(256, 256, 64), cell=(1e-9, 1e-9, 1e-9), seed=4, amp=0.01, eps_b=649.0,
               T=300.0, layers=[(0, 32, 2), (32, 64, 1)], radius=20,
               fields=[2e8 - 1e7 * i for i in range(41)] + [-1.9e8 + 1e7 * i for i in range(40)])


def rhombohedral_start(shape_xyz, p, noise, seed) -> np.ndarray:
    """Uniform P along [111] with magnitude p plus uniform noise in [-noise, noise] (heating branch)."""
    P = uniform_P(shape_xyz, noise, seed, np.float64)
    P += p / np.sqrt(3.0)
    return P.astype(np.float32)


def sweep_members(n=48, tmin=180.0, tmax=450.0, seed=0) -> list:
    """Members of the uneven temperature sweep: n/2 temperatures evenly spread in [tmin, tmax],
    a cooling branch (random start) and a heating branch ([111] start), cube edges from
    batch_sizes(n, seed=seed)."""
    sizes = batch_sizes(n, seed=seed)
    half = n // 2
    temps = [tmin + (tmax - tmin) * i / max(half - 1, 1) for i in range(half)]
    out = []
    for b, branch in enumerate(("cooling", "heating")):
        for i, T in enumerate(temps):
            k = b * half + i
            out.append(dict(L=sizes[k], T=T, branch=branch, seed=100 + k))
    return out


#: 64x64x32 PbTiO3-on-SrTiO3 bilayers for the learned warm start: T ~ U(250, 350) K,
#: Ez ~ U(-150, 150) MV/m, thickness ratio t_PTO : t_STO ~ U(0.25, 0.75) of the 32 layers
#: (PbTiO3 on top), eps_B = 649, 1 nm cells, +-0.01 C/m^2 random starts; seed 5, 10 % held out.
CONFIG5 = dict(shape=(64, 64, 32), cell=(1e-9, 1e-9, 1e-9), seed=5, amp=0.01, eps_b=649.0, n=2000,
               held_out=0.1, T=(250.0, 350.0), Ez=(-1.5e8, 1.5e8), ratio=(0.25, 0.75), tol=1e-6,
               dt_star=0.004)


def bilayer_points(n=2000, seed=5, T=(250.0, 350.0), Ez=(-1.5e8, 1.5e8), ratio=(0.25, 0.75), nz=32):
    """Seeded (T, Ez, thickness) points: t_PTO = round(nz r / (1 + r)) layers on top of nz - t_PTO
    SrTiO3 layers, r the PbTiO3:SrTiO3 thickness ratio; each point carries its own start seed."""
    g = np.random.Generator(np.random.Philox(seed))
    out = []
    for i in range(n):
        t, e, r = g.uniform(*T), g.uniform(*Ez), g.uniform(*ratio)
        t_pto = int(round(nz * r / (1.0 + r)))
        out.append(dict(T=float(t), Ez=float(e), ratio=float(r), t_pto=t_pto, seed=10_000 + seed * 100_000 + i))
    return out


def bilayer_map(shape_xyz, t_pto) -> np.ndarray:
    """SrTiO3 (id 2) below, PbTiO3 (id 1) in the top t_pto layers."""
    nz = shape_xyz[2]
    return layer_map(shape_xyz, [(0, nz - t_pto, 2), (nz - t_pto, nz, 1)])


#: The AC hysteresis sample of Sec. 4.4 (Fig. 3): 128 nm x 128 nm, 12 nm SrTiO3 below 20 nm
#: PbTiO3, 1 nm cells, eps_B = 649, 300 K.  The 4 nm vacuum cap of the paper's sample is the open
#: boundary above the grid (P = 0 outside).  Start: +0.7 C/m^2 along z in PbTiO3 plus +-0.01 C/m^2
#: noise (seed 6).  Out-of-plane field of amplitude 400 MV/m (the DC loop spans about +-400 MV/m);
#: the AC frequencies span the paper's 0.0017 - 0.174 MHz; the DC loop steps 20 MV/m.
CONFIG_AC = dict(shape=(128, 128, 32), cell=(1e-9, 1e-9, 1e-9), seed=6, amp=0.01, p_up=0.7, eps_b=649.0,
                 T=300.0, layers=[(0, 12, 2), (12, 32, 1)], E0=4e8,
                 freqs_mhz=[0.174, 0.0552, 0.0174, 0.0055, 0.0017],
                 dc_fields=[4e8 - 2e7 * i for i in range(41)] + [-3.8e8 + 2e7 * i for i in range(40)])

#: PbTiO3 with the gradient coefficients of the strain-skyrmion study (Sec. 4.4, Ref. [36]):
#: G11 = 3.46e-10, G12 = 0, G44 = G'44 = 1.73e-10 N m^4 C^-2; Landau terms of Table 1.
PTO_SKX = dict(PTO, G11=3.46e-10, G12=0.0, G44=1.73e-10, G44p=1.73e-10)
#: SrTiO3 of Table 1 with the same gradient coefficients (its Table 1 entries are blank).
STO_SKX = dict(STO, G11=3.46e-10, G12=0.0, G44=1.73e-10, G44p=1.73e-10)

#: The strain-skyrmion sample of Sec. 4.4 (Fig. 4): 40 x 40 x 32 nm^3 PbTiO3 on a 40 x 40 x 8 nm^3
#: SrTiO3 layer in vacuum, 0.5 nm cells (80 x 80 x 80), 300 K, eps_B = 45 (the paper gives none for
#: this sample; 45 is its PbTiO3 cube value), r_s = 1.0 ... 1.8 applied to PbTiO3, each r_s starting
#: from the state relaxed at the one before, the first from a +-0.01 C/m^2 random start (seed 7).
CONFIG_SKX = dict(shape=(80, 80, 80), cell=(0.5e-9, 0.5e-9, 0.5e-9), seed=7, amp=0.01, eps_b=45.0, T=300.0,
                  layers=[(0, 16, 2), (16, 80, 1)], r_s=[1.0 + 0.1 * i for i in range(9)])

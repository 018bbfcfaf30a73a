"""Material presets for users of the library (Table 1 of the paper, SI units).

Field names are those of ``tdgl_material`` (include/tdgl.h).  SrTiO3's alpha1 prefactor is read
as 4.05e7 N m^2 C^-2 (Table 1 prints "405", which gives an unphysical permittivity); its
sixth-order and gradient entries are blank in Table 1 and are set to 0 and to the PbTiO3
gradient coefficients respectively.
"""
from __future__ import annotations


def material(**kw) -> dict:
    rec = dict(a1_form=0, a0=0.0, T0=0.0, coth_A=0.0, coth_Ts=0.0, coth_T1=1.0, a11_0=0.0, a11_T=0.0,
               a11_Tref=0.0, a12=0.0, a111_0=0.0, a111_T=0.0, a111_Tref=0.0, a112=0.0, a123=0.0,
               G11=0.0, G12=0.0, G44=0.0, G44p=0.0, r_s=1.0)
    unknown = set(kw) - set(rec)
    if unknown:
        raise KeyError(f"unknown material fields {sorted(unknown)}")
    rec.update(kw)
    return rec


# Table 1, BaTiO3
BTO = material(a0=3.34e5, T0=381.0, a11_0=-2.02e8, a11_T=4.69e6, a11_Tref=393.0, a12=3.23e8,
               a111_0=2.76e9, a111_T=-5.52e7, a111_Tref=393.0, a112=4.47e9, a123=4.91e9,
               G11=5.1e-10, G12=-2.0e-11, G44=2.0e-11, G44p=2.0e-11)
# Table 1, PbTiO3
PTO = material(a0=3.85e5, T0=752.0, a11_0=-7.3e7, a12=7.5e8, a111_0=2.6e8, a112=6.1e8, a123=-3.7e9,
               G11=1.038e-10, G44=5.19e-11, G44p=5.19e-11)
# Table 1, SrTiO3 (see module docstring for the readings)
STO = material(a1_form=1, coth_A=4.05e7, coth_Ts=54.0, coth_T1=30.0, a11_0=1.7e9, a12=1.37e9,
               G11=1.038e-10, G44=5.19e-11, G44p=5.19e-11)

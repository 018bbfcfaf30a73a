"""ORACLE (test infrastructure).  Table 1 coefficients evaluated at a temperature.

Follows Table 1 (the temperature forms of alpha1, alpha11, alpha111) and the strain form of
Sec. 4.4, where the quadratic term is written (T - Tc)(alpha0 (Px^2 + Py^2) + r_s alpha0 Pz^2):
the z quadratic coefficient is r_s * alpha1.
"""
from __future__ import annotations

import math


def alpha1(m: dict, T: float) -> float:
    """alpha1(T) for the three forms of a material record (linear, coth, constant)."""
    form = int(m["a1_form"])
    if form == 0:
        return m["a0"] * (T - m["T0"])
    if form == 1:
        coth = lambda v: math.cosh(v) / math.sinh(v)
        return m["coth_A"] * (coth(m["coth_Ts"] / T) - coth(m["coth_Ts"] / m["coth_T1"]))
    if form == 2:
        return m["a0"]
    raise ValueError(f"unknown alpha1 form {form}")


def coefficients(m: dict, T: float) -> dict:
    """All Landau and gradient coefficients of one material at temperature T (SI)."""
    a1 = alpha1(m, T)
    return dict(
        a1x=a1, a1y=a1, a1z=m["r_s"] * a1,
        a11=m["a11_0"] + m["a11_T"] * (T - m["a11_Tref"]),
        a12=m["a12"],
        a111=m["a111_0"] + m["a111_T"] * (T - m["a111_Tref"]),
        a112=m["a112"], a123=m["a123"],
        G11=m["G11"], G12=m["G12"], G44=m["G44"], G44p=m["G44p"],
    )

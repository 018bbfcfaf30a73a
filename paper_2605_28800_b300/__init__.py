"""B300-native explicit TDGL (Landau-Khalatnikov) step for ferroelectric polarization.

The compute path is libtdgl.so (hand-written CUDA for sm_103a, C ABI in include/tdgl.h);
``tdgl`` is its thin ctypes binding.  Material presets follow Table 1 of the paper.
"""
from . import tdgl
from .tdgl import Batch, Context, Sim, TdglError, TERM_ALL, TERM_ELEC, TERM_EXT, TERM_GRAD, TERM_LANDAU
from .materials import BTO, PTO, STO, material

__all__ = ["tdgl", "Batch", "Context", "Sim", "TdglError", "TERM_ALL", "TERM_ELEC", "TERM_EXT", "TERM_GRAD",
           "TERM_LANDAU", "BTO", "PTO", "STO", "material"]

"""FP64 CPU oracle for one explicit TDGL (Landau-Khalatnikov) step of a ferroelectric polarization field.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or execute anything in this package.  The
product path (``paper_2605_28800_b300``) never imports it and shares no code with it.

It computes, in SI units and float64, exactly the discrete system that the CUDA path computes in
normalized float32:

* ``material.coefficients``  Table 1 coefficients evaluated at a temperature (with the strain
  form of Sec. 4.4 for the z quadratic term).
* ``landau``                 Eq. 3 energy density and its field -dF/dP.
* ``gradient``               a discrete form of Eq. 4 (faces + central-difference cross terms
                             with mirror ghosts at free surfaces) and its exact field.
* ``tensor`` / ``electrostatics``  Eqs. 5-6: the cell-averaged interaction tensor (Newell
                             near field, Gauss-Legendre far field) and the field as a direct
                             O(N^2) sum or as a zero-padded FFT convolution (numpy FFT).
* ``system.System``          Eq. 2 total field and energy, the forward Euler step of Eq. 1 with
                             L = 1, and a relaxation loop.

Parity status: every function is pinned by a ``-m "not gpu"`` test against closed forms,
brute force or paper-printed values (see tests/test_oracle_*.py).
"""
from .material import coefficients
from .system import System, TERM_LANDAU, TERM_GRAD, TERM_ELEC, TERM_EXT, TERM_ALL

__all__ = ["coefficients", "System", "TERM_LANDAU", "TERM_GRAD", "TERM_ELEC", "TERM_EXT", "TERM_ALL"]

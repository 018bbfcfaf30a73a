"""ORACLE (test infrastructure).  Total field, energies and the explicit TDGL step.

Eq. 2: F = F_Land + F_Grad + F_Elec + F_Ext; Eq. 7: F_Ext = -int E_ext . P, so the external
field enters the effective field as +E_ext.  A time-dependent excitation (Sec. 3; the AC loops of
Sec. 4.4) is E_ext(t) = E_ext + E_ac sin(2 pi f t + phase), taken at the time of each step.  Eq. 1 with L = 1 (Sec. 2), integrated with the
forward Euler rule (the simplest of the explicit schemes named in Sec. 3; Heun, RK45 and AB3M2
below are the three the paper lists):
    P <- P + dt * L * (h_Land + h_Grad + E_el + E_ext)      on material cells;
vacuum cells keep P = 0 (Sec. 2: P = 0 outside the sample).
"""
from __future__ import annotations

import numpy as np

from . import electrostatics as _es
from . import gradient as _grad
from . import landau as _landau
from . import tensor as _tensor
from .material import coefficients

TERM_LANDAU, TERM_GRAD, TERM_ELEC, TERM_EXT = 1, 2, 4, 8
TERM_ALL = 15
_COEF_KEYS = ("a1x", "a1y", "a1z", "a11", "a12", "a111", "a112", "a123", "G11", "G12", "G44", "G44p")


class System:
    """A finite sample on an (nx, ny, nz) grid of (dx, dy, dz) cells, SI units, float64.

    mat: uint8 (nz, ny, nx) material ids (0 = vacuum); materials: {id: material record}.
    conv: 'fft' (zero-padded FFT) or 'direct' (O(N^2) sum) for the electrostatic field.
    """

    def __init__(self, shape, cell, mat, materials, T, eps_b=1.0, E_ext=(0.0, 0.0, 0.0),
                 terms=TERM_ALL, conv="fft", octant=None, L=1.0, E_ac=(0.0, 0.0, 0.0), freq=0.0,
                 phase=0.0):
        self.shape = tuple(int(v) for v in shape)
        self.cell = tuple(float(v) for v in cell)
        nx, ny, nz = self.shape
        self.mat = np.asarray(mat, dtype=np.uint8).reshape(nz, ny, nx)
        self.m = self.mat > 0
        self.materials = dict(materials)
        self.eps_b = float(eps_b)
        self.E_ext = np.asarray(E_ext, dtype=np.float64).reshape(3)
        self.E_ac = np.asarray(E_ac, dtype=np.float64).reshape(3)
        self.freq, self.phase = float(freq), float(phase)
        self.terms = int(terms)
        self.L = float(L)
        self.V = self.cell[0] * self.cell[1] * self.cell[2]
        self.conv = conv
        self._octant = octant
        self._convolver = None
        self._Nfull = None
        self.set_temperature(T)

    # -- parameters -------------------------------------------------------------------------
    def set_temperature(self, T):
        self.T = float(T)
        self.coef = {k: np.zeros(self.mat.shape) for k in _COEF_KEYS}
        for mid, rec in self.materials.items():
            sel = self.mat == mid
            if not np.any(sel):
                continue
            c = coefficients(rec, self.T)
            for k in _COEF_KEYS:
                self.coef[k][sel] = c[k]

    def _tensor_octant(self):
        if self._octant is None:
            self._octant = _tensor.octant(self.shape, self.cell)
        return self._octant

    def applied_field(self, t=0.0):
        """E_ext(t), V/m (3,)."""
        return self.E_ext + self.E_ac * np.sin(2.0 * np.pi * self.freq * t + self.phase)

    # -- fields -----------------------------------------------------------------------------
    def electrostatic_field(self, P):
        P = np.asarray(P, dtype=np.float64)
        if self.conv == "direct":
            if self._Nfull is None:
                self._Nfull = _tensor.full(self.shape, self.cell, self._tensor_octant())
            return _es.direct(P, self._Nfull, self.eps_b)
        if self._convolver is None:
            self._convolver = _es.FFTConvolver(self.shape, self.cell, self._tensor_octant())
        return self._convolver.apply(P, self.eps_b)

    def fields(self, P, t=0.0):
        """Dict of the four field contributions and their sum at time t, each (3, nz, ny, nx), V/m."""
        P = np.asarray(P, dtype=np.float64)
        z = np.zeros(P.shape)
        out = {"landau": z, "grad": z, "elec": z, "ext": z}
        if self.terms & TERM_LANDAU:
            out["landau"] = np.where(self.m, _landau.field(P, self.coef), 0.0)
        if self.terms & TERM_GRAD:
            out["grad"], _ = _grad.field_and_energy(P, self.mat, self.coef, self.cell)
        if self.terms & TERM_ELEC:
            out["elec"] = self.electrostatic_field(P)
        if self.terms & TERM_EXT:
            out["ext"] = np.where(self.m, self.applied_field(t)[:, None, None, None], 0.0)
        out["total"] = np.where(self.m, out["landau"] + out["grad"] + out["elec"] + out["ext"], 0.0)
        return out

    def energy(self, P, t=0.0):
        """Energy terms of Eq. 2 in joules at time t: land, grad, elec, ext, total."""
        P = np.asarray(P, dtype=np.float64)
        e = dict(land=0.0, grad=0.0, elec=0.0, ext=0.0)
        if self.terms & TERM_LANDAU:
            e["land"] = self.V * float(np.sum(np.where(self.m, _landau.energy_density(P, self.coef), 0.0)))
        if self.terms & TERM_GRAD:
            _, e["grad"] = _grad.field_and_energy(P, self.mat, self.coef, self.cell)
        if self.terms & TERM_ELEC:
            e["elec"] = _es.energy(self.electrostatic_field(P), P, self.V)
        if self.terms & TERM_EXT:
            e["ext"] = -self.V * float(np.sum(np.where(self.m, np.tensordot(self.applied_field(t), P, 1), 0.0)))
        e["total"] = e["land"] + e["grad"] + e["elec"] + e["ext"]
        return e

    # -- dynamics ---------------------------------------------------------------------------
    def step(self, P, dt, t=0.0):
        """One forward Euler step of Eq. 1 from time t; returns the new P (float64)."""
        P = np.asarray(P, dtype=np.float64)
        Pn = P + dt * self.L * self.fields(P, t)["total"]
        return np.where(self.m, Pn, 0.0)

    def heun_step(self, P, dt, t=0.0):
        """One step of Heun's method (Sec. 3): predictor P~ = P + dt h(P, t), then
        P + dt/2 (h(P, t) + h(P~, t + dt))."""
        P = np.asarray(P, dtype=np.float64)
        h0 = self.fields(P, t)["total"]
        Pt = np.where(self.m, P + dt * self.L * h0, 0.0)
        h1 = self.fields(Pt, t + dt)["total"]
        return np.where(self.m, P + 0.5 * dt * self.L * (h0 + h1), 0.0)

    # Runge-Kutta-Fehlberg 4(5) (Fehlberg 1969): nodes, stage matrix, fourth- and fifth-order weights
    RKF_C = (0.0, 1 / 4, 3 / 8, 12 / 13, 1.0, 1 / 2)
    RKF_A = ((), (1 / 4,), (3 / 32, 9 / 32), (1932 / 2197, -7200 / 2197, 7296 / 2197),
             (439 / 216, -8.0, 3680 / 513, -845 / 4104), (-8 / 27, 2.0, -3544 / 2565, 1859 / 4104, -11 / 40))
    RKF_B4 = (25 / 216, 0.0, 1408 / 2565, 2197 / 4104, -1 / 5, 0.0)
    RKF_B5 = (16 / 135, 0.0, 6656 / 12825, 28561 / 56430, -9 / 50, 2 / 55)

    def rkf45_step(self, P, dt, t=0.0):
        """One Runge-Kutta-Fehlberg step (the RK45 of Sec. 3): returns (P4, P5), the fourth-order
        solution that advances and the fifth-order one whose difference estimates the local error."""
        P = np.asarray(P, dtype=np.float64)
        k = []
        for i in range(6):
            Pi = P + dt * self.L * sum(a * kj for a, kj in zip(self.RKF_A[i], k)) if i else P
            k.append(self.fields(np.where(self.m, Pi, 0.0), t + self.RKF_C[i] * dt)["total"])
        P4 = P + dt * self.L * sum(b * kj for b, kj in zip(self.RKF_B4, k))
        P5 = P + dt * self.L * sum(b * kj for b, kj in zip(self.RKF_B5, k))
        return np.where(self.m, P4, 0.0), np.where(self.m, P5, 0.0)

    def ab3m2_run(self, P, dt, n, t0=0.0):
        """n steps of the Adams pair (the AB3M2 of Sec. 3) in predict-evaluate-correct-evaluate
        form: predictor Adams-Bashforth with the newest q = min(step + 1, 3) derivatives,
        corrector Adams-Moulton with q - 1 past derivatives (the trapezoid rule on the first step,
        so that step is Heun's method), then the derivative at the new state."""
        P = np.asarray(P, dtype=np.float64)
        f = lambda Q, t: self.fields(np.where(self.m, Q, 0.0), t)["total"]
        hist = [f(P, t0)]                                   # newest first
        AB = {1: (1.0,), 2: (3 / 2, -1 / 2), 3: (23 / 12, -16 / 12, 5 / 12)}
        AM = {1: (1 / 2, 1 / 2), 2: (5 / 12, 8 / 12, -1 / 12), 3: (5 / 12, 8 / 12, -1 / 12)}
        for i in range(n):
            t = t0 + i * dt
            q = len(hist)
            Pp = P + dt * self.L * sum(c * h for c, h in zip(AB[q], hist))
            fs = f(Pp, t + dt)
            P = np.where(self.m, P + dt * self.L * sum(c * h for c, h in zip(AM[q], [fs] + hist)), 0.0)
            hist = [f(P, t + dt)] + hist[:2]
        return P

    def run(self, P, dt, n, t0=0.0, method="euler"):
        if method == "ab3m2":
            return self.ab3m2_run(P, dt, n, t0)
        if method == "rk45":
            f = lambda Q, dt_, t: self.rkf45_step(Q, dt_, t)[0]
        else:
            f = self.heun_step if method == "heun" else self.step
        for i in range(n):
            P = f(P, dt, t0 + i * dt)
        return P

    def relax(self, P, dt, tol, P0, max_steps, check_every=16):
        """Step until max|P_new - P| / P0 < tol on a checked step (every check_every steps).

        Returns (P, steps_taken, converged)."""
        P = np.asarray(P, dtype=np.float64)
        steps = 0
        while steps < max_steps:
            Pn = self.step(P, dt)
            steps += 1
            if steps % check_every == 0 or steps == max_steps:
                if float(np.max(np.abs(Pn - P))) / P0 < tol:
                    return Pn, steps, True
            P = Pn
        return P, steps, False

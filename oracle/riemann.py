"""Exact Riemann solver for the frozen limit of the model.

TEST INFRASTRUCTURE ONLY.

With Q = I = 0 and 1/tau = 0, eqs. 1-4 reduce to the Euler equations of an
ideal gas (gamma) plus a passively advected vibrational energy: E_nu / rho is
constant along particle paths, so it jumps only at the contact.  The solver
below is written from the gas-dynamics mathematics of the Riemann problem:

* the star pressure p* solves f_L(p) + f_R(p) + (u_R - u_L) = 0 with
  f_K(p) = (p - p_K) sqrt(A_K / (p + B_K)),  A_K = 2 / ((gamma+1) rho_K),
           B_K = (gamma-1)/(gamma+1) p_K                 (shock, p > p_K)
  f_K(p) = 2 c_K / (gamma-1) [(p/p_K)^((gamma-1)/(2 gamma)) - 1]  (rarefaction);
* u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2;
* shock densities from the Rankine-Hugoniot adiabat, fan states from the
  isentrope and the Riemann invariant u +- 2c/(gamma-1).
"""
from __future__ import annotations

import math

import numpy as np


class Riemann:
    def __init__(self, gamma, rhoL, uL, pL, rhoR, uR, pR, evL=0.0, evR=0.0):
        self.g = gamma
        self.L = (rhoL, uL, pL)
        self.R = (rhoR, uR, pR)
        self.ev = (evL, evR)           # specific vibrational energy each side
        self.cL = math.sqrt(gamma * pL / rhoL)
        self.cR = math.sqrt(gamma * pR / rhoR)
        if 2.0 * (self.cL + self.cR) / (gamma - 1.0) <= uR - uL:
            raise ValueError("vacuum is generated; not handled")
        self.pstar, self.ustar = self._star()

    def _f(self, p, rhoK, pK, cK):
        g = self.g
        if p > pK:
            A = 2.0 / ((g + 1.0) * rhoK)
            B = (g - 1.0) / (g + 1.0) * pK
            s = math.sqrt(A / (p + B))
            return (p - pK) * s, s * (1.0 - 0.5 * (p - pK) / (B + p))
        e = (g - 1.0) / (2.0 * g)
        return (2.0 * cK / (g - 1.0)) * ((p / pK) ** e - 1.0), (p / pK) ** (-(g + 1.0) / (2.0 * g)) / (rhoK * cK)

    def _star(self):
        (rL, uL, pL), (rR, uR, pR) = self.L, self.R
        du = uR - uL
        # two-rarefaction initial guess
        g = self.g
        z = (g - 1.0) / (2.0 * g)
        p = ((self.cL + self.cR - 0.5 * (g - 1.0) * du) /
             (self.cL / pL ** z + self.cR / pR ** z)) ** (1.0 / z)
        p = max(p, 1e-12)
        for _ in range(100):
            fL, dL = self._f(p, rL, pL, self.cL)
            fR, dR = self._f(p, rR, pR, self.cR)
            pn = p - (fL + fR + du) / (dL + dR)
            pn = max(pn, 1e-14)
            if abs(pn - p) <= 1e-15 * (pn + p):
                p = pn
                break
            p = pn
        fL, _ = self._f(p, rL, pL, self.cL)
        fR, _ = self._f(p, rR, pR, self.cR)
        return p, 0.5 * (uL + uR) + 0.5 * (fR - fL)

    def star_densities(self):
        g = self.g
        out = []
        for (rK, uK, pK) in (self.L, self.R):
            ratio = self.pstar / pK
            if self.pstar > pK:
                gm = (g - 1.0) / (g + 1.0)
                out.append(rK * (ratio + gm) / (gm * ratio + 1.0))
            else:
                out.append(rK * ratio ** (1.0 / g))
        return tuple(out)

    def wave_speeds(self):
        """(left wave head, left wave tail, contact, right tail, right head);
        for a shock head == tail == the shock speed."""
        g = self.g
        rsL, rsR = self.star_densities()
        (rL, uL, pL), (rR, uR, pR) = self.L, self.R
        if self.pstar > pL:
            sL = uL - self.cL * math.sqrt((g + 1) / (2 * g) * self.pstar / pL + (g - 1) / (2 * g))
            lh = lt = sL
        else:
            lh = uL - self.cL
            lt = self.ustar - math.sqrt(g * self.pstar / rsL)
        if self.pstar > pR:
            sR = uR + self.cR * math.sqrt((g + 1) / (2 * g) * self.pstar / pR + (g - 1) / (2 * g))
            rh = rt = sR
        else:
            rh = uR + self.cR
            rt = self.ustar + math.sqrt(g * self.pstar / rsR)
        return lh, lt, self.ustar, rt, rh

    def sample(self, xi: float):
        """Primitive state (rho, u, p, e_nu) at similarity coordinate xi = x / t."""
        g = self.g
        rsL, rsR = self.star_densities()
        lh, lt, c, rt, rh = self.wave_speeds()
        if xi < c:
            rK, uK, pK = self.L
            cK = self.cL
            ev = self.ev[0]
            if xi < lh:
                return rK, uK, pK, ev
            if xi >= lt:
                return rsL, self.ustar, self.pstar, ev
            # inside the left fan
            u = 2.0 / (g + 1.0) * (cK + 0.5 * (g - 1.0) * uK + xi)
            cc = 2.0 / (g + 1.0) * (cK + 0.5 * (g - 1.0) * (uK - xi))
            rho = rK * (cc / cK) ** (2.0 / (g - 1.0))
            return rho, u, pK * (cc / cK) ** (2.0 * g / (g - 1.0)), ev
        rK, uK, pK = self.R
        cK = self.cR
        ev = self.ev[1]
        if xi > rh:
            return rK, uK, pK, ev
        if xi <= rt:
            return rsR, self.ustar, self.pstar, ev
        u = 2.0 / (g + 1.0) * (-cK + 0.5 * (g - 1.0) * uK + xi)
        cc = 2.0 / (g + 1.0) * (cK - 0.5 * (g - 1.0) * (uK - xi))
        rho = rK * (cc / cK) ** (2.0 / (g - 1.0))
        return rho, u, pK * (cc / cK) ** (2.0 * g / (g - 1.0)), ev

    def sample_array(self, xi: np.ndarray) -> np.ndarray:
        return np.array([self.sample(float(x)) for x in np.ravel(xi)]).T

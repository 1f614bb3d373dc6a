"""Static spherical star (Tolman-Oppenheimer-Volkoff): initial data for the
fluid tests and the benchmark, computed with scipy (it holds none of the
evolution's arithmetic): the TOV equations in the areal radius r for a cold polytrope P = K rho^Gamma, eps = K rho^(Gamma-1) /
(Gamma-1), together with d ln rbar / dr = 1 / (r sqrt(1 - 2m/r)) for the
isotropic radius rbar, matched at the surface R to the exterior
Schwarzschild solution in isotropic coordinates (rbar(R) = (sqrt(R^2 - 2MR)
+ R - M)/2, alpha = e^nu with nu(R) = ln(1 - 2M/R)/2).  In isotropic
coordinates gamma_ij = psi^4 delta_ij with psi^2 = r / rbar."""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp
from scipy.interpolate import CubicSpline


class TOV:
    def __init__(self, rho_c=1.28e-3, K=100.0, Gamma=2.0):
        self.K, self.G = K, Gamma
        Pc = K * rho_c ** Gamma

        def rhs(r, y):
            P, m, nu, lrb = y
            P = max(P, 0.0)
            rho = (P / K) ** (1.0 / Gamma)
            e = rho + P / (Gamma - 1.0)
            den = r * (r - 2.0 * m)
            dnu = (m + 4.0 * math.pi * r ** 3 * P) / den
            return [-(e + P) * dnu, 4.0 * math.pi * r * r * e, dnu, 1.0 / (r * math.sqrt(1.0 - 2.0 * m / r))]

        def surface(r, y):
            return y[0] - 1e-14 * Pc
        surface.terminal = True
        r0 = 1e-6
        e_c = rho_c + Pc / (Gamma - 1.0)
        y0 = [Pc, 4.0 / 3.0 * math.pi * r0 ** 3 * e_c, 0.0, math.log(r0)]
        sol = solve_ivp(rhs, (r0, 50.0), y0, events=surface, rtol=1e-12, atol=1e-16, dense_output=True,
                        max_step=0.01)
        R = sol.t_events[0][0]
        yR = sol.y_events[0][0]
        M = yR[1]
        self.R, self.M = R, M
        rbR = 0.5 * (math.sqrt(R * R - 2.0 * M * R) + R - M)
        dnu = 0.5 * math.log(1.0 - 2.0 * M / R) - yR[2]
        dlrb = math.log(rbR) - yR[3]
        r = np.linspace(r0, R, 20001)
        Y = sol.sol(r)
        rb = np.exp(Y[3] + dlrb)
        self.Rbar = rbR
        P = np.maximum(Y[0], 0.0)
        self._rho = CubicSpline(rb, (P / K) ** (1.0 / Gamma))
        self._psi2 = CubicSpline(rb, r / rb)
        self._nu = CubicSpline(rb, Y[2] + dnu)

    def fields(self, rbar):
        """(rho, psi, alpha) at isotropic radii rbar (array)."""
        rbar = np.asarray(rbar, dtype=np.float64)
        inside = rbar < self.Rbar
        rc = np.clip(rbar, 1e-6, self.Rbar)
        rho = np.where(inside, np.maximum(self._rho(rc), 0.0), 0.0)
        psi = np.where(inside, np.sqrt(self._psi2(rc)), 1.0 + self.M / (2.0 * np.maximum(rbar, 1e-12)))
        ha = self.M / (2.0 * np.maximum(rbar, 1e-12))
        alpha = np.where(inside, np.exp(self._nu(rc)), (1.0 - ha) / (1.0 + ha))
        return rho, psi, alpha


def tov_patch_data(p, star=None, rho_floor=None, centre=(0.0, 0.0, 0.0)):
    """Z4c fields (isotropic coordinates: W = psi^-2, conformally flat, the
    static lapse, zero shift and extrinsic curvature) and fluid primitives
    (rho, eps on the cold polytrope, at rest) of the star centred at `centre`
    on patch p; rho is at least rho_floor (an array or number) outside the
    star."""
    import initial_data as idd
    star = star or TOV()
    z, y, x = np.meshgrid(p.axis(2) - centre[2], p.axis(1) - centre[1], p.axis(0) - centre[0], indexing="ij")
    rho, psi, al = star.fields(np.sqrt(x * x + y * y + z * z))
    u = idd.minkowski(p)
    u[0] = psi ** -2
    u[18] = al
    prim = np.zeros((5,) + p.shape[1:])
    prim[0] = np.maximum(rho, rho_floor if rho_floor is not None else 0.0)
    prim[1] = star.K * prim[0] ** (star.G - 1.0) / (star.G - 1.0)
    return u, prim

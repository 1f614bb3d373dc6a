"""Exact solution of the special-relativistic Riemann problem of an ideal gas
P = (G - 1) rho eps with no tangential velocity, written for the tests from
the definitions (no code shared with the oracle):

* across a rarefaction the flow is an isentropic simple wave, P = K rho^G,
  with dv/dP = -/+ (1 - v^2) / (rho h c_s) for the wave moving to the left /
  right (h = 1 + eps + P/rho, c_s^2 = G P / (rho h)); inside the fan the
  state at x/t = xi is the one whose characteristic speed (v -/+ c_s) /
  (1 -/+ v c_s) equals xi;
* across a shock of speed V the Rankine-Hugoniot conditions hold for the
  fluxes of D = rho W, S = rho h W^2 v and tau = rho h W^2 - P - D in the
  frame of the lab: [D (v - V)] = 0, [S (v - V) + P] = 0,
  [(tau + D)(v - V) + P v] = 0; at a given post-shock pressure they give
  the post-shock (rho, v) and V in closed form (the Taub adiabat and the
  mass flux through the shock);
* the intermediate pressure is the root of v*_L(P) - v*_R(P); the contact
  moves with v*.
"""
import math

import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq


class Gas:
    def __init__(self, G):
        self.G = G

    def h(self, rho, P):
        return 1.0 + self.G / (self.G - 1.0) * P / rho

    def cs(self, rho, P):
        return math.sqrt(self.G * P / (rho * self.h(rho, P)))


def _rarefaction_v(gas, rho0, P0, v0, P, sign):
    """Velocity behind a rarefaction reaching pressure P (sign -1: the wave
    moves left, +1: right)."""
    K = P0 / rho0 ** gas.G

    def rhs(lp, y):
        p = math.exp(lp)
        rho = (p / K) ** (1.0 / gas.G)
        return [sign * p * (1.0 - y[0] ** 2) / (rho * gas.h(rho, p) * gas.cs(rho, p))]
    if P == P0:
        return v0
    sol = solve_ivp(rhs, (math.log(P0), math.log(P)), [v0], method="DOP853", rtol=1e-12, atol=1e-14)
    return float(sol.y[0, -1])


def _shock(gas, rho0, P0, v0, P, sign):
    """Post-shock (rho, v) and shock speed V for post-shock pressure P > P0.

    The jump conditions give the Taub adiabat [h^2] = (h0/rho0 + h/rho)[P],
    quadratic in h for the ideal gas (rho = G P / ((G - 1)(h - 1))); the
    invariant mass flux j = W_V rho W (V - v), the same on both sides, has
    j^2 = [P] / (h0/rho0 - h/rho) and the sign of the wave; j on the
    upstream side is quadratic in V, and on the downstream side gives v.
    The momentum and energy conditions are then checked as residuals."""
    G = gas.G
    h0 = gas.h(rho0, P0)
    dp = P - P0
    k = (G - 1.0) * dp / (G * P)
    c = h0 * h0 + h0 * dp / rho0
    h = (-k + math.sqrt(k * k + 4.0 * (1.0 - k) * c)) / (2.0 * (1.0 - k))
    rho = G * P / ((G - 1.0) * (h - 1.0))
    j2 = dp / (h0 / rho0 - h / rho)
    j = sign * math.sqrt(j2)
    W0 = 1.0 / math.sqrt(1.0 - v0 * v0)
    D0 = rho0 * W0
    V = (D0 * D0 * v0 + sign * math.sqrt(j2) * math.sqrt(j2 + rho0 * rho0)) / (D0 * D0 + j2)
    WV = 1.0 / math.sqrt(1.0 - V * V)
    q = j / (WV * rho)
    v = (V - q * math.sqrt(1.0 + q * q - V * V)) / (1.0 + q * q)

    def flux(r, u, p):
        W = 1.0 / math.sqrt(1.0 - u * u)
        hh = gas.h(r, p)
        return np.array([r * W * (u - V), r * hh * W * W * u * (u - V) + p,
                         (r * hh * W * W - p) * (u - V) + p * u])
    f0, f1 = flux(rho0, v0, P0), flux(rho, v, P)
    scale = np.abs(f0).max() + np.abs(f1).max()
    if np.abs(f1 - f0).max() > 1e-10 * scale:
        raise RuntimeError("shock conditions not met")
    return rho, v, V


def _side_v(gas, state, P, sign):
    rho0, P0, v0 = state
    if P <= P0:
        return _rarefaction_v(gas, rho0, P0, v0, P, sign)
    return _shock(gas, rho0, P0, v0, P, sign)[1]


def solve(gas, left, right):
    """left, right = (rho, P, v).  Returns a function of xi = x/t giving
    (rho, P, v) and the intermediate pressure and velocity."""
    f = lambda P: _side_v(gas, left, P, -1.0) - _side_v(gas, right, P, 1.0)
    lo, hi = 1e-6 * min(left[1], right[1]), 10.0 * max(left[1], right[1])
    Ps = brentq(f, lo, hi, xtol=1e-14, rtol=1e-13)
    vs = _side_v(gas, left, Ps, -1.0)

    def star_rho(state, sign):
        rho0, P0, v0 = state
        if Ps <= P0:
            return rho0 * (Ps / P0) ** (1.0 / gas.G)
        return _shock(gas, rho0, P0, v0, Ps, sign)[0]

    rhoL_s, rhoR_s = star_rho(left, -1.0), star_rho(right, 1.0)

    def lam(rho, P, v, sign):
        c = gas.cs(rho, P)
        return (v + sign * c) / (1.0 + sign * v * c)

    def side(state, sign, rho_s, xi):
        rho0, P0, v0 = state
        if Ps <= P0:  # rarefaction: head at the outer state's speed, tail at the star state's
            head = lam(rho0, P0, v0, sign)
            tail = lam(rho_s, Ps, vs, sign)
            if (xi - head) * sign >= 0:
                return rho0, P0, v0
            if (xi - tail) * sign <= 0:
                return rho_s, Ps, vs
            K = P0 / rho0 ** gas.G
            g = lambda p: lam((p / K) ** (1.0 / gas.G), p, _rarefaction_v(gas, rho0, P0, v0, p, sign), sign) - xi
            p = brentq(g, min(Ps, P0), max(Ps, P0), xtol=1e-14)
            return (p / K) ** (1.0 / gas.G), p, _rarefaction_v(gas, rho0, P0, v0, p, sign)
        V = _shock(gas, rho0, P0, v0, Ps, sign)[2]
        if (xi - V) * sign >= 0:
            return rho0, P0, v0
        return rho_s, Ps, vs

    def at(xi):
        if xi < vs:
            return side(left, -1.0, rhoL_s, xi)
        return side(right, 1.0, rhoR_s, xi)
    return at, Ps, vs

"""Exact solution of the Riemann problem for the 1D Euler equations of an
ideal gamma-law gas (TEST INFRASTRUCTURE: pins the oracle on the Sod tube).

Method (the classical one, as in Toro, "Riemann Solvers and Numerical Methods
for Fluid Dynamics", ch. 4): the star pressure p* is the root of
    f(p) = f_L(p) + f_R(p) + (u_R - u_L),
where f_K is the shock Rankine-Hugoniot relation for p > p_K and the
rarefaction isentrope for p <= p_K; u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2.
The self-similar solution is then sampled at xi = (x - x0) / t. The root is
bracketed and found with scipy's brentq.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _fk(p, rho, pk, gamma):
    """Velocity change across the K wave as a function of the star pressure."""
    c = math.sqrt(gamma * pk / rho)
    if p > pk:   # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    # rarefaction
    return 2.0 * c / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(left, right, gamma=1.4):
    """(p*, u*) for left/right primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    du = ur - ul
    f = lambda p: _fk(p, rl, pl, gamma) + _fk(p, rr, pr, gamma) + du
    lo, hi = 1e-14, max(pl, pr)
    while f(hi) < 0.0:
        hi *= 2.0
    ps = brentq(f, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_fk(ps, rr, pr, gamma) - _fk(ps, rl, pl, gamma))
    return ps, us


def sample(xi, left, right, gamma=1.4):
    """Primitive state (rho, u, p) of the exact solution at similarity
    coordinate xi = x/t (scalar or array)."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    ps, us = star_state(left, right, gamma)
    out = np.zeros((3, xi.size))
    g = gamma
    for n, s in enumerate(xi):
        if s <= us:
            rho, u, p = left
            c = math.sqrt(g * p / rho)
            if ps > p:   # left shock
                S = u - c * math.sqrt((g + 1) / (2 * g) * ps / p + (g - 1) / (2 * g))
                if s < S:
                    out[:, n] = (rho, u, p)
                else:
                    q = ps / p
                    out[:, n] = (rho * (q + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * q + 1), us, ps)
            else:        # left rarefaction
                cs = c * (ps / p) ** ((g - 1) / (2 * g))
                head, tail = u - c, us - cs
                if s < head:
                    out[:, n] = (rho, u, p)
                elif s > tail:
                    out[:, n] = (rho * (ps / p) ** (1 / g), us, ps)
                else:
                    w = 2 / (g + 1) + (g - 1) / ((g + 1) * c) * (u - s)
                    out[:, n] = (rho * w ** (2 / (g - 1)), 2 / (g + 1) * (c + (g - 1) / 2 * u + s),
                                 p * w ** (2 * g / (g - 1)))
        else:
            rho, u, p = right
            c = math.sqrt(g * p / rho)
            if ps > p:   # right shock
                S = u + c * math.sqrt((g + 1) / (2 * g) * ps / p + (g - 1) / (2 * g))
                if s > S:
                    out[:, n] = (rho, u, p)
                else:
                    q = ps / p
                    out[:, n] = (rho * (q + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * q + 1), us, ps)
            else:        # right rarefaction
                cs = c * (ps / p) ** ((g - 1) / (2 * g))
                head, tail = u + c, us + cs
                if s > head:
                    out[:, n] = (rho, u, p)
                elif s < tail:
                    out[:, n] = (rho * (ps / p) ** (1 / g), us, ps)
                else:
                    w = 2 / (g + 1) - (g - 1) / ((g + 1) * c) * (u - s)
                    out[:, n] = (rho * w ** (2 / (g - 1)), 2 / (g + 1) * (-c + (g - 1) / 2 * u + s),
                                 p * w ** (2 * g / (g - 1)))
    return out

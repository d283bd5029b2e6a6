"""Sedov-Taylor point blast: the similarity constant xi0 in
R(t) = xi0 (E t^2 / rho0)^(1/5) (TEST INFRASTRUCTURE: pins the blast radius).

Derivation used here (spherical symmetry, strong shock into gas at rest).
With lambda = r / R(t), R' = dR/dt = 2R / (5t) and R'' = -(3/2) R'^2 / R,
write u = R' f(lambda), rho = rho0 g(lambda), p = rho0 R'^2 h(lambda).
Mass, momentum and entropy conservation become
    g f' + (f - lambda) g'                  = -2 g f / lambda
    (f - lambda) f' + h' / g                 = (3/2) f
    -gamma (f - lambda) g'/g + (f - lambda) h'/h = 3
with strong-shock values at lambda = 1:
    f = 2/(gamma+1), g = (gamma+1)/(gamma-1), h = 2/(gamma+1).
Energy: E = 4 pi rho0 R'^2 R^3 I = (16 pi / 25) rho0 (R^5 / t^2) I with
I = int_0^1 (g f^2 / 2 + h / (gamma - 1)) lambda^2 dlambda, hence
xi0 = (25 / (16 pi I))^(1/5). The ODEs are integrated inward with scipy's
solve_ivp (a library integrator used as one step).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp


def _rhs(lam, y, gamma):
    f, g, h = y
    a = f - lam
    M = np.array([[g, a, 0.0],
                  [a, 0.0, 1.0 / g],
                  [0.0, -gamma * a / g, a / h]])
    b = np.array([-2.0 * g * f / lam, 1.5 * f, 3.0])
    return np.linalg.solve(M, b)


def profiles(gamma: float = 1.4, lam_min: float = 1e-4, n: int = 2001):
    """(lambda, f, g, h) on a grid from 1 down to lam_min."""
    y0 = [2.0 / (gamma + 1.0), (gamma + 1.0) / (gamma - 1.0), 2.0 / (gamma + 1.0)]
    lam = np.linspace(1.0, lam_min, n)
    sol = solve_ivp(_rhs, (1.0, lam_min), y0, t_eval=lam, args=(gamma,),
                    rtol=1e-11, atol=1e-13, method="LSODA")
    if not sol.success:
        raise RuntimeError(sol.message)
    return sol.t, sol.y[0], sol.y[1], sol.y[2]


def xi0(gamma: float = 1.4) -> float:
    """Similarity constant of the spherical blast for ratio of specific heats gamma."""
    lam, f, g, h = profiles(gamma)
    integrand = (0.5 * g * f * f + h / (gamma - 1.0)) * lam * lam
    I = -np.trapezoid(integrand, lam)       # lam decreases
    return (25.0 / (16.0 * math.pi * I)) ** 0.2


def shock_radius(t: float, energy: float = 1.0, rho0: float = 1.0, gamma: float = 1.4) -> float:
    return xi0(gamma) * (energy * t * t / rho0) ** 0.2

"""Flux functions, LLF fluxes and maximum speeds for the oracle
(test infrastructure only).

Arrays carry the component axis first: u has shape (ncomp, ...).

Sources:
  * LLF flux F(uL, uR; n) = (f(uL) + f(uR))/2 . n - lambda/2 (uR - uL),
    Sec. 3, eq. (fluxLLF).
  * KPP flux f(u) = (sin u, cos u), Sec. 5.3.2.
  * Euler: p = (gamma - 1)(rho E - |rho v|^2 / (2 rho)), Sec. 5.2; sound
    speed c = sqrt(max(0, gamma p / rho)), Sec. 5.2.2.
  * Max speeds are deferred by the paper to its references (Sec. 2.2).
    Readings used here: advection |v.n|; Burgers max(|uL|,|uR|) |nx + ny|;
    KPP 1 (|f'(u).n| <= 1); Euler the two-rarefaction upper bound of
    Guermond & Popov (J. Comput. Phys. 321, 2016) for 1 < gamma <= 5/3.
"""
from __future__ import annotations

import numpy as np

ADV, BURGERS, KPP, EULER = 0, 1, 2, 3


def flux(kind: int, u: np.ndarray, prob: dict):
    """Physical flux components (fx, fy), each with the shape of u."""
    if kind == ADV:
        return prob["vx"] * u, prob["vy"] * u
    if kind == BURGERS:
        return 0.5 * u * u, 0.5 * u * u
    if kind == KPP:
        return np.sin(u), np.cos(u)
    if kind == EULER:
        g = prob["gamma_gas"]
        rho, mx, my, E = u[0], u[1], u[2], u[3]
        vx, vy = mx / rho, my / rho
        p = (g - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho)
        fx = np.stack([mx, mx * vx + p, my * vx, (E + p) * vx])
        fy = np.stack([my, mx * vy, my * vy + p, (E + p) * vy])
        return fx, fy
    raise ValueError(kind)


def normal_flux(kind, u, nx, ny, prob):
    fx, fy = flux(kind, u, prob)
    return fx * nx + fy * ny


def pressure(u, g):
    return (g - 1.0) * (u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / u[0])


def sound_speed(u, g):
    return np.sqrt(np.maximum(0.0, g * pressure(u, g) / u[0]))


def max_speed(kind, uL, uR, nx, ny, prob):
    """Upper bound lambda_LR of the maximum wave speed of the 1D Riemann
    problem (uL, uR) in direction n = (nx, ny), |n| = 1."""
    if kind == ADV:
        return np.abs(prob["vx"] * nx + prob["vy"] * ny) * np.ones_like(uL[0])
    if kind == BURGERS:
        return np.maximum(np.abs(uL[0]), np.abs(uR[0])) * abs(nx + ny)
    if kind == KPP:
        return np.ones_like(uL[0])
    if kind == EULER:
        g = prob["gamma_gas"]
        rL, rR = uL[0], uR[0]
        vL = (uL[1] * nx + uL[2] * ny) / rL
        vR = (uR[1] * nx + uR[2] * ny) / rR
        pL, pR = pressure(uL, g), pressure(uR, g)
        aL = np.sqrt(g * pL / rL)
        aR = np.sqrt(g * pR / rR)
        # two-rarefaction pressure p_TR >= p* for 1 < gamma <= 5/3
        expo = (g - 1.0) / (2.0 * g)
        num = aL + aR - 0.5 * (g - 1.0) * (vR - vL)
        den = aL * pL ** (-expo) + aR * pR ** (-expo)
        ptr = np.where(num > 0.0, np.maximum(num, 0.0) / den, 0.0) ** (1.0 / expo)
        cg = (g + 1.0) / (2.0 * g)
        lam1 = vL - aL * np.sqrt(1.0 + cg * np.maximum(0.0, (ptr - pL) / pL))
        lam3 = vR + aR * np.sqrt(1.0 + cg * np.maximum(0.0, (ptr - pR) / pR))
        return np.maximum(np.abs(lam1), np.abs(lam3))
    raise ValueError(kind)


def llf(kind, uL, uR, nx, ny, prob, lam=None):
    """LLF flux F(uL, uR; n), eq. (fluxLLF); returns (F, lambda)."""
    if lam is None:
        lam = max_speed(kind, uL, uR, nx, ny, prob)
    F = 0.5 * (normal_flux(kind, uL, nx, ny, prob) + normal_flux(kind, uR, nx, ny, prob)) \
        - 0.5 * lam * (uR - uL)
    return F, lam


def node_speed(kind, u, prob):
    """Bound on the maximum speed at a state over all directions, used for
    lambda_e in nu_e = lambda_e h_e / (2p) (eq. (stab:WENO))."""
    if kind == ADV:
        return np.hypot(prob["vx"], prob["vy"]) * np.ones_like(u[0])
    if kind == BURGERS:
        return np.sqrt(2.0) * np.abs(u[0])
    if kind == KPP:
        return np.ones_like(u[0])
    if kind == EULER:
        g = prob["gamma_gas"]
        return np.hypot(u[1], u[2]) / u[0] + sound_speed(u, g)
    raise ValueError(kind)

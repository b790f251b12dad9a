"""Pins for the oracle's Euler parts (CPU).

  * the LLF speed is an upper bound of the exact maximum wave speed of the
    1D Riemann problem; the exact speeds come from the textbook exact
    Riemann solver (Toro, Ch. 4: Newton iteration for p*), written here;
  * identical states give lambda = |v.n| + c;
  * Appendix A limiter: ubar + alpha f / m keeps rho > 0 and p > 0 for
    random admissible ubar and arbitrary f;
  * conservation on a periodic mesh and positivity (Sec. 5.2: rho > 0,
    p > 0) of every Bernstein coefficient after WENO-L steps;
  * the blast wave stays positive (zero violations)."""
import math

import numpy as np
import pytest

import inputs
from inputs import Mesh, Problem
import oracle.physics as ph
import oracle.scheme as S

G = 1.4


def exact_max_speed(rL, uL, pL, rR, uR, pR, g=G):
    """Max |wave speed| of the exact 1D Euler Riemann problem (no vacuum)."""
    aL, aR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    AL, BL = 2.0 / ((g + 1) * rL), (g - 1) / (g + 1) * pL
    AR, BR = 2.0 / ((g + 1) * rR), (g - 1) / (g + 1) * pR

    def fk(p, rk, pk, ak, A, B):
        """Toro's pressure function f_K and its derivative."""
        if p > pk:
            q = math.sqrt(A / (p + B))
            return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
        r = (p / pk) ** ((g - 1) / (2 * g))
        return 2 * ak / (g - 1) * (r - 1.0), (p / pk) ** (-(g + 1) / (2 * g)) / (rk * ak)

    p = max(1e-8, 0.5 * (pL + pR))
    for _ in range(200):
        f1, d1 = fk(p, rL, pL, aL, AL, BL)
        f2, d2 = fk(p, rR, pR, aR, AR, BR)
        F = f1 + f2 + (uR - uL)
        dp = F / (d1 + d2)
        pn = max(1e-12, p - dp)
        if abs(pn - p) < 1e-14 * p:
            p = pn
            break
        p = pn
    ps = p
    if ps > pL:
        SL = uL - aL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
    else:
        SL = uL - aL
    if ps > pR:
        SR = uR + aR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
    else:
        SR = uR + aR
    return max(abs(SL), abs(SR))


def test_riemann_solver_sanity():
    # Sod: p* = 0.30313, left rarefaction head -1.18322, right shock 1.75216
    s = exact_max_speed(1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    assert abs(s - 1.75216) < 2e-4


def test_llf_speed_is_upper_bound():
    rng = inputs.SplitMix64(77)
    prob = Problem(flux=inputs.FLUX_EULER).as_dict()
    for _ in range(400):
        rL, rR = rng.uniform(0.05, 2.0), rng.uniform(0.05, 2.0)
        pL, pR = rng.uniform(0.01, 2.0), rng.uniform(0.01, 2.0)
        uL, uR = rng.uniform(-1.5, 1.5), rng.uniform(-1.5, 1.5)
        vt = rng.uniform(-1, 1)
        th = rng.uniform(0, 2 * math.pi)
        nx, ny = math.cos(th), math.sin(th)
        # build 2D states with normal velocity u and tangential vt
        def cons(r, un, p):
            vx, vy = un * nx - vt * ny, un * ny + vt * nx
            return inputs.euler_primitive_to_conserved(np.array([r]), np.array([vx]),
                                                       np.array([vy]), np.array([p]))
        UL, UR = cons(rL, uL, pL), cons(rR, uR, pR)
        lam = ph.max_speed(ph.EULER, UL, UR, nx, ny, prob)[0]
        # vacuum generation: the bound falls back to the rarefaction heads
        if 2 * (math.sqrt(G * pL / rL) + math.sqrt(G * pR / rR)) / (G - 1) <= uR - uL:
            continue
        ex = exact_max_speed(rL, uL, pL, rR, uR, pR)
        assert lam >= ex * (1 - 1e-12), (lam, ex)
        assert lam <= 3.0 * ex + 1e-12


def test_llf_speed_identical_states():
    prob = Problem(flux=inputs.FLUX_EULER).as_dict()
    U = inputs.euler_primitive_to_conserved(np.array([0.7]), np.array([0.3]),
                                            np.array([-0.4]), np.array([0.9]))
    lam = ph.max_speed(ph.EULER, U, U, 0.6, 0.8, prob)[0]
    c = math.sqrt(G * 0.9 / 0.7)
    assert abs(lam - (abs(0.3 * 0.6 - 0.4 * 0.8) + c)) < 1e-14


def test_appendix_a_positivity():
    prob = Problem(flux=inputs.FLUX_EULER).as_dict()
    rng = inputs.SplitMix64(5)
    n = 2000
    rho = rng.array(n, 1e-3, 2.0)
    vx, vy = rng.array(n, -3, 3), rng.array(n, -3, 3)
    p = rng.array(n, 1e-6, 2.0)
    ub = inputs.euler_primitive_to_conserved(rho, vx, vy, p)
    f = np.stack([rng.array(n, -5, 5) for _ in range(4)])
    m = rng.array(n, 0.01, 1.0)
    a = S.euler_alpha(ub, f, m, prob)
    us = ub + a * f / m
    assert np.all((a >= 0) & (a <= 1))
    assert np.all(us[0] > 0)
    assert np.all(ph.pressure(us, G) > 0)
    # alpha = 1 whenever the unlimited state is admissible with margin
    u1 = ub + f / m
    ok = (u1[0] > 1e-9 * ub[0]) & (u1[0] * u1[3] - 0.5 * (u1[1] ** 2 + u1[2] ** 2)
                                    > 1e-9 * (ub[0] * ub[3] - 0.5 * (ub[1] ** 2 + ub[2] ** 2)))
    assert np.all(a[ok & (np.abs(f).max(axis=0) / m < 1e-3)] == 1.0)


def test_euler_conservation_and_positivity_periodic():
    mesh = Mesh(6, 5, 2, 0.0, 1.2, 0.0, 1.0)
    prob = Problem(flux=inputs.FLUX_EULER, mode=inputs.MODE_WENO_L).as_dict()
    u = inputs.random_euler_state(mesh, 31)
    m0 = S.mass(mesh, u)
    u1, t, st = S.run(mesh, prob, u, 4)
    m1 = S.mass(mesh, u1)
    assert np.all(np.abs(m1 - m0) <= 1e-13 * np.abs(m0).max())
    assert st["violations"] == 0


@pytest.mark.parametrize("p", [1, 2, 3])
def test_euler_blast_positivity(p):
    mesh, prob, u0 = inputs.euler_blast_config(8, 8, p)
    u1, t, st = S.run(mesh, prob, u0, 8)
    assert st["violations"] == 0
    assert np.all(u1[0] > 0) and np.all(ph.pressure(u1, G) > 0)


def test_euler_quadrant_small():
    mesh, prob, u0 = inputs.euler_quadrant_config(8, 8, 3)
    u1, t, st = S.run(mesh, prob, u0, 4)
    assert st["violations"] == 0

"""Pins of the oracle's nonlinear parts: the Euler and KPP fluxes, the
Appendix-A positivity factors and the volume / boundary integrals of a
nonlinear flux (CPU).

What fixes each expected value:
  * Euler flux (Sec. 5.2): the Rankine-Hugoniot conditions of exact shocks
    built from the textbook normal-shock relations for a given Mach number
    (density and pressure ratios of a moving normal shock), in a rotated
    frame with a tangential velocity; the eigenvalues v.n - c, v.n, v.n,
    v.n + c of the flux Jacobian (taken by complex-step differentiation of
    the oracle's own flux), and the Jacobian itself against the textbook
    matrices of the 2D Euler equations;
  * Appendix A: the factors alpha_i are the LARGEST admissible ones.  The
    test derives them from the definition of the limited state
    u* = ubar + alpha f / m alone: rho* is linear in alpha, and
    P(alpha) = rho* E* - |m*|^2 / 2 is a quadratic whose coefficients are
    read off three evaluations; on [0, 1] its linear minorant is
    P(0) + alpha (P'(0) + min(0, P''/2)), so alpha^p is where that minorant
    reaches the margin eps P(0), and alpha^rho where rho* reaches eps rho_bar;
  * the nonlinear-flux residual eq. (weak:galerkin): the oracle's weak form
    with face terms (a high-order rule in place of the default p + 2 points)
    against a strong-form global assembly sum_e int phi_i div f(u_h) with
    the fluxes' Jacobians written from their definitions (tests/bruteforce.py);
  * KPP flux orientation: a small smooth perturbation of a constant state
    travels with the characteristic velocity f'(u) = (cos u, -sin u).
"""
import math

import numpy as np
import pytest

import inputs
from inputs import Mesh, Problem
import oracle.physics as ph
import oracle.scheme as S
from tests.bruteforce import Brute


def _euler_prob(g=1.4):
    return Problem(flux=inputs.FLUX_EULER, gamma_gas=g).as_dict()


def _cons(rho, vx, vy, p, g):
    E = p / (g - 1.0) + 0.5 * rho * (vx * vx + vy * vy)
    return np.array([rho, rho * vx, rho * vy, E], dtype=np.float64)


# --------------------------------------------------------------------------
# Euler flux: exact shocks
# --------------------------------------------------------------------------
@pytest.mark.parametrize("g", [1.4, 5.0 / 3.0, 1.2])
def test_euler_flux_rankine_hugoniot(g):
    """f(u_L).n - f(u_R).n = s (u_L - u_R) for a normal shock moving with
    speed s along n into the state u_R (textbook normal-shock relations:
    rho_L / rho_R = (g+1) M^2 / ((g-1) M^2 + 2),
    p_L / p_R = 1 + 2 g (M^2 - 1) / (g + 1), M the upstream Mach number in
    the shock frame; the tangential velocity is continuous)."""
    prob = _euler_prob(g)
    rng = inputs.SplitMix64(1701)
    for _ in range(200):
        M = rng.uniform(1.05, 6.0)
        rR, pR = rng.uniform(0.1, 3.0), rng.uniform(0.05, 5.0)
        vR = rng.uniform(-2.0, 2.0)           # normal velocity ahead of the shock
        vt = rng.uniform(-2.0, 2.0)           # tangential velocity (both sides)
        th = rng.uniform(0.0, 2.0 * math.pi)
        nx, ny = math.cos(th), math.sin(th)
        cR = math.sqrt(g * pR / rR)
        s = vR + M * cR                       # shock speed along n
        rL = rR * (g + 1.0) * M * M / ((g - 1.0) * M * M + 2.0)
        pL = pR * (1.0 + 2.0 * g * (M * M - 1.0) / (g + 1.0))
        wL = (M * cR) * rR / rL               # relative speed behind the shock
        vL = s - wL

        def state(r, vn, p):
            return _cons(r, vn * nx - vt * ny, vn * ny + vt * nx, p, g)

        uL, uR = state(rL, vL, pL), state(rR, vR, pR)
        FL = ph.normal_flux(ph.EULER, uL[:, None], nx, ny, prob)[:, 0]
        FR = ph.normal_flux(ph.EULER, uR[:, None], nx, ny, prob)[:, 0]
        lhs, rhs = FL - FR, s * (uL - uR)
        scale = np.abs(FL).max() + np.abs(FR).max() + abs(s) * np.abs(uL).max()
        assert np.abs(lhs - rhs).max() <= 1e-13 * scale, (lhs, rhs)


def _jac_complex_step(u, nx, ny, prob):
    """d (f(u).n) / du by complex-step differentiation (exact to rounding
    for a flux built from + - * /)."""
    h = 1e-30
    J = np.zeros((4, 4))
    for j in range(4):
        up = u.astype(np.complex128)
        up[j] += 1j * h
        J[:, j] = ph.normal_flux(ph.EULER, up[:, None], nx, ny, prob)[:, 0].imag / h
    return J


def _jac_textbook(u, nx, ny, g):
    """n_x A_x + n_y A_y of the 2D Euler equations in conserved variables
    (rho, rho v_x, rho v_y, E), with q2 = |v|^2 and total enthalpy
    H = (E + p) / rho, written from the standard form of the Jacobians."""
    rho, mx, my, E = u
    vx, vy = mx / rho, my / rho
    q2 = vx * vx + vy * vy
    p = (g - 1.0) * (E - 0.5 * rho * q2)
    H = (E + p) / rho
    k = 0.5 * (g - 1.0) * q2
    Ax = np.array([
        [0.0, 1.0, 0.0, 0.0],
        [k - vx * vx, (3.0 - g) * vx, -(g - 1.0) * vy, g - 1.0],
        [-vx * vy, vy, vx, 0.0],
        [vx * (k - H), H - (g - 1.0) * vx * vx, -(g - 1.0) * vx * vy, g * vx]])
    Ay = np.array([
        [0.0, 0.0, 1.0, 0.0],
        [-vx * vy, vy, vx, 0.0],
        [k - vy * vy, -(g - 1.0) * vx, (3.0 - g) * vy, g - 1.0],
        [vy * (k - H), -(g - 1.0) * vx * vy, H - (g - 1.0) * vy * vy, g * vy]])
    return nx * Ax + ny * Ay


@pytest.mark.parametrize("g", [1.4, 5.0 / 3.0])
def test_euler_flux_jacobian(g):
    """The Jacobian of the oracle's normal flux has the eigenvalues
    v.n - c, v.n (twice), v.n + c and equals the textbook matrix."""
    prob = _euler_prob(g)
    rng = inputs.SplitMix64(1702)
    for _ in range(100):
        rho, p = rng.uniform(0.1, 3.0), rng.uniform(0.05, 5.0)
        vx, vy = rng.uniform(-2, 2), rng.uniform(-2, 2)
        th = rng.uniform(0.0, 2.0 * math.pi)
        nx, ny = math.cos(th), math.sin(th)
        u = _cons(rho, vx, vy, p, g)
        J = _jac_complex_step(u, nx, ny, prob)
        vn, c = vx * nx + vy * ny, math.sqrt(g * p / rho)
        ev = np.sort(np.linalg.eigvals(J).real)
        ref = np.sort([vn - c, vn, vn, vn + c])
        assert np.abs(ev - ref).max() <= 1e-9 * (abs(vn) + c), (ev, ref)
        Jt = _jac_textbook(u, nx, ny, g)
        assert np.abs(J - Jt).max() <= 1e-13 * np.abs(Jt).max()


def test_euler_flux_pins_catch_planted_mistakes(monkeypatch):
    """Each plausible mistake in the Euler flux fails one of the pins above:
    an energy flux E v instead of (E + p) v, and swapped momentum-flux
    entries (rho v_x v_y placed in the wrong component)."""
    g = 1.4
    prob = _euler_prob(g)
    u = _cons(0.9, 0.4, -0.7, 1.3, g)
    nx, ny = 0.6, 0.8
    good = _jac_complex_step(u, nx, ny, prob)
    Jt = _jac_textbook(u, nx, ny, g)
    assert np.abs(good - Jt).max() <= 1e-13 * np.abs(Jt).max()
    orig = ph.flux

    def no_p_energy(kind, w, pr):
        fx, fy = orig(kind, w, pr)
        if kind == ph.EULER:
            rho, mx, my, E = w
            fx = fx.copy()
            fy = fy.copy()
            fx[3] = E * mx / rho
            fy[3] = E * my / rho
        return fx, fy

    def swapped(kind, w, pr):
        fx, fy = orig(kind, w, pr)
        if kind == ph.EULER:
            fx = fx.copy()
            fx[[1, 2]] = fx[[2, 1]]
        return fx, fy

    for bad in (no_p_energy, swapped):
        monkeypatch.setattr(ph, "flux", bad)
        J = _jac_complex_step(u, nx, ny, prob)
        assert np.abs(J - Jt).max() > 1e-3
        monkeypatch.setattr(ph, "flux", orig)


# --------------------------------------------------------------------------
# Appendix A: sharpness of the positivity factors
# --------------------------------------------------------------------------
def _largest_admissible(ub, f, m, eps):
    """The largest alpha in [0, 1] whose limited state ubar + alpha f / m
    keeps rho* >= eps rho_bar and the linear minorant of P(alpha) on [0, 1]
    at or above eps P(0), from the definition of the state alone."""
    def P(a):
        us = ub + a * f / m
        return us[0] * us[3] - 0.5 * (us[1] ** 2 + us[2] ** 2)

    P0, P1, Pm = P(0.0), P(1.0), P(-1.0)
    c2 = 0.5 * (P1 + Pm) - P0            # coefficient of alpha^2
    c1 = 0.5 * (P1 - Pm)                 # coefficient of alpha
    slope = c1 + min(0.0, c2)            # alpha^2 >= ... on [0, 1]: c2 alpha^2 >= min(0, c2) alpha
    a_p = 1.0
    if P0 + slope < eps * P0:
        a_p = (eps - 1.0) * P0 / slope
    a_r = 1.0
    if ub[0] + f[0] / m < eps * ub[0]:
        a_r = (eps - 1.0) * ub[0] * m / f[0]
    return min(a_r, a_p), P


def test_appendix_a_factors_are_largest():
    prob = Problem(flux=inputs.FLUX_EULER).as_dict()
    eps = prob["pos_eps"]
    g = prob["gamma_gas"]
    rng = inputs.SplitMix64(1703)
    n_lim = 0
    for _ in range(3000):
        ub = _cons(rng.uniform(1e-3, 2.0), rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(1e-6, 2.0), g)
        f = np.array([rng.uniform(-5, 5) for _ in range(4)])
        m = rng.uniform(0.01, 1.0)
        a = float(S.euler_alpha(ub[:, None], f[:, None], np.array([m]), prob)[0])
        ref, P = _largest_admissible(ub, f, m, eps)
        assert abs(a - ref) <= 1e-10 * max(ref, 1e-300) + 1e-15, (a, ref)
        # admissible with the exact quadratic and the density margin
        us = ub + a * f / m
        assert us[0] >= eps * ub[0] * (1.0 - 1e-12)
        assert P(a) >= eps * P(0.0) * (1.0 - 1e-9)
        n_lim += a < 1.0
    assert n_lim > 1000


def test_appendix_a_pin_catches_planted_mistakes(monkeypatch):
    """A limiter that cuts too much or too little fails the sharpness pin:
    a flipped sign inside the min{0, ...} term, and alpha^rho taken from the
    pressure-scaled flux."""
    prob = Problem(flux=inputs.FLUX_EULER).as_dict()
    eps = prob["pos_eps"]
    rng = inputs.SplitMix64(1704)
    cases = []
    for _ in range(400):
        ub = _cons(rng.uniform(1e-3, 2.0), rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(1e-6, 2.0), 1.4)
        f = np.array([rng.uniform(-5, 5) for _ in range(4)])
        cases.append((ub, f, rng.uniform(0.01, 1.0)))

    def mismatches(alpha_fn):
        bad = 0
        for ub, f, m in cases:
            ref, _ = _largest_admissible(ub, f, m, eps)
            a = float(alpha_fn(ub[:, None], f[:, None], np.array([m]), prob)[0])
            bad += abs(a - ref) > 1e-10 * max(ref, 1e-300) + 1e-15
        return bad

    assert mismatches(S.euler_alpha) == 0

    def flipped_min(ub, f, m, pr):
        rho, mx, my, E = ub
        fr, fmx, fmy, fE = f
        e = pr["pos_eps"]
        thr = m * rho * (1.0 - e)
        a_rho = np.where(thr + fr < 0.0, -thr / np.where(fr == 0.0, 1.0, fr), 1.0)
        Q = (1.0 - e) * m * (0.5 * (mx * mx + my * my) - rho * E)
        R = rho * fE + E * fr - (mx * fmx + my * fmy) + np.minimum(0.0, -(fE * fr - 0.5 * (fmx * fmx + fmy * fmy))) / m
        a_p = np.where(R < Q, Q / np.where(R == 0.0, 1.0, R), 1.0)
        return np.clip(np.minimum(a_rho, a_p), 0.0, 1.0)

    def pressure_from_scaled_flux(ub, f, m, pr):
        # alpha^rho first, then alpha^p evaluated on the already scaled flux
        e = pr["pos_eps"]
        thr = m * ub[0] * (1.0 - e)
        a_rho = np.where(thr + f[0] < 0.0, -thr / np.where(f[0] == 0.0, 1.0, f[0]), 1.0)
        a_p = S.euler_alpha(ub, a_rho * f, m, pr)
        return np.clip(a_rho * a_p, 0.0, 1.0)

    assert mismatches(flipped_min) > 20
    assert mismatches(pressure_from_scaled_flux) > 5
    # a factor 1 % below the largest admissible one is not sharp
    assert mismatches(lambda *a: 0.99 * S.euler_alpha(*a)) > 200


# --------------------------------------------------------------------------
# nonlinear-flux residual: weak form with face terms vs strong form
# --------------------------------------------------------------------------
def _kpp_jac(uq):
    u = uq[0]
    return np.cos(u)[None, None, :], -np.sin(u)[None, None, :]


def _euler_jac_field(g):
    def jac(uq):
        nq = uq.shape[1]
        Ax = np.zeros((4, 4, nq))
        Ay = np.zeros((4, 4, nq))
        for q in range(nq):
            Ax[:, :, q] = _jac_textbook(uq[:, q], 1.0, 0.0, g)
            Ay[:, :, q] = _jac_textbook(uq[:, q], 0.0, 1.0, g)
        return Ax, Ay
    return jac


def _smooth_euler_state(mesh, seed, g=1.4):
    """A smooth admissible Euler state with seeded phases (rho in [0.7, 1.3])."""
    rng = inputs.SplitMix64(seed)
    X, Y = inputs.node_coords(mesh)
    L = mesh.x1 - mesh.x0

    def wave(a):
        kx, ky = rng.randint(1, 2), rng.randint(1, 2)
        ph_ = rng.uniform(0.0, 2.0 * math.pi)
        return a * np.sin(2 * math.pi * (kx * (X - mesh.x0) + ky * (Y - mesh.y0)) / L + ph_)

    rho = 1.0 + wave(0.3)
    vx, vy = 0.4 + wave(0.3), -0.2 + wave(0.3)
    p = 1.0 + wave(0.3)
    return inputs.euler_primitive_to_conserved(rho, vx, vy, p, g)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("bc", [inputs.BC_PERIODIC, inputs.BC_FIXED])
def test_kpp_residual_weak_equals_strong(p, bc):
    """Gathered oracle element residuals (weak form, interior face terms of
    f_h, boundary faces with the LLF flux F(u_h, u_hat; n)) equal
    -(a + b) of eq. (weak:galerkin) assembled in strong form, for the KPP
    flux f(u) = (sin u, cos u) with Jacobian (cos u, -sin u)."""
    n = 3 if bc == inputs.BC_PERIODIC else 2
    mesh = Mesh(n, n, p, 0.0, 1.0, 0.0, 1.0, bc, bc)
    ub = 1.1
    prob = Problem(flux=inputs.FLUX_KPP, ubc=(ub, 0, 0, 0), umin=0.0, umax=5.0).as_dict()
    u = inputs.random_scalar_state(mesh, 61 + p, 0.5, 3.0, 0.7)
    nq = 2 * p + 12
    om = S.OracleMesh(mesh, nq=nq)
    W = S.element_residual(om, om.blocks(u), prob)
    r_or = om.gather(W)[0]
    bf = Brute(n, n, p, 0.0, 1.0, 0.0, 1.0, bc == inputs.BC_PERIODIC, nq=nq)
    a = bf.galerkin_strong_system(u.reshape(1, -1), _kpp_jac)[0]
    fn = lambda w, nx_, ny_: np.sin(w) * nx_ + np.cos(w) * ny_
    # LLF with the KPP speed bound 1 (|f'(u).n| <= 1), eq. (fluxLLF)
    Fllf = lambda w, v, nx_, ny_: 0.5 * (fn(w, nx_, ny_) + fn(v, nx_, ny_)) - 0.5 * (v - w)
    b = bf.boundary_term(u.ravel(), fn, Fllf, ub)
    ref = -(a + b)
    assert np.abs(r_or - ref).max() <= 1e-12 * np.abs(ref).max(), np.abs(r_or - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("bc", [inputs.BC_PERIODIC, inputs.BC_OUTFLOW])
def test_euler_residual_weak_equals_strong(p, bc):
    """As above for the Euler flux: periodic (b = 0) and OUTFLOW sides
    (u_hat = u_h, so F(u_h, u_h; n) = f(u_h).n and b = 0)."""
    g = 1.4
    n = 3 if bc == inputs.BC_PERIODIC else 2
    mesh = Mesh(n, n, p, 0.0, 1.0, 0.0, 1.0, bc, bc)
    prob = _euler_prob(g)
    u = _smooth_euler_state(mesh, 71 + p)
    nq = 2 * p + 14
    om = S.OracleMesh(mesh, nq=nq)
    W = S.element_residual(om, om.blocks(u), prob)
    r_or = om.gather(W)
    bf = Brute(n, n, p, 0.0, 1.0, 0.0, 1.0, bc == inputs.BC_PERIODIC, nq=nq)
    a = bf.galerkin_strong_system(u.reshape(4, -1), _euler_jac_field(g))
    ref = -a
    for c in range(4):
        sc = np.abs(ref).max()
        assert np.abs(r_or[c] - ref[c]).max() <= 1e-11 * sc, (c, np.abs(r_or[c] - ref[c]).max() / sc)


def test_residual_pin_catches_planted_flux_mistakes(monkeypatch):
    """The weak/strong comparison fails with the KPP components swapped or
    the Euler energy flux missing its pressure work."""
    p, n = 2, 3
    mesh = Mesh(n, n, p)
    nq = 2 * p + 12
    om = S.OracleMesh(mesh, nq=nq)
    bf = Brute(n, n, p, 0.0, 1.0, 0.0, 1.0, True, nq=nq)
    orig = ph.flux

    def kpp_swapped(kind, w, pr):
        if kind == ph.KPP:
            return np.cos(w), np.sin(w)
        return orig(kind, w, pr)

    u = inputs.random_scalar_state(mesh, 63, 0.5, 3.0, 0.7)
    prob = Problem(flux=inputs.FLUX_KPP).as_dict()
    ref = -bf.galerkin_strong_system(u.reshape(1, -1), _kpp_jac)[0]
    monkeypatch.setattr(ph, "flux", kpp_swapped)
    bad = om.gather(S.element_residual(om, om.blocks(u), prob))[0]
    monkeypatch.setattr(ph, "flux", orig)
    assert np.abs(bad - ref).max() > 1e-3 * np.abs(ref).max()

    def euler_no_p(kind, w, pr):
        fx, fy = orig(kind, w, pr)
        if kind == ph.EULER:
            rho, mx, my, E = w
            fx = fx.copy()
            fy = fy.copy()
            fx[3] = E * mx / rho
            fy[3] = E * my / rho
        return fx, fy

    ue = _smooth_euler_state(mesh, 73)
    prob = _euler_prob()
    ref = -bf.galerkin_strong_system(ue.reshape(4, -1), _euler_jac_field(1.4))
    monkeypatch.setattr(ph, "flux", euler_no_p)
    bad = om.gather(S.element_residual(om, om.blocks(ue), prob))
    monkeypatch.setattr(ph, "flux", orig)
    assert np.abs(bad[3] - ref[3]).max() > 1e-3 * np.abs(ref[3]).max()


# --------------------------------------------------------------------------
# KPP: orientation of the flux through the motion of a small perturbation
# --------------------------------------------------------------------------
def test_kpp_small_perturbation_travels_with_characteristic_velocity():
    """On a periodic box a smooth bump of amplitude 1e-3 on the constant
    state u_b moves, to first order in the amplitude, with
    f'(u_b) = (cos u_b, -sin u_b); its centroid after time t is displaced by
    t f'(u_b) (within 5 %)."""
    ubg = 1.0
    mesh = Mesh(32, 32, 2, 0.0, 2.0, 0.0, 2.0)
    X, Y = inputs.node_coords(mesh)
    r2 = (X - 1.0) ** 2 + (Y - 1.0) ** 2
    u0 = (ubg + 1e-3 * np.exp(-r2 / 0.05))[None]
    prob = Problem(flux=inputs.FLUX_KPP, mode=inputs.MODE_HO, flux_limiter=S.FL_NONE,
                   umin=0.0, umax=5.0, cfl=0.2).as_dict()

    def centroid(u):
        w = u[0] - ubg
        return (w * X).sum() / w.sum(), (w * Y).sum() / w.sum()

    u1, t, _ = S.run(mesh, prob, u0, 60)
    c0, c1 = centroid(u0), centroid(u1)
    vx, vy = (c1[0] - c0[0]) / t, (c1[1] - c0[1]) / t
    ex, ey = math.cos(ubg), -math.sin(ubg)
    assert abs(vx - ex) <= 0.05 and abs(vy - ey) <= 0.05, (vx, vy, ex, ey)

"""Pins of the subcell pseudo time step of Lemma 1, eq. (dtmaxsubcell), used
by the unlimited-flux variant (option OPT_SUBCELL_DT with the flux limiter
off), against what the mathematics fixes:

  * closed forms: for advection with v = (1, 0) every boundary node's
    |c_ie| lambda_0i adds up to the inflow plus outflow length 2h, so
    dt_e = min(h/(p+1), m_0^e / (2h)) with m_0^e = (p-1)^2 h^2/(p+1)^2 for
    p >= 2, and dt_e = (1/2) min(h/2, h^2/(2h)) = h/4 for Q1 (s = 2); for
    v = (1, 1)/sqrt 2 and Q1 only the corners (0,0) and (1,1) see a speed
    (lambda = 1, |c| = h/sqrt 2), so dt_e = (1/2) min(sqrt2 h/4, h^2/(sqrt2 h));
  * Lemma 1 itself: with dt_e = dt_e^max the unlimited intermediate
    average ubar^e of eq. (uebar) stays in G for any admissible nodal data
    (scalar fluxes on periodic meshes, Q1..Q4), and rho, p stay positive
    for Euler; the macrocell bound of eq. (dtmaxcell) does not guarantee
    this for the unlimited fluxes: adversarial column data leave G with
    it, so the check has teeth;
  * a Burgers case where u_0^e (the interior mean) differs from the cell
    average, so the speeds lambda_0i depend on which one is taken.
"""
import math

import numpy as np
import pytest

import inputs
from inputs import Mesh, Problem
import oracle.scheme as S
from oracle import physics as ph


def _adv(vx, vy, p, n=4):
    mesh = Mesh(n, n, p)
    prob = Problem(flux=inputs.FLUX_ADVECTION, vx=vx, vy=vy, flux_limiter=0, options=S.OPT_SUBCELL_DT)
    return mesh, prob


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_closed_form_axis_aligned_advection(p):
    mesh, prob = _adv(1.0, 0.0, p)
    om = S.OracleMesh(mesh)
    u = inputs.random_scalar_state(mesh, 3, 0.0, 1.0, 0.5)
    dte = S.subcell_time_steps(om, om.blocks(u), prob.as_dict())
    h = om.h
    if p == 1:
        expect = h / 4
    else:
        m0 = (p - 1) ** 2 * h * h / (p + 1) ** 2
        expect = min(h / (p + 1), m0 / (2 * h))
    assert np.allclose(dte, expect, rtol=1e-14, atol=0)


def test_closed_form_diagonal_advection_q1():
    mesh, prob = _adv(1 / math.sqrt(2), 1 / math.sqrt(2), 1)
    om = S.OracleMesh(mesh)
    u = inputs.random_scalar_state(mesh, 4, 0.0, 1.0, 0.5)
    dte = S.subcell_time_steps(om, om.blocks(u), prob.as_dict())
    # corners (0,0), (1,1): |c| lambda = (h/sqrt2) * 1, corners (1,0), (0,1): 0;
    # sum sqrt2 h, node term (h^2/4)/(h/sqrt2) = sqrt2 h/4, m_0 = |K| = h^2
    h = om.h
    expect = 0.5 * min(h * math.sqrt(2) / 4, h * h / (math.sqrt(2) * h))
    assert np.allclose(dte, expect, rtol=1e-14, atol=0)


def test_closed_form_burgers_uses_interior_mean():
    """Q2 Burgers with 1 on every interior node and 0.1 elsewhere: u_0^e = 1
    (not the cell mean 0.2), lambda_0i = max(|u_0|, |u_i|) |nx + ny| = 1 on
    edge nodes, sqrt 2 on the corners (0,0) and (2,2), 0 on the other two;
    sum = 4 h/3 + 2 (sqrt2 h/3) sqrt2 = 8h/3 and dt_e = min(h/3, h/6,
    (h^2/9) / (8h/3)) = h/24."""
    mesh = Mesh(4, 4, 2)
    gx, gy = np.meshgrid(np.arange(mesh.nnx), np.arange(mesh.nny), indexing="xy")
    u = np.where((gx % 2 == 1) & (gy % 2 == 1), 1.0, 0.1)[None]
    prob = Problem(flux=inputs.FLUX_BURGERS, flux_limiter=0, options=S.OPT_SUBCELL_DT)
    om = S.OracleMesh(mesh)
    dte = S.subcell_time_steps(om, om.blocks(u), prob.as_dict())
    assert np.allclose(dte, om.h / 24, rtol=1e-14, atol=0)


def _step_states(mesh, seed, lo, hi):
    """Discontinuous nodal data: every coefficient drawn independently."""
    rng = inputs.SplitMix64(inputs.BASE_SEED + 500 + seed)
    return np.array([[rng.uniform(lo, hi) for _ in range(mesh.nnx)] for _ in range(mesh.nny)])[None]


def _column_pattern(mesh, lo, hi):
    """Adversarial data for a flow along x: hi on the face columns gx = p, 3p,
    5p, ..., lo elsewhere, so elements alternate between full outflow and full
    inflow through their x faces."""
    gx = np.arange(mesh.nnx)
    row = np.where(gx % (2 * mesh.p) == mesh.p, hi, lo)
    return np.broadcast_to(row, (mesh.nny, mesh.nnx)).copy()[None]


def _worst_excursion(om, base, u, opts, lo, hi):
    prob = Problem(options=opts, **base).as_dict()
    _, info = S.fe_stage(om, prob, u, 0.0)
    ube = info["ube"][0]
    return max(lo - ube.min(), ube.max() - hi, 0.0)


@pytest.mark.parametrize("flux", [inputs.FLUX_ADVECTION, inputs.FLUX_BURGERS, inputs.FLUX_KPP])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lemma1_unlimited_average_stays_in_G(flux, p):
    mesh = Mesh(6, 4, p, 0.0, 1.5, 0.0, 1.0)
    lo, hi = (0.0, 1.0) if flux != inputs.FLUX_KPP else (math.pi / 4, 3.5 * math.pi)
    base = dict(flux=flux, vx=0.8, vy=-0.6, umin=lo, umax=hi, mode=inputs.MODE_HO, flux_limiter=0)
    om = S.OracleMesh(mesh)
    cases = [_step_states(mesh, seed + 10 * p + 100 * flux, lo, hi) for seed in range(6)]
    cases += [_column_pattern(mesh, lo, hi), _column_pattern(mesh, hi, lo)]
    worst = max(_worst_excursion(om, base, u, S.OPT_SUBCELL_DT, lo, hi) for u in cases)
    assert worst <= 1e-13 * max(abs(lo), abs(hi), 1.0)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_macrocell_bound_is_not_enough_for_unlimited_fluxes(p):
    """The same check with the macrocell bound fails on the column pattern, so
    the subcell check above has teeth."""
    mesh = Mesh(6, 4, p, 0.0, 1.5, 0.0, 1.0)
    base = dict(flux=inputs.FLUX_ADVECTION, vx=1.0, vy=0.0, umin=0.0, umax=1.0, mode=inputs.MODE_HO,
                flux_limiter=0)
    om = S.OracleMesh(mesh)
    u = _column_pattern(mesh, 0.0, 1.0)
    assert _worst_excursion(om, base, u, 0, 0.0, 1.0) > 0.05
    assert _worst_excursion(om, base, u, S.OPT_SUBCELL_DT, 0.0, 1.0) <= 1e-15


@pytest.mark.parametrize("p", [1, 2, 3])
def test_lemma1_euler_positivity(p):
    mesh = Mesh(5, 4, p, 0.0, 1.25, 0.0, 1.0)
    om = S.OracleMesh(mesh)
    prob = Problem(flux=inputs.FLUX_EULER, mode=inputs.MODE_HO, flux_limiter=0, options=S.OPT_SUBCELL_DT,
                   umin=0.0, umax=0.0).as_dict()
    for seed in range(4):
        rng = inputs.SplitMix64(inputs.BASE_SEED + 900 + seed + 10 * p)
        shape = (mesh.nny, mesh.nnx)
        prim = [np.array([[rng.uniform(a, b) for _ in range(shape[1])] for _ in range(shape[0])])
                for a, b in ((0.05, 2.0), (-3.0, 3.0), (-3.0, 3.0), (0.01, 5.0))]
        u = inputs.euler_primitive_to_conserved(*prim)
        _, info = S.fe_stage(om, prob, u, 0.0)
        ube = info["ube"]
        assert ube[0].min() > 0.0
        assert ph.pressure(ube, 1.4).min() > 0.0

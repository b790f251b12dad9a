"""Pins of the Q1-variant element contributions of eq. (aecQ1) (option
OPT_AEC_Q1) against what the mathematics fixes:

  * conservation: sum_i f_i^e = 0 in every element (the three terms vanish
    separately: sum_i (phi_i - m_i^e/|K_e|) = 0, sum_i m_i^e (u_i - u^e) = 0,
    and the consistent and lumped masses have equal row sums), for every
    flux and degree;
  * a closed form of the divergence term: Q1 advection with v = (1, 0) and
    nodal data u_j = x_j y_j reproduces f_h = (xy, 0) exactly, div f_h = y,
    and int (phi_i - 1/4) y over an element is -h^3/24 on its bottom nodes
    and +h^3/24 on its top nodes, whatever the element's position;
  * the low-order time derivative: one LO stage is u + dt udot^L exactly
    (eq. (fe-update) with eq. (weak:low2));
  * gamma_e = 0 (LO) gives f_i^e = 0.
"""
import math

import numpy as np
import pytest

import inputs
from inputs import Mesh, Problem
import oracle.scheme as S


def _case(flux, p, mode=inputs.MODE_WENO_L):
    mesh = Mesh(6, 5, p, 0.0, 1.2, 0.0, 1.0)
    if flux == inputs.FLUX_EULER:
        mesh = Mesh(6, 5, p, 0.0, 1.2, 0.0, 1.0, inputs.BC_OUTFLOW, inputs.BC_OUTFLOW)
        prob = Problem(flux=flux, mode=mode, flux_limiter=0, options=S.OPT_AEC_Q1, umin=0.0, umax=0.0)
        return mesh, prob, inputs.random_euler_state(mesh, 30 + p)
    lo, hi = (0.0, 1.0) if flux != inputs.FLUX_KPP else (math.pi / 4, 3.5 * math.pi)
    prob = Problem(flux=flux, vx=0.8, vy=-0.6, umin=lo, umax=hi, mode=mode, flux_limiter=0, options=S.OPT_AEC_Q1,
                   w_lin=0.2)
    return mesh, prob, inputs.random_scalar_state(mesh, 20 + p + 10 * flux, lo, hi, 0.4)


@pytest.mark.parametrize("flux", [inputs.FLUX_ADVECTION, inputs.FLUX_BURGERS, inputs.FLUX_KPP, inputs.FLUX_EULER])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_element_contributions_sum_to_zero(flux, p):
    mesh, prob, u = _case(flux, p)
    om = S.OracleMesh(mesh)
    dt = S.time_step(om, prob.as_dict(), u)
    _, info = S.fe_stage(om, prob.as_dict(), u, dt)
    fie = info["fie"]
    scale = np.abs(fie).max()
    assert scale > 0.0
    assert np.abs(fie.sum(axis=2)).max() <= 1e-13 * scale


def test_divergence_term_closed_form_q1():
    mesh = Mesh(3, 2, 1, 0.25, 1.75, -0.5, 0.5, inputs.BC_OUTFLOW, inputs.BC_OUTFLOW)
    X, Y = inputs.node_coords(mesh)
    u = (X * Y)[None]
    prob = Problem(flux=inputs.FLUX_ADVECTION, vx=1.0, vy=0.0).as_dict()
    om = S.OracleMesh(mesh)
    D = S.flux_divergence_term(om, om.blocks(u), prob)[0]          # (E, 4), local nodes (a, b)
    h = om.h
    expect = np.array([-1.0, -1.0, 1.0, 1.0]) * h ** 3 / 24        # b = 0, 0, 1, 1
    assert np.allclose(D, expect[None, :], rtol=0, atol=1e-15)


@pytest.mark.parametrize("flux", [inputs.FLUX_BURGERS, inputs.FLUX_KPP, inputs.FLUX_EULER])
def test_lo_stage_is_u_plus_dt_udot_low(flux):
    mesh, prob, u = _case(flux, 1)
    om = S.OracleMesh(mesh)
    dt = S.time_step(om, prob.as_dict(), u)
    _, info = S.fe_stage(om, prob.as_dict(), u, dt)
    prob.mode = inputs.MODE_LO
    ulo, info_lo = S.fe_stage(om, prob.as_dict(), u, dt)
    assert np.array_equal(info_lo["ube"], info["ube"])
    udl = info["udot_l"].reshape(u.shape)
    ref = u + dt * udl
    assert np.abs(ulo - ref).max() <= 1e-13 * np.abs(u).max()


def test_gamma_zero_gives_no_contribution():
    mesh, prob, u = _case(inputs.FLUX_KPP, 1)
    om = S.OracleMesh(mesh)
    U = om.blocks(u)
    ue = S.cell_averages(om, U)
    dte = np.full(om.E, 1e-3)
    fie, _ = S.aec_q1(om, U, ue, ue, dte, np.zeros(om.E), prob.as_dict())
    assert np.array_equal(fie, np.zeros_like(fie))


def test_mass_correction_closed_form_q1():
    """Constant u (so D = 0 and u_i = u^e), dt_e = 1, and ubar^e - u = 1 in
    one element only: udot^L = 1/4 on that element's nodes (each Q1 node has
    four elements).  Its right neighbour sees udot^L = (1/4, 0) along x and
    constant along y, so (M udot^L)_i - m_i^e udot^L_i = h^2/24 - h^2/16 =
    -h^2/48 on its left nodes and h^2/48 on its right nodes, and f_i^e is
    minus that."""
    mesh = Mesh(4, 4, 1)
    om = S.OracleMesh(mesh)
    u = np.full((1, om.nny, om.nnx), 0.5)
    U = om.blocks(u)
    ue = S.cell_averages(om, U)
    ube = ue.copy()
    e0 = 1 * mesh.nx + 1
    ube[0, e0] += 1.0
    prob = Problem(flux=inputs.FLUX_ADVECTION, vx=1.0, vy=0.0).as_dict()
    fie, _ = S.aec_q1(om, U, ue, ube, np.ones(om.E), np.ones(om.E), prob)
    h2 = om.h ** 2
    right = fie[0, e0 + 1]                       # local nodes (a, b): (0,0), (1,0), (0,1), (1,1)
    assert np.allclose(right, [h2 / 48, -h2 / 48, h2 / 48, -h2 / 48], rtol=0, atol=1e-16)

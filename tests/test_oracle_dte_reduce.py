"""Pins of the pseudo-time-step reduction of the remark after eq.
(dtmaxcell) (option OPT_DTE_REDUCE, unlimited averages of eq. (uebar)):
where the macrocell dt_e lets ubar^e leave G, dt_e is decreased as much as
necessary to bring it back (CPU).

What fixes each expected value:
  * a closed form: advection along x of the column pattern (value 1 on the
    face columns gx = p, 3p, ..., 0 elsewhere) gives every even element
    u^e = 1/(p+1), f^H_W = 0, f^H_E = 1 and dt_e = h/2, so
    ubar^e = 1/(p+1) - 1/2 < 0 for p >= 2; the largest admissible dt_e is
    h/(p+1), where ubar^e = 0; the odd elements stay inside and keep h/2;
  * invariance: data whose averages stay in G are not touched (same bits);
  * Euler: after the reduction every ubar^e has rho > 0 and p > 0, and each
    reduced dt_e is the largest one the Appendix-A criterion admits, derived
    here from the definition of the moved state (rho linear, rho E - |m|^2/2
    quadratic in the step);
  * end to end: WENO-L with the flux limiter off on the column pattern
    leaves G at the nodes with the macrocell dt_e and stays in G with the
    reduced one.
"""
import math

import numpy as np
import pytest

import inputs
from inputs import Mesh, Problem
import oracle.physics as ph
import oracle.scheme as S


def _column_pattern(mesh, lo, hi):
    gx = np.arange(mesh.nnx)
    row = np.where(gx % (2 * mesh.p) == mesh.p, hi, lo)
    return np.broadcast_to(row, (mesh.nny, mesh.nnx)).copy()[None]


def _adv(p, opts=0, mode=inputs.MODE_HO):
    mesh = Mesh(6, 4, p, 0.0, 1.5, 0.0, 1.0)
    prob = Problem(flux=inputs.FLUX_ADVECTION, vx=1.0, vy=0.0, umin=0.0, umax=1.0, mode=mode,
                   flux_limiter=S.FL_NONE, options=opts).as_dict()
    return mesh, prob


@pytest.mark.parametrize("p", [2, 3, 4])
def test_column_pattern_closed_form(p):
    mesh, prob = _adv(p)
    om = S.OracleMesh(mesh)
    u = _column_pattern(mesh, 0.0, 1.0)
    _, info0 = S.fe_stage(om, prob, u, 0.0)
    even = (om.EX % 2) == 0
    assert info0["ubar_outside"] == int(even.sum())
    assert np.allclose(info0["ube"][0][even], 1.0 / (p + 1) - 0.5, rtol=0, atol=1e-14)
    prob["options"] = S.OPT_DTE_REDUCE
    _, info = S.fe_stage(om, prob, u, 0.0)
    h = om.h
    assert info["dte_reduced"] == int(even.sum())
    assert np.allclose(info["dte"][even], h / (p + 1), rtol=1e-14, atol=0)
    assert np.array_equal(info["dte"][~even], info0["dte"][~even])
    assert np.allclose(info["dte"][~even], h / 2, rtol=1e-15, atol=0)
    ube = info["ube"][0]
    assert np.all(np.abs(ube[even]) <= 1e-15)
    assert ube.min() >= -1e-15 and ube.max() <= 1.0 + 1e-15


@pytest.mark.parametrize("flux", [inputs.FLUX_ADVECTION, inputs.FLUX_BURGERS, inputs.FLUX_KPP])
def test_no_change_where_averages_stay_in_G(flux):
    mesh = Mesh(8, 6, 2, 0.0, 4.0 / 3.0, 0.0, 1.0)
    lo, hi = (0.0, 1.0) if flux != inputs.FLUX_KPP else (math.pi / 4, 3.5 * math.pi)
    base = dict(flux=flux, vx=0.8, vy=-0.45, umin=lo, umax=hi, mode=inputs.MODE_WENO_L, flux_limiter=S.FL_NONE)
    u = inputs.random_scalar_state(mesh, 31, lo, hi, 0.8)
    a, ia = S.fe_stage(mesh, Problem(**base).as_dict(), u, 1e-4)
    b, ib = S.fe_stage(mesh, Problem(options=S.OPT_DTE_REDUCE, **base).as_dict(), u, 1e-4)
    assert ia["ubar_outside"] == 0 and ib["dte_reduced"] == 0
    assert np.array_equal(a, b)


def _euler_columns(p, rlo, v, pres):
    mesh = Mesh(6, 4, p, 0.0, 1.5, 0.0, 1.0)
    gx = np.arange(mesh.nnx)
    rho = np.broadcast_to(np.where(gx % (2 * p) == p, 1.0, rlo), (mesh.nny, mesh.nnx))
    u = inputs.euler_primitive_to_conserved(rho, np.full(rho.shape, v), np.zeros(rho.shape),
                                            np.full(rho.shape, pres))
    return mesh, u


def _largest_step(ue, g, eps):
    """Largest alpha in [0, 1] with ue + alpha g admissible by the
    Appendix-A criterion, from the definition of the moved state."""
    def P(a):
        w = ue + a * g
        return w[0] * w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2)
    P0, P1, Pm = P(0.0), P(1.0), P(-1.0)
    slope = 0.5 * (P1 - Pm) + min(0.0, 0.5 * (P1 + Pm) - P0)
    a_p = 1.0 if P0 + slope >= eps * P0 else (eps - 1.0) * P0 / slope
    a_r = 1.0 if ue[0] + g[0] >= eps * ue[0] else (eps - 1.0) * ue[0] / g[0]
    return min(a_p, a_r)


@pytest.mark.parametrize("p,rlo,v,pres", [(2, 1e-2, 3.0, 1e-2), (2, 1e-4, 1.0, 1e-3), (3, 1e-3, 2.0, 0.1)])
def test_euler_reduction_positive_and_largest(p, rlo, v, pres):
    mesh, u = _euler_columns(p, rlo, v, pres)
    prob = Problem(flux=inputs.FLUX_EULER, mode=inputs.MODE_HO, flux_limiter=S.FL_NONE).as_dict()
    om = S.OracleMesh(mesh)
    _, i0 = S.fe_stage(om, prob, u, 0.0)
    assert i0["ubar_outside"] > 0
    out0 = ~S.in_domain(prob, i0["ube"])
    prob["options"] = S.OPT_DTE_REDUCE
    _, i1 = S.fe_stage(om, prob, u, 0.0)
    ube = i1["ube"]
    assert i1["dte_reduced"] == i0["ubar_outside"]
    assert np.all(ube[0] > 0.0) and np.all(ph.pressure(ube, 1.4) > 0.0)
    # each reduced step is the largest admissible one
    ue = i0["ue"]
    eps = prob["pos_eps"]
    for e in np.nonzero(out0)[0]:
        g = i0["ube"][:, e] - ue[:, e]            # the move at the macrocell dt_e
        ref = _largest_step(ue[:, e], g, eps)
        assert abs(i1["dte"][e] / i0["dte"][e] - ref) <= 1e-12, (e, i1["dte"][e] / i0["dte"][e], ref)
    assert np.array_equal(i1["dte"][~out0], i0["dte"][~out0])


def test_weno_l_without_flux_limiter_is_idp_with_the_reduction():
    p = 2
    mesh, prob = _adv(p, mode=inputs.MODE_WENO_L)
    om = S.OracleMesh(mesh)
    u = _column_pattern(mesh, 0.0, 1.0)
    dt = 0.5 * om.h / (p + 1)            # below every reduced dt_e (theta <= 1)
    out0, i0 = S.ssp_stage(om, prob, u, u, dt, 0.0, 1.0)
    assert i0["violations"] > 0
    prob["options"] = S.OPT_DTE_REDUCE
    out1, i1 = S.ssp_stage(om, prob, u, u, dt, 0.0, 1.0)
    assert i1["violations"] == 0 and i1["dte_reduced"] > 0

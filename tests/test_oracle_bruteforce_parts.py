"""Brute-force pins of the oracle's stage intermediates on small meshes (CPU).

Each intermediate is recomputed here from its defining integral with the
basis functions evaluated from the Bernstein formula, or for LGL meshes the
Lagrange product formula at the closed-form Lobatto points, and a high-order
Gauss rule (tests/bruteforce.py), element by element, independently of the
oracle's tables and operator algebra (m_i^e = int phi_i per node):
  * u^e = (1/|K_e|) int_K u_h, eq. (ueold);
  * f^H_ee' = (1/|S|) int_S f_h . n with the group flux f_h = sum_j f(u_j)
    phi_j, eq. (hoflux), for every flux (Euler included);
  * f_i^e of eq. (aec) as printed (periodic mesh: g_i^e = 0): m_i^e (u_i -
    u^e) + dt_e [ int grad phi_i . (f(u_h) - f_h) - int (phi_i - m_i^e/|K|)
    div f_h - s_h^e(phi_i, u_h) - int phi_i (udot_h - udot_i) ], with the
    sensor gamma_e, nu_e, g_h, udot and dt_e taken from the oracle (each
    pinned elsewhere) and the integrals by quadrature.
"""
import numpy as np
import pytest

import inputs
from inputs import Mesh, Problem
import oracle.physics as ph
import oracle.scheme as S
from tests.bruteforce import Brute

NQ = 12


def _flux(kind, U, prob):
    fx, fy = ph.flux(kind, U, prob)
    return np.asarray(fx), np.asarray(fy)


def _case(kind, p, basis=0):
    mesh = Mesh(3, 3, p, basis=basis)  # periodic
    if kind == inputs.FLUX_EULER:
        prob = Problem(flux=kind, mode=inputs.MODE_WENO, flux_limiter=S.FL_NONE)
        u = inputs.random_euler_state(mesh, 90 + p)
    else:
        prob = Problem(flux=kind, vx=0.7, vy=-0.3, mode=inputs.MODE_WENO, flux_limiter=S.FL_NONE,
                       umin=0.0, umax=4.0, w_lin=0.2)
        u = inputs.random_scalar_state(mesh, 80 + p + 10 * kind, 0.2, 2.0, 0.5)
    return mesh, prob.as_dict(), u


FLUXES = [inputs.FLUX_ADVECTION, inputs.FLUX_BURGERS, inputs.FLUX_KPP, inputs.FLUX_EULER]


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("kind", FLUXES)
@pytest.mark.parametrize("p", [1, 2, 3])
def test_cell_averages_by_quadrature(kind, p, basis):
    mesh, prob, u = _case(kind, p, basis)
    bf = Brute(mesh.nx, mesh.ny, p, mesh.x0, mesh.x1, mesh.y0, mesh.y1, True, nq=NQ, basis=basis)
    xi, eta, W = bf.quad2()
    B = bf.basis_at(xi, eta)
    nc = u.shape[0]
    uf = u.reshape(nc, -1)
    _, info = S.fe_stage(mesh, prob, u, 1e-4)
    for ex, ey in bf.elements():
        e = ey * mesh.nx + ex
        ids = [bf.gid(ex, ey, a, b) for (a, b) in bf.local()]
        for c in range(nc):
            uq = sum(uf[c, j] * B[l][0] for l, j in enumerate(ids))
            avg = np.sum(W * uq) / (bf.h * bf.h)
            assert abs(info["ue"][c, e] - avg) <= 1e-14 * max(1.0, abs(avg))


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("kind", FLUXES)
@pytest.mark.parametrize("p", [1, 2, 3])
def test_high_order_facet_fluxes_by_quadrature(kind, p, basis):
    """f^H on every canonical facet (x-facets: normal +x at x = i h; y-facets:
    +y at y = j h) as the face mean of the group flux."""
    mesh, prob, u = _case(kind, p, basis)
    om = S.OracleMesh(mesh)
    FHx, FHy = S.high_order_facets(om, u, prob)
    nc = u.shape[0]
    uf = u.reshape(nc, -1)
    bf = Brute(mesh.nx, mesh.ny, p, mesh.x0, mesh.x1, mesh.y0, mesh.y1, True, nq=NQ, basis=basis)
    s = bf.xq
    # face of element (ex, ey) at its west side (xi = 0) is the canonical
    # x-facet (ey, ex); its south side (eta = 0) the y-facet (ex, ey)
    for ex, ey in bf.elements():
        ids = [bf.gid(ex, ey, a, b) for (a, b) in bf.local()]
        fx, fy = _flux(kind, uf[:, ids], prob)            # nodal fluxes f(u_j), (nc, n2)
        for side, (xi, eta), (nx_, ny_), val in (
                ("W", (np.zeros_like(s), s), (1.0, 0.0), FHx[:, ey * om.nfx + ex]),
                ("S", (s, np.zeros_like(s)), (0.0, 1.0), FHy[:, ex * om.nfy + ey])):
            Bf = bf.basis_at(xi, eta)
            fh = sum((fx[:, l] * nx_ + fy[:, l] * ny_)[:, None] * Bf[l][0][None, :] for l in range(len(ids)))
            mean = (fh * bf.wq[None, :]).sum(axis=1)      # (1/|S|) int_S over the unit face parameter
            assert np.abs(val - mean).max() <= 1e-13 * max(1.0, np.abs(mean).max()), (side, val, mean)


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("kind", FLUXES)
@pytest.mark.parametrize("p", [1, 2])
def test_element_contributions_from_eq_aec(kind, p, basis):
    mesh, prob, u = _case(kind, p, basis)
    nc = u.shape[0]
    # the same high-order rule on both sides for the integrals of f(u_h)
    # (the stage's default p + 2 points are exact only for polynomial fluxes)
    om = S.OracleMesh(mesh, nq=NQ)
    _, info = S.fe_stage(om, prob, u, 1e-4)
    fie, dte, gam, nu = info["fie"], info["dte"], info["gamma"], info["nu"]
    ue = info["ue"]
    gx, gy, ud = info["gx"], info["gy"], info["udot"]
    bf = Brute(mesh.nx, mesh.ny, p, mesh.x0, mesh.x1, mesh.y0, mesh.y1, True, nq=NQ, basis=basis)
    xi, eta, W = bf.quad2()
    B = bf.basis_at(xi, eta)
    h = bf.h
    loc = bf.local()
    uf = u.reshape(nc, -1)
    for ex, ey in bf.elements():
        e = ey * mesh.nx + ex
        ids = [bf.gid(ex, ey, a, b) for (a, b) in bf.local()]
        n2 = len(ids)
        U = uf[:, ids]
        uq = np.array([sum(U[c, l] * B[l][0] for l in range(n2)) for c in range(nc)])
        uxq = np.array([sum(U[c, l] * B[l][1] for l in range(n2)) for c in range(nc)])
        uyq = np.array([sum(U[c, l] * B[l][2] for l in range(n2)) for c in range(nc)])
        fxq, fyq = _flux(kind, uq, prob)                   # f(u_h) at the points
        fxn, fyn = _flux(kind, U, prob)                    # f(u_j) at the nodes
        fhx = np.array([sum(fxn[c, l] * B[l][0] for l in range(n2)) for c in range(nc)])
        fhy = np.array([sum(fyn[c, l] * B[l][0] for l in range(n2)) for c in range(nc)])
        divfh = np.array([sum(fxn[c, l] * B[l][1] + fyn[c, l] * B[l][2] for l in range(n2)) for c in range(nc)])
        G = gx.reshape(nc, -1)[:, ids]
        Gy = gy.reshape(nc, -1)[:, ids]
        gxq = np.array([sum(G[c, l] * B[l][0] for l in range(n2)) for c in range(nc)])
        gyq = np.array([sum(Gy[c, l] * B[l][0] for l in range(n2)) for c in range(nc)])
        UD = ud.reshape(nc, -1)[:, ids]
        udq = np.array([sum(UD[c, l] * B[l][0] for l in range(n2)) for c in range(nc)])
        for i in range(n2):
            v, vx, vy = B[i]
            me = bf.mass_e(*loc[i])
            vol = np.sum(W * (vx * (fxq - fhx) + vy * (fyq - fhy)), axis=1)
            div = np.sum(W * (v - me / (h * h)) * divfh, axis=1)
            stab = nu[e] * np.sum(W * (vx * (uxq - gam[e] * gxq) + vy * (uyq - gam[e] * gyq)), axis=1)
            mass = np.sum(W * v * (udq - UD[:, i][:, None]), axis=1)
            ref = me * (U[:, i] - ue[:, e]) + dte[e] * (vol - div - stab - mass)
            sc = np.abs(fie[:, e, :]).max(axis=1) + 1e-300
            assert np.all(np.abs(fie[:, e, i] - ref) <= 1e-11 * sc), (e, i, fie[:, e, i], ref)

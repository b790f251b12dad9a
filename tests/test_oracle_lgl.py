"""Pins of the oracle on the Lagrange basis at the Legendre-Gauss-Lobatto
points, the collocated spectral-element basis the paper's concluding section
names as the next step (CPU).

The scheme is written with m_i^e = int phi_i throughout (eqs. (ueold),
(hoflux), (aec), (eq:SSPupdate)), so on an LGL mesh the oracle runs the same
stage with the Lagrange tables, the lumped masses |K| w_a w_b and the face
weights w_a.  What fixes each expected value:
  * the Lobatto points and weights: their closed forms (Simpson for p = 2,
    +-1/sqrt(5) for p = 3, +-sqrt(3/7) for p = 4), and the rule's exactness
    for polynomials of degree 2p - 1 (and not 2p);
  * the 1D tables: the Lagrange product formula evaluated independently
    (tests/bruteforce.py) and integrated with a high-order Gauss rule;
    continuation maps reproduce any polynomial of degree p;
  * p = 1: the Lagrange basis at the two Lobatto points is the Bernstein
    basis, so every stage equals the Bernstein oracle's;
  * mass conservation, free-stream preservation and the invariant domain;
  * the HO scheme with nodal initial data converges at the optimal rate
    p + 1 on the smooth 1D advection problem of Sec. 5.1.1 (y-independent).
The intermediates u^e, f^H and f_i^e are pinned by brute force in
tests/test_oracle_bruteforce_parts.py (basis 1).
"""
import math

import numpy as np
import pytest
from scipy.special import roots_legendre

import inputs
from inputs import Mesh, Problem
import oracle.scheme as S
import oracle.tables as T
from tests.bruteforce import LOBATTO, Brute, lagr


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lobatto_points_closed_form(p):
    x, w = T.lgl_points(p)
    xr, wr = LOBATTO[p]
    assert np.abs(x - np.array(xr)).max() <= 2e-16
    assert np.abs(w - np.array(wr)).max() <= 2e-16


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lobatto_rule_exact_to_degree_2p_minus_1(p):
    x, w = T.lgl_points(p)
    for k in range(2 * p):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) <= 1e-15
    assert abs(np.dot(w, x ** (2 * p)) - 1.0 / (2 * p + 1)) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_tables_by_quadrature(p):
    t = T.lgl_tables(p)
    n = p + 1
    xn = np.array(LOBATTO[p][0])
    g, wg = roots_legendre(2 * p + 4)
    xg, wg = 0.5 * (g + 1.0), 0.5 * wg
    L = [lagr(p, a, xg) for a in range(n)]
    dL = [lagr(p, a, xg, 1) for a in range(n)]
    M = np.array([[np.dot(wg, L[a] * L[b]) for b in range(n)] for a in range(n)])
    C = np.array([[np.dot(wg, dL[a] * L[b]) for b in range(n)] for a in range(n)])
    D = np.array([[np.dot(wg, dL[a] * dL[b]) for b in range(n)] for a in range(n)])
    for key, ref in (("M", M), ("C", C), ("D", D), ("S", None)):
        if ref is not None:
            assert np.abs(t[key] - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max()), key
    assert np.abs(t["S"][0] - M).max() <= 1e-14 and np.abs(t["S"][1] - D).max() <= 1e-12
    # the Lagrange property at the nodes and the node values at the ends
    B = np.array([[lagr(p, a, np.array([xb]))[0] for a in range(n)] for xb in t["xn"]])
    assert np.abs(B - np.eye(n)).max() <= 1e-14
    assert np.array_equal(t["B0"].round(14), np.eye(n)[0]) and np.array_equal(t["B1"].round(14), np.eye(n)[p])
    # values and derivatives at the stage's quadrature points
    Bq = np.array([[lagr(p, a, np.array([x]))[0] for a in range(n)] for x in t["xq"]])
    dBq = np.array([[lagr(p, a, np.array([x]), 1)[0] for a in range(n)] for x in t["xq"]])
    assert np.abs(t["Bq"] - Bq).max() <= 1e-13 and np.abs(t["dBq"] - dBq).max() <= 1e-12
    # int l_a = w_a, and continuation reproduces polynomials of degree p
    assert np.abs(t["M"].sum(axis=1) - np.array(LOBATTO[p][1])).max() <= 1e-15
    rng = np.random.default_rng(p)
    q = np.polynomial.Polynomial(rng.standard_normal(p + 1))
    assert np.abs(t["Ep"] @ q(xn + 1.0) - q(xn)).max() <= 1e-12 * np.abs(q(xn)).max()
    assert np.abs(t["Em"] @ q(xn - 1.0) - q(xn)).max() <= 1e-12 * np.abs(q(xn)).max()


def _cases():
    out = []
    for flux, mode, fl, bc in ((0, 3, 1, 0), (1, 2, 1, 2), (2, 3, 0, 2), (0, 1, 0, 1), (0, 0, 2, 0),
                               (3, 3, 1, 1), (3, 2, 0, 0)):
        out.append((flux, mode, fl, bc))
    return out


def _setup(flux, mode, fl, bc, p, basis, nx=5, ny=4):
    mesh = Mesh(nx, ny, p, 0.0, nx / ny, 0.0, 1.0, bc, bc, basis)
    if flux == inputs.FLUX_EULER:
        prob = Problem(flux=flux, mode=mode, flux_limiter=fl, ubc=(1.0, 0.1, -0.2, 2.5))
        u = inputs.random_euler_state(mesh, 40)
    else:
        lo, hi = (0.0, 1.0) if flux != inputs.FLUX_KPP else (math.pi / 4, 3.5 * math.pi)
        prob = Problem(flux=flux, mode=mode, flux_limiter=fl, vx=0.8, vy=-0.45, umin=lo, umax=hi,
                       ubc=(lo, 0, 0, 0), w_lin=0.2)
        u = inputs.random_scalar_state(mesh, 41, lo, hi, 0.4)
    return mesh, prob.as_dict(), u


@pytest.mark.parametrize("case", _cases())
def test_q1_lgl_equals_bernstein(case):
    """The two Lobatto points of p = 1 make the Lagrange basis the Bernstein
    one: same tables, masses and face weights, so the same stage."""
    mb, prob, u = _setup(*case, 1, 0)
    ml, _, _ = _setup(*case, 1, 1)
    dt = 0.5 * S.time_step(mb, prob, u)
    rb, ib = S.ssp_stage(S.OracleMesh(mb), prob, u, u, dt, 0.75, 0.25)
    rl, il = S.ssp_stage(S.OracleMesh(ml), prob, u, u, dt, 0.75, 0.25)
    sc = np.abs(rb).reshape(rb.shape[0], -1).max(axis=1)[:, None]
    assert (np.abs(rb - rl).reshape(rb.shape[0], -1) / sc).max() <= 1e-13
    for k in ("ue", "dte", "ube", "beta"):
        assert np.allclose(ib[k], il[k], rtol=1e-13, atol=1e-14), k


@pytest.mark.parametrize("case", [c for c in _cases() if c[0] != inputs.FLUX_EULER or (c[1], c[2]) == (3, 1)])
@pytest.mark.parametrize("p", [2, 3])
def test_lgl_conservation_and_invariant_domain(case, p):
    """Random data; Euler only with both limiters (positivity is not claimed
    for the unlimited WENO scheme)."""
    flux, mode, fl, bc = case
    mesh, prob, u = _setup(flux, mode, fl, bc, p, 1)
    u0 = u.copy()
    out, _, st = S.run(mesh, prob, u, 3)
    assert st["violations"] == 0
    if bc == 0:
        m0, m1 = S.mass(mesh, u0), S.mass(mesh, out)
        assert np.all(np.abs(m1 - m0) <= 1e-13 * np.maximum(1.0, np.abs(m0)))
    if flux == inputs.FLUX_EULER:
        assert np.all(out[0] > 0)
    elif mode in (0, 3):
        assert out.min() >= prob["umin"] and out.max() <= prob["umax"]


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("flux", [0, 3])
def test_lgl_free_stream(p, flux):
    mesh = Mesh(4, 4, p, basis=1)
    if flux == inputs.FLUX_EULER:
        prob = Problem(flux=3, mode=3).as_dict()
        u = np.broadcast_to(np.array([1.3, 0.4, -0.2, 2.9])[:, None, None], (4, mesh.nny, mesh.nnx)).copy()
    else:
        prob = Problem(flux=0, mode=3, vx=0.8, vy=-0.45).as_dict()
        u = np.full((1, mesh.nny, mesh.nnx), 0.37)
    out, _, _ = S.run(mesh, prob, u, 2)
    assert np.abs(out - u).max() <= 1e-14 * np.abs(u).max()


def test_subcell_bound_refused_on_lgl():
    mesh, prob, u = _setup(0, 3, 0, 0, 2, 1)
    prob["options"] = S.OPT_SUBCELL_DT
    with pytest.raises(ValueError):
        S.fe_stage(mesh, prob, u, 1e-4)


def _gauss(x):
    return np.exp(-100.0 * (x - 0.5) ** 2)


def _l2_error_1d(N, p, tend):
    """HO scheme (no limiting), Sec. 5.1.1 setting: v = (1, 0), nodal
    initial data u_j = u0(x_j), dt = h/12, k_g = k_u = 10; L2 error of u_h
    against the translated profile by a high-order Gauss rule."""
    mesh = Mesh(N, 1, p, 0.0, 1.0, 0.0, 1.0 / N, basis=1)
    prob = Problem(flux=0, vx=1.0, vy=0.0, mode=1, flux_limiter=S.FL_NONE, k_g=10, k_u=10).as_dict()
    X, _ = inputs.node_coords(mesh)
    u = _gauss(X)[None].copy()
    om = S.OracleMesh(mesh)
    dt = om.h / 12.0
    nsteps = int(round(tend / dt))
    for _ in range(nsteps):
        un = u
        for (a, b) in S.SSP3:
            u, _ = S.ssp_stage(om, prob, u, un, dt, a, b)
    bf = Brute(N, 1, p, 0.0, 1.0, 0.0, 1.0 / N, True, nq=p + 6, basis=1)
    xi, eta, W = bf.quad2()
    B = bf.basis_at(xi, eta)
    uf = u.reshape(-1)
    err = 0.0
    for ex, ey in bf.elements():
        ids = [bf.gid(ex, ey, a, b) for (a, b) in bf.local()]
        uq = sum(uf[j] * B[l][0] for l, j in enumerate(ids))
        xe = ((ex + xi) * bf.h - nsteps * dt) % 1.0
        err += np.sum(W * (uq - _gauss(xe)) ** 2)
    return math.sqrt(err * N)


@pytest.mark.parametrize("p,Ns,rate", [(2, (32, 64), 2.8), (3, (16, 32), 3.6)])
def test_lgl_ho_converges_at_optimal_rate(p, Ns, rate):
    e = [_l2_error_1d(N, p, 0.25) for N in Ns]
    assert math.log2(e[0] / e[1]) >= rate, e


@pytest.mark.parametrize("basis", [inputs.BASIS_BERNSTEIN, inputs.BASIS_LGL])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_blast_deposit_is_the_stated_energy(basis, p):
    """The blast recipe sizes its deposit with the basis's integral weights,
    so sum_i m_i u_i of the energy exceeds the background's by exactly the
    stated 0.25 in either basis (m_i: the oracle's lumped masses)."""
    mesh, prob, u0 = inputs.euler_blast_config(8, 8, p, basis=basis)
    bg = inputs.euler_primitive_to_conserved(np.ones(u0.shape[1:]), np.zeros(u0.shape[1:]),
                                             np.zeros(u0.shape[1:]), np.full(u0.shape[1:], 1e-6), 1.4)
    d = S.mass(mesh, u0) - S.mass(mesh, bg)
    assert abs(d[3] - 0.25) <= 1e-14 and np.abs(d[:3]).max() == 0.0


@pytest.mark.parametrize("p", [2, 3])
def test_lgl_blast_positivity(p):
    mesh, prob, u0 = inputs.euler_blast_config(8, 8, p, basis=inputs.BASIS_LGL)
    u1, t, st = S.run(mesh, prob.as_dict(), u0, 6)
    assert st["violations"] == 0
    assert np.all(u1[0] > 0)
    e_int = u1[3] - 0.5 * (u1[1] ** 2 + u1[2] ** 2) / u1[0]
    assert np.all(e_int > 0)

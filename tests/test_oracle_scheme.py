"""Pins for the oracle's stage (CPU only).

What fixes each expected value:
  * Theorem of Sec. 4 (MCL with alpha = beta = 1 equals CG-WENO): the
    oracle's limited-form update must equal a brute-force Galerkin
    right-hand side assembled in strong form (tests/bruteforce.py);
  * the same theorem implies independence from the pseudo time steps;
  * zero-sum property eq. (zerosum) and global conservation;
  * free-stream preservation;
  * the LO cell average is a finite-volume LLF update, eq. (uebar2);
  * Theorem 1 / eq. (fAlim) / eq. (slimit2): invariant-domain preservation;
  * sensor special cases (data that every candidate reproduces gives
    gamma = 1) and a brute-force semi-norm, eq. (WENO:norm);
  * the Richardson projection converges to the consistent L2 projection.
"""
import math

import numpy as np
import pytest

import inputs
from inputs import Mesh, Problem
import oracle.scheme as S
import oracle.physics as ph
from tests.bruteforce import Brute, bern


def _prob(**kw):
    p = Problem()
    for k, v in kw.items():
        setattr(p, k, v)
    return p.as_dict()


def _brute_rhs(mesh: Mesh, prob: dict, u2d, gamma, nu):
    """Brute-force CG-WENO right-hand side M_L^-1[r - M_C udot + M_L udot],
    r = -(a + b + s_h), with the same fixed Richardson counts (scalar)."""
    per = mesh.bc_x == inputs.BC_PERIODIC
    bf = Brute(mesh.nx, mesh.ny, mesh.p, mesh.x0, mesh.x1, mesh.y0, mesh.y1, per)
    MC, K, Gx, Gy = bf.matrices()
    m = MC.sum(axis=1)
    u = u2d.ravel()
    bgx, bgy = Gx @ u, Gy @ u
    gx, gy = bgx / m, bgy / m
    for _ in range(prob["k_g"]):
        gx = gx + (bgx - MC @ gx) / m
        gy = gy + (bgy - MC @ gy) / m
    if prob["flux"] == inputs.FLUX_ADVECTION:
        vx, vy = prob["vx"], prob["vy"]
        dflux = lambda w: (vx * np.ones_like(w), vy * np.ones_like(w))
        fn = lambda w, nx_, ny_: (vx * nx_ + vy * ny_) * w
        lam = lambda w, ub, nx_, ny_: abs(vx * nx_ + vy * ny_)
    else:  # Burgers
        dflux = lambda w: (w, w)
        fn = lambda w, nx_, ny_: 0.5 * w * w * (nx_ + ny_)
        lam = lambda w, ub, nx_, ny_: np.maximum(np.abs(w), abs(ub)) * abs(nx_ + ny_)
    Fllf = lambda w, ub, nx_, ny_: 0.5 * (fn(w, nx_, ny_) + fn(ub, nx_, ny_)) \
        - 0.5 * lam(w, ub, nx_, ny_) * (ub - w)
    a = bf.galerkin_strong(u, dflux)
    if mesh.bc_x == inputs.BC_OUTFLOW:
        b = np.zeros_like(a)
    else:
        b = bf.boundary_term(u, fn, Fllf, prob["ubc"][0])
    s = bf.element_stab(u, gx, gy, nu, gamma)
    r = -(a + b + s)
    ud = r / m
    for _ in range(prob["k_u"]):
        ud = ud + (r - MC @ ud) / m
    return (r - MC @ ud + m * ud) / m


CASES = [
    # (p, bc, flux, mode, k_g, k_u)
    (1, inputs.BC_PERIODIC, inputs.FLUX_ADVECTION, inputs.MODE_HO, 1, 0),
    (2, inputs.BC_PERIODIC, inputs.FLUX_ADVECTION, inputs.MODE_WENO, 1, 0),
    (3, inputs.BC_PERIODIC, inputs.FLUX_ADVECTION, inputs.MODE_WENO, 0, 2),
    (2, inputs.BC_FIXED, inputs.FLUX_ADVECTION, inputs.MODE_WENO, 2, 1),
    (2, inputs.BC_OUTFLOW, inputs.FLUX_ADVECTION, inputs.MODE_HO, 1, 0),
    (2, inputs.BC_PERIODIC, inputs.FLUX_BURGERS, inputs.MODE_WENO, 1, 1),
    # Burgers volume integrand has degree 3p per direction: the (p+2)-point
    # rule is exact for p <= 3 only
    (3, inputs.BC_PERIODIC, inputs.FLUX_BURGERS, inputs.MODE_HO, 1, 0),
    (4, inputs.BC_PERIODIC, inputs.FLUX_ADVECTION, inputs.MODE_WENO, 1, 1),
]


@pytest.mark.parametrize("p,bc,flux,mode,kg,ku", CASES)
def test_theorem_mcl_equals_cgweno(p, bc, flux, mode, kg, ku):
    """Sec. 4 Theorem: with alpha = beta = 1 the limited form reproduces
    the stabilised CG-WENO scheme eq. (weak:stab2)."""
    mesh = Mesh(3, 3, p, 0.0, 1.0, 0.0, 1.0, bc, bc)
    prob = _prob(flux=flux, vx=0.7, vy=-0.4, mode=mode, flux_limiter=S.FL_NONE,
                 k_g=kg, k_u=ku, ubc=(0.3, 0, 0, 0))
    u = inputs.random_scalar_state(mesh, 11 + p, 0.1, 0.9)
    dt = 1e-3
    ufe, info = S.fe_stage(mesh, prob, u, dt)
    rhs_o = (ufe - u).ravel() / dt
    gamma = info["gamma"]
    rhs_b = _brute_rhs(mesh, prob, u[0], gamma, info["nu"])
    scale = np.abs(rhs_b).max()
    assert np.abs(rhs_o - rhs_b).max() <= 1e-10 * scale, np.abs(rhs_o - rhs_b).max() / scale


def test_pseudo_time_step_independence(monkeypatch):
    """With beta = 1 and alpha = 1, dt_e cancels (proof of the Theorem)."""
    mesh = Mesh(4, 4, 2)
    prob = _prob(mode=inputs.MODE_WENO, flux_limiter=S.FL_NONE)
    u = inputs.random_scalar_state(mesh, 5)
    u1, _ = S.fe_stage(mesh, prob, u, 2e-3)
    orig = S.pseudo_time_steps
    monkeypatch.setattr(S, "pseudo_time_steps", lambda om, lo, pr: 0.37 * orig(om, lo, pr))
    u2, _ = S.fe_stage(mesh, prob, u, 2e-3)
    assert np.abs(u1 - u2).max() <= 1e-14 * np.abs(u).max()


@pytest.mark.parametrize("flux", [inputs.FLUX_ADVECTION, inputs.FLUX_BURGERS, inputs.FLUX_KPP])
def test_zero_sum_element_contributions(flux):
    """eq. (zerosum): sum_i f_i^e = 0 away from the boundary."""
    mesh = Mesh(4, 5, 3, 0.0, 1.0, 0.0, 1.25)
    prob = _prob(flux=flux, mode=inputs.MODE_WENO_L, umin=0.0, umax=4.0)
    u = inputs.random_scalar_state(mesh, 3, 0.5, 3.0)
    _, info = S.fe_stage(mesh, prob, u, 1e-4)
    fie = info["fie"]
    assert np.abs(fie.sum(axis=2)).max() <= 1e-14 * np.abs(fie).max() * fie.shape[2]
    assert np.abs(fie).max() > 0


@pytest.mark.parametrize("flux", [inputs.FLUX_ADVECTION, inputs.FLUX_BURGERS, inputs.FLUX_KPP])
@pytest.mark.parametrize("mode", [inputs.MODE_LO, inputs.MODE_WENO, inputs.MODE_WENO_L])
def test_global_conservation_periodic(flux, mode):
    """P3: sum_i m_i u_i is constant on periodic meshes (zero-sum f_i^e and
    antisymmetric facet fluxes)."""
    mesh = Mesh(6, 6, 2)
    prob = _prob(flux=flux, mode=mode, umin=0.0, umax=1.0,
                 flux_limiter=S.FL_LOW if mode == inputs.MODE_LO else S.FL_LIMITED)
    u = inputs.random_scalar_state(mesh, 9, 0.0, 1.0, 0.3)
    m0 = S.mass(mesh, u)
    u1, t, st = S.run(mesh, prob, u, 5)
    m1 = S.mass(mesh, u1)
    assert abs(m1[0] - m0[0]) <= 2e-15 * 30 * abs(m0[0])
    assert st["violations"] == 0


@pytest.mark.parametrize("flux", [inputs.FLUX_ADVECTION, inputs.FLUX_BURGERS, inputs.FLUX_KPP,
                                  inputs.FLUX_EULER])
@pytest.mark.parametrize("mode", [inputs.MODE_LO, inputs.MODE_HO, inputs.MODE_WENO,
                                  inputs.MODE_WENO_L])
def test_free_stream(flux, mode):
    """P4: a constant state stays constant."""
    mesh = Mesh(3, 4, 2, 0.0, 0.75, 0.0, 1.0, inputs.BC_OUTFLOW, inputs.BC_OUTFLOW)
    if flux == inputs.FLUX_EULER:
        c = inputs.euler_primitive_to_conserved(np.array(0.8), np.array(0.3),
                                                np.array(-0.2), np.array(0.6))
        u = np.broadcast_to(c[:, None, None], (4, mesh.nny, mesh.nnx)).copy()
        prob = _prob(flux=flux, mode=mode, w_lin=1e-3)
    else:
        u = np.full((1, mesh.nny, mesh.nnx), 0.42)
        prob = _prob(flux=flux, mode=mode, umin=0.0, umax=1.0)
    u1, _, _ = S.run(mesh, prob, u, 3)
    assert np.abs(u1 - u).max() <= 1e-13 * np.abs(u).max()


def test_low_order_average_is_fv_llf():
    """P6: ubar^{e,L} is the finite-volume LLF update of the cell averages
    with dt_e from eq. (dtmaxcell), written here as a plain element loop."""
    mesh = Mesh(5, 4, 2, 0.0, 1.25, 0.0, 1.0, inputs.BC_FIXED, inputs.BC_FIXED)
    vx, vy = 0.8, -0.35
    prob = _prob(flux=inputs.FLUX_ADVECTION, vx=vx, vy=vy, mode=inputs.MODE_LO,
                 flux_limiter=S.FL_LOW, ubc=(0.25, 0, 0, 0))
    u = inputs.random_scalar_state(mesh, 21)
    _, info = S.fe_stage(mesh, prob, u, 1e-3)
    p, h = mesh.p, mesh.h
    ue = np.zeros((mesh.ny, mesh.nx))
    for ey in range(mesh.ny):
        for ex in range(mesh.nx):
            ue[ey, ex] = u[0, ey * p:ey * p + p + 1, ex * p:ex * p + p + 1].mean()
    for ey in range(mesh.ny):
        for ex in range(mesh.nx):
            tot_lam, tot_F = 0.0, 0.0
            for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                jx, jy = ex + dx, ey + dy
                inside = 0 <= jx < mesh.nx and 0 <= jy < mesh.ny
                uR = ue[jy, jx] if inside else 0.25
                vn = vx * dx + vy * dy
                lam = abs(vn)
                tot_lam += lam
                tot_F += 0.5 * vn * (ue[ey, ex] + uR) - 0.5 * lam * (uR - ue[ey, ex])
            dte = h / tot_lam
            e = ey * mesh.nx + ex
            assert abs(info["dte"][e] - dte) <= 1e-15 * dte
            assert abs(info["ubL"][0, e] - (ue[ey, ex] - dte / h * tot_F)) <= 1e-15
    # LO stays within the range of the data and the boundary value
    lo = min(u.min(), 0.25)
    hi = max(u.max(), 0.25)
    u1, _, st = S.run(mesh, prob, u, 4)
    assert u1.min() >= lo - 1e-15 and u1.max() <= hi + 1e-15


@pytest.mark.parametrize("fl", [S.FL_LIMITED, S.FL_LOW])
def test_idp_weno_l_hump_and_disk(fl):
    """P9 / Theorem 1: zero bound violations with the flux and slope limiters."""
    mesh, prob, u0 = inputs.advection_config(16, 16, 2, flux_limiter=fl)
    u1, t, st = S.run(mesh, prob, u0, 15)
    assert st["violations"] == 0
    assert u1.min() >= 0.0 and u1.max() <= 1.0


def test_idp_kpp_small():
    mesh, prob, u0 = inputs.kpp_config(16, 16, 2)
    u1, t, st = S.run(mesh, prob, u0, 6)
    assert st["violations"] == 0
    assert u1.min() >= math.pi / 4 and u1.max() <= 3.5 * math.pi


def test_flux_limited_averages_in_bounds():
    """eq. (fAlim) keeps every ubar^e in [umin, umax] whenever ubar^{e,L} is."""
    mesh = Mesh(8, 8, 2)
    prob = _prob(mode=inputs.MODE_WENO_L, umin=0.0, umax=1.0, vx=1.0, vy=0.5)
    for seed in range(4):
        u = inputs.random_scalar_state(mesh, 100 + seed, 0.0, 1.0, 0.0)
        _, info = S.fe_stage(mesh, prob, u, 1e-3)
        assert info["ubL"].min() >= 0.0 and info["ubL"].max() <= 1.0
        assert info["ube"].min() >= -1e-15 and info["ube"].max() <= 1.0 + 1e-15
        ubi = info["ube"][:, :, None] + info["beta"][None, :, None] * info["fie"] / (mesh.h ** 2 / 9)
        assert ubi.min() >= -1e-14 and ubi.max() <= 1.0 + 1e-14


def test_sensor_linear_data_is_smooth():
    """Every candidate reproduces a global linear function, so u* = u_h and
    gamma_e = 1; linear data equal their Bernstein coefficients."""
    mesh = Mesh(5, 5, 3, 0.0, 1.0, 0.0, 1.0, inputs.BC_OUTFLOW, inputs.BC_OUTFLOW)
    X, Y = inputs.node_coords(mesh)
    u = (0.3 + 0.5 * X - 0.2 * Y)[None]
    om = S.OracleMesh(mesh)
    g = S.sensor(om, om.blocks(u), _prob())
    assert np.all(g > 1.0 - 1e-12)
    # a jump is flagged
    u2 = np.where(X > 0.5, 1.0, 0.0)[None]
    g2 = S.sensor(om, om.blocks(u2), _prob())
    assert g2.min() < 0.2
    assert np.all(g2[(om.EX == 0) | (om.EX == 4)] > 1.0 - 1e-12)


def test_seminorm_brute_force():
    """eq. (WENO:norm) on a square: sum_{1<=|k|<=p} h^{2|k|-2} int |D^k v|^2
    equals c^T A c, checked by direct quadrature of derivatives."""
    from scipy.special import roots_legendre
    p = 3
    om = S.OracleMesh(Mesh(2, 2, p, 0.0, 0.5, 0.0, 0.5))
    h = om.h
    rng = inputs.SplitMix64(7)
    c = rng.array(om.n2, -1, 1)
    t, w = roots_legendre(8)
    xq, wq = 0.5 * (t + 1), 0.5 * w
    XI, ETA = np.meshgrid(xq, xq, indexing="xy")
    W = np.outer(wq, wq)
    tot = 0.0
    for k1 in range(p + 1):
        for k2 in range(p + 1):
            if 1 <= k1 + k2 <= p:
                d = sum(c[b * (p + 1) + a] * bern(p, a, XI, k1) * bern(p, b, ETA, k2)
                        for b in range(p + 1) for a in range(p + 1)) / h ** (k1 + k2)
                tot += h ** (2 * (k1 + k2) - 2) * np.sum(W * d * d) * h * h
    assert abs(c @ om.A2 @ c - tot) <= 1e-12 * tot


def test_gradient_projection_richardson_limit():
    """k_g Richardson sweeps converge to the consistent L2 projection."""
    # p = 1: M_L^-1 M_C has spectrum in [1/9, 1], so 400 sweeps converge
    mesh = Mesh(3, 3, 1)
    bf = Brute(3, 3, 1, 0.0, 1.0, 0.0, 1.0, True)
    MC, K, Gx, Gy = bf.matrices()
    u = inputs.random_scalar_state(mesh, 4)
    om = S.OracleMesh(mesh)
    gx, gy = S.gradient_projection(om, om.blocks(u), _prob(k_g=400))
    ref = np.linalg.solve(MC, Gx @ u.ravel())
    assert np.abs(gx[0] - ref).max() <= 1e-12 * np.abs(ref).max()
    mesh = Mesh(3, 3, 2)
    bf = Brute(3, 3, 2, 0.0, 1.0, 0.0, 1.0, True)
    MC, K, Gx, Gy = bf.matrices()
    u = inputs.random_scalar_state(mesh, 4)
    om = S.OracleMesh(mesh)
    gx1, _ = S.gradient_projection(om, om.blocks(u), _prob(k_g=1))
    m = MC.sum(axis=1)
    b = Gx @ u.ravel()
    g0 = b / m
    assert np.abs(gx1[0] - (g0 + (b - MC @ g0) / m)).max() <= 1e-12 * np.abs(g0).max()


def test_lumped_masses_partition():
    for bc in (inputs.BC_PERIODIC, inputs.BC_FIXED):
        mesh = Mesh(3, 5, 3, 0.0, 0.6, 0.0, 1.0, bc, bc)
        om = S.OracleMesh(mesh)
        assert abs(om.mi.sum() - 0.6) <= 1e-15


def test_slope_limiter_is_maximal():
    """eq. (slimit2): beta_e is the largest factor keeping every
    ubar_i^e = ubar^e + beta f_i^e / m_i^e in [umin, umax]: when beta_e < 1
    some node sits on a bound."""
    mesh = Mesh(8, 8, 3)
    prob = _prob(mode=inputs.MODE_WENO_L, umin=0.0, umax=1.0)
    u = inputs.random_scalar_state(mesh, 41, 0.0, 1.0, 0.2)
    _, info = S.fe_stage(mesh, prob, u, 1e-3)
    m = mesh.h ** 2 / 16
    beta, ube, fie = info["beta"], info["ube"][0], info["fie"][0]
    ubi = ube[:, None] + beta[:, None] * fie / m
    gap = np.minimum(ubi - 0.0, 1.0 - ubi).min(axis=1)
    assert np.all(gap >= -1e-14)
    lim = beta < 1.0
    assert lim.sum() > 5
    assert np.all(gap[lim] <= 1e-13)


def test_flux_limiter_is_maximal():
    """eq. (fAlim): |fbar^A| <= |f^A| with equal sign, and whenever the flux
    is cut the intermediate state u_ee' of one side sits on a bound."""
    mesh = Mesh(5, 4, 2, 0.0, 1.25, 0.0, 1.0, inputs.BC_FIXED, inputs.BC_FIXED)
    om = S.OracleMesh(mesh)
    prob = _prob(umin=0.0, umax=1.0)
    rng = inputs.SplitMix64(8)
    ubL = rng.array(om.E, 0.0, 1.0)[None, :]
    dte = rng.array(om.E, 0.01, 0.05)
    for axis, nf in (("x", om.ny * om.nfx), ("y", om.nx * om.nfy)):
        fA = rng.array(nf, -3.0, 3.0)[None, :]
        fb = S.flux_limit(om, fA, ubL, dte, prob, axis)[0]
        assert np.all(fb * fA[0] >= 0) and np.all(np.abs(fb) <= np.abs(fA[0]))
        # side states u_ee' = ubar^{e,L} +- |dK| dt_e fbar / |K|
        k = S._facet_kind(om, axis)
        cut = np.abs(fb) < np.abs(fA[0])
        assert cut.sum() > 3
        for f in np.nonzero(cut)[0]:
            if axis == "x":
                ey, i = divmod(f, om.nfx)
                L = ey * om.nx + i - 1 if i > 0 else -1
                R = ey * om.nx + i if i < om.nx else -1
            else:
                ex, j = divmod(f, om.nfy)
                L = (j - 1) * om.nx + ex if j > 0 else -1
                R = j * om.nx + ex if j < om.ny else -1
            states = []
            if L >= 0:
                states.append(ubL[0, L] + 4 * dte[L] / om.h * fb[f])
            if R >= 0:
                states.append(ubL[0, R] - 4 * dte[R] / om.h * fb[f])
            d = min(min(abs(s - 0.0), abs(s - 1.0)) for s in states)
            assert d <= 1e-13
            assert all(-1e-14 <= s <= 1 + 1e-14 for s in states)

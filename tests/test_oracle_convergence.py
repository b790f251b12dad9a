"""Convergence pin of the oracle against the paper's Table 1 (CPU).

A y-independent run on an N x 1 periodic mesh reproduces the 1D setting of
Sec. 5.1.1: u0 = exp(-100 (x - 0.5)^2), v = (1, 0), t = 1, L2-projected
initial data.  The time step is the paper's omega_CFL = 0.5 of the subcell
bound of Lemma 1 for P2 without flux limiting (dt = h/12), and the two
mass-matrix solves are run close to convergence (k_g = k_u = 10), as the
paper solves them.

Expected values (tests/golden/table1_advection_1d_l2.txt):
  * P2 WENO: the L2 errors at 1/h = 32 and 64 agree with the paper's within
    25 %, and the rate between them is third order;
  * P2 WENO-L: bound clipping of the Bernstein coefficients limits the rate
    to about 2.4 (paper: 2.38);
  * P1 WENO: at least the optimal rate 2 on 1/h = 64 -> 128 (the paper
    reports superconvergence there; its sensor candidates are not given, so
    this is the bound checked).
"""
import os

import numpy as np
import pytest
from scipy.special import roots_legendre

import inputs
import oracle.scheme as S
from tests.bruteforce import bern

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_advection_1d_l2.txt")


def _golden():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    return {int(r[0]): [float(v) for v in r[1:]] for r in rows}


def _f(x):
    return np.exp(-100.0 * (x - 0.5) ** 2)


def _quad(om):
    t, w = roots_legendre(om.p + 5)
    xq, wq = 0.5 * (t + 1.0), 0.5 * w
    XI, ETA = np.meshgrid(xq, xq, indexing="xy")
    return XI.ravel(), ETA.ravel(), np.outer(wq, wq).ravel() * om.h * om.h


def l2_projection(om):
    XI, ETA, W = _quad(om)
    n = om.n1
    rhs = np.zeros(om.N)
    MC = np.zeros((om.N, om.N))
    for e in range(om.E):
        X = om.x0 + (om.EX[e] + XI) * om.h
        fv = _f(X)
        ids = om.conn[e]
        phis = [bern(om.p, a, XI) * bern(om.p, b, ETA) for b in range(n) for a in range(n)]
        for li, i in enumerate(ids):
            rhs[i] += np.sum(W * fv * phis[li])
            for lj, j in enumerate(ids):
                MC[i, j] += np.sum(W * phis[li] * phis[lj])
    return np.linalg.solve(MC, rhs)


def l2_error(om, c):
    XI, ETA, W = _quad(om)
    n = om.n1
    tot = 0.0
    for e in range(om.E):
        X = om.x0 + (om.EX[e] + XI) * om.h
        uh = sum(c[om.conn[e, b * n + a]] * bern(om.p, a, XI) * bern(om.p, b, ETA)
                 for b in range(n) for a in range(n))
        tot += np.sum(W * (uh - _f(X)) ** 2)
    return np.sqrt(tot / (om.h * om.ny))


def run_1d(N, p, mode):
    mesh = inputs.Mesh(N, 1, p, 0.0, 1.0, 0.0, 1.0 / N)
    om = S.OracleMesh(mesh)
    prob = inputs.Problem(flux=inputs.FLUX_ADVECTION, vx=1.0, vy=0.0, mode=mode,
                          flux_limiter=S.FL_NONE, cfl=1.0 / 6.0, umin=0.0, umax=1.0,
                          k_g=10, k_u=10, w_lin=1e-3).as_dict()
    c0 = l2_projection(om).reshape(1, om.nny, om.nnx)
    u, t, st = S.run(om, prob, c0, 100000, t_end=1.0)
    assert abs(t - 1.0) < 1e-12
    return l2_error(om, u.ravel())


@pytest.mark.slow
def test_table1_p2_weno():
    gold = _golden()
    e32 = run_1d(32, 2, inputs.MODE_WENO)
    e64 = run_1d(64, 2, inputs.MODE_WENO)
    for N, e in ((32, e32), (64, e64)):
        ref = gold[N][2]
        assert abs(e - ref) <= 0.25 * ref, (N, e, ref)
    eoc = np.log2(e32 / e64)
    assert 3.0 <= eoc <= 4.2, eoc


@pytest.mark.slow
def test_table1_p2_weno_l_clipping_rate():
    e32 = run_1d(32, 2, inputs.MODE_WENO_L)
    e64 = run_1d(64, 2, inputs.MODE_WENO_L)
    eoc = np.log2(e32 / e64)
    assert 2.0 <= eoc <= 2.7, eoc
    # clipping makes the limited P2 errors larger than the unlimited ones
    assert e64 > 5 * _golden()[64][2]


@pytest.mark.slow
def test_table1_p1_weno_rate():
    e64 = run_1d(64, 1, inputs.MODE_WENO)
    e128 = run_1d(128, 1, inputs.MODE_WENO)
    assert np.log2(e64 / e128) >= 2.0

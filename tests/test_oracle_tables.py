"""Pins for the oracle's exact 1D Bernstein tables (CPU).

Each check uses a fact fixed by the mathematics independently of the
oracle's polynomial arithmetic: closed forms from the Bernstein literature,
integration by parts, partition of unity (Sec. 2.1 of the paper), and
direct evaluation of the defining formula."""
from math import comb

import numpy as np
import pytest

from oracle.tables import tables


def bern(p, a, x):
    return comb(p, a) * x ** a * (1.0 - x) ** (p - a)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_partition_of_unity_and_nonnegativity(p):
    T = tables(p)
    x = np.linspace(0.0, 1.0, 37)
    vals = np.array([[bern(p, a, xx) for a in range(p + 1)] for xx in x])
    assert np.all(vals >= 0.0)
    assert np.allclose(vals.sum(axis=1), 1.0, atol=1e-15)
    assert np.allclose(T["Bq"].sum(axis=1), 1.0, atol=1e-15)
    assert np.allclose(T["dBq"].sum(axis=1), 0.0, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_mass_closed_form(p):
    # int_0^1 B_a B_b = C(p,a) C(p,b) / ((2p+1) C(2p, a+b))
    T = tables(p)
    for a in range(p + 1):
        for b in range(p + 1):
            ref = comb(p, a) * comb(p, b) / ((2 * p + 1) * comb(2 * p, a + b))
            assert abs(T["M"][a, b] - ref) <= 1e-16
    # int B_a = 1/(p+1): lumped mass m_i^e = |K|/|N_e| (Sec. 3)
    assert np.allclose(T["M"].sum(axis=1), 1.0 / (p + 1), atol=1e-16)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_derivative_tables_by_parts(p):
    T = tables(p)
    C, D, S = T["C"], T["D"], T["S"]
    n = p + 1
    # integration by parts: C[a,b] + C[b,a] = B_a B_b |_0^1
    e0 = np.zeros(n); e0[0] = 1.0
    e1 = np.zeros(n); e1[p] = 1.0
    assert np.allclose(C + C.T, np.outer(e1, e1) - np.outer(e0, e0), atol=1e-14)
    # sum_a B_a' = 0 kills the first index
    assert np.allclose(C.sum(axis=0), 0.0, atol=1e-14)
    assert np.allclose(D.sum(axis=0), 0.0, atol=1e-13)
    assert np.allclose(D, D.T)
    assert np.allclose(S[0], T["M"])
    assert np.allclose(S[1], D)
    # the p-th derivative of B_a is the constant p! C(p,a) (-1)^(p-a)
    from math import factorial
    cst = np.array([factorial(p) * comb(p, a) * (-1) ** (p - a) for a in range(n)], dtype=float)
    assert np.allclose(S[p], np.outer(cst, cst), rtol=1e-14)
    # numeric check of D against a fine midpoint rule of finite differences
    x = (np.arange(4000) + 0.5) / 4000
    eps = 1e-6
    d = np.array([[(bern(p, a, xx + eps) - bern(p, a, xx - eps)) / (2 * eps) for xx in x]
                  for a in range(n)])
    assert np.allclose(D, d @ d.T / len(x), atol=1e-5)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gauss_rule_exactness(p):
    T = tables(p)
    nq = T["nq"]
    for k in range(2 * nq):
        assert abs(np.dot(T["wq"], T["xq"] ** k) - 1.0 / (k + 1)) < 1e-15
    xq = T["xq"]
    for a in range(p + 1):
        assert np.allclose(T["Bq"][:, a], [bern(p, a, x) for x in xq], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_neighbour_continuation(p):
    # Ep[:, a] are the Bernstein coefficients on [0,1] of B_a(x - 1)
    T = tables(p)
    x = np.linspace(-0.3, 1.3, 17)
    for a in range(p + 1):
        lhs = np.array([sum(T["Ep"][b, a] * bern(p, b, xx) for b in range(p + 1)) for xx in x])
        rhs = np.array([comb(p, a) * (xx - 1) ** a * (2 - xx) ** (p - a) for xx in x])
        assert np.allclose(lhs, rhs, atol=1e-12)
        lhs = np.array([sum(T["Em"][b, a] * bern(p, b, xx) for b in range(p + 1)) for xx in x])
        rhs = np.array([comb(p, a) * (xx + 1) ** a * (-xx) ** (p - a) for xx in x])
        assert np.allclose(lhs, rhs, atol=1e-12)

"""Exact 1D Bernstein tables for the oracle (test infrastructure only).

Every polynomial is held as a list of exact rational monomial coefficients
(``fractions.Fraction``); integrals over [0, 1] are taken term by term
(int_0^1 x^n dx = 1/(n+1)), so each table entry is the exact rational
number rounded once to float64.  Gauss-Legendre nodes come from
``numpy.polynomial.legendre.leggauss`` (a library primitive).

Definitions (Sec. 2.1 of the paper, Bernstein basis of degree p on [0, 1]):
    B_a(x) = C(p, a) x^a (1 - x)^(p - a),  a = 0..p.
The 2D basis on the unit square is the tensor product B_a(xi) B_b(eta).
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import comb

import numpy as np


def bern_poly(p: int, a: int) -> list:
    """Monomial coefficients of B_a^p(x), exact."""
    c = [Fraction(0)] * (p + 1)
    for k in range(p - a + 1):
        c[a + k] += Fraction(comb(p, a) * comb(p - a, k) * (-1) ** k)
    return c


def poly_deriv(c: list, k: int = 1) -> list:
    for _ in range(k):
        c = [c[n] * n for n in range(1, len(c))] or [Fraction(0)]
    return c


def poly_mul(c1: list, c2: list) -> list:
    out = [Fraction(0)] * (len(c1) + len(c2) - 1)
    for i, a in enumerate(c1):
        for j, b in enumerate(c2):
            out[i + j] += a * b
    return out


def poly_int01(c: list) -> Fraction:
    return sum((cn / (n + 1) for n, cn in enumerate(c)), Fraction(0))


def poly_eval_exact(c: list, x: float) -> float:
    """Evaluate at a float point exactly, then round once."""
    xf = Fraction(x)
    acc = Fraction(0)
    for cn in reversed(c):
        acc = acc * xf + cn
    return float(acc)


def poly_shift(c: list, s: int) -> list:
    """Coefficients of q(x) = c(x + s) (binomial expansion, exact)."""
    out = [Fraction(0)] * len(c)
    for n, cn in enumerate(c):
        for k in range(n + 1):
            out[k] += cn * comb(n, k) * Fraction(s) ** (n - k)
    return out


def monomial_to_bernstein(c: list, p: int) -> list:
    """Bernstein coefficients on [0,1] of a polynomial of degree <= p given
    by monomial coefficients, using x^m = sum_{b>=m} C(b,m)/C(p,m) B_b(x)."""
    out = [Fraction(0)] * (p + 1)
    for m, cm in enumerate(c):
        if cm == 0:
            continue
        for b in range(m, p + 1):
            out[b] += cm * Fraction(comb(b, m), comb(p, m))
    return out


@lru_cache(maxsize=None)
def tables(p: int, nq: int | None = None) -> dict:
    """All 1D tables the oracle needs for degree p (float64 numpy arrays).

    M[a,b]   = int B_a B_b                  (1D mass)
    C[a,b]   = int B_a' B_b                 (derivative on the first index)
    D[a,b]   = int B_a' B_b'                (1D stiffness)
    S[k][a,b]= int B_a^(k) B_b^(k), k=0..p  (semi-norm blocks)
    xq, wq   : nq-point Gauss-Legendre rule on [0,1] (default nq = p + 2)
    Bq[q,a]  = B_a(xq[q]);  dBq[q,a] = B_a'(xq[q])
    Ep[b,a]  : Bernstein coefficients on [0,1] of B_a(x - 1)  (east neighbour
               polynomial continued onto [0,1])
    Em[b,a]  : the same for B_a(x + 1)  (west neighbour)
    """
    if nq is None:
        nq = p + 2
    polys = [bern_poly(p, a) for a in range(p + 1)]
    n = p + 1
    M = np.zeros((n, n))
    C = np.zeros((n, n))
    D = np.zeros((n, n))
    S = np.zeros((p + 1, n, n))
    for a in range(n):
        for b in range(n):
            M[a, b] = float(poly_int01(poly_mul(polys[a], polys[b])))
            C[a, b] = float(poly_int01(poly_mul(poly_deriv(polys[a]), polys[b])))
            D[a, b] = float(poly_int01(poly_mul(poly_deriv(polys[a]), poly_deriv(polys[b]))))
            for k in range(p + 1):
                S[k, a, b] = float(poly_int01(poly_mul(poly_deriv(polys[a], k),
                                                       poly_deriv(polys[b], k))))
    xg, wg = np.polynomial.legendre.leggauss(nq)
    xq = 0.5 * (xg + 1.0)
    wq = 0.5 * wg
    Bq = np.array([[poly_eval_exact(polys[a], x) for a in range(n)] for x in xq])
    dBq = np.array([[poly_eval_exact(poly_deriv(polys[a]), x) for a in range(n)] for x in xq])
    Ep = np.zeros((n, n))
    Em = np.zeros((n, n))
    for a in range(n):
        bp = monomial_to_bernstein(poly_shift(polys[a], -1), p)   # B_a(x - 1)
        bm = monomial_to_bernstein(poly_shift(polys[a], +1), p)   # B_a(x + 1)
        for b in range(n):
            Ep[b, a] = float(bp[b])
            Em[b, a] = float(bm[b])
    return dict(p=p, nq=nq, M=M, C=C, D=D, S=S, xq=xq, wq=wq, Bq=Bq, dBq=dBq, Ep=Ep, Em=Em,
                B1=np.array([poly_eval_exact(polys[a], 1.0) for a in range(n)]),
                B0=np.array([poly_eval_exact(polys[a], 0.0) for a in range(n)]),
                wl=np.full(n, 1.0 / n), xn=np.arange(n) / p, basis="bernstein")


# ---------------------------------------------------------------------------
# Lagrange basis at the Legendre-Gauss-Lobatto points (the collocated LGL
# spectral-element basis the paper's concluding section names as the next
# step).  The nodes on [-1, 1] are -1, 1 and the roots of P_p'; the weights
# are 2 / (p (p + 1) P_p(x_j)^2).  The polynomials are held as float64
# monomial coefficients (numpy.polynomial.polynomial, a library primitive);
# every integral is an exact Gauss-Legendre sum of a polynomial of degree
# at most 2p, so each table entry is accurate to rounding.
# ---------------------------------------------------------------------------
def lgl_points(p: int):
    """LGL nodes and weights on [0, 1] (weights sum to 1), ascending."""
    P = np.polynomial.legendre.Legendre.basis(p)
    inner = np.sort(np.real(P.deriv().roots())) if p >= 2 else np.zeros(0)
    xs = np.concatenate(([-1.0], inner, [1.0]))
    # one Newton polish of the interior roots on P_p'
    dP, d2P = P.deriv(), P.deriv(2)
    for _ in range(3):
        xs[1:-1] = xs[1:-1] - dP(xs[1:-1]) / d2P(xs[1:-1])
    w = 2.0 / (p * (p + 1) * P(xs) ** 2)
    return 0.5 * (xs + 1.0), 0.5 * w


def lagrange_polys(xn):
    """Monomial coefficients (ascending) of the Lagrange polynomials l_a
    with l_a(xn[b]) = delta_ab."""
    npoly = np.polynomial.polynomial
    out = []
    for a in range(len(xn)):
        c = np.array([1.0])
        for b in range(len(xn)):
            if b != a:
                c = npoly.polymul(c, np.array([-xn[b], 1.0]) / (xn[a] - xn[b]))
        out.append(c)
    return out


@lru_cache(maxsize=None)
def lgl_tables(p: int, nq: int | None = None) -> dict:
    """The tables of ``tables`` for the Lagrange basis at the LGL points:
    same keys and meanings with l_a in place of B_a; Ep[b, a] = l_a(xn[b] - 1)
    and Em[b, a] = l_a(xn[b] + 1) (a Lagrange coefficient is the value at
    the node); wl[a] = int_0^1 l_a (the LGL weight); xn the nodes."""
    if nq is None:
        nq = p + 2
    npoly = np.polynomial.polynomial
    xn, wl = lgl_points(p)
    L = lagrange_polys(xn)
    n = p + 1
    xg, wg = np.polynomial.legendre.leggauss(p + 2)      # exact to degree 2p + 3
    xg, wg = 0.5 * (xg + 1.0), 0.5 * wg

    def der(c, k):
        return npoly.polyder(c, k) if k > 0 else c

    def integ(c1, c2):
        return float(np.dot(wg, npoly.polyval(xg, c1) * npoly.polyval(xg, c2)))

    M = np.array([[integ(L[a], L[b]) for b in range(n)] for a in range(n)])
    C = np.array([[integ(der(L[a], 1), L[b]) for b in range(n)] for a in range(n)])
    D = np.array([[integ(der(L[a], 1), der(L[b], 1)) for b in range(n)] for a in range(n)])
    S = np.array([[[integ(der(L[a], k), der(L[b], k)) for b in range(n)] for a in range(n)]
                  for k in range(p + 1)])
    xq, wq = np.polynomial.legendre.leggauss(nq)
    xq, wq = 0.5 * (xq + 1.0), 0.5 * wq
    Bq = np.array([[npoly.polyval(x, L[a]) for a in range(n)] for x in xq])
    dBq = np.array([[npoly.polyval(x, der(L[a], 1)) for a in range(n)] for x in xq])
    Ep = np.array([[npoly.polyval(xn[b] - 1.0, L[a]) for a in range(n)] for b in range(n)])
    Em = np.array([[npoly.polyval(xn[b] + 1.0, L[a]) for a in range(n)] for b in range(n)])
    return dict(p=p, nq=nq, M=M, C=C, D=D, S=S, xq=xq, wq=wq, Bq=Bq, dBq=dBq, Ep=Ep, Em=Em,
                B1=np.array([npoly.polyval(1.0, L[a]) for a in range(n)]),
                B0=np.array([npoly.polyval(0.0, L[a]) for a in range(n)]),
                wl=wl, xn=xn, basis="lgl")


def basis_tables(p: int, nq: int | None = None, basis: int = 0) -> dict:
    """Tables of the Bernstein basis (basis 0) or the LGL Lagrange basis (1)."""
    return lgl_tables(p, nq) if basis == 1 else tables(p, nq)


def bern_eval(p: int, a: int, x: np.ndarray, k: int = 0) -> np.ndarray:
    """k-th derivative of B_a^p at points x (float evaluation, Horner)."""
    c = [float(v) for v in poly_deriv(bern_poly(p, a), k)]
    out = np.zeros_like(np.asarray(x, dtype=np.float64))
    for cn in reversed(c):
        out = out * x + cn
    return out

"""Brute-force global assembly for pinning the oracle (test code only).

Everything here is written from the definitions in Sec. 2 of the paper,
independently of oracle/: basis functions evaluated from the Bernstein
formula (or, for LGL meshes, the Lagrange product formula at the textbook
closed-form Lobatto points), global matrices assembled element by element
with a high-order Gauss rule from scipy, and the Galerkin form a(v, u) taken
in its STRONG form  sum_e int_K v div f(u_h)  (the oracle uses the weak form
with face terms; the two agree only if both are right)."""
from math import comb, sqrt

import numpy as np
from scipy.special import roots_legendre

# Legendre-Gauss-Lobatto points and weights on [0, 1] in closed form
# (textbook values: Simpson for p = 2; +-1/sqrt(5) and +-sqrt(3/7) on [-1, 1])
LOBATTO = {
    1: ([0.0, 1.0], [0.5, 0.5]),
    2: ([0.0, 0.5, 1.0], [1 / 6, 2 / 3, 1 / 6]),
    3: ([0.0, 0.5 * (1 - 1 / sqrt(5)), 0.5 * (1 + 1 / sqrt(5)), 1.0], [1 / 12, 5 / 12, 5 / 12, 1 / 12]),
    4: ([0.0, 0.5 * (1 - sqrt(3 / 7)), 0.5, 0.5 * (1 + sqrt(3 / 7)), 1.0],
        [1 / 20, 49 / 180, 16 / 45, 49 / 180, 1 / 20]),
}


def lagr(p, a, x, k=0):
    """k-th derivative (k <= 1) of the Lagrange polynomial l_a at the
    Lobatto points of degree p, from the product formula."""
    xn = LOBATTO[p][0]
    x = np.asarray(x, dtype=np.float64)
    others = [b for b in range(p + 1) if b != a]
    if k == 0:
        out = np.ones_like(x)
        for b in others:
            out = out * (x - xn[b]) / (xn[a] - xn[b])
        return out
    out = np.zeros_like(x)
    for c in others:
        term = np.full_like(x, 1.0 / (xn[a] - xn[c]))
        for b in others:
            if b != c:
                term = term * (x - xn[b]) / (xn[a] - xn[b])
        out = out + term
    return out


def bern(p, a, x, k=0):
    """k-th derivative of B_a^p at x via the derivative recursion."""
    if k == 0:
        if a < 0 or a > p:
            return np.zeros_like(x)
        return comb(p, a) * x ** a * (1.0 - x) ** (p - a)
    return p * (bern(p - 1, a - 1, x, k - 1) - bern(p - 1, a, x, k - 1))


class Brute:
    def __init__(self, nx, ny, p, x0, x1, y0, y1, periodic, nq=None, basis=0):
        self.nx, self.ny, self.p = nx, ny, p
        self.basis = basis
        self.h = (x1 - x0) / nx
        self.x0, self.y0 = x0, y0
        self.periodic = periodic
        self.nnx = nx * p + (0 if periodic else 1)
        self.nny = ny * p + (0 if periodic else 1)
        self.N = self.nnx * self.nny
        nq = nq or (2 * p + 3)
        t, w = roots_legendre(nq)
        self.xq = 0.5 * (t + 1.0)
        self.wq = 0.5 * w

    def gid(self, ex, ey, a, b):
        gx, gy = ex * self.p + a, ey * self.p + b
        if self.periodic:
            gx %= self.nnx
            gy %= self.nny
        return gy * self.nnx + gx

    def elements(self):
        for ey in range(self.ny):
            for ex in range(self.nx):
                yield ex, ey

    def local(self):
        p = self.p
        return [(a, b) for b in range(p + 1) for a in range(p + 1)]

    def phi1(self, a, x, k=0):
        """1D basis function a (or its derivative) at reference points."""
        return lagr(self.p, a, x, k) if self.basis == 1 else bern(self.p, a, x, k)

    def mass_e(self, a, b):
        """m_i^e = int_K phi_i for local node (a, b): |K|/(p+1)^2 (Bernstein)
        or |K| w_a w_b (LGL)."""
        if self.basis == 1:
            w = LOBATTO[self.p][1]
            return self.h * self.h * w[a] * w[b]
        return self.h * self.h / (self.p + 1) ** 2

    def basis_at(self, xi, eta):
        """values, d/dx, d/dy of all local basis functions at reference points."""
        p, h = self.p, self.h
        f = self.phi1
        out = []
        for (a, b) in self.local():
            v = f(a, xi) * f(b, eta)
            dx = f(a, xi, 1) * f(b, eta) / h
            dy = f(a, xi) * f(b, eta, 1) / h
            out.append((v, dx, dy))
        return out

    def quad2(self):
        XI, ETA = np.meshgrid(self.xq, self.xq, indexing="xy")
        W = np.outer(self.wq, self.wq)
        return XI.ravel(), ETA.ravel(), W.ravel() * self.h * self.h

    def matrices(self):
        N = self.N
        MC = np.zeros((N, N))
        K = np.zeros((N, N))
        Gx = np.zeros((N, N))   # int phi_i d_x phi_j
        Gy = np.zeros((N, N))
        xi, eta, W = self.quad2()
        B = self.basis_at(xi, eta)
        for ex, ey in self.elements():
            ids = [self.gid(ex, ey, a, b) for (a, b) in self.local()]
            for li, i in enumerate(ids):
                for lj, j in enumerate(ids):
                    MC[i, j] += np.sum(W * B[li][0] * B[lj][0])
                    K[i, j] += np.sum(W * (B[li][1] * B[lj][1] + B[li][2] * B[lj][2]))
                    Gx[i, j] += np.sum(W * B[li][0] * B[lj][1])
                    Gy[i, j] += np.sum(W * B[li][0] * B[lj][2])
        return MC, K, Gx, Gy

    def element_stab(self, u, gx, gy, nu, gamma):
        """s_i = sum_e nu_e int_K grad phi_i . (grad u_h - gamma_e g_h), eq. (stab:WENO)."""
        s = np.zeros(self.N)
        xi, eta, W = self.quad2()
        B = self.basis_at(xi, eta)
        for ex, ey in self.elements():
            e = ey * self.nx + ex
            ids = [self.gid(ex, ey, a, b) for (a, b) in self.local()]
            ux = sum(u[j] * B[l][1] for l, j in enumerate(ids))
            uy = sum(u[j] * B[l][2] for l, j in enumerate(ids))
            gxq = sum(gx[j] * B[l][0] for l, j in enumerate(ids))
            gyq = sum(gy[j] * B[l][0] for l, j in enumerate(ids))
            for l, i in enumerate(ids):
                s[i] += nu[e] * np.sum(W * (B[l][1] * (ux - gamma[e] * gxq)
                                             + B[l][2] * (uy - gamma[e] * gyq)))
        return s

    def galerkin_strong(self, u, dflux):
        """a(phi_i, u_h) = sum_e int_K phi_i div f(u_h) with div f = f'(u).grad u."""
        a = np.zeros(self.N)
        xi, eta, W = self.quad2()
        B = self.basis_at(xi, eta)
        for ex, ey in self.elements():
            ids = [self.gid(ex, ey, aa, bb) for (aa, bb) in self.local()]
            uq = sum(u[j] * B[l][0] for l, j in enumerate(ids))
            ux = sum(u[j] * B[l][1] for l, j in enumerate(ids))
            uy = sum(u[j] * B[l][2] for l, j in enumerate(ids))
            fpx, fpy = dflux(uq)
            div = fpx * ux + fpy * uy
            for l, i in enumerate(ids):
                a[i] += np.sum(W * B[l][0] * div)
        return a

    def galerkin_strong_system(self, U, jac):
        """a(phi_i, u_h) = sum_e int_K phi_i div f(u_h) for a system, with
        div f = A_x(u_h) d_x u_h + A_y(u_h) d_y u_h; U has shape (nc, N) and
        jac(uq) returns the flux Jacobians (A_x, A_y), each (nc, nc, nq)."""
        nc = U.shape[0]
        a = np.zeros((nc, self.N))
        xi, eta, W = self.quad2()
        B = self.basis_at(xi, eta)
        for ex, ey in self.elements():
            ids = [self.gid(ex, ey, aa, bb) for (aa, bb) in self.local()]
            uq = np.array([sum(U[c, j] * B[l][0] for l, j in enumerate(ids)) for c in range(nc)])
            ux = np.array([sum(U[c, j] * B[l][1] for l, j in enumerate(ids)) for c in range(nc)])
            uy = np.array([sum(U[c, j] * B[l][2] for l, j in enumerate(ids)) for c in range(nc)])
            Ax, Ay = jac(uq)
            div = np.einsum("abq,bq->aq", Ax, ux) + np.einsum("abq,bq->aq", Ay, uy)
            for l, i in enumerate(ids):
                a[:, i] += np.sum(W * B[l][0] * div, axis=1)
        return a

    def boundary_term(self, u, flux_n, F_llf, ub):
        """b(phi_i, u_h, u_hat) = int_dOmega phi_i [F(u_h, u_hat; n) - f(u_h).n] ds."""
        b = np.zeros(self.N)
        if self.periodic:
            return b
        p, h = self.p, self.h
        for ex, ey in self.elements():
            sides = []
            if ex == 0:
                sides.append(("W", (-1.0, 0.0)))
            if ex == self.nx - 1:
                sides.append(("E", (1.0, 0.0)))
            if ey == 0:
                sides.append(("S", (0.0, -1.0)))
            if ey == self.ny - 1:
                sides.append(("N", (0.0, 1.0)))
            for side, (nx_, ny_) in sides:
                s = self.xq
                if side == "W":
                    xi, eta = np.zeros_like(s), s
                elif side == "E":
                    xi, eta = np.ones_like(s), s
                elif side == "S":
                    xi, eta = s, np.zeros_like(s)
                else:
                    xi, eta = s, np.ones_like(s)
                B = self.basis_at(xi, eta)
                ids = [self.gid(ex, ey, aa, bb) for (aa, bb) in self.local()]
                uq = sum(u[j] * B[l][0] for l, j in enumerate(ids))
                val = F_llf(uq, ub, nx_, ny_) - flux_n(uq, nx_, ny_)
                for l, i in enumerate(ids):
                    b[i] += np.sum(self.wq * h * B[l][0] * val)
        return b

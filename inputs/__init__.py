"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module generates inputs only: mesh descriptions, problem parameters
and initial Bernstein coefficient arrays.  It holds none of the scheme's
arithmetic (no fluxes, no residuals, no limiters), so the oracle and the
CUDA path can both consume its output without sharing method code.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014), written out
here from its published definition.

Layout conventions (both sides rely on them):
  * global node (gx, gy) stores Bernstein coefficient u[c, gy, gx];
    x is the fastest index;
  * a periodic direction of n elements has n*p nodes, a non-periodic one
    n*p + 1;
  * nodal points are the uniform sub-grid x0 + gx*h/p (Sec. 2.1 of the
    paper: Bernstein nodes of a uniform quadrilateral mesh), and
    initialisation takes u_j(0) = u_0(x_j) (Sec. 5, numerical results).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

MASK64 = (1 << 64) - 1

BC_PERIODIC = 0
BC_OUTFLOW = 1
BC_FIXED = 2
BC_WALL = 3

FLUX_ADVECTION = 0
FLUX_BURGERS = 1
FLUX_KPP = 2
FLUX_EULER = 3

MODE_LO = 0
MODE_HO = 1
MODE_WENO = 2
MODE_WENO_L = 3
# element basis: Bernstein (the paper's) or Lagrange at the LGL points
BASIS_BERNSTEIN, BASIS_LGL = 0, 1

FP64 = 0
FP32_MIXED = 1

BASE_SEED = 2509046731


class SplitMix64:
    """splitmix64 counter-based generator (public-domain reference definition)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1)) if hi > lo else lo

    def array(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        return np.array([self.uniform(lo, hi) for _ in range(n)], dtype=np.float64)


@dataclass
class Mesh:
    nx: int
    ny: int
    p: int
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    bc_x: int = BC_PERIODIC
    bc_y: int = BC_PERIODIC
    basis: int = BASIS_BERNSTEIN

    @property
    def nnx(self) -> int:
        return self.nx * self.p + (0 if self.bc_x == BC_PERIODIC else 1)

    @property
    def nny(self) -> int:
        return self.ny * self.p + (0 if self.bc_y == BC_PERIODIC else 1)

    @property
    def h(self) -> float:
        return (self.x1 - self.x0) / self.nx

    def as_dict(self) -> dict:
        return asdict(self)


@dataclass
class Problem:
    """Problem parameters; defaults follow the paper where it states them."""
    flux: int = FLUX_ADVECTION
    vx: float = 1.0
    vy: float = 0.5
    gamma_gas: float = 1.4            # Sec. 5.2: gamma = 1.4
    mode: int = MODE_WENO_L
    flux_limiter: int = 1
    umin: float = 0.0
    umax: float = 1.0
    pos_eps: float = 1e-10            # Euler positivity margin
    q: float = 1.0                    # Sec. 5: q = 1 unless stated
    r: float = 2.0                    # Sec. 2.2: r = 2 (Jiang-Shu default)
    weno_eps: float = 1e-12
    w_lin: float = 1e-3               # Sec. 5.4: default 1e-3; Sec. 5.3 uses 0.2 (2D scalar)
    gamma_eps: float = 1e-12
    cfl: float = 0.2
    k_g: int = 1
    k_u: int = 1
    lambda_floor: float = 1e-12
    options: int = 0                  # bits as in cgl_problem.options
    ubc: tuple = (0.0, 0.0, 0.0, 0.0)
    # optional per-side boundary table {side: boundary_side(...)} for the
    # sides W, E, S, N; None: the mesh's bc_x / bc_y with the state ubc
    boundary: dict | None = None

    @property
    def ncomp(self) -> int:
        return 4 if self.flux == FLUX_EULER else 1

    def as_dict(self) -> dict:
        d = asdict(self)
        d["ubc"] = tuple(float(v) for v in self.ubc)
        return d


def _lobatto_offsets(p: int) -> np.ndarray:
    """Positions in [0, 1] of the p + 1 Legendre-Gauss-Lobatto points
    (0, 1 and the roots of P_p', by numpy's root finder), ascending; used
    only to place the nodal points of LGL meshes."""
    if p == 1:
        return np.array([0.0, 1.0])
    inner = np.sort(np.real(np.polynomial.legendre.Legendre.basis(p).deriv().roots()))
    return 0.5 * (np.concatenate(([-1.0], inner, [1.0])) + 1.0)


def node_coords(mesh: Mesh):
    """Physical coordinates of the nodal points, arrays of shape (nny, nnx):
    the uniform points x0 + k h/p for Bernstein meshes, the LGL points of
    each element for LGL meshes."""
    h = mesh.h
    hy = (mesh.y1 - mesh.y0) / mesh.ny
    gx = np.arange(mesh.nnx)
    gy = np.arange(mesh.nny)
    if getattr(mesh, "basis", BASIS_BERNSTEIN) == BASIS_LGL:
        off = _lobatto_offsets(mesh.p)
        x = mesh.x0 + ((gx // mesh.p) + off[gx % mesh.p]) * h
        y = mesh.y0 + ((gy // mesh.p) + off[gy % mesh.p]) * hy
    else:
        x = mesh.x0 + gx * (h / mesh.p)
        y = mesh.y0 + gy * (hy / mesh.p)
    return np.meshgrid(x, y, indexing="xy")


# --------------------------------------------------------------------------
# initial data recipes
# --------------------------------------------------------------------------

def _hump_and_slotted_disk(X, Y, rng: SplitMix64):
    """Cosine hump plus slotted disk with seeded centres, values in [0, 1]."""
    for _ in range(1000):
        c1 = (rng.uniform(0.2, 0.8), rng.uniform(0.2, 0.8))
        c2 = (rng.uniform(0.2, 0.8), rng.uniform(0.2, 0.8))
        r1 = rng.uniform(0.1, 0.18)
        r2 = rng.uniform(0.1, 0.18)
        slot = rng.uniform(0.02, 0.05)
        if math.hypot(c1[0] - c2[0], c1[1] - c2[1]) > r1 + r2 + 0.02:
            break
    rr = np.hypot(X - c1[0], Y - c1[1]) / r1
    u = np.where(rr < 1.0, 0.5 * (1.0 + np.cos(np.pi * np.minimum(rr, 1.0))), 0.0)
    in_disk = np.hypot(X - c2[0], Y - c2[1]) <= r2
    in_slot = (np.abs(X - c2[0]) <= slot) & (Y <= c2[1] + 0.5 * r2)
    u = np.where(in_disk & ~in_slot, 1.0, u)
    return u


def advection_config(nx=32, ny=32, p=2, seed_index=1, **prob):
    """2D linear advection, velocity (1, 0.5), periodic unit square."""
    mesh = Mesh(nx, ny, p)
    problem = Problem(flux=FLUX_ADVECTION, vx=1.0, vy=0.5, umin=0.0, umax=1.0, cfl=0.2,
                      w_lin=0.2)
    for k, v in prob.items():
        setattr(problem, k, v)
    X, Y = node_coords(mesh)
    u0 = _hump_and_slotted_disk(X, Y, SplitMix64(BASE_SEED + seed_index))
    return mesh, problem, u0[None, :, :].copy()


def kpp_config(nx=256, ny=256, p=2, basis=BASIS_BERNSTEIN, **prob):
    """KPP problem: f(u) = (sin u, cos u) on (-2,2)x(-2.5,1.5), u0 = 7pi/2 in r<=1
    else pi/4 (Sec. 5.3.2), fixed boundary state pi/4."""
    mesh = Mesh(nx, ny, p, -2.0, 2.0, -2.5, 1.5, BC_FIXED, BC_FIXED, basis)
    lo, hi = math.pi / 4, 3.5 * math.pi
    problem = Problem(flux=FLUX_KPP, umin=lo, umax=hi, cfl=0.2, w_lin=0.2,
                      ubc=(lo, 0.0, 0.0, 0.0))
    for k, v in prob.items():
        setattr(problem, k, v)
    X, Y = node_coords(mesh)
    u0 = np.where(np.hypot(X, Y) <= 1.0, hi, lo)
    return mesh, problem, u0[None, :, :].copy()


def euler_primitive_to_conserved(rho, vx, vy, p, gamma=1.4):
    """Input recipe helper: ideal-gas conserved variables from primitives."""
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)
    return np.stack([rho, rho * vx, rho * vy, E])


def euler_quadrant_config(nx=512, ny=512, p=3, seed_index=3, basis=BASIS_BERNSTEIN, **prob):
    """Four-quadrant Riemann data on the unit square, outflow boundaries."""
    mesh = Mesh(nx, ny, p, 0.0, 1.0, 0.0, 1.0, BC_OUTFLOW, BC_OUTFLOW, basis)
    problem = Problem(flux=FLUX_EULER, w_lin=1e-3, cfl=0.2, umin=0.0, umax=0.0)
    for k, v in prob.items():
        setattr(problem, k, v)
    rng = SplitMix64(BASE_SEED + seed_index)
    quad = []
    for _ in range(4):
        quad.append((rng.uniform(0.14, 1.5), rng.uniform(-0.7, 1.2),
                     rng.uniform(-0.7, 1.2), rng.uniform(0.14, 1.5)))
    X, Y = node_coords(mesh)
    qi = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int)
    prim = np.zeros((4,) + X.shape)
    for k in range(4):
        for c in range(4):
            prim[c][qi == k] = quad[k][c]
    u0 = euler_primitive_to_conserved(prim[0], prim[1], prim[2], prim[3], problem.gamma_gas)
    return mesh, problem, u0


def euler_blast_config(nx=2048, ny=2048, p=2, energy=0.25, basis=BASIS_BERNSTEIN, **prob):
    """Near-vacuum blast: rho=1, v=0, p=1e-6 background, total energy excess
    `energy` deposited on the nodes of the closed central 2x2 cell block."""
    assert nx % 2 == 0 and ny % 2 == 0
    mesh = Mesh(nx, ny, p, 0.0, 1.0, 0.0, 1.0, BC_OUTFLOW, BC_OUTFLOW, basis)
    problem = Problem(flux=FLUX_EULER, w_lin=1e-3, cfl=0.2, umin=0.0, umax=0.0)
    for k, v in prob.items():
        setattr(problem, k, v)
    g = problem.gamma_gas
    shape = (mesh.nny, mesh.nnx)
    u0 = euler_primitive_to_conserved(np.ones(shape), np.zeros(shape), np.zeros(shape),
                                      np.full(shape, 1e-6), g)
    cx, cy = nx // 2, ny // 2
    gx0, gx1 = (cx - 1) * p, (cx + 1) * p
    gy0, gy1 = (cy - 1) * p, (cy + 1) * p
    # integral weight of each block node, summed over the cells containing it:
    # |K|/(p+1)^2 per cell for Bernstein basis functions (Sec. 3), |K| w_a w_b
    # for the Lagrange basis at the LGL points (w: the Lobatto weights on
    # [0, 1], 1 / (p (p+1) P_p(x_a)^2) there); counted here only to size the
    # deposit.
    h = mesh.h
    if basis == BASIS_LGL:
        xa = _lobatto_offsets(p)
        wa = 1.0 / (p * (p + 1) * np.polynomial.legendre.Legendre.basis(p)(2.0 * xa - 1.0) ** 2)
        wcell = h * h * np.outer(wa, wa)
    else:
        wcell = np.full((p + 1, p + 1), h * h / (p + 1) ** 2)
    w = np.zeros(shape)
    for ey in range(cy - 2, cy + 2):
        for ex in range(cx - 2, cx + 2):
            w[ey * p:(ey + 1) * p + 1, ex * p:(ex + 1) * p + 1] += wcell
    block = np.zeros(shape, dtype=bool)
    block[gy0:gy1 + 1, gx0:gx1 + 1] = True
    total_w = w[block].sum()
    u0[3][block] += energy / total_w
    return mesh, problem, u0


def boundary_side(kind, state=(0.0, 0.0, 0.0, 0.0), kind_hi=None, state_hi=None, s0=math.inf, s1=0.0):
    """Boundary data of one side: points whose coordinate along the side lies
    below s0 + s1 t take (kind, state), the others (kind_hi, state_hi)
    (default: the same)."""
    kh = kind if kind_hi is None else kind_hi
    sh = state if state_hi is None else state_hi
    return {"kind": (int(kind), int(kh)),
            "state": (tuple(float(v) for v in state), tuple(float(v) for v in sh)),
            "s0": float(s0), "s1": float(s1)}


def dmr_states(gamma=1.4):
    """Post-shock and pre-shock states of the double Mach reflection (Sec. 5.4
    of the paper): (rho, vx, vy, p) = (8, 8.25 cos 30deg, -8.25 sin 30deg,
    116.5) and (1.4, 0, 0, 1), as conserved variables."""
    a = math.radians(30.0)
    post = euler_primitive_to_conserved(np.array(8.0), np.array(8.25 * math.cos(a)),
                                        np.array(-8.25 * math.sin(a)), np.array(116.5), gamma)
    pre = euler_primitive_to_conserved(np.array(1.4), np.array(0.0), np.array(0.0), np.array(1.0), gamma)
    return tuple(float(v) for v in post), tuple(float(v) for v in pre)


def dmr_config(ny=192, p=2, **prob):
    """Double Mach reflection on (0,4) x (0,1) with 4 ny x ny elements (Sec.
    5.4): post-shock state for x < 1/6 + y/sqrt(3), pre-shock state elsewhere
    (nodal values); boundary: W inflow (post-shock), E outflow, S post-shock
    inflow for x < 1/6 and reflecting wall for x >= 1/6, N post-shock inflow
    for x < 1/6 + (1 + 20 t)/sqrt(3) and pre-shock inflow beyond.  The
    paper's meshes: Q1 with ny = 384 and Q2 with ny = 192 (591,745 nodes)."""
    mesh = Mesh(4 * ny, ny, p, 0.0, 4.0, 0.0, 1.0, BC_OUTFLOW, BC_OUTFLOW)
    problem = Problem(flux=FLUX_EULER, w_lin=1e-3, q=1.0, cfl=0.2, umin=0.0, umax=0.0)
    for k, v in prob.items():
        setattr(problem, k, v)
    post, pre = dmr_states(problem.gamma_gas)
    r3 = math.sqrt(3.0)
    problem.boundary = {
        "W": boundary_side(BC_FIXED, post),
        "E": boundary_side(BC_OUTFLOW),
        "S": boundary_side(BC_FIXED, post, BC_WALL, post, s0=1.0 / 6.0),
        "N": boundary_side(BC_FIXED, post, BC_FIXED, pre, s0=1.0 / 6.0 + 1.0 / r3, s1=20.0 / r3),
    }
    X, Y = node_coords(mesh)
    left = X < 1.0 / 6.0 + Y / r3
    u0 = np.zeros((4,) + X.shape)
    for c in range(4):
        u0[c] = np.where(left, post[c], pre[c])
    return mesh, problem, u0


def batched_instances(n=256, seed_index=4, nmin=16, nmax=128, pmax=4):
    """Independent periodic instances of uneven size and degree: advection or
    Burgers, step + cosine hump initial data clipped to [0, 1]."""
    rng = SplitMix64(BASE_SEED + seed_index)
    out = []
    for _ in range(n):
        N = rng.randint(nmin, nmax)
        p = rng.randint(1, pmax)
        flux = FLUX_ADVECTION if rng.uniform() < 0.5 else FLUX_BURGERS
        ang = rng.uniform(0.0, 2.0 * math.pi)
        spd = rng.uniform(0.5, 1.0)
        mesh = Mesh(N, N, p)
        problem = Problem(flux=flux, vx=spd * math.cos(ang), vy=spd * math.sin(ang),
                          umin=0.0, umax=1.0, cfl=0.2, w_lin=0.2)
        X, Y = node_coords(mesh)
        ax, bx = sorted((rng.uniform(0.1, 0.9), rng.uniform(0.1, 0.9)))
        ay, by = sorted((rng.uniform(0.1, 0.9), rng.uniform(0.1, 0.9)))
        sv = rng.uniform(0.6, 1.0)
        hc = (rng.uniform(0.2, 0.8), rng.uniform(0.2, 0.8))
        hr = rng.uniform(0.1, 0.25)
        ha = rng.uniform(0.2, 0.4)
        step = np.where((X >= ax) & (X <= bx) & (Y >= ay) & (Y <= by), sv, 0.0)
        rr = np.hypot(X - hc[0], Y - hc[1]) / hr
        hump = np.where(rr < 1.0, ha * 0.5 * (1.0 + np.cos(np.pi * np.minimum(rr, 1.0))), 0.0)
        u0 = np.clip(step + hump, 0.0, 1.0)[None, :, :].copy()
        out.append((mesh, problem, u0))
    return out


def random_scalar_state(mesh: Mesh, seed: int, lo=0.0, hi=1.0, smooth_frac=0.5):
    """Random coefficients in [lo, hi]: a smooth wave plus seeded noise.
    Used by parity tests to exercise every limiter branch."""
    rng = SplitMix64(seed)
    X, Y = node_coords(mesh)
    L = mesh.x1 - mesh.x0
    kx, ky = rng.randint(1, 3), rng.randint(1, 3)
    ph = rng.uniform(0.0, 2 * math.pi)
    wave = 0.5 + 0.5 * np.sin(2 * np.pi * (kx * (X - mesh.x0) / L + ky * (Y - mesh.y0) / L) + ph)
    noise = rng.array(X.size).reshape(X.shape)
    u = smooth_frac * wave + (1.0 - smooth_frac) * noise
    return (lo + (hi - lo) * u)[None, :, :].copy()


def random_euler_state(mesh: Mesh, seed: int, gamma=1.4):
    """Random admissible Euler coefficients (rho, p in [0.2, 1.5], |v| <= 1)."""
    rng = SplitMix64(seed)
    n = mesh.nnx * mesh.nny
    rho = rng.array(n, 0.2, 1.5).reshape(mesh.nny, mesh.nnx)
    vx = rng.array(n, -1.0, 1.0).reshape(mesh.nny, mesh.nnx)
    vy = rng.array(n, -1.0, 1.0).reshape(mesh.nny, mesh.nnx)
    p = rng.array(n, 0.2, 1.5).reshape(mesh.nny, mesh.nnx)
    return euler_primitive_to_conserved(rho, vx, vy, p, gamma)

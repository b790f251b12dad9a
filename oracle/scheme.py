"""Plain FP64 CPU oracle of one SSP-RK stage of the element-based convex
limited CG-WENO scheme (Kuzmin, Hajduk, Vedral, arXiv 2509.04673).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this package.  It
shares no code with the CUDA path.

The stage follows the paper's summary of the algorithm (Sec. 4.3, steps
1-5), on a uniform mesh of square Q_p Bernstein elements, with dense
per-element matrices (no sum factorisation):

  1. cell averages u^e                                    eq. (ueold)
  2. facet speeds lambda_ee', pseudo time steps
     dt_e = |K_e| / sum |S_ee'| lambda_ee'               eq. (dtmaxcell)
     low-order cell fluxes f^L = F(u^e, u^e'; n)          Sec. 4, f^L
     low-order averages ubar^{e,L}                        eq. (uelowFCT)
  3. WENO sensor gamma_e                                  eqs. (WENO:alpha), (WENO:norm)
     viscosity nu_e = lambda_e h / (2p)                   eq. (stab:WENO)
  4. gradient projection g_h (consistent mass solved by
     lumped-preconditioned Richardson, k_g sweeps)        Sec. 2.2
  5. target residual r = -(a + b + s_h) and udot (k_u
     Richardson sweeps)                                   eqs. (weak:stab2), Sec. 4.3 step 2
  6. high-order facet fluxes f^H, antidiffusive fluxes
     f^A = f^L - f^H, flux limiter                        eqs. (hoflux), (flim), (fAlim), App. A
  7. limited averages ubar^e                              eq. (uelim)
  8. element contributions f_i^e                          eqs. (aec), (aecb)
  9. slope limiter beta_e                                 eqs. (slimit1), (slimit2), App. A
 10. SSP update u_i^SSP                                   eq. (eq:SSPupdate)

Readings of points the paper leaves open are listed in the design notes
and restated at each use below.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import physics as ph
from .tables import basis_tables

BC_PERIODIC, BC_OUTFLOW, BC_FIXED, BC_WALL = 0, 1, 2, 3
OPT_SUBCELL_DT = 4
OPT_AEC_Q1 = 8
OPT_DTE_REDUCE = 16
SIDES = ("W", "E", "S", "N")
# SSP-RK3 stage times t + c dt of the Shu-Osher stages
SSP3_C = (0.0, 1.0, 0.5)
MODE_LO, MODE_HO, MODE_WENO, MODE_WENO_L = 0, 1, 2, 3
FL_NONE, FL_LIMITED, FL_LOW = 0, 1, 2


def op2(Ax: np.ndarray, Ay: np.ndarray) -> np.ndarray:
    """2D tensor operator T[i, j] = Ax[a, c] * Ay[b, d] for local nodes
    i = b*(p+1) + a and j = d*(p+1) + c (x index fastest)."""
    n = Ax.shape[0]
    T = np.zeros((n * n, n * n))
    for b in range(n):
        for a in range(n):
            for d in range(n):
                for c in range(n):
                    T[b * n + a, d * n + c] = Ax[a, c] * Ay[b, d]
    return T


class OracleMesh:
    """Index sets of a uniform nx x ny mesh of degree-p squares (Table 1 of
    the paper: N_e, E_i, B_e) and dense element operators.  The basis is the
    paper's Bernstein basis, or (basis 1) the Lagrange basis at the LGL
    points, the collocated spectral-element basis of the concluding section:
    the scheme is written with m_i^e = int phi_i throughout, so the same
    stage runs on either basis with its own tables, lumped masses and face
    weights."""

    def __init__(self, mesh, nq=None):
        """nq: Gauss points per direction for the integrals of nonlinear
        functions (default p + 2, reading R7; the pins use a high-order rule
        to compare the weak form with a strong-form assembly)."""
        m = mesh if isinstance(mesh, dict) else mesh.as_dict()
        self.basis = int(m.get("basis", 0))
        self.nx, self.ny, self.p = int(m["nx"]), int(m["ny"]), int(m["p"])
        self.x0, self.x1, self.y0, self.y1 = m["x0"], m["x1"], m["y0"], m["y1"]
        self.bc_x, self.bc_y = int(m["bc_x"]), int(m["bc_y"])
        p, nx, ny = self.p, self.nx, self.ny
        self.h = (self.x1 - self.x0) / nx
        hy = (self.y1 - self.y0) / ny
        if abs(hy - self.h) > 1e-12 * abs(self.h):
            raise ValueError("square elements required")
        self.px = self.bc_x == BC_PERIODIC
        self.py = self.bc_y == BC_PERIODIC
        self.nnx = nx * p + (0 if self.px else 1)
        self.nny = ny * p + (0 if self.py else 1)
        self.N = self.nnx * self.nny
        self.E = nx * ny
        n = p + 1
        self.n1, self.n2 = n, n * n
        # N_e: global node index of local node (a, b) of element (ex, ey)
        ex = np.arange(nx)
        ey = np.arange(ny)
        conn = np.zeros((ny, nx, n, n), dtype=np.int64)  # [ey, ex, b, a]
        for b in range(n):
            for a in range(n):
                gx = ex * p + a
                gy = ey * p + b
                if self.px:
                    gx = gx % self.nnx
                if self.py:
                    gy = gy % self.nny
                conn[:, :, b, a] = gy[:, None] * self.nnx + gx[None, :]
        self.conn = conn.reshape(self.E, self.n2)
        # B_e: face neighbours W, E, S, N (-1 on a non-periodic boundary)
        EX, EY = np.meshgrid(ex, ey, indexing="xy")
        EX, EY = EX.ravel(), EY.ravel()

        def nb(dx, dy):
            jx, jy = EX + dx, EY + dy
            ok = np.ones_like(jx, dtype=bool)
            if self.px:
                jx = jx % nx
            else:
                ok &= (jx >= 0) & (jx < nx)
            if self.py:
                jy = jy % ny
            else:
                ok &= (jy >= 0) & (jy < ny)
            return np.where(ok, jy * nx + jx, -1)

        self.nbr = np.stack([nb(-1, 0), nb(1, 0), nb(0, -1), nb(0, 1)], axis=1)
        self.EX, self.EY = EX, EY
        # canonical facets: x-facet (ey, i) at x = x0 + i h between elements
        # (i-1, ey) [L] and (i, ey) [R]; y-facet (j, ex) between (ex, j-1) and (ex, j)
        self.nfx = nx if self.px else nx + 1
        self.nfy = ny if self.py else ny + 1
        # element -> facet indices (flat) for W, E, S, N
        self.fW = EY * self.nfx + EX
        self.fE = EY * self.nfx + ((EX + 1) % nx if self.px else EX + 1)
        self.fS = EX * self.nfy + EY          # y-facets stored [ex, j]
        self.fN = EX * self.nfy + ((EY + 1) % ny if self.py else EY + 1)
        # local node lists of the four faces (position along the face = index)
        a_idx = np.arange(n)
        self.face_nodes = {
            "W": a_idx * n + 0, "E": a_idx * n + p,
            "S": 0 * n + a_idx, "N": p * n + a_idx,
        }
        self._ops(nq)
        # lumped masses m_i^e = int_{K_e} phi_i and m_i = sum_{e in E_i} m_i^e
        # (Sec. 3).  Bernstein: |K| / (p+1)^2 for every i (kept as the scalar
        # me); LGL: |K| w_a w_b with the LGL weights, per local node (me_i).
        if self.basis == 0:
            self.me = self.h * self.h / self.n2
            self.me_i = np.full(self.n2, self.me)
            self.mi = np.bincount(self.conn.ravel(), minlength=self.N) * self.me
            # (m_i^e / |K_e|) |S| = h / (p+1)^2: the weight of the facet fluxes in eq. (aecb)
            self.kface = np.full(self.n2, self.h / self.n2)
        else:
            wl = self.T["wl"]
            self.me_i = self.h * self.h * np.outer(wl, wl).ravel()   # index b*n + a
            self.me = self.me_i
            self.mi = np.bincount(self.conn.ravel(), weights=np.tile(self.me_i, self.E), minlength=self.N)
            self.kface = self.h * np.outer(wl, wl).ravel()
        self.xn = self.T["xn"]

    def cell_mean(self, U):
        """(1/|K_e|) sum_i m_i^e U_i over the last axis (n2 values)."""
        if self.basis == 0:
            return U.mean(axis=-1)
        return U @ (self.me_i / (self.h * self.h))

    def face_mean(self, F):
        """(1/|S|) int_S f_h over one face from the values of f at its p + 1
        nodes (last axis): Bernstein 1/(p+1) each, LGL the weights w_a."""
        if self.basis == 0:
            return F.mean(axis=-1)
        return F @ self.T["wl"]

    def _ops(self, nq=None):
        T = basis_tables(self.p, nq, self.basis)
        self.T = T
        h, p, n = self.h, self.p, self.n1
        M, C, D = T["M"], T["C"], T["D"]
        self.Mass2 = h * h * op2(M, M)                      # int phi_i phi_j
        self.Stiff2 = op2(D, M) + op2(M, D)                 # int grad phi_i . grad phi_j
        self.Gx2 = h * op2(C, M)                            # int d_x phi_i phi_j
        self.Gy2 = h * op2(M, C)
        self.Bx2 = h * op2(C.T, M)                          # int phi_i d_x phi_j
        self.By2 = h * op2(M, C.T)
        nq = T["nq"]
        Bq, dBq, wq = T["Bq"], T["dBq"], T["wq"]
        self.Phi = np.zeros((nq * nq, self.n2))
        self.dPx = np.zeros((nq * nq, self.n2))
        self.dPy = np.zeros((nq * nq, self.n2))
        self.Wq = np.zeros(nq * nq)
        for q2 in range(nq):
            for q1 in range(nq):
                q = q2 * nq + q1
                self.Wq[q] = wq[q1] * wq[q2]
                for d in range(n):
                    for c in range(n):
                        j = d * n + c
                        self.Phi[q, j] = Bq[q1, c] * Bq[q2, d]
                        self.dPx[q, j] = dBq[q1, c] * Bq[q2, d]
                        self.dPy[q, j] = Bq[q1, c] * dBq[q2, d]
        # semi-norm (WENO:norm): sum over multi-indices 1 <= k1 + k2 <= p;
        # on a square the h-weights cancel, leaving reference integrals
        S = T["S"]
        A2 = np.zeros((self.n2, self.n2))
        for k1 in range(p + 1):
            for k2 in range(p + 1):
                if 1 <= k1 + k2 <= p:
                    A2 += op2(S[k1], S[k2])
        self.A2 = A2
        # continuation of neighbour polynomials onto K_e (x or y direction)
        I = np.eye(n)
        self.ExtW = op2(T["Em"], I)    # west neighbour lies on [-1, 0]
        self.ExtE = op2(T["Ep"], I)    # east neighbour lies on [1, 2]
        self.ExtS = op2(I, T["Em"])
        self.ExtN = op2(I, T["Ep"])

    # -- helpers ------------------------------------------------------------
    def blocks(self, u):
        """Element coefficient blocks, shape (nc, E, n2)."""
        return u.reshape(u.shape[0], -1)[:, self.conn]

    def gather(self, vals):
        """Sum of element vectors (nc, E, n2) into nodes (nc, N), eq. (mcl) sum over E_i."""
        out = np.zeros((vals.shape[0], self.N))
        for c in range(vals.shape[0]):
            out[c] = np.bincount(self.conn.ravel(), weights=vals[c].ravel(), minlength=self.N)
        return out


@dataclass
class StageOut:
    u: np.ndarray
    info: dict


def _prob(prob):
    return prob if isinstance(prob, dict) else prob.as_dict()


def boundary_table(om: OracleMesh, prob, nc):
    """Boundary data of the four sides W, E, S, N as
    {side: (kinds, states, s0, s1)}.  The part of a side whose coordinate
    (y on W and E, x on S and N) lies below s(t) = s0 + s1 t takes
    (kinds[0], states[0]), the rest (kinds[1], states[1]).  Without a
    "boundary" entry each non-periodic side takes its axis's bc and the
    state ubc everywhere (Sec. 2: weakly imposed data u_hat)."""
    b = prob.get("boundary")
    tab = {}
    for side in SIDES:
        if b is None:
            bc = om.bc_x if side in ("W", "E") else om.bc_y
            st = np.asarray(prob["ubc"][:nc], dtype=np.float64)
            tab[side] = ((bc, bc), (st, st), math.inf, 0.0)
        else:
            sd = b[side]
            kinds = tuple(int(k) for k in sd["kind"])
            states = tuple(np.asarray(list(x)[:nc], dtype=np.float64) for x in sd["state"])
            tab[side] = (kinds, states, float(sd["s0"]), float(sd["s1"]))
    return tab


def side_hi(spec, pos, ts):
    """True where a boundary point at coordinate pos lies at or above the
    split s0 + s1 ts of its side (stage time ts)."""
    _, _, s0, s1 = spec
    sp = s0 if s1 == 0.0 else s0 + s1 * ts
    return np.asarray(pos) >= sp


def side_is_plain(spec):
    """A side that is OUTFLOW everywhere: F(u, u; n) = f(u).n."""
    return spec[0][0] == BC_OUTFLOW and spec[0][1] == BC_OUTFLOW


def external_state(side, spec, hi, Uin):
    """u_hat at boundary points of one side from the interior states Uin
    (nc, ...): FIXED gives the side's state, OUTFLOW the interior state and
    WALL the interior state with the normal momentum reversed,
    m - 2 (m.n) n (a reflecting wall; the sides' normals are +-x, +-y)."""
    Uin = np.asarray(Uin, dtype=np.float64)
    out = Uin.copy()
    hi = np.broadcast_to(hi, Uin.shape[1:])
    for slot, sel in ((0, ~hi), (1, hi)):
        if not sel.any():
            continue
        kind, state = spec[0][slot], spec[1][slot]
        if kind == BC_FIXED:
            out[:, sel] = state[:, None]
        elif kind == BC_WALL:
            comp = 1 if side in ("W", "E") else 2
            out[comp, sel] = -Uin[comp, sel]
    return out


def cell_averages(om: OracleMesh, U):
    """u^e = (1/|K_e|) sum_i m_i^e u_i, eq. (ueold): the mean of the (p+1)^2
    Bernstein coefficients, the LGL-weighted mean of the nodal values."""
    return om.cell_mean(U)


def facet_states(om: OracleMesh, ue, prob, t=0.0):
    """Left/right cell states of the canonical x- and y-facets; on a
    non-periodic boundary the external state is u_hat of the side at the
    facet midpoint and time t, taken from the cell's own average (FIXED: the
    side's state; OUTFLOW: the average itself, the reading F(u, u; n) =
    f(u).n; WALL: the average with reversed normal momentum)."""
    nc = ue.shape[0]
    tab = boundary_table(om, prob, nc)
    nx, ny, h = om.nx, om.ny, om.h
    ue3 = ue.reshape(nc, ny, nx)
    out = {}
    # x-facets [ey, i]
    L = np.zeros((nc, ny, om.nfx))
    R = np.zeros((nc, ny, om.nfx))
    if om.px:
        R[:] = ue3
        L[:] = np.roll(ue3, 1, axis=2)
    else:
        R[:, :, :nx] = ue3
        L[:, :, 1:] = ue3
        ymid = om.y0 + (np.arange(ny) + 0.5) * h
        for side, col, dst in (("W", 0, (L, 0)), ("E", nx - 1, (R, nx))):
            spec = tab[side]
            own = ue3[:, :, col]
            dst[0][:, :, dst[1]] = external_state(side, spec, side_hi(spec, ymid, t), own)
    out["x"] = (L.reshape(nc, -1), R.reshape(nc, -1))
    # y-facets stored [ex, j]
    ueT = ue3.transpose(0, 2, 1)   # [c, ex, ey]
    L = np.zeros((nc, nx, om.nfy))
    R = np.zeros((nc, nx, om.nfy))
    if om.py:
        R[:] = ueT
        L[:] = np.roll(ueT, 1, axis=2)
    else:
        R[:, :, :ny] = ueT
        L[:, :, 1:] = ueT
        xmid = om.x0 + (np.arange(nx) + 0.5) * h
        for side, row, dst in (("S", 0, (L, 0)), ("N", ny - 1, (R, ny))):
            spec = tab[side]
            own = ueT[:, :, row]
            dst[0][:, :, dst[1]] = external_state(side, spec, side_hi(spec, xmid, t), own)
    out["y"] = (L.reshape(nc, -1), R.reshape(nc, -1))
    return out


def _facet_kind(om, axis):
    """Per canonical facet: 0 interior/periodic, -1 low boundary (element on
    the R side), +1 high boundary (element on the L side)."""
    if axis == "x":
        nf, per, n_other, ncell = om.nfx, om.px, om.ny, om.nx
        k = np.zeros((n_other, nf), dtype=int)
    else:
        nf, per, n_other, ncell = om.nfy, om.py, om.nx, om.ny
        k = np.zeros((n_other, nf), dtype=int)
    if not per:
        k[:, 0] = -1
        k[:, ncell] = 1
    return k.ravel()


def low_order_facets(om: OracleMesh, ue, prob, t=0.0):
    """lambda_ee' and f^L_ee' = F(u^e, u^e'; n_ee') on canonical facets
    (normal +x or +y), Sec. 3 eq. (uebar2) and Sec. 4 (f^L).  Boundary facets
    use the cell's outward normal and are stored with the canonical sign."""
    kind = prob["flux"]
    st = facet_states(om, ue, prob, t)
    res = {}
    for axis, (nx_, ny_) in (("x", (1.0, 0.0)), ("y", (0.0, 1.0))):
        L, R = st[axis]
        fk = _facet_kind(om, axis)
        F, lam = ph.llf(kind, L, R, nx_, ny_, prob)
        # low boundary: element is R, outward normal -n, external state is L
        lo = fk == -1
        if lo.any():
            Fo, lo_lam = ph.llf(kind, R[:, lo], L[:, lo], -nx_, -ny_, prob)
            F[:, lo] = -Fo
            lam[lo] = lo_lam
        res[axis] = (F, lam, fk)
    return res


def pseudo_time_steps(om: OracleMesh, lo, prob):
    """dt_e = |K_e| / sum_{e'} |S_ee'| lambda_ee', eq. (dtmaxcell); the speed
    sum is floored at lambda_floor (reading for zero-speed regions)."""
    lamx, lamy = lo["x"][1], lo["y"][1]
    s = lamx[om.fW] + lamx[om.fE] + lamy[om.fS] + lamy[om.fN]
    s = np.maximum(s, prob["lambda_floor"])
    return om.h * om.h / (om.h * s)


def subcell_time_steps(om: OracleMesh, U, prob):
    """dt_e^max of Lemma 1, eq. (dtmaxsubcell), the pseudo time step of the
    unlimited-flux variant (Sec. 4.3, step 4: flux limiter deactivated):

      dt_e = (1/s) min{ min_{i in N_e^b} m_i^e / (|c_ie| lambda_0i),
                        m_0^e / sum_{i in N_e^b} |c_ie| lambda_0i }

    N_e^b: the nodes on the element boundary; u_0^e: the mass-weighted mean
    of the interior nodes, m_0^e their mass; c_ie = int_{dK_e} phi_i n ds
    (|S|/(p+1) times the outward normal of each face through node i, so a
    corner node gets the diagonal); lambda_0i: the speed bound of the
    Riemann problem (u_0^e, u_i) along c_ie/|c_ie|; s = 1.  Without interior
    nodes (Q1): u_0^e = u^e, m_0^e = |K_e| and s = 2 (the lemma's second
    case).  Readings: a node term with zero speed is dropped, and the sum is
    floored at lambda_floor |S| (as eq. (dtmaxcell) floors its speed sum)."""
    if om.basis != 0:
        raise ValueError("the subcell bound of Lemma 1 is stated for Bernstein elements")
    kind = prob["flux"]
    p, n, h = om.p, om.n1, om.h
    nc = U.shape[0]
    me = om.me
    a_idx = np.arange(n * n) % n
    b_idx = np.arange(n * n) // n
    cx = np.where(a_idx == 0, -1.0, np.where(a_idx == p, 1.0, 0.0))
    cy = np.where(b_idx == 0, -1.0, np.where(b_idx == p, 1.0, 0.0))
    bnd = (cx != 0.0) | (cy != 0.0)
    if p >= 2:
        inner = ~bnd
        u0 = U[:, :, inner].mean(axis=2)                  # equal masses m_i^e
        m0 = inner.sum() * me
        s_fac = 1.0
    else:
        u0 = U.mean(axis=2)
        m0 = h * h
        s_fac = 2.0
    norm = np.sqrt(cx * cx + cy * cy)
    best = np.full(om.E, np.inf)
    total = np.zeros(om.E)
    for i in np.nonzero(bnd)[0]:
        c_abs = (h / (p + 1)) * norm[i]
        nx_, ny_ = cx[i] / norm[i], cy[i] / norm[i]
        lam = ph.max_speed(kind, u0, U[:, :, i], nx_, ny_, prob)
        w = c_abs * lam
        total = total + w
        with np.errstate(divide="ignore"):
            best = np.minimum(best, np.where(w > 0.0, me / np.where(w > 0.0, w, 1.0), np.inf))
    total = np.maximum(total, prob["lambda_floor"] * h)
    return np.minimum(best, m0 / total) / s_fac


def outward_sum(om: OracleMesh, Fx, Fy):
    """sum_{e'} of the outward canonical facet values of each element."""
    return Fx[:, om.fE] - Fx[:, om.fW] + Fy[:, om.fN] - Fy[:, om.fS]


def _seminorm2(V, A2):
    """Squared semi-norm c^T A c of each row of V.  A annihilates constants
    (the semi-norm has no k = 0 term), so each row is shifted by its first
    entry first: exact algebra that gives exact zeros for constant data and
    avoids cancellation for nearly constant data."""
    Vc = V - V[:, :1]
    return np.einsum("ei,ij,ej->e", Vc, A2, Vc)


def sensor(om: OracleMesh, U, prob):
    """WENO smoothness sensor gamma_e, eqs. (WENO:alpha), (WENO:norm).

    Readings: candidate 0 is u_h^e; candidates 1..n_e are the face
    neighbours' polynomials continued onto K_e (the semi-norm ignores the
    constant shift that would restore u^e's mean); missing neighbours on a
    non-periodic boundary are dropped, w_0 = 1 - n_e w_lin; r-th power of the
    semi-norm, absolute epsilon; ratio = num / (den + gamma_eps); systems
    take the minimum over components."""
    nc = U.shape[0]
    A2 = om.A2
    w_lin, r, eps, q, geps = prob["w_lin"], prob["r"], prob["weno_eps"], prob["q"], prob["gamma_eps"]
    gam = np.ones(om.E)
    exts = (om.ExtW, om.ExtE, om.ExtS, om.ExtN)
    for c in range(nc):
        # constants do not change any semi-norm, so every block is shifted by
        # its first coefficient before it is continued or compared (exact
        # algebra; keeps flat data exactly flat)
        U0 = U[c] - U[c][:, :1]
        cands = [U0]
        present = [np.ones(om.E, dtype=bool)]
        for k in range(4):
            nb = om.nbr[:, k]
            ok = nb >= 0
            Un = U[c][np.where(ok, nb, 0)]
            Un = Un - Un[:, :1]
            cands.append(Un @ exts[k].T)
            present.append(ok)
        ne = sum(pr.astype(float) for pr in present[1:])
        wt = []
        for l, (Ul, pr) in enumerate(zip(cands, present)):
            sig = np.maximum(_seminorm2(Ul, A2), 0.0)
            wl = (1.0 - ne * w_lin) if l == 0 else w_lin * pr
            wt.append(wl / (sig ** (0.5 * r) + eps))
        tot = sum(wt)
        # u_h^e - u_h^{e,*} = sum_{l>=1} omega_l (u_h^e - u_{h,l}^e) since
        # sum_l omega_l = 1 (no cancellation against omega_0 ~ 1)
        dlt = sum((w / tot)[:, None] * (U0 - Ul) for w, Ul in zip(wt[1:], cands[1:]))
        num = np.sqrt(np.maximum(_seminorm2(dlt, A2), 0.0))
        den = np.sqrt(np.maximum(_seminorm2(U0, A2), 0.0))
        ratio = num / (den + geps)
        gam = np.minimum(gam, 1.0 - np.minimum(1.0, ratio) ** q)
    return gam


def element_speed(om: OracleMesh, U, prob):
    """lambda_e = max over the element's coefficients of the state's speed bound."""
    return ph.node_speed(prob["flux"], U, prob).max(axis=1)


def gradient_projection(om: OracleMesh, U, prob):
    """g_h: L2 projection of grad u_h, M_C g = b with b_i = sum_e int phi_i grad u_h,
    solved by x0 = M_L^-1 b, x <- x + M_L^-1 (b - M_C x) (k_g sweeps)."""
    nc = U.shape[0]
    bx = om.gather(U @ om.Bx2.T)
    by = om.gather(U @ om.By2.T)
    gx = bx / om.mi
    gy = by / om.mi
    for _ in range(int(prob["k_g"])):
        gx = gx + (bx - om.gather(om.blocks(gx) @ om.Mass2.T)) / om.mi
        gy = gy + (by - om.gather(om.blocks(gy) @ om.Mass2.T)) / om.mi
    return gx, gy


def _face_geometry(om: OracleMesh):
    """(name, outward normal, facet-kind test, facet index array) per face."""
    return (("W", (-1.0, 0.0)), ("E", (1.0, 0.0)), ("S", (0.0, -1.0)), ("N", (0.0, 1.0)))


def boundary_face_mask(om: OracleMesh, name):
    if name == "W":
        return (om.EX == 0) & (not om.px)
    if name == "E":
        return (om.EX == om.nx - 1) & (not om.px)
    if name == "S":
        return (om.EY == 0) & (not om.py)
    return (om.EY == om.ny - 1) & (not om.py)


def element_residual(om: OracleMesh, U, prob, t=0.0):
    """W_i^e = int grad phi_i . f(u_h) - sum_{interior faces} int phi_i f_h.n
              - sum_{faces on dOmega} int phi_i F(u_h, u_hat; n).

    Summed over e in E_i this is -(a + b)(phi_i) of eq. (weak:galerkin):
    interior face terms of the continuous f_h cancel, and the derivation of
    the Theorem in Sec. 4 turns the remaining pieces into a and b.  The
    volume integral and the boundary integral of the nonlinear F use the
    (p+2)-point Gauss rule per direction (reading: quadrature is not fixed
    by the paper); f_h face integrals are exact (face mass matrix)."""
    kind = prob["flux"]
    nc = U.shape[0]
    h, n = om.h, om.n1
    T = om.T
    Uq = U @ om.Phi.T                                   # (nc, E, nq^2)
    fx, fy = ph.flux(kind, Uq, prob)
    W = h * ((fx * om.Wq) @ om.dPx + (fy * om.Wq) @ om.dPy)
    M = T["M"]
    tab = boundary_table(om, prob, nc)
    for name, (nxo, nyo) in _face_geometry(om):
        fn = om.face_nodes[name]
        Uf = U[:, :, fn]                                 # (nc, E, n) face coefficients
        bmask = boundary_face_mask(om, name)
        bmask = np.broadcast_to(bmask, (om.E,))
        # interior: int_S phi_i f_h.n = h sum_d M[b, d] f(u_d).n
        fnrm = ph.normal_flux(kind, Uf, nxo, nyo, prob)
        term = h * fnrm @ M.T
        if bmask.any():
            spec = tab[name]
            # boundary: int_S phi_i F(u_h, u_hat; n) ds by Gauss quadrature,
            # u_hat taken at each Gauss point of the face at time t
            Ufq = Uf[:, bmask] @ T["Bq"].T               # (nc, nb, nq)
            if side_is_plain(spec):
                Fq = ph.normal_flux(kind, Ufq, nxo, nyo, prob)
            else:
                # coordinate along the side of the Gauss points
                cell = (om.EY if name in ("W", "E") else om.EX)[bmask]
                o0 = om.y0 if name in ("W", "E") else om.x0
                pos = (o0 + cell * h)[:, None] + T["xq"][None, :] * h
                ext = external_state(name, spec, side_hi(spec, pos, t), Ufq)
                Fq, _ = ph.llf(kind, Ufq, ext, nxo, nyo, prob)
            term_b = h * (Fq * T["wq"]) @ T["Bq"]        # (nc, nb, n)
            term[:, bmask] = term_b
        W[:, :, fn] -= term
    return W


def high_order_facets(om: OracleMesh, u, prob, t=0.0):
    """f^H_ee' on canonical facets, eq. (hoflux): the face average of f_h.n,
    (1/(p+1)) sum_{j on S} f(u_j).n (Bernstein face integrals equal
    |S|/(p+1)); on a boundary side that is not OUTFLOW everywhere the
    average LLF flux f^d_ee' with the nodal Riemann data (u_j, u_hat_j),
    u_hat_j taken at time t and at the node's position on the element's face,
    x_e + k h/p (unwrapped: on a periodic direction the last node of the last
    element lies at x1, not at its periodic image x0)."""
    kind = prob["flux"]
    nc = u.shape[0]
    p, nx, ny = om.p, om.nx, om.ny
    tab = boundary_table(om, prob, nc)
    hn = om.h / p
    uu = u.reshape(nc, om.nny, om.nnx)
    b = np.arange(p + 1)
    # x-facets [ey, i]: face nodes gx = i p, gy = ey p + b
    GX = (np.arange(om.nfx) * p) % om.nnx
    GY = np.arange(ny)[:, None] * p + b[None, :]
    # positions along a side: the unwrapped node of the face, x_e + k h/p
    # (Bernstein) or x_e + xn_k h (LGL)
    if om.basis == 0:
        posy = om.y0 + GY * hn
    else:
        posy = om.y0 + (np.arange(ny)[:, None] + om.xn[None, :]) * om.h
    if om.py:
        GY = GY % om.nny
    Uf = uu[:, GY[:, None, :], GX[None, :, None]]            # (nc, ny, nfx, p+1)
    Fx = om.face_mean(ph.normal_flux(kind, Uf, 1.0, 0.0, prob))
    if not om.px:
        for side, i, sgn in (("W", 0, -1.0), ("E", nx, 1.0)):
            spec = tab[side]
            if side_is_plain(spec):
                continue
            Ub = Uf[:, :, i, :]
            ext = external_state(side, spec, side_hi(spec, posy, t), Ub)
            Fj, _ = ph.llf(kind, Ub, ext, sgn, 0.0, prob)
            Fx[:, :, i] = sgn * om.face_mean(Fj)
    # y-facets [ex, j]: face nodes gy = j p, gx = ex p + b
    GY = (np.arange(om.nfy) * p) % om.nny
    GX = np.arange(nx)[:, None] * p + b[None, :]
    if om.basis == 0:
        posx = om.x0 + GX * hn
    else:
        posx = om.x0 + (np.arange(nx)[:, None] + om.xn[None, :]) * om.h
    if om.px:
        GX = GX % om.nnx
    Uf = uu[:, GY[None, :, None], GX[:, None, :]]            # (nc, nx, nfy, p+1)
    Fy = om.face_mean(ph.normal_flux(kind, Uf, 0.0, 1.0, prob))
    if not om.py:
        for side, j, sgn in (("S", 0, -1.0), ("N", ny, 1.0)):
            spec = tab[side]
            if side_is_plain(spec):
                continue
            Ub = Uf[:, :, j, :]
            ext = external_state(side, spec, side_hi(spec, posx, t), Ub)
            Fj, _ = ph.llf(kind, Ub, ext, 0.0, sgn, prob)
            Fy[:, :, j] = sgn * om.face_mean(Fj)
    return Fx.reshape(nc, -1), Fy.reshape(nc, -1)


def euler_alpha(ubar, f, m, prob):
    """Appendix A correction factor bounds alpha_i = min(alpha_i^rho, alpha_i^p)
    for states ubar (4, ...) modified by ubar + alpha f / m.

    Reading of strict positivity: the admissible set keeps a margin,
    rho* >= eps rho_bar and the pressure constraint uses (1 - eps) Q_i."""
    eps = prob["pos_eps"]
    rho, mx, my, E = ubar[0], ubar[1], ubar[2], ubar[3]
    fr, fmx, fmy, fE = f[0], f[1], f[2], f[3]
    thr = m * rho * (1.0 - eps)
    with np.errstate(divide="ignore", invalid="ignore"):
        a_rho = np.where(thr + fr < 0.0, -thr / np.where(fr == 0.0, 1.0, fr), 1.0)
        Q = (1.0 - eps) * m * (0.5 * (mx * mx + my * my) - rho * E)
        Rr = rho * fE + E * fr - (mx * fmx + my * fmy) \
            + np.minimum(0.0, fE * fr - 0.5 * (fmx * fmx + fmy * fmy)) / m
        a_p = np.where(Rr < Q, Q / np.where(Rr == 0.0, 1.0, Rr), 1.0)
    return np.clip(np.minimum(a_rho, a_p), 0.0, 1.0)


def flux_limit(om: OracleMesh, fA, ubL, dte, prob, axis):
    """Limited antidiffusive facet fluxes fbar^A, eq. (fAlim) for scalars
    (global bounds) and Appendix A with N = 2 for Euler.  fA is canonical
    (flux from the L cell to the R cell)."""
    nc = fA.shape[0]
    fk = _facet_kind(om, axis)
    nx, ny = om.nx, om.ny
    if axis == "x":
        nf = om.nfx
        iy, ii = np.meshgrid(np.arange(ny), np.arange(nf), indexing="ij")
        iy, ii = iy.ravel(), ii.ravel()
        Lx = (ii - 1) % nx if om.px else ii - 1
        Rx = ii % nx if om.px else ii
        Le = np.where(Lx >= 0, iy * nx + np.clip(Lx, 0, nx - 1), -1)
        Re = np.where(Rx < nx, iy * nx + np.clip(Rx, 0, nx - 1), -1)
        if not om.px:
            Le[fk == -1] = -1
            Re[fk == 1] = -1
    else:
        nf = om.nfy
        ix, jj = np.meshgrid(np.arange(nx), np.arange(nf), indexing="ij")
        ix, jj = ix.ravel(), jj.ravel()
        Ly = (jj - 1) % ny if om.py else jj - 1
        Ry = jj % ny if om.py else jj
        Le = np.where(Ly >= 0, np.clip(Ly, 0, ny - 1) * nx + ix, -1)
        Re = np.where(Ry < ny, np.clip(Ry, 0, ny - 1) * nx + ix, -1)
        if not om.py:
            Le[fk == -1] = -1
            Re[fk == 1] = -1
    hasL, hasR = Le >= 0, Re >= 0
    Lc, Rc = np.where(hasL, Le, 0), np.where(hasR, Re, 0)
    h = om.h
    if prob["flux"] != ph.EULER:
        umin, umax = prob["umin"], prob["umax"]
        Qp = np.maximum(0.0, (h / 4.0) * (umax - ubL[0]) / dte)
        Qm = np.minimum(0.0, (h / 4.0) * (umin - ubL[0]) / dte)
        inf = np.inf
        # f^A >= 0: L gains, R loses; f^A < 0: L loses, R gains
        fmax = np.minimum(np.where(hasL, Qp[Lc], inf), np.where(hasR, -Qm[Rc], inf))
        fmin = np.maximum(np.where(hasL, Qm[Lc], -inf), np.where(hasR, -Qp[Rc], -inf))
        a = fA[0]
        return np.where(a >= 0.0, np.minimum(a, fmax), np.maximum(a, fmin))[None, :]
    # Euler, Appendix A with N = 2: u_1 = ubar^{L,L} + alpha fA / m_1,
    # m_1 = |K| / (|dK| dt_L); u_2 = ubar^{R,L} - alpha fA / m_2
    alpha = np.ones(fA.shape[1])
    mL = (h / 4.0) / dte[Lc]
    aL = euler_alpha(ubL[:, Lc], fA, mL, prob)
    alpha = np.where(hasL, np.minimum(alpha, aL), alpha)
    mR = (h / 4.0) / dte[Rc]
    aR = euler_alpha(ubL[:, Rc], -fA, mR, prob)
    alpha = np.where(hasR, np.minimum(alpha, aR), alpha)
    return alpha[None, :] * fA


def slope_limit(om: OracleMesh, fie, ube, prob):
    """beta_e = min_i beta_{i,e}, eqs. (slimit1)-(slimit2) for scalars with
    global bounds; Appendix A with N = |N_e| for Euler.  Clamped to [0, 1]."""
    m = om.me
    if prob["flux"] != ph.EULER:
        umin, umax = prob["umin"], prob["umax"]
        f = fie[0]
        gp = m * (umax - ube[0])[:, None]
        gm = m * (umin - ube[0])[:, None]
        with np.errstate(divide="ignore", invalid="ignore"):
            bp = np.minimum(1.0, gp / np.where(f > 0, f, 1.0))
            bm = np.minimum(1.0, gm / np.where(f < 0, f, -1.0))
        b = np.where(f > 0, bp, np.where(f < 0, bm, 1.0))
        return np.clip(b.min(axis=1), 0.0, 1.0)
    ub = np.broadcast_to(ube[:, :, None], fie.shape)
    return euler_alpha(ub, fie, m, prob).min(axis=1)


def in_domain(prob, ub):
    """Per element: is the average ub (nc, E) in G?  Scalars: umin <= ub <=
    umax; Euler: rho > 0 and rho E - |m|^2/2 > 0 (p > 0)."""
    if prob["flux"] == ph.EULER:
        return (ub[0] > 0.0) & (ub[0] * ub[3] - 0.5 * (ub[1] ** 2 + ub[2] ** 2) > 0.0)
    return (ub[0] >= prob["umin"]) & (ub[0] <= prob["umax"])


def reduced_time_steps(prob, ue, osum, rs):
    """The strategy of the remark after eq. (dtmaxcell) for the unlimited
    averages of eq. (uebar), ubar^e(r) = u^e - r S_e with r = dt_e / h and
    S_e the outward sum of the facet fluxes f^H: where ubar^e(rs) leaves G,
    the largest r in [0, rs] with ubar^e(r) in G (returned as r).  Scalars:
    the bound that is crossed, solved exactly (u^e itself lies in G).  Euler
    (reading): the largest r allowed by the positivity criterion of
    Appendix A for the state u^e moved by r S_e: rho >= eps rho^e and the
    linear minorant of rho E - |m|^2/2 at least eps times its value at u^e,
    i.e. r = rs alpha(u^e, -rs S_e, m = 1)."""
    keep = in_domain(prob, ue - rs * osum)
    if prob["flux"] == ph.EULER:
        alpha = euler_alpha(ue, -rs[None, :] * osum, np.ones_like(rs), prob)
        return np.where(keep, rs, rs * alpha)
    umin, umax = prob["umin"], prob["umax"]
    d = osum[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        r_hi = np.where(d < 0.0, (umax - ue[0]) / np.where(d < 0.0, -d, 1.0), np.inf)
        r_lo = np.where(d > 0.0, (ue[0] - umin) / np.where(d > 0.0, d, 1.0), np.inf)
    r = np.maximum(np.minimum(rs, np.minimum(r_hi, r_lo)), 0.0)
    return np.where(keep, rs, r)


def fe_stage(mesh, prob, u, dt, t=0.0):
    """One forward-Euler stage u -> u^SSP, eq. (eq:SSPupdate), with all
    intermediates.  u has shape (nc, nny, nnx); t is the stage time, which
    only time-dependent boundary data use."""
    prob = _prob(prob)
    om = mesh if isinstance(mesh, OracleMesh) else OracleMesh(mesh)
    kind, mode, fl = prob["flux"], int(prob["mode"]), int(prob["flux_limiter"])
    nc = u.shape[0]
    uf = u.reshape(nc, -1)
    U = om.blocks(u)
    ue = cell_averages(om, U)
    lo = low_order_facets(om, ue, prob, t)
    dte = pseudo_time_steps(om, lo, prob)
    if int(prob.get("options", 0)) & OPT_SUBCELL_DT:
        dte = subcell_time_steps(om, U, prob)
    FLx, FLy = lo["x"][0], lo["y"][0]
    ubL = ue - (dte / om.h) * outward_sum(om, FLx, FLy)          # eq. (uelowFCT)
    info = dict(ue=ue, dte=dte, ubL=ubL, ubar_outside=0, dte_reduced=0)
    need_ho = mode != MODE_LO or fl != FL_LOW
    if need_ho:
        FHx, FHy = high_order_facets(om, u, prob, t)
    # limited cell averages, eq. (uelim)
    if fl == FL_LOW:
        ube = ubL.copy()
    elif fl == FL_NONE:
        osum = outward_sum(om, FHx, FHy)
        rs = dte / om.h
        ube = ue - rs * osum                                      # eq. (uebar)
        info["ubar_outside"] = int(np.count_nonzero(~in_domain(prob, ube)))
        if int(prob.get("options", 0)) & OPT_DTE_REDUCE:
            # remark after eq. (dtmaxcell): decrease dt_e where ubar^e left G
            rs2 = reduced_time_steps(prob, ue, osum, rs)
            info["dte_reduced"] = int(np.count_nonzero(rs2 < rs))
            dte = rs2 * om.h
            ube = ue - rs2 * osum
            info["dte"] = dte
    else:
        fAx = FLx - FHx
        fAy = FLy - FHy
        fbx = flux_limit(om, fAx, ubL, dte, prob, "x")
        fby = flux_limit(om, fAy, ubL, dte, prob, "y")
        ube = ubL + (dte / om.h) * outward_sum(om, fbx, fby)
    info["ube"] = ube
    theta = dt / dte
    me = om.me
    if mode == MODE_LO:
        beta = np.zeros(om.E)
        fie = np.zeros_like(U)
        gamma = np.zeros(om.E)
    elif int(prob.get("options", 0)) & OPT_AEC_Q1:
        gamma = sensor(om, U, prob) if mode in (MODE_WENO, MODE_WENO_L) else np.ones(om.E)
        fie, udl = aec_q1(om, U, ue, ube, dte, gamma, prob)
        beta = slope_limit(om, fie, ube, prob) if mode == MODE_WENO_L else np.ones(om.E)
        info.update(gamma=gamma, udot_l=udl, fie=fie)
    else:
        gamma = sensor(om, U, prob) if mode in (MODE_WENO, MODE_WENO_L) else np.ones(om.E)
        lam_e = element_speed(om, U, prob)
        nu = lam_e * om.h / (2.0 * om.p)
        gx, gy = gradient_projection(om, U, prob)
        Gx, Gy = om.blocks(gx.reshape(u.shape)), om.blocks(gy.reshape(u.shape))
        W = element_residual(om, U, prob, t)
        s = nu[None, :, None] * (U @ om.Stiff2.T
                                 - gamma[None, :, None] * (Gx @ om.Gx2.T + Gy @ om.Gy2.T))
        Rl = W - s
        r = om.gather(Rl)
        ud = r / om.mi
        for _ in range(int(prob["k_u"])):
            ud = ud + (r - om.gather(om.blocks(ud.reshape(u.shape)) @ om.Mass2.T)) / om.mi
        UD = om.blocks(ud.reshape(u.shape))
        fHsum = outward_sum(om, FHx, FHy)
        # eq. (aec) with eq. (aecb) folded in (see element_residual)
        fie = me * (U - ue[:, :, None]) + dte[None, :, None] * (
            Rl + om.kface * fHsum[:, :, None] - UD @ om.Mass2.T + me * UD)
        if mode == MODE_WENO_L:
            beta = slope_limit(om, fie, ube, prob)
        else:
            beta = np.ones(om.E)
        info.update(gamma=gamma, nu=nu, gx=gx, gy=gy, r=r, udot=ud, fie=fie)
    info["beta"] = beta
    info["theta"] = theta
    # eq. (eq:SSPupdate): m_i u_i = sum_e m_i^e [(1 - dt/dt_e) u_i + (dt/dt_e) ubar_i^e]
    ubi = ube[:, :, None] + beta[None, :, None] * fie / me
    w = me * ((1.0 - theta)[None, :, None] * U + theta[None, :, None] * ubi)
    unew = om.gather(w) / om.mi
    return unew.reshape(u.shape), info


def low_order_time_derivative(om: OracleMesh, U, ube, dte):
    """udot^L_i of the low-order scheme, eq. (weak:low2):
    m_i udot^L_i = sum_{e in E_i} m_i^e (ubar^e - u_i) / dt_e, with the
    stage's intermediate averages ubar^e (reading for the 'low-order
    approximation to the time derivative' of eq. (aecQ1))."""
    w = om.me * (ube[:, :, None] - U) / dte[None, :, None]
    return om.gather(w) / om.mi


def flux_divergence_term(om: OracleMesh, U, prob):
    """D_i = int_{K_e} (phi_i - m_i^e/|K_e|) div f_h dx of eq. (aecQ1), with
    f_h = sum_j f(u_j) phi_j (eq. (gfe)): sum_j (B_ij - (m_i^e/|K_e|) c_j) . f(u_j),
    B_ij = int phi_i grad phi_j, c_j = int grad phi_j = sum_i B_ij."""
    fx, fy = ph.flux(prob["flux"], U, prob)             # (nc, E, n2) nodal fluxes
    cx = om.Bx2.sum(axis=0)
    cy = om.By2.sum(axis=0)
    return fx @ om.Bx2.T + fy @ om.By2.T - (om.me / (om.h * om.h)) * (fx @ cx + fy @ cy)[:, :, None]


def aec_q1(om: OracleMesh, U, ue, ube, dte, gamma, prob):
    """Element contributions of eq. (aecQ1), the Q1 variant of Sec. 5.3:
      f_i^e = gamma_e ( m_i^e (u_i - u^e) - dt_e [ int (phi_i - m_i^e/|K_e|) div f_h
                                                  + int phi_i (udot^L_h - udot^L_i) ] )
    with f_h = sum_j f(u_j) phi_j (eq. (gfe)), so that
    int phi_i div f_h = sum_j int phi_i grad phi_j . f(u_j) and
    int div f_h = sum_j c_j . f(u_j), c_j = int grad phi_j; the last term is
    (M udot^L)_i - m_i^e udot^L_i with the consistent element mass matrix M.
    Written for any p; the paper applies it to Q1."""
    D = flux_divergence_term(om, U, prob)
    udl = low_order_time_derivative(om, U, ube, dte)
    UDL = om.blocks(udl.reshape((U.shape[0], om.nny, om.nnx)))
    inner = D + UDL @ om.Mass2.T - om.me * UDL
    return gamma[None, :, None] * (om.me * (U - ue[:, :, None]) - dte[None, :, None] * inner), udl


def bound_check(prob, u, clamp=True):
    """Invariant-domain check after a stage.  Scalars in IDP modes (LO,
    WENO-L): values outside [umin, umax] by more than a rounding tolerance are
    violations; all are clamped to the bounds.  Euler: count coefficients
    with rho <= 0 or p <= 0."""
    prob = _prob(prob)
    if prob["flux"] == ph.EULER:
        rho = u[0]
        pr = ph.pressure(u, prob["gamma_gas"])
        return u, int(np.count_nonzero((rho <= 0) | (pr <= 0))), 0
    if int(prob["mode"]) not in (MODE_LO, MODE_WENO_L):
        return u, 0, 0
    lo, hi = prob["umin"], prob["umax"]
    tol = 1e-12 * max(abs(lo), abs(hi), 1.0)
    viol = int(np.count_nonzero((u < lo - tol) | (u > hi + tol)))
    nclamp = int(np.count_nonzero((u < lo) | (u > hi)))
    if clamp:
        u = np.clip(u, lo, hi)
    return u, viol, nclamp


SSP3 = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))


def ssp_stage(mesh, prob, u, un, dt, a, b, t=0.0):
    """u_out = a u^n + b FE(u) with FE taken at stage time t, then the
    invariant-domain check (clamp)."""
    ufe, info = fe_stage(mesh, prob, u, dt, t)
    out = a * un + b * ufe if a != 0.0 else b * ufe
    out, viol, ncl = bound_check(prob, out)
    info["violations"] = viol
    info["clamps"] = ncl
    return out, info


def time_step(mesh, prob, u, t=0.0):
    """Global dt = cfl * min_e dt_e from the state u, eq. (cflglob) scaled by
    omega_CFL (Sec. 5)."""
    prob = _prob(prob)
    om = mesh if isinstance(mesh, OracleMesh) else OracleMesh(mesh)
    U = om.blocks(u)
    ue = cell_averages(om, U)
    if int(prob.get("options", 0)) & OPT_SUBCELL_DT:
        return prob["cfl"] * subcell_time_steps(om, U, prob).min()
    lo = low_order_facets(om, ue, prob, t)
    return prob["cfl"] * pseudo_time_steps(om, lo, prob).min()


def run(mesh, prob, u, nsteps, t_end=math.inf, t=0.0, collect=False):
    """SSP-RK3 (Shu-Osher form) with adaptive dt; returns (u, t, stats)."""
    prob = _prob(prob)
    om = mesh if isinstance(mesh, OracleMesh) else OracleMesh(mesh)
    stats = dict(violations=0, clamps=0, steps=0, dts=[])
    for _ in range(nsteps):
        if t >= t_end:
            break
        dt = min(time_step(om, prob, u, t), t_end - t)
        un = u
        for (a, b), c in zip(SSP3, SSP3_C):
            u, info = ssp_stage(om, prob, u, un, dt, a, b, t if c == 0.0 else t + c * dt)
            stats["violations"] += info["violations"]
            stats["clamps"] += info["clamps"]
        t += dt
        stats["steps"] += 1
        stats["dts"].append(dt)
    return u, t, stats


def mass(mesh, u):
    """Global conservation sum sum_i m_i u_i per component (FP64)."""
    om = mesh if isinstance(mesh, OracleMesh) else OracleMesh(mesh)
    return (u.reshape(u.shape[0], -1) * om.mi[None, :]).sum(axis=1)

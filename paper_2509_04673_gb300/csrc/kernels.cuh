// kernels.cuh — CUDA kernels of one SSP-RK stage of the element-based
// convex-limited CG-WENO scheme (Kuzmin, Hajduk, Vedral, arXiv 2509.04673),
// following the order of the algorithm summary in Sec. 4.3:
//
//   k_pre          cell averages u^e of the element and its face neighbours
//                  (eq. (ueold)), facet speeds, dt_e (eq. (dtmaxcell)), f^L,
//                  ubar^{e,L} (eq. (uelowFCT)), WENO sensor gamma_e (eqs.
//                  (WENO:alpha), (WENO:norm)), nu_e (eq. (stab:WENO)), block
//                  minimum of dt_e
//   k_dt_final     global dt = omega_CFL min_e dt_e (eq. (cflglob), Sec. 5)
//   k_grad_rhs     right-hand side of the g_h projection, int phi_i grad u_h,
//                  as a tiled separable stencil, and its lumped iterate
//   k_mass_sweep   lumped-preconditioned Richardson sweep with M_C applied
//                  as a tiled separable stencil
//   k_res_ev       element residual: Galerkin part of eq. (weak:stab2) with
//                  boundary terms (eqs. (aec), (aecb)) and s_h (eq. (stab:WENO))
//   k_gather_init  node-centric sum over E_i of the element residuals in a
//                  fixed order (deterministic), and its lumped iterate
//   k_update_ev    facet fluxes f^H (eq. (hoflux)), flux limiter (eq. (fAlim),
//                  Appendix A), ubar^e (eq. (uelim)), f_i^e (eq. (aec)),
//                  beta_e (eqs. (slimit1), (slimit2), Appendix A), element
//                  contributions of eq. (eq:SSPupdate)
//   k_final        node gather, SSP-RK combination, invariant-domain check;
//                  on the last stage of a step also t += dt
//
// One thread per element (or node; the stencils use 32 x 16 node tiles).
// Kernels are templated on the bulk precision R (double, or float in the
// mixed form), the degree P and the physics policy Ph. Cell averages, dt_e,
// the facet flux limiter, limiter bound gaps and positivity factors are
// float64 in both forms.
//
// Element vectors (ER, EW and the no-allocation scratch) are stored
// component-major, [local node i][field v][element e]: a warp of consecutive
// elements writes, and a warp of consecutive nodes reads, contiguous runs.
#pragma once

#include "common.cuh"

namespace cgl {

// element-vector layout: value v of local node i of element e, NV values
DEV long long ev_at(long long E, int e, int i, int v, int NV) { return (long long)(i * NV + v) * E + e; }


// Programmatic dependent launch: every kernel of a stage first lets the next
// kernel of the stream be scheduled (it launches once all blocks of this one
// are resident) and then waits until the previous kernel has completed and
// its writes are visible.  Each kernel calls this first, in every thread,
// before any global memory access; for a kernel launched without the
// programmatic-serialisation attribute both instructions do nothing.
DEV void pdl_begin() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// k_pre waits first and lets the next kernel be scheduled only then: when
// k_grad_rhs / k_grad_sweep (which need only u) start, the kernel that last
// wrote u has completed, so they can run beside k_pre.
DEV void pdl_wait_then_trigger() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// the gradient kernels wait for k_pre only before they exit, so that they
// complete after it and later kernels may rely on both
DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }


template <int P>
struct Dim {
    static constexpr int N1 = P + 1, N2 = N1 * N1, NQ = P + 2;
};

// device counters: invariant-domain violations, rounding clamps, theta > 1,
// non-finite values, unlimited averages ubar^e outside G (flux limiter off),
// pseudo time steps reduced by the remark after eq. (dtmaxcell)
// (slot CNT_IMPORT: non-finite values of the last host copy into the state;
// CNT_REFUSED: pipelined host copies refused for a non-finite value since the
// last cgl_sync)
enum { CNT_VIOL = 0, CNT_CLAMP = 1, CNT_CFL = 2, CNT_NONFINITE = 3, CNT_UBAR = 4, CNT_DTE_RED = 5, CNT_IMPORT = 6,
       CNT_REFUSED = 7, CNT_N = 8 };

// global node of local (a, b) in element (ex, ey); periodic wrap at the far side
DEV long long node_of(const MeshDev& m, int ex, int ey, int a, int b) {
    int gx = ex * m.p + a, gy = ey * m.p + b;
    if (m.px && gx == m.nnx) gx = 0;
    if (m.py && gy == m.nny) gy = 0;
    return (long long)gy * m.nnx + gx;
}

// the global node indices of element (ex, ey), degree P = m.p: the columns
// and row offsets are formed once per element (only the last column and row
// can wrap, in a periodic direction), so that each node index is one add;
// the same indices as node_of
template <int P>
struct ElemNodes {
    int gx[P + 1];
    long long row[P + 1];
    DEV ElemNodes(const MeshDev& m, int ex, int ey) {
#pragma unroll
        for (int a = 0; a <= P; ++a) gx[a] = ex * P + a;
        if (m.px && gx[P] == m.nnx) gx[P] = 0;
#pragma unroll
        for (int b = 0; b <= P; ++b) {
            int gy = ey * P + b;
            if (b == P && m.py && gy == m.nny) gy = 0;
            row[b] = (long long)gy * m.nnx;
        }
    }
    DEV long long operator()(int a, int b) const { return row[b] + gx[a]; }
};

// face neighbour (0 W, 1 E, 2 S, 3 N) or -1 on a non-periodic boundary
DEV int neighbour(const MeshDev& m, int ex, int ey, int dir) {
    int jx = ex, jy = ey;
    if (dir == 0) jx = ex - 1;
    else if (dir == 1) jx = ex + 1;
    else if (dir == 2) jy = ey - 1;
    else jy = ey + 1;
    if (jx < 0 || jx >= m.nx) {
        if (!m.px) return -1;
        jx = (jx + m.nx) % m.nx;
    }
    if (jy < 0 || jy >= m.ny) {
        if (!m.py) return -1;
        jy = (jy + m.ny) % m.ny;
    }
    return jy * m.nx + jx;
}

// coordinates (jx, jy) of the face neighbour of element (ex, ey) in
// direction dir (0 W, 1 E, 2 S, 3 N), wrapped on periodic directions; only
// meaningful where neighbour() is >= 0 (no integer division)
DEV void neighbour_xy(const MeshDev& m, int ex, int ey, int dir, int& jx, int& jy) {
    jx = ex + (dir == 0 ? -1 : dir == 1 ? 1 : 0);
    jy = ey + (dir == 2 ? -1 : dir == 3 ? 1 : 0);
    jx = jx < 0 ? jx + m.nx : (jx >= m.nx ? jx - m.nx : jx);
    jy = jy < 0 ? jy + m.ny : (jy >= m.ny ? jy - m.ny : jy);
}

// ---------------------------------------------------------------------------
// boundary data u_hat on the sides d = 0..3 (W, E, S, N), Sec. 2.  The
// positions and the split are evaluated in float64 with explicit rounding
// (no contraction), so that a point that lies exactly on a split (a node at
// x = 1/6 on a mesh of width 1/192) takes the same side as the plain
// evaluation s0 + s1 (t + c dt) and x0 + k hn.
// ---------------------------------------------------------------------------
DEV bool side_plain(const ProbDev& pr, int d) { return (pr.plain_mask >> d) & 1; }
DEV bool side_split(const ProbDev& pr, int d) { return (pr.split_mask >> d) & 1; }

// slot (0 below the split, 1 at or above it) of a point at coordinate pos
// of a side with two parts
DEV int side_slot(const ProbDev& pr, int d, double pos) {
    const SideDev& sd = pr.side[d];
    double sp = sd.s0;
    if (sd.s1 != 0.0) {
        double ts = *pr.t_dev;
        if (pr.tc != 0.0) ts = __dadd_rn(ts, __dmul_rn(pr.tc, *pr.dt_dev));
        sp = __dadd_rn(sd.s0, __dmul_rn(sd.s1, ts));
    }
    return pos < sp ? 0 : 1;
}

// coordinate along side d of node k (0..p) of the face of element (ex, ey):
// x0 + g h/p (Bernstein), x_e + xn_k h (LGL)
DEV double side_node_pos(const MeshDev& m, int d, int ex, int ey, int k) {
    const int c = (d < 2) ? ey : ex;
    if (m.basis) {
        const double xk = c_tabd[PMAX + 1 + m.p].xn[k];
        return __dadd_rn(__dadd_rn((d < 2) ? m.y0 : m.x0, __dmul_rn((double)c, m.h)), __dmul_rn(xk, m.h));
    }
    const int g = c * m.p + k;
    return __dadd_rn((d < 2) ? m.y0 : m.x0, __dmul_rn((double)g, m.hn));
}

// coordinate along side d of the midpoint of the face of element (ex, ey)
DEV double side_mid_pos(const MeshDev& m, int d, int ex, int ey) {
    const int c = (d < 2) ? ey : ex;
    return __dadd_rn((d < 2) ? m.y0 : m.x0, __dmul_rn((double)c + 0.5, m.h));
}

// coordinate along side d of the Gauss point x_q (on [0,1]) of that face
DEV double side_quad_pos(const MeshDev& m, int d, int ex, int ey, double xq) {
    const int c = (d < 2) ? ey : ex;
    return __dadd_rn(__dadd_rn((d < 2) ? m.y0 : m.x0, __dmul_rn((double)c, m.h)), __dmul_rn(xq, m.h));
}

// u_hat from the interior state u: FIXED -> the side's state, OUTFLOW -> u,
// WALL -> u with the normal momentum reversed, m - 2 (m.n) n (Euler; the
// normals of the sides are +-x and +-y)
template <class T, int NC>
DEV void ext_state(const ProbDev& pr, int d, int slot, const T* u, T* uh) {
    const SideDev& sd = pr.side[d];
    const int kind = sd.kind[slot];
#pragma unroll
    for (int c = 0; c < NC; ++c) uh[c] = (kind == BC_FIXED) ? PV<T>::side_state(sd, slot, c) : u[c];
    if constexpr (NC == 4) {
        if (kind == BC_WALL) {
            if (d < 2) uh[1] = -u[1];
            else uh[2] = -u[2];
        }
    }
}

// 2D launches: elements as (x: ex, y: ey), nodes as (x: gx, y: gy); no
// integer division by runtime sizes in the kernels
DEV bool elem_of_thread(const MeshDev& m, int& ex, int& ey, int& e) {
    ex = blockIdx.x * blockDim.x + threadIdx.x;
    ey = blockIdx.y * blockDim.y + threadIdx.y;
    e = ey * m.nx + ex;
    return ex < m.nx && ey < m.ny;
}

DEV bool node_of_thread(const MeshDev& m, int& gx, int& gy, long long& node) {
    gx = blockIdx.x * blockDim.x + threadIdx.x;
    gy = blockIdx.y * blockDim.y + threadIdx.y;
    node = (long long)gy * m.nnx + gx;
    return gx < m.nnx && gy < m.nny;
}

template <class R, int P, int NC>
DEV void load_block(const R* __restrict__ u, const MeshDev& m, int ex, int ey,
                    R (&U)[NC][Dim<P>::N2]) {
    constexpr int N1 = P + 1;
    const ElemNodes<P> en(m, ex, ey);
#pragma unroll
    for (int b = 0; b < N1; ++b)
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            const long long g = en(a, b);
#pragma unroll
            for (int c = 0; c < NC; ++c) U[c][b * N1 + a] = u[c * m.NN + g];
        }
}

// element mean of the coefficients as float64: plain sum for double data;
// for float data a compensated (Neumaier) float sum widened once, accurate
// to ~1e-14 relative without per-node float64 arithmetic
template <int N>
DEV double block_mean(const double (&v)[N]) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) s += v[i];
    return s * (1.0 / N);
}
template <int N>
DEV double block_mean(const float (&v)[N]) {
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float t = s + v[i];
        c += (fabsf(s) >= fabsf(v[i])) ? ((s - t) + v[i]) : ((v[i] - t) + s);
        s = t;
    }
    return ((double)s + (double)c) * (1.0 / N);
}

// u^e of eq. (ueold), (1/|K_e|) sum_i m_i^e u_i: the mean of the Bernstein
// coefficients, or on an LGL mesh (float64 form) the nodal values weighted
// by w_a w_b
template <class R, int P>
DEV double cell_mean(const MeshDev& m, const R (&v)[Dim<P>::N2]) {
    if constexpr (sizeof(R) == 8) {
        if (m.basis) {
            constexpr int N1 = P + 1;
            const Tab<double>& T = c_tabd[PMAX + 1 + P];
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < N1; ++b) {
                double r = 0.0;
#pragma unroll
                for (int a = 0; a < N1; ++a) r += T.wl[a] * v[b * N1 + a];
                s += T.wl[b] * r;
            }
            return s;
        }
    }
    return block_mean<Dim<P>::N2>(v);
}

// b^e_i = (int phi_i d_x u_h, int phi_i d_y u_h), sum-factorised, into EV
// at ev_at(E, e, i, v, 2NC), v = dim*NC + c
template <class R, int P, int NC>
DEV void grad_vectors(const MeshDev& m, const R (&U)[NC][Dim<P>::N2], R h, long long E, int e,
                      R* __restrict__ EV) {
    constexpr int N1 = P + 1, N2 = Dim<P>::N2, NV = 2 * NC;
    const Tab<R>& T = tab_of<R>(m, P);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        R Y[N1][N1], Z[N1][N1];
#pragma unroll
        for (int d = 0; d < N1; ++d)
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                R sx = R(0), sy = R(0);
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    sx += T.C[k][a] * U[c][d * N1 + k];
                    sy += T.M[a][k] * U[c][d * N1 + k];
                }
                Y[d][a] = sx;
                Z[d][a] = sy;
            }
#pragma unroll
        for (int b = 0; b < N1; ++b)
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                R sx = R(0), sy = R(0);
#pragma unroll
                for (int d = 0; d < N1; ++d) {
                    sx += T.M[b][d] * Y[d][a];
                    sy += T.C[d][b] * Z[d][a];
                }
                EV[ev_at(E, e, b * N1 + a, c, NV)] = h * sx;
                EV[ev_at(E, e, b * N1 + a, NC + c, NV)] = h * sy;
            }
    }
}

// ---------------------------------------------------------------------------
// low-order facet quantities of element e on its four faces in the canonical
// orientation (normal +x for W/E, +y for S/N): lambda and F^L = F(u^L, u^R)
// with f^L of Sec. 4; on a non-periodic boundary the external state is
// u_hat (FIXED) or u^e itself (OUTFLOW) and the cell's outward normal is used.
// ---------------------------------------------------------------------------
// upper bound of the facet speed, evaluated in precision RS: float64, or in
// float with a 2^-20 relative inflation so that it stays an upper bound
template <class Ph, class RS>
DEV double facet_speed(const double* uL, const double* uR, double nx, double ny, const ProbDev& pr) {
    if (sizeof(RS) == 8) return Ph::template max_speed<double>(uL, uR, nx, ny, pr);
    float fL[Ph::NC], fR[Ph::NC];
#pragma unroll
    for (int c = 0; c < Ph::NC; ++c) {
        fL[c] = (float)uL[c];
        fR[c] = (float)uR[c];
    }
    float l = Ph::template max_speed<float>(fL, fR, (float)nx, (float)ny, pr);
    return (double)l * (1.0 + 0x1p-20);
}

template <class Ph, class R>
DEV void lo_facets(const MeshDev& m, const ProbDev& pr, const int (&nb)[4], int ex, int ey,
                   const double (&us)[Ph::NC], const double (&fxs)[Ph::NC], const double (&fys)[Ph::NC],
                   const double (&uo)[4][Ph::NC], const double (&fxo)[4][Ph::NC],
                   const double (&fyo)[4][Ph::NC], double (&lam)[4], double (&FL)[4][Ph::NC]) {
    constexpr int NC = Ph::NC;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const double cnx = (d < 2) ? 1.0 : 0.0, cny = (d < 2) ? 0.0 : 1.0;
        const bool self_is_L = (d == 1 || d == 3);
        if (nb[d] >= 0) {
            const double* uL = self_is_L ? us : uo[d];
            const double* uR = self_is_L ? uo[d] : us;
            const double* fxL = self_is_L ? fxs : fxo[d];
            const double* fyL = self_is_L ? fys : fyo[d];
            const double* fxR = self_is_L ? fxo[d] : fxs;
            const double* fyR = self_is_L ? fyo[d] : fys;
            double l = facet_speed<Ph, R>(uL, uR, cnx, cny, pr);
            lam[d] = l;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                double nL = fxL[c] * cnx + fyL[c] * cny;
                double nR = fxR[c] * cnx + fyR[c] * cny;
                FL[d][c] = 0.5 * (nL + nR) - 0.5 * l * (uR[c] - uL[c]);
            }
        } else {
            // external state u_hat at the facet midpoint from the cell average
            const int slot = side_split(pr, d) ? side_slot(pr, d, side_mid_pos(m, d, ex, ey)) : 0;
            const int kind = pr.side[d].kind[slot];
            double ux[NC];
            ext_state<double, NC>(pr, d, slot, us, ux);
            const double sg = self_is_L ? 1.0 : -1.0;
            // f(u_hat) (FIXED, WALL) or the cell's own f(u^e) (OUTFLOW)
            double fxx[NC], fyx[NC];
            if (kind != BC_OUTFLOW) {
                R ubR[NC], fxR[NC], fyR[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) ubR[c] = R(ux[c]);
                Ph::template flux<R>(ubR, fxR, fyR, pr);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    fxx[c] = (double)fxR[c];
                    fyx[c] = (double)fyR[c];
                }
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    fxx[c] = fxs[c];
                    fyx[c] = fys[c];
                }
            }
            const double nx = sg * cnx, ny = sg * cny;
            double l = facet_speed<Ph, R>(us, ux, nx, ny, pr);
            lam[d] = l;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                double nL = fxs[c] * nx + fys[c] * ny;
                double nR = fxx[c] * nx + fyx[c] * ny;
                double F = 0.5 * (nL + nR) - 0.5 * l * (ux[c] - us[c]);
                FL[d][c] = sg * F;
            }
        }
    }
}

// cell average u^e (float64) and f(u^e) (evaluated in the bulk precision R,
// widened) of the block of element (jx, jy)
template <class R, int P, class Ph>
DEV void cell_state(const R* __restrict__ u, const MeshDev& m, const ProbDev& pr, int jx, int jy,
                    double (&avg)[Ph::NC], double (&fx)[Ph::NC], double (&fy)[Ph::NC]) {
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    R U[NC][N2];
    load_block<R, P, NC>(u, m, jx, jy, U);
    R aR[NC], fxR[NC], fyR[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        avg[c] = cell_mean<R, P>(m, U[c]);
        aR[c] = R(avg[c]);
    }
    Ph::template flux<R>(aR, fxR, fyR, pr);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        fx[c] = (double)fxR[c];
        fy[c] = (double)fyR[c];
    }
}

// x^e for the exponents other than the defaults r = 2, q = 1 of the sensor
// (eqs. (WENO:alpha), (stab:WENO)): out of line, so that the sensor's hot
// code, which the default exponents take, stays small in the instruction
// cache (the same powf / pow as an inlined call)
static __device__ __noinline__ float pow_rare(float x, float e) { return powf(x, e); }
static __device__ __noinline__ double pow_rare(double x, double e) { return pow(x, e); }

// the float64 Appendix-A factor where the float32 certificate of the
// FP32-mixed form could not show alpha = 1 (rare): out of line, so that the
// unrolled node loop of the slope limiter carries a call per node instead of
// a copy of the float64 formula (measured: k_update_el 5.52 -> 5.41 ms per
// three blast steps; in k_facet, at its 73-register cap, the call measured
// slower, 4.66 -> 5.80 ms, so the facet limiter keeps it inline, as does the
// FP64 form, where it runs everywhere)
static __device__ __noinline__ double euler_alpha_rare(const double* ub, const double* f, double m, double eps) {
    return euler_alpha<double>(ub, f, m, eps);
}
template <class R>
DEV double euler_alpha_of(const double* ub, const double* f, double m, double eps) {
    if constexpr (sizeof(R) == 4) return euler_alpha_rare(ub, f, m, eps);
    else return euler_alpha<double>(ub, f, m, eps);
}

// quadratic form of the semi-norm matrix A; A annihilates constants, so the
// block is shifted by its first coefficient first (exact zeros for constant
// data, no cancellation for nearly constant data).  a2b: the basis's offset
// in the packed matrices (a2_base; 0 for Bernstein)
template <class R, int P>
DEV R qform(const R (&v)[Dim<P>::N2], int a2b = 0) {
    constexpr int N2 = Dim<P>::N2;
    constexpr int off = A2_OFF[P];
    // d = v - v_0 (d_0 = 0); A symmetric: s = sum_i d_i (A_ii d_i + 2 sum_{j>i} A_ij d_j)
    R d[N2];
#pragma unroll
    for (int i = 0; i < N2; ++i) d[i] = v[i] - v[0];
    R s = R(0);
#pragma unroll
    for (int i = 1; i < N2; ++i) {
        R t = R(0);
#pragma unroll
        for (int j = i + 1; j < N2; ++j) t += TabSel<R>::A2(a2b + off + i * N2 + j) * d[j];
        s += d[i] * (TabSel<R>::A2(a2b + off + i * N2 + i) * d[i] + R(2) * t);
    }
    return s;
}

// neighbour polynomial continued onto K_e: dir 0 W (Em in x), 1 E (Ep in x),
// 2 S (Em in y), 3 N (Ep in y)
template <class R, int P>
DEV void continue_nb(const Tab<R>& T, int dir, const R (&src)[Dim<P>::N2], R (&dst)[Dim<P>::N2]) {
    constexpr int N1 = P + 1;
#pragma unroll
    for (int b = 0; b < N1; ++b)
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            R s = R(0);
            if (dir < 2) {
#pragma unroll
                for (int c = 0; c < N1; ++c)
                    s += (dir == 0 ? T.Em[a][c] : T.Ep[a][c]) * src[b * N1 + c];
            } else {
#pragma unroll
                for (int d = 0; d < N1; ++d)
                    s += (dir == 2 ? T.Em[b][d] : T.Ep[b][d]) * src[d * N1 + a];
            }
            dst[b * N1 + a] = s;
        }
}

template <class R, int P, class Ph>
DEV void load_comp(const R* __restrict__ u, const MeshDev& m, int ex, int ey, int c, R (&V)[Dim<P>::N2]) {
    constexpr int N1 = P + 1;
    const ElemNodes<P> en(m, ex, ey);
    const R* __restrict__ uc = u + (long long)c * m.NN;
#pragma unroll
    for (int b = 0; b < N1; ++b)
#pragma unroll
        for (int a = 0; a < N1; ++a) V[b * N1 + a] = uc[en(a, b)];
}

// WENO smoothness sensor gamma_e, eq. (WENO:alpha), minimum over components.
// Every block is shifted by its first coefficient (constants do not change
// semi-norms) and u_h^e - u_h^{e,*} is formed as sum_{l>=1} omega_l
// (u_h^e - u_{h,l}^e), using sum_l omega_l = 1.
template <class R, int P, class Ph>
DEV R sensor(const MeshDev& m, const ProbDev& pr, const R* __restrict__ u,
             const R (&U)[Ph::NC][Dim<P>::N2], const int (&nb)[4], int ex, int ey) {
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    const R wl = PV<R>::w_lin(pr), eps = PV<R>::weno_eps(pr), geps = PV<R>::gamma_eps(pr);
    const bool r2 = (pr.r == 2.0);
    const R rh = R(0.5 * pr.r);
    const Tab<R>& T = tab_of<R>(m, P);
    const int a2b = a2_base<R>(m);
    int ne = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) ne += (nb[d] >= 0);
    R gam = R(1);
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
        R U0[N2];
#pragma unroll
        for (int i = 0; i < N2; ++i) U0[i] = U[c][i] - U[c][0];
        R sig0 = fmax(qform<R, P>(U0, a2b), R(0));
        R wt[5];
        wt[0] = (R(1) - R(ne) * wl) / ((r2 ? sig0 : pow_rare(sig0, rh)) + eps);
#pragma unroll 1
        for (int d = 0; d < 4; ++d) {
            wt[d + 1] = R(0);
            if (nb[d] >= 0) {
                R V[N2], W[N2];
                int jx, jy;
                neighbour_xy(m, ex, ey, d, jx, jy);
                load_comp<R, P, Ph>(u, m, jx, jy, c, V);
                const R v0 = V[0];
#pragma unroll
                for (int i = 0; i < N2; ++i) V[i] -= v0;
                continue_nb<R, P>(T, d, V, W);
                R sg = fmax(qform<R, P>(W, a2b), R(0));
                wt[d + 1] = wl / ((r2 ? sg : pow_rare(sg, rh)) + eps);
            }
        }
        R tot = (((wt[0] + wt[1]) + wt[2]) + wt[3]) + wt[4];
        R Dl[N2];
#pragma unroll
        for (int i = 0; i < N2; ++i) Dl[i] = R(0);
#pragma unroll 1
        for (int d = 0; d < 4; ++d) {
            if (nb[d] >= 0) {
                R V[N2], W[N2];
                int jx, jy;
                neighbour_xy(m, ex, ey, d, jx, jy);
                load_comp<R, P, Ph>(u, m, jx, jy, c, V);
                const R v0 = V[0];
#pragma unroll
                for (int i = 0; i < N2; ++i) V[i] -= v0;
                continue_nb<R, P>(T, d, V, W);
                R wd = wt[d + 1] / tot;
#pragma unroll
                for (int i = 0; i < N2; ++i) Dl[i] += wd * (U0[i] - W[i]);
            }
        }
        R num = sqrt(fmax(qform<R, P>(Dl, a2b), R(0)));
        R den = sqrt(sig0);
        R ratio = num / (den + geps);
        R gc = R(1) - (pr.q == 1.0 ? fmin(R(1), ratio) : pow_rare(fmin(R(1), ratio), PV<R>::q(pr)));
        gam = fmin(gam, gc);
    }
    return gam;
}

// scalar sensor with the four neighbour blocks already in registers (V[d]
// holds the raw block of neighbour d when nb[d] >= 0); same arithmetic as
// sensor() with NC = 1
template <class R, int P>
DEV R sensor_scalar(const ProbDev& pr, const R (&U)[Dim<P>::N2], const R (&V)[4][Dim<P>::N2],
                    const int (&nb)[4]) {
    constexpr int N2 = Dim<P>::N2;
    const R wl = PV<R>::w_lin(pr), eps = PV<R>::weno_eps(pr), geps = PV<R>::gamma_eps(pr);
    const bool r2 = (pr.r == 2.0);
    const R rh = R(0.5 * pr.r);
    int ne = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) ne += (nb[d] >= 0);
    R U0[N2];
#pragma unroll
    for (int i = 0; i < N2; ++i) U0[i] = U[i] - U[0];
    R sig0 = fmax(qform<R, P>(U0), R(0));
    R wt[5];
    wt[0] = (R(1) - R(ne) * wl) / ((r2 ? sig0 : pow_rare(sig0, rh)) + eps);
    // the continued candidates, each formed once and kept for both passes
    R W[4][N2];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        wt[d + 1] = R(0);
        if (nb[d] >= 0) {
            R Vc[N2];
#pragma unroll
            for (int i = 0; i < N2; ++i) Vc[i] = V[d][i] - V[d][0];
            continue_nb<R, P>(TabSel<R>::t(P), d, Vc, W[d]);
            R sg = fmax(qform<R, P>(W[d]), R(0));
            wt[d + 1] = wl / ((r2 ? sg : pow_rare(sg, rh)) + eps);
        }
    }
    R tot = (((wt[0] + wt[1]) + wt[2]) + wt[3]) + wt[4];
    const R rtot = R(1) / tot;  // one division for the four weights omega_l
    R Dl[N2];
#pragma unroll
    for (int i = 0; i < N2; ++i) Dl[i] = R(0);
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        if (nb[d] >= 0) {
            R wd = wt[d + 1] * rtot;
#pragma unroll
            for (int i = 0; i < N2; ++i) Dl[i] += wd * (U0[i] - W[d][i]);
        }
    }
    R num = sqrt(fmax(qform<R, P>(Dl), R(0)));
    R den = sqrt(sig0);
    R ratio = num / (den + geps);
    return R(1) - (pr.q == 1.0 ? fmin(R(1), ratio) : pow_rare(fmin(R(1), ratio), PV<R>::q(pr)));
}

// float-float mean of N floats: compensated (Neumaier) sum, then a division
// by N whose remainder is taken exactly with an FMA; hi + lo carries about
// 1e-14 relative accuracy without float64 arithmetic
// (explicit round-to-nearest intrinsics throughout: the compiler never
// contracts or reorders them, so every kernel that inlines these helpers
// computes the same bits)
template <int N>
DEV void ff_mean(const float (&v)[N], float& hi, float& lo) {
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float t = __fadd_rn(s, v[i]);
        const float e = (fabsf(s) >= fabsf(v[i])) ? __fadd_rn(__fsub_rn(s, t), v[i])
                                                   : __fadd_rn(__fsub_rn(v[i], t), s);
        c = __fadd_rn(c, e);
        s = t;
    }
    const float h = __fadd_rn(s, c);
    const float l = __fsub_rn(c, __fsub_rn(h, s));
    const float k = 1.0f / N;
    const float q = __fmul_rn(h, k);
    const float r = __fmaf_rn(-q, (float)N, h);
    hi = q;
    lo = __fmul_rn(__fadd_rn(r, l), k);
}

// (ah + al) - (bh + bl) rounded to float (TwoSum on the high parts)
DEV float ff_diff(float ah, float al, float bh, float bl) {
    const float s = __fsub_rn(ah, bh);
    const float bb = __fsub_rn(s, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(-bh, bb));
    return __fadd_rn(s, __fadd_rn(err, __fsub_rn(al, bl)));
}

// error-free sum a + b = s + t (Knuth's TwoSum)
DEV void two_sum(float a, float b, float& s, float& t) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// ((a - b) + c) - d as a float-float pair hi + lo (relative error ~2^-44)
DEV void ff_sum4(float a, float b, float c, float d, float& hi, float& lo) {
    float s1, t1, s2, t2, s3, t3;
    two_sum(a, -b, s1, t1);
    two_sum(s1, c, s2, t2);
    two_sum(s2, -d, s3, t3);
    hi = s3;
    lo = __fadd_rn(__fadd_rn(t1, t2), t3);
}

// sum of N floats as a float-float pair hi + lo: Knuth's TwoSum into a
// running sum with the rounding errors collected separately (relative error
// of hi + lo about N^2 2^-48 of the sum of magnitudes)
template <int N>
DEV void ff_sum(const float (&v)[N], float& hi, float& lo) {
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float t, e;
        two_sum(s, v[i], t, e);
        c = __fadd_rn(c, e);
        s = t;
    }
    two_sum(s, c, hi, lo);
}

// LLF flux value 0.5 (nL + nR) - 0.5 lambda jump, with a fixed evaluation order
DEV float llf_value(float nL, float nR, float lam, float jump) {
    return __fmaf_rn(__fmul_rn(-0.5f, lam), jump, __fmul_rn(0.5f, __fadd_rn(nL, nR)));
}

// ---------------------------------------------------------------------------
// k_pre: dt_e, ubar^{e,L}, gamma_e, nu_e
// ---------------------------------------------------------------------------
// block-wide minimum of positive doubles folded into *bits with an integer
// atomicMin on the bit pattern (order independent, hence deterministic)
DEV void block_min_to(double v, unsigned long long* bits) {
    __shared__ unsigned long long sm[32];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y;
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_down_sync(0xffffffffu, b, o);
        b = w < b ? w : b;
    }
    if ((t & 31) == 0) sm[t >> 5] = b;
    __syncthreads();
    if (t < 32) {
        b = (t < (nt >> 5)) ? sm[t] : 0x7ff0000000000000ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long w = __shfl_down_sync(0xffffffffu, b, o);
            b = w < b ? w : b;
        }
        if (t == 0) atomicMin(bits, b);
    }
}

// ---------------------------------------------------------------------------
// k_pre: per element u^e and the face neighbours' u^{e'} (from their blocks,
// eq. (ueold)), f(u^e), lambda_e, the facet speeds and f^L, dt_e (eq.
// (dtmaxcell)), ubar^{e,L} (eq. (uelowFCT)), the flux-limiter capacities,
// gamma_e (eqs. (WENO:alpha), (WENO:norm)), nu_e, the element vectors of the
// g_h right-hand side, and (stage 1) the block minimum of dt_e.
// ---------------------------------------------------------------------------
// FP32-mixed form of pre_at: cell means as float-float pairs, low-order
// facet fluxes formed in float (their flux part is float-accurate anyway,
// the jump term comes from float-float differences), float facet fluxes and
// flux-limiter capacities (rounded toward zero, so they stay admissible)
// stored for the update pass; float64 for u^e, the speed-sum reciprocal,
// dt_e, ubar^{e,L} and the bound gaps.
template <class R, int NC>
struct CompVec {
    R v[NC];
};

// pseudo time step dt_e^max of Lemma 1, eq. (dtmaxsubcell), for the
// unlimited-flux variant (option OPT_SUBCELL_DT with the flux limiter off):
//   dt_e = (1/s) min{ min_{i on dK_e} m_i^e / (|c_ie| lambda_0i),
//                     m_0^e / sum_{i on dK_e} |c_ie| lambda_0i }
// with u_0^e the mean of the interior coefficients (m_0^e their mass),
// c_ie = int_{dK_e} phi_i n ds = |S|/(p+1) times the sum of the outward
// normals of the faces through node i, lambda_0i the speed bound of
// (u_0^e, u_i) along c_ie/|c_ie|, s = 1; for Q1 (no interior node) u_0^e =
// u^e, m_0^e = |K_e| and s = 2.  A node term with zero speed is dropped and
// the sum is floored at lambda_floor |S|.  Float64 from the element's
// coefficients; out of line (not on the default path).
template <class R, int P, class Ph>
__device__ __noinline__ double subcell_dt(const R* __restrict__ u, const MeshDev& m, const ProbDev& pr, int ex,
                                          int ey) {
    constexpr int NC = Ph::NC, N1 = P + 1, N2 = N1 * N1;
    R Ub[NC][N2];
    load_block<R, P, NC>(u, m, ex, ey, Ub);
    double u0[NC];
    double m0, sfac;
    if constexpr (P >= 2) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double acc = 0.0;
            for (int b = 1; b < P; ++b)
                for (int a = 1; a < P; ++a) acc += (double)Ub[c][b * N1 + a];
            u0[c] = acc / (double)((P - 1) * (P - 1));
        }
        m0 = (double)((P - 1) * (P - 1)) * m.me;
        sfac = 1.0;
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double acc = 0.0;
            for (int i = 0; i < N2; ++i) acc += (double)Ub[c][i];
            u0[c] = acc / (double)N2;
        }
        m0 = m.h * m.h;
        sfac = 2.0;
    }
    const double cface = m.h / (double)N1;
    double best = __longlong_as_double(0x7ff0000000000000LL), total = 0.0;
    for (int b = 0; b < N1; ++b)
        for (int a = 0; a < N1; ++a) {
            const double cx = (a == 0) ? -1.0 : (a == P) ? 1.0 : 0.0;
            const double cy = (b == 0) ? -1.0 : (b == P) ? 1.0 : 0.0;
            if (cx == 0.0 && cy == 0.0) continue;
            const double nrm = sqrt(cx * cx + cy * cy);
            double ui[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) ui[c] = (double)Ub[c][b * N1 + a];
            const double lam = Ph::template max_speed<double>(u0, ui, cx / nrm, cy / nrm, pr);
            const double w = (cface * nrm) * lam;
            total += w;
            if (w > 0.0) best = fmin(best, m.me / w);
        }
    total = fmax(total, pr.lambda_floor * m.h);
    return fmin(best, m0 / total) / sfac;
}

// low-order quantities of a boundary facet of the FP32-mixed k_pre: the
// speed bound (inflated like the interior ones) and F(u^e, u_hat; n) in the
// canonical orientation, u_hat of side d at the facet midpoint in float-float
// (FIXED: the side's state; OUTFLOW: u^e; WALL: u^e with reversed normal
// momentum); uh, ul: the element's float-float mean, fn: its flux along the
// facet axis; returns [F_0 .. F_{NC-1}, lambda]
template <class Ph>
__device__ __noinline__ CompVec<float, Ph::NC + 1> boundary_facet_lo(const MeshDev& m, const ProbDev& pr, int d,
                                                                    int ex, int ey, float sg,
                                                                    CompVec<float, Ph::NC> uh,
                                                                    CompVec<float, Ph::NC> ul,
                                                                    CompVec<float, Ph::NC> fn) {
    constexpr int NC = Ph::NC;
    const bool xf = d < 2;
    const float inflate = 1.0f + 0x1p-20f;
    const float cnx = xf ? 1.f : 0.f, cny = xf ? 0.f : 1.f;
    const int slot = side_split(pr, d) ? side_slot(pr, d, side_mid_pos(m, d, ex, ey)) : 0;
    const SideDev& sd = pr.side[d];
    const int kind = sd.kind[slot];
    float xh[NC], xl[NC], xfx[NC], xfy[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        xh[c] = (kind == BC_FIXED) ? sd.st_f[slot][c] : uh.v[c];
        xl[c] = (kind == BC_FIXED) ? sd.st_lo_f[slot][c] : ul.v[c];
    }
    if constexpr (NC == 4) {
        if (kind == BC_WALL) {
            const int cn = xf ? 1 : 2;
            xh[cn] = -xh[cn];
            xl[cn] = -xl[cn];
        }
    }
    Ph::template flux<float>(xh, xfx, xfy, pr);
    const float l = __fmul_rn(Ph::template max_speed<float>(uh.v, xh, sg * cnx, sg * cny, pr), inflate);
    CompVec<float, NC + 1> out;
    out.v[NC] = l;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float ns = sg * fn.v[c];
        const float nx = sg * (xf ? xfx[c] : xfy[c]);
        const float Fo = llf_value(ns, nx, l, ff_diff(xh[c], xl[c], uh.v[c], ul.v[c]));
        out.v[c] = sg * Fo;
    }
    return out;
}

// SUB: pseudo time steps from the subcell bound of Lemma 1 (a separate
// instantiation, so that the default kernels carry none of its code).
// LO (systems): the low-order part only: the element's own float-float mean
// comes from k_avg like its neighbours' (the same ff_mean of the same block,
// hence the same bits), no coefficient block is loaded, and gamma_e, nu_e
// are left to k_sens
template <int P, class Ph, bool SUB = false, bool LO = false>
DEV double pre_at_mixed(const MeshDev& m, const ProbDev& pr, const float* __restrict__ u,
                        double* __restrict__ ue_out, double* __restrict__ dte_out,
                        double* __restrict__ ubl_out, double* __restrict__ gam_out,
                        double* __restrict__ nu_out, float* __restrict__ q_out,
                        float* __restrict__ fl_out, float* __restrict__ EV, float* __restrict__ cf_out,
                        float* __restrict__ avg, int ex, int ey, int e, const float* __restrict__ cq = nullptr) {
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    static_assert(!LO || NC > 1, "the low-order-only form reads the means of k_avg (systems)");
    int nb[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) nb[d] = neighbour(m, ex, ey, d);
    float U[LO ? 1 : NC][LO ? 1 : N2];
    if constexpr (!LO) load_block<float, P, NC>(u, m, ex, ey, U);
    float uh[NC], ul[NC], fxs[NC], fys[NC];
    double ued[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if constexpr (LO) {
            uh[c] = avg[(2 * c) * m.E + e];
            ul[c] = avg[(2 * c + 1) * m.E + e];
        } else {
            ff_mean<N2>(U[c], uh[c], ul[c]);
        }
        ued[c] = (double)uh[c] + (double)ul[c];
        ue_out[c * m.E + e] = ued[c];
    }
    // LO: the fluxes of the means and the speed parts were formed by k_avg
    constexpr int NQP = LO ? Ph::NPART_OR_1 : 1;
    float qs[NQP], qn[4][NQP];
    if constexpr (LO) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            fxs[c] = cq[c * m.E + e];
            fys[c] = cq[(NC + c) * m.E + e];
        }
#pragma unroll
        for (int k = 0; k < NQP; ++k) qs[k] = cq[(2 * NC + k) * m.E + e];
    } else {
        Ph::template flux<float>(uh, fxs, fys, pr);
    }
    // neighbours: means, fluxes (and, for scalars, the blocks for the sensor)
    float oh[4][NC], ol[4][NC], ofx[4][NC], ofy[4][NC];
    // scalars at p <= 2 keep the neighbour blocks for the sensor; at p >= 3
    // the sensor reloads them (registers, hence occupancy, matter more)
    constexpr bool keepV = (NC == 1) && (P <= 2);
    float V1[keepV ? 4 : 1][keepV ? N2 : 1];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        if (nb[d] >= 0) {
            if constexpr (NC > 1) {
                // systems: the neighbours' float-float means from k_avg
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    oh[d][c] = avg[(2 * c) * m.E + nb[d]];
                    ol[d][c] = avg[(2 * c + 1) * m.E + nb[d]];
                }
                if constexpr (LO) {
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        ofx[d][c] = cq[c * m.E + nb[d]];
                        ofy[d][c] = cq[(NC + c) * m.E + nb[d]];
                    }
#pragma unroll
                    for (int k = 0; k < NQP; ++k) qn[d][k] = cq[(2 * NC + k) * m.E + nb[d]];
                }
            } else {
                int jx, jy;
                neighbour_xy(m, ex, ey, d, jx, jy);
                float B[NC][N2];
                load_block<float, P, NC>(u, m, jx, jy, B);
#pragma unroll
                for (int c = 0; c < NC; ++c) ff_mean<N2>(B[c], oh[d][c], ol[d][c]);
                if constexpr (keepV) {
#pragma unroll
                    for (int i = 0; i < N2; ++i) V1[d][i] = B[0][i];
                }
            }
            if constexpr (!LO) Ph::template flux<float>(oh[d], ofx[d], ofy[d], pr);
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) oh[d][c] = ol[d][c] = ofx[d][c] = ofy[d][c] = 0.f;
            if constexpr (keepV) {
#pragma unroll
                for (int i = 0; i < N2; ++i) V1[d][i] = 0.f;
            }
        }
    }
    // canonical facet fluxes F(u^L, u^R; n), n = +x (W, E) or +y (S, N)
    const float inflate = 1.0f + 0x1p-20f;
    float lam[4], F[4][NC];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const bool xf = d < 2;
        const float cnx = xf ? 1.f : 0.f, cny = xf ? 0.f : 1.f;
        const bool self_is_L = (d == 1 || d == 3);
        if (nb[d] >= 0) {
            const float* Lh = self_is_L ? uh : oh[d];
            const float* Ll = self_is_L ? ul : ol[d];
            const float* Rh = self_is_L ? oh[d] : uh;
            const float* Rl = self_is_L ? ol[d] : ul;
            const float* fL = xf ? (self_is_L ? fxs : ofx[d]) : (self_is_L ? fys : ofy[d]);
            const float* fR = xf ? (self_is_L ? ofx[d] : fxs) : (self_is_L ? ofy[d] : fys);
            float ls;
            if constexpr (LO) {
                const float* qL = self_is_L ? qs : qn[d];
                const float* qR = self_is_L ? qn[d] : qs;
                ls = Ph::facet_speed_parts(qL, qR, xf ? 0 : 1, PV<float>::gam(pr));
            } else {
                ls = Ph::template max_speed<float>(Lh, Rh, cnx, cny, pr);
            }
            const float l = __fmul_rn(ls, inflate);
            lam[d] = l;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                F[d][c] = llf_value(fL[c], fR[c], l, ff_diff(Rh[c], Rl[c], Lh[c], Ll[c]));
        } else {
            // boundary facet: out of line (rare; keeps the hot code small)
            CompVec<float, NC> vh, vl, vf;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                vh.v[c] = uh[c];
                vl.v[c] = ul[c];
                vf.v[c] = xf ? fxs[c] : fys[c];
            }
            const CompVec<float, NC + 1> o =
                boundary_facet_lo<Ph>(m, pr, d, ex, ey, self_is_L ? 1.f : -1.f, vh, vl, vf);
            lam[d] = o.v[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) F[d][c] = o.v[c];
        }
    }
    float sf = __fadd_rn(__fadd_rn(__fadd_rn(lam[0], lam[1]), lam[2]), lam[3]);
    sf = fmaxf(sf, pr.lambda_floor_f);
    // dt_e / h = 1 / s: float reciprocal refined by one float64 Newton step
    // (relative error ~2^-46, far inside the 2^-20 inflation of the speeds;
    // GB300's float64 divide is a long sequence on its narrow float64 pipe)
    double s, rs;
    if constexpr (SUB) {
        // Lemma 1 bound; the float speed sum is rounded up (a float dt_e no
        // larger than the bound)
        rs = subcell_dt<float, P, Ph>(u, m, pr, ex, ey) * m.inv_h;
        s = 1.0 / rs;
        sf = __double2float_ru(s);
    } else {
        s = (double)sf;
        const double r0 = (double)__frcp_rn(sf);
        rs = fma(r0, fma(-s, r0, 1.0), r0);
    }
    const double dte = m.h * rs;
    dte_out[e] = dte;
    dte_out[m.E + e] = rs;
    dte_out[2 * m.E + e] = s * m.inv_h;
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int c = 0; c < NC; ++c) fl_out[((long long)e * 4 + d) * NC + c] = F[d][c];
    const float s4 = 0.25f * sf;  // |K| / (|dK| dt_e), exact
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        // facet flux sum (F_E - F_W) + F_N - F_S as a float-float pair, widened once
        float osh, osl;
        ff_sum4(F[1][c], F[0][c], F[3][c], F[2][c], osh, osl);
        const double os = (double)osh + (double)osl;
        const double bl = ued[c] - rs * os;
        ubl_out[c * m.E + e] = bl;
        if (NC == 1) {
            // capacities (s/4)(umax - bl) >= 0 and (s/4)(umin - bl) <= 0: bound
            // gaps in float64, both factors and the product rounded toward zero
            // (smaller magnitudes stay admissible)
            q_out[e] = __fmul_rz(s4, fmaxf(0.f, __double2float_rz(pr.umax - bl)));
            q_out[m.E + e] = __fmul_rz(s4, fminf(0.f, __double2float_rz(pr.umin - bl)));
            // the float-float mean, for the element contributions of k_update_ev
            avg[e] = uh[0];
            avg[m.E + e] = ul[0];
        } else {
            // float copies for the certificate of the facet limiter (euler_alpha_is_one)
            cf_out[(1 + c) * m.E + e] = (float)bl;
        }
    }
    cf_out[e] = sf;  // the float speed sum (dt_e in float for k_update_ev)
    if constexpr (LO) {
        return dte;
    } else {
    float gam;
    if (pr.mode == MODE_WENO || pr.mode == MODE_WENO_L) {
        if constexpr (keepV) {
            float U1[N2];
#pragma unroll
            for (int i = 0; i < N2; ++i) U1[i] = U[0][i];
            gam = sensor_scalar<float, P>(pr, U1, V1, nb);
        } else {
            gam = sensor<float, P, Ph>(m, pr, u, U, nb, ex, ey);
        }
    } else {
        gam = (pr.mode == MODE_HO) ? 1.f : 0.f;
    }
    gam_out[e] = (double)gam;
    float lm = 0.f;
#pragma unroll
    for (int i = 0; i < N2; ++i) {
        float ui[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ui[c] = U[c][i];
        lm = fmaxf(lm, Ph::template node_speed<float>(ui, pr));
    }
    nu_out[e] = (double)(lm * (m.h_f * (0.5f / P)));
    if (EV) grad_vectors<float, P, NC>(m, U, m.h_f, m.E, e, EV);
    return dte;
    }
}

template <class R, int P, class Ph, bool SUB = false>
DEV double pre_at(const MeshDev& m, const ProbDev& pr, const R* __restrict__ u, double* __restrict__ ue_out,
                  double* __restrict__ dte_out, double* __restrict__ ubl_out,
                  double* __restrict__ gam_out, double* __restrict__ nu_out,
                  R* __restrict__ q_out, R* __restrict__ fl_out, R* __restrict__ EV,
                  float* __restrict__ cf_out, float* __restrict__ avg, int ex, int ey, int e) {
    if constexpr (sizeof(R) == 4) {
        return pre_at_mixed<P, Ph, SUB>(m, pr, u, ue_out, dte_out, ubl_out, gam_out, nu_out, q_out, fl_out, EV,
                                        cf_out, avg, ex, ey, e);
    } else {
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    double dte;
    {
        int nb[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) nb[d] = neighbour(m, ex, ey, d);
        R U[NC][N2];
        load_block<R, P, NC>(u, m, ex, ey, U);
        double us[NC], fxs[NC], fys[NC];
        {
            R aR[NC], fxR[NC], fyR[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                us[c] = cell_mean<R, P>(m, U[c]);
                aR[c] = R(us[c]);
                ue_out[c * m.E + e] = us[c];
            }
            Ph::template flux<R>(aR, fxR, fyR, pr);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                fxs[c] = (double)fxR[c];
                fys[c] = (double)fyR[c];
            }
        }
        double uo[4][NC], fxo[4][NC], fyo[4][NC];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            if (nb[d] >= 0) {
                int jx, jy;
                neighbour_xy(m, ex, ey, d, jx, jy);
                cell_state<R, P, Ph>(u, m, pr, jx, jy, uo[d], fxo[d], fyo[d]);
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) uo[d][c] = fxo[d][c] = fyo[d][c] = 0.0;
            }
        }
        double lam[4], FL[4][NC];
        lo_facets<Ph, R>(m, pr, nb, ex, ey, us, fxs, fys, uo, fxo, fyo, lam, FL);
        double s = ((lam[0] + lam[1]) + lam[2]) + lam[3];
        s = fmax(s, pr.lambda_floor);
        // dt_e = |K| / (|S| sum lambda) = h / s; dt_e / h = 1 / s
        double rs = 1.0 / s;
        if constexpr (SUB) {
            // Lemma 1 bound instead (the unlimited-flux variant)
            rs = subcell_dt<R, P, Ph>(u, m, pr, ex, ey) * m.inv_h;
            s = 1.0 / rs;
        }
        dte = m.h * rs;
        dte_out[e] = dte;
        dte_out[m.E + e] = rs;              // dt_e / h
        dte_out[2 * m.E + e] = s * m.inv_h; // 1 / dt_e
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int c = 0; c < NC; ++c) fl_out[((long long)e * 4 + d) * NC + c] = FL[d][c];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double os = ((FL[1][c] - FL[0][c]) + FL[3][c]) - FL[2][c];
            double bl = us[c] - rs * os;
            ubl_out[c * m.E + e] = bl;
            if (NC == 1) {
                // admissible antidiffusive capacities of eq. (fAlim):
                // (|K|/|dK|)(umax - ubar^{e,L})/dt_e = (s/4)(umax - ubar^{e,L}) >= 0, and
                // (s/4)(umin - ubar^{e,L}) <= 0
                q_out[e] = fmax(0.0, (0.25 * s) * (pr.umax - bl));
                q_out[m.E + e] = fmin(0.0, (0.25 * s) * (pr.umin - bl));
            }
        }
        double gam;
        if (pr.mode == MODE_WENO || pr.mode == MODE_WENO_L) {
            gam = (double)sensor<R, P, Ph>(m, pr, u, U, nb, ex, ey);
        } else {
            gam = (pr.mode == MODE_HO) ? 1.0 : 0.0;
        }
        gam_out[e] = gam;
        R lm = R(0);
#pragma unroll
        for (int i = 0; i < N2; ++i) {
            R ui[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) ui[c] = U[c][i];
            lm = fmax(lm, Ph::template node_speed<R>(ui, pr));
        }
        nu_out[e] = (double)lm * (m.h * (0.5 / m.p));
        if (EV) grad_vectors<R, P, NC>(m, U, PV<R>::h(m), m.E, e, EV);
    }
    return dte;
    }
}

// k_avg (FP32-mixed systems): float-float cell means of every element, read
// by k_pre_lo for the element and its four face neighbours instead of their
// coefficient blocks; avg[(2c) E + e] = high part, avg[(2c+1) E + e] = low
// part of component c.  Beside them the quantities of the mean's state that
// every facet of the cell needs, formed once per cell: cq[c E + e] = f_x(u^e)
// and cq[(NC + c) E + e] = f_y(u^e) (the flux of the high parts), then the
// speed parts of the two-rarefaction bound.
template <int P, class Ph>
__global__ void k_avg(MeshDev m, ProbDev pr, const float* __restrict__ u, float* __restrict__ avg,
                      float* __restrict__ cq) {
    pdl_begin();
    int ex, ey, e;
    if (!elem_of_thread(m, ex, ey, e)) return;
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    float U[NC][N2];
    load_block<float, P, NC>(u, m, ex, ey, U);
    float uh[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float hi, lo;
        ff_mean<N2>(U[c], hi, lo);
        avg[(2 * c) * m.E + e] = hi;
        avg[(2 * c + 1) * m.E + e] = lo;
        uh[c] = hi;
    }
    float fx[NC], fy[NC], q[Ph::NPART_OR_1];
    Ph::template flux<float>(uh, fx, fy, pr);
    Ph::speed_parts(uh, PV<float>::gam(pr), q);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        cq[c * m.E + e] = fx[c];
        cq[(NC + c) * m.E + e] = fy[c];
    }
#pragma unroll
    for (int k = 0; k < Ph::NPART_OR_1; ++k) cq[(2 * NC + k) * m.E + e] = q[k];
}

// Resident blocks of 128 threads per SM requested from the compiler for the
// one-thread-per-element kernels (a register cap of 65536 / (128 n)),
// chosen by measurement on GB300 (time per launch against the uncapped
// form): FP32-mixed Euler at p = 2 (blast 2048^2 Q2) k_pre_lo 5 (-13 %),
// k_facet 7 (-25 %), k_res_ev and k_update_el 4 (-8 %, -13 %); at p = 3
// (quadrants 512^2 Q3) k_pre_lo 5 (-9 %), k_facet 6 (-17 %), the residual
// and the update uncapped (3 blocks: +18 %, +7 %); the FP64 Euler p = 2
// residual and update 3; every other instantiation 1 (the compiler's choice).
enum { EK_PRE_LO = 0, EK_FACET, EK_RES, EK_UPD };
template <int P, int NC, int RSZ>
constexpr int elem_blocks(int k) {
    if (NC > 1 && P == 2) {
        if (RSZ == 8) return (k == EK_RES || k == EK_UPD) ? 3 : 1;
        return k == EK_PRE_LO ? 5 : k == EK_FACET ? 7 : 4;
    }
    if (NC > 1 && P == 3 && RSZ == 4) return k == EK_PRE_LO ? 5 : k == EK_FACET ? 6 : 1;
    return 1;
}

template <class R, int P, class Ph, bool SUB = false>
__global__ void k_pre(MeshDev m, ProbDev pr, const R* __restrict__ u, double* __restrict__ ue_out,
                      double* __restrict__ dte_out, double* __restrict__ ubl_out,
                      double* __restrict__ gam_out, double* __restrict__ nu_out,
                      R* __restrict__ q_out, R* __restrict__ fl_out, R* __restrict__ EV,
                      float* __restrict__ cf_out, float* __restrict__ avg,
                      unsigned long long* __restrict__ dtbits) {
    pdl_wait_then_trigger();
    int ex, ey, e;
    double dte = __longlong_as_double(0x7ff0000000000000LL);
    if (elem_of_thread(m, ex, ey, e))
        dte = pre_at<R, P, Ph, SUB>(m, pr, u, ue_out, dte_out, ubl_out, gam_out, nu_out, q_out, fl_out, EV, cf_out,
                                    avg, ex, ey, e);
    if (dtbits) block_min_to(dte, dtbits);
}

// FP32-mixed systems: the low-order part of k_pre (cell states from k_avg,
// facet speeds and f^L, dt_e, ubar^{e,L}, the float copies for the facet
// limiter's certificate); gamma_e and nu_e come from k_sens
template <int P, class Ph, bool SUB = false>
__global__ void __launch_bounds__(128, elem_blocks<P, Ph::NC, 4>(EK_PRE_LO)) k_pre_lo(MeshDev m, ProbDev pr, const float* __restrict__ u, double* __restrict__ ue_out,
                         double* __restrict__ dte_out, double* __restrict__ ubl_out,
                         float* __restrict__ fl_out, float* __restrict__ cf_out, float* __restrict__ avg,
                         const float* __restrict__ cq, unsigned long long* __restrict__ dtbits) {
    pdl_wait_then_trigger();
    int ex, ey, e;
    double dte = __longlong_as_double(0x7ff0000000000000LL);
    if (elem_of_thread(m, ex, ey, e))
        dte = pre_at_mixed<P, Ph, SUB, true>(m, pr, u, ue_out, dte_out, ubl_out, nullptr, nullptr, nullptr, fl_out,
                                             nullptr, cf_out, avg, ex, ey, e, cq);
    if (dtbits) block_min_to(dte, dtbits);
}

// FP32-mixed systems: the WENO sensor gamma_e (eqs. (WENO:alpha),
// (WENO:norm)) and nu_e (eq. (stab:WENO)) with one thread per element and
// component.  A block holds K_SENS_TX consecutive elements of one row, one
// warp per component (threadIdx.y = c): each thread evaluates the scalar
// sensor of its component (the arithmetic of sensor() for that component),
// the block takes gamma_e = min over the components and the node speeds of
// nu_e from the element blocks it stages in shared memory.
constexpr int K_SENS_TX = 32;
template <int P, class Ph>
__global__ void __launch_bounds__(K_SENS_TX * Ph::NC) k_sens(MeshDev m, ProbDev pr, const float* __restrict__ u,
                                                             double* __restrict__ gam_out,
                                                             double* __restrict__ nu_out) {
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2, TX = K_SENS_TX;
    __shared__ float sU[NC][N2][TX];
    __shared__ float sG[NC][TX], sL[NC][TX];
    pdl_wait_then_trigger();
    const int tx = threadIdx.x, c = threadIdx.y;
    const int ex = blockIdx.x * TX + tx, ey = blockIdx.y;
    const bool valid = ex < m.nx;
    float gam = 1.f;
    if (valid) {
        int nb[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) nb[d] = neighbour(m, ex, ey, d);
        const float* uc = u + c * m.NN;
        float U[1][N2];
        load_comp<float, P, Ph>(u, m, ex, ey, c, U[0]);
#pragma unroll
        for (int i = 0; i < N2; ++i) sU[c][i][tx] = U[0][i];
        if (pr.mode == MODE_WENO || pr.mode == MODE_WENO_L) {
            if constexpr (P <= 2) {
                float V[4][N2];
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    if (nb[d] >= 0) {
                        int jx, jy;
                        neighbour_xy(m, ex, ey, d, jx, jy);
                        load_comp<float, P, Ph>(u, m, jx, jy, c, V[d]);
                    } else {
#pragma unroll
                        for (int i = 0; i < N2; ++i) V[d][i] = 0.f;
                    }
                }
                gam = sensor_scalar<float, P>(pr, U[0], V, nb);
            } else {
                // one component as a scalar field (neighbour blocks reloaded,
                // fewer live registers at p >= 3)
                gam = sensor<float, P, PhysAdv>(m, pr, uc, U, nb, ex, ey);
            }
        } else {
            gam = (pr.mode == MODE_HO) ? 1.f : 0.f;
        }
    }
    sG[c][tx] = gam;
    __syncthreads();
    float lm = 0.f;
    if (valid) {
        // the nodes of this component's thread, in a loop that is not
        // unrolled: one copy of the node-speed code (the unrolled form with a
        // test per node put nine copies in the instruction cache; measured
        // k_sens 8.21 -> 7.24 ms per three blast steps with the reciprocal
        // of the weight sum below)
#pragma unroll 1
        for (int i = c; i < N2; i += NC) {
            float ui[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) ui[k] = sU[k][i][tx];
            lm = fmaxf(lm, Ph::template node_speed<float>(ui, pr));
        }
    }
    sL[c][tx] = lm;
    __syncthreads();
    if (c == 0 && valid) {
        float g = 1.f, l = 0.f;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            g = fminf(g, sG[k][tx]);
            l = fmaxf(l, sL[k][tx]);
        }
        const int e = ey * m.nx + ex;
        gam_out[e] = (double)g;
        nu_out[e] = (double)(l * (m.h_f * (0.5f / P)));
    }
}

// global dt from the block minima folded into the bit pattern by k_pre
// dt = min(cfl * min_e dt_e, t_end - t), never negative
static __global__ void k_dt_final(unsigned long long* bits, double cfl, const double* t,
                                  const double* t_end, double* dt) {
    pdl_begin();
    double d = cfl * __longlong_as_double((long long)*bits);
    *bits = 0x7ff0000000000000ull;  // ready for the next reduction
    double rem = *t_end - *t;
    if (rem < d) d = rem > 0.0 ? rem : 0.0;
    *dt = d;
}

// ---------------------------------------------------------------------------
// node-centric gathers over E_i in a fixed order (lower neighbour first in
// each direction): deterministic, no atomics.
// ---------------------------------------------------------------------------
// elements containing node (gx, gy): at most two per direction (lower one
// first), with the node's local index in each; compile-time P
template <int P>
struct NodeC {
    int ex0, ex1, a0, a1, nxc;
    int ey0, ey1, b0, b1, nyc;
};

template <int P>
DEV NodeC<P> node_c(const MeshDev& m, int gx, int gy) {
    NodeC<P> c;
    int ex = gx / P, a = gx - ex * P;
    if (a == 0) {
        const bool lo = (ex > 0) || m.px, hi = ex < m.nx;
        c.ex0 = lo ? (ex == 0 ? m.nx - 1 : ex - 1) : ex;
        c.a0 = lo ? P : 0;
        c.ex1 = ex;
        c.a1 = 0;
        c.nxc = (int)lo + (int)hi;
    } else {
        c.ex0 = c.ex1 = ex;
        c.a0 = c.a1 = a;
        c.nxc = 1;
    }
    int ey = gy / P, b = gy - ey * P;
    if (b == 0) {
        const bool lo = (ey > 0) || m.py, hi = ey < m.ny;
        c.ey0 = lo ? (ey == 0 ? m.ny - 1 : ey - 1) : ey;
        c.b0 = lo ? P : 0;
        c.ey1 = ey;
        c.b1 = 0;
        c.nyc = (int)lo + (int)hi;
    } else {
        c.ey0 = c.ey1 = ey;
        c.b0 = c.b1 = b;
        c.nyc = 1;
    }
    return c;
}

// 1/|E_i| for |E_i| in {1, 2, 4} (exact powers of two)
template <class R>
DEV R inv_count(int n) {
    return n == 4 ? R(0.25) : (n == 2 ? R(0.5) : R(1));
}

// 1 / m_i on an LGL mesh (float64 form): m_i = sum over the cnt elements
// containing node i of h^2 w_a w_b, with the node's local indices (a0, b0)
// in the first of them; the LGL weights are symmetric (w_0 = w_p), so a
// shared node has the same weight in every element containing it
template <int P>
DEV double inv_lumped_lgl(const MeshDev& m, int cnt, int a0, int b0) {
    const Tab<double>& T = c_tabd[PMAX + 1 + P];
    return inv_count<double>(cnt) * (m.inv_h2 * (T.iwl[a0] * T.iwl[b0]));
}


// s[v] = sum over E_i of the element vectors at node (gx, gy), fixed order
template <class R, int P, int NV>
DEV void gather_at(const MeshDev& m, const R* __restrict__ EV, const NodeC<P>& c, R (&s)[NV]) {
    constexpr int N1 = P + 1, N2 = N1 * N1;
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = R(0);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        if (j < c.nyc) {
            const int ey = j ? c.ey1 : c.ey0, b = j ? c.b1 : c.b0;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (i < c.nxc) {
                    const int ex = i ? c.ex1 : c.ex0, a = i ? c.a1 : c.a0;
                    const int e = ey * m.nx + ex;
#pragma unroll
                    for (int v = 0; v < NV; ++v) s[v] += EV[ev_at(m.E, e, b * N1 + a, v, NV)];
                }
            }
        }
    }
}

// sum over E_i of element vectors; out[v*NN + node]; if xout, also x = sum / m_i
template <class R, int P, int NV>
DEV void gather_init_at(MeshDev m, const R* __restrict__ EV, R* __restrict__ bout,
                              R* __restrict__ xout, int gx, int gy, long long node) {
    const NodeC<P> c = node_c<P>(m, gx, gy);
    R s[NV];
    gather_at<R, P, NV>(m, EV, c, s);
    const R inv_mi = is_lgl<R>(m) ? R(inv_lumped_lgl<P>(m, c.nxc * c.nyc, c.a0, c.b0))
                                  : PV<R>::inv_me(m) * inv_count<R>(c.nxc * c.nyc);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if (bout) bout[v * m.NN + node] = s[v];
        if (xout) xout[v * m.NN + node] = s[v] * inv_mi;
    }
}

template <class R, int P, int NV>
__global__ void k_gather_init(MeshDev m, const R* __restrict__ EV, R* __restrict__ bout,
                              R* __restrict__ xout) {
    pdl_begin();
    int gx, gy;
    long long node;
    if (!node_of_thread(m, gx, gy, node)) return;
    gather_init_at<R, P, NV>(m, EV, bout, xout, gx, gy, node);
}




// explicitly rounded multiply-add and multiply (no contraction choices left
// to the compiler, so the per-node and the tiled stencils give equal bits)
DEV float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }
DEV double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }
DEV float mul_r(float a, float b) { return __fmul_rn(a, b); }
DEV double mul_r(double a, double b) { return __dmul_rn(a, b); }

// Richardson update x + (b - h^2 s) / m_i with s = (M (x) M) x at the node
template <class R>
DEV R sweep_value(R x, R b, R s, R h2, R inv_mi) {
    return fma_r(fma_r(-h2, s, b), inv_mi, x);
}

// ---------------------------------------------------------------------------
// node-centric application of the assembled linear operators. On a uniform
// mesh, sum_{e in E_i} of an element operator A^e = Ax (x) Ay is a separable
// stencil over the (2p+1)^2 nodes around node i: along x the weight of offset
// k is sum over the (at most two) elements containing i of Ax[a_e][k + a_e]
// (a_e = local index of i in e); likewise along y.
// ---------------------------------------------------------------------------
// 1D weights of the assembled mass (WHICH 0: M[a][c]) or of the derivative on
// the trial index (WHICH 1: C[c][a] = int B_c' B_a) for offsets -P..P. The
// node's first containing element has local index a0 (0..P); a second one
// (n == 2, a shared vertex) has local index 0. Built from compile-time table
// entries by selects (no runtime-indexed arrays).
template <class R, int P, int WHICH>
DEV R wtab(const Tab<R>& T, int a, int c) {
    return (WHICH == 0) ? T.M[a][c] : T.C[c][a];
}

template <class R, int P, int WHICH>
DEV void weights_1d(const Tab<R>& T, int n, int a0, int /*a1*/, R (&w)[2 * P + 1]) {
#pragma unroll
    for (int k = 0; k < 2 * P + 1; ++k) {
        const int off = k - P;
        R s = R(0);
#pragma unroll
        for (int aa = 0; aa <= P; ++aa) {
            const int cc = off + aa;
            if (cc >= 0 && cc <= P) s = (a0 == aa) ? wtab<R, P, WHICH>(T, aa, cc) : s;
        }
        if (off >= 0 && off <= P) s += (n == 2) ? wtab<R, P, WHICH>(T, 0, off) : R(0);
        w[k] = s;
    }
}

// indices of the 2P+1 nodes at offsets -P..P around g along a direction of
// n nodes (periodic wrap; clamped where only zero weights reach)
template <int P>
DEV void offsets_1d(int g, int n, int periodic, int (&idx)[2 * P + 1]) {
#pragma unroll
    for (int k = 0; k < 2 * P + 1; ++k) {
        int x = g + k - P;
        if (periodic) x = x < 0 ? x + n : (x >= n ? x - n : x);
        else x = x < 0 ? 0 : (x >= n ? n - 1 : x);
        idx[k] = x;
    }
}

// g_h right-hand side b_i = sum_e int phi_i grad u_h (x: derivative weights
// along x, mass along y; y: the reverse) and the lumped first iterate b / m_i;
// b and g hold [x components (NC)][y components (NC)]
template <class R, int P, int NC>
DEV void grad_rhs_at(MeshDev m, const R* __restrict__ u, R* __restrict__ bout, R* __restrict__ gout,
                     int gx, int gy, long long node) {
    const Tab<R>& T = tab_of<R>(m, P);
    const NodeC<P> c = node_c<P>(m, gx, gy);
    R wMx[2 * P + 1], wCx[2 * P + 1], wMy[2 * P + 1], wCy[2 * P + 1];
    weights_1d<R, P, 0>(T, c.nxc, c.a0, c.a1, wMx);
    weights_1d<R, P, 1>(T, c.nxc, c.a0, c.a1, wCx);
    weights_1d<R, P, 0>(T, c.nyc, c.b0, c.b1, wMy);
    weights_1d<R, P, 1>(T, c.nyc, c.b0, c.b1, wCy);
    int cols[2 * P + 1], rows[2 * P + 1];
    offsets_1d<P>(gx, m.nnx, m.px, cols);
    offsets_1d<P>(gy, m.nny, m.py, rows);
    R sx[NC], sy[NC];
#pragma unroll
    for (int v = 0; v < NC; ++v) sx[v] = sy[v] = R(0);
#pragma unroll
    for (int ky = 0; ky < 2 * P + 1; ++ky) {
        const long long row = (long long)rows[ky] * m.nnx;
        R tx[NC], ty[NC];
#pragma unroll
        for (int v = 0; v < NC; ++v) tx[v] = ty[v] = R(0);
#pragma unroll
        for (int kx = 0; kx < 2 * P + 1; ++kx) {
            const long long idx = row + cols[kx];
#pragma unroll
            for (int v = 0; v < NC; ++v) {
                const R x = u[v * m.NN + idx];
                tx[v] = fma_r(wCx[kx], x, tx[v]);
                ty[v] = fma_r(wMx[kx], x, ty[v]);
            }
        }
#pragma unroll
        for (int v = 0; v < NC; ++v) {
            sx[v] = fma_r(wMy[ky], tx[v], sx[v]);
            sy[v] = fma_r(wCy[ky], ty[v], sy[v]);
        }
    }
    const R h = PV<R>::h(m);
    const R inv_mi = is_lgl<R>(m) ? R(inv_lumped_lgl<P>(m, c.nxc * c.nyc, c.a0, c.b0))
                                  : mul_r(PV<R>::inv_me(m), inv_count<R>(c.nxc * c.nyc));
#pragma unroll
    for (int v = 0; v < NC; ++v) {
        const R bx = mul_r(h, sx[v]), by = mul_r(h, sy[v]);
        bout[v * m.NN + node] = bx;
        bout[(NC + v) * m.NN + node] = by;
        gout[v * m.NN + node] = mul_r(bx, inv_mi);
        gout[(NC + v) * m.NN + node] = mul_r(by, inv_mi);
    }
}

// one lumped-preconditioned Richardson sweep for NV fields,
// x_out = x_in + (b - M_C x_in) / m_i, with M_C applied as a stencil
template <class R, int P, int NV>
DEV void mass_sweep_at(MeshDev m, const R* __restrict__ xin, const R* __restrict__ b, R* __restrict__ xout,
                       int gx, int gy, long long node) {
    const Tab<R>& T = tab_of<R>(m, P);
    const NodeC<P> c = node_c<P>(m, gx, gy);
    R wx[2 * P + 1], wy[2 * P + 1];
    weights_1d<R, P, 0>(T, c.nxc, c.a0, c.a1, wx);
    weights_1d<R, P, 0>(T, c.nyc, c.b0, c.b1, wy);
    int cols[2 * P + 1], rows[2 * P + 1];
    offsets_1d<P>(gx, m.nnx, m.px, cols);
    offsets_1d<P>(gy, m.nny, m.py, rows);
    R s[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = R(0);
#pragma unroll
    for (int ky = 0; ky < 2 * P + 1; ++ky) {
        const long long row = (long long)rows[ky] * m.nnx;
        R t[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) t[v] = R(0);
#pragma unroll
        for (int kx = 0; kx < 2 * P + 1; ++kx) {
            const long long idx = row + cols[kx];
#pragma unroll
            for (int v = 0; v < NV; ++v) t[v] = fma_r(wx[kx], xin[v * m.NN + idx], t[v]);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] = fma_r(wy[ky], t[v], s[v]);
    }
    const R h2 = PV<R>::h2(m);
    const R inv_mi = is_lgl<R>(m) ? R(inv_lumped_lgl<P>(m, c.nxc * c.nyc, c.a0, c.b0))
                                  : mul_r(PV<R>::inv_me(m), inv_count<R>(c.nxc * c.nyc));
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const long long k = v * m.NN + node;
        xout[k] = sweep_value(xin[k], b[k], s[v], h2, inv_mi);
    }
}

// ---------------------------------------------------------------------------
// Tiled forms of the two stencils: a block of 32 x 8 threads owns a tile of
// 32 x 16 nodes, stages one field of the tile plus a halo of p nodes in
// shared memory (coalesced rows, periodic wrap, zeros outside a
// non-periodic mesh, where every weight that reaches them is 0), applies
// the 1D operator along x for all halo rows, then along y.  The weights of
// a node depend only on its class along each direction (local index 1..p-1
// inside an element, an interior vertex shared by two elements, or a
// boundary vertex); the class tables are built per block from the element
// tables with the same additions as weights_1d.  Same arithmetic, in the
// same order with the same roundings, as grad_rhs_at / mass_sweep_at.
// ---------------------------------------------------------------------------
constexpr int ST_TX = 32, ST_TY = 16, ST_BY = 8;

// class of node g along a direction of n nodes: 1..P-1 inside an element,
// 0 vertex shared by two elements, P lower boundary vertex, P+1 upper one
template <int P>
DEV int node_class(int g, int n, int periodic) {
    const int a = g % P;
    if (a != 0) return a;
    if (!periodic) {
        if (g == 0) return P;
        if (g == n - 1) return P + 1;
    }
    return 0;
}

// local index of a node of class cls in the first element containing it
// (a shared vertex: p in the lower element; a low / high boundary vertex:
// 0 / p; inside an element: cls)
template <int P>
DEV int class_index(int cls) {
    return (cls == 0 || cls == P + 1) ? P : (cls == P ? 0 : cls);
}

// weight of offset off (-P..P) for a node of class cls (WHICH 0: mass,
// 1: derivative on the trial index), as weights_1d computes it
template <class R, int P, int WHICH>
DEV R class_weight(const Tab<R>& T, int cls, int off) {
    // first containing element and the node's local index in it
    const int a0 = (cls == 0 || cls == P + 1) ? P : (cls == P ? 0 : cls);
    const bool two = cls == 0;
    R s = R(0);
    const int cc = off + a0;
    if (cc >= 0 && cc <= P) s = wtab<R, P, WHICH>(T, a0, cc);
    if (two && off >= 0 && off <= P) s += wtab<R, P, WHICH>(T, 0, off);
    return s;
}

// stage one field (rows gy0-P.., columns gx0-P..) of the tile in shared memory
// a node index on a periodic direction of n nodes taken into [0, n) (the
// fused stencils, halo 2p): one period covers every node of a tile and its
// halo on meshes at least a tile wide; a narrower mesh (down to one element)
// takes the remainder, so a staged halo value is always a node of the mesh
DEV int wrap_periodic(int g, int n) {
    g = g < 0 ? g + n : (g >= n ? g - n : g);
    if ((unsigned)g >= (unsigned)n) g = ((g % n) + n) % n;
    return g;
}

template <class R, int P, int BY, int TY = ST_TY>
DEV void stage_tile(const MeshDev& m, const R* __restrict__ x, R (*xs)[ST_TX + 2 * P], int gx0, int gy0, int tid) {
    constexpr int HX = ST_TX + 2 * P, HY = TY + 2 * P;
    for (int i = tid; i < HX * HY; i += ST_TX * BY) {
        const int r = i / HX, c = i - r * HX;
        int gy = gy0 - P + r, gx = gx0 - P + c;
        // one period on periodic directions: a halo of p never needs more on a
        // mesh of at least one element (p nodes) per side; a position still
        // outside after it (two periods away, on a mesh narrower than the
        // tile) feeds no output of the tile and is not read
        if (m.py) gy = gy < 0 ? gy + m.nny : (gy >= m.nny ? gy - m.nny : gy);
        if (m.px) gx = gx < 0 ? gx + m.nnx : (gx >= m.nnx ? gx - m.nnx : gx);
        const bool in = (unsigned)gy < (unsigned)m.nny && (unsigned)gx < (unsigned)m.nnx;
        // through L2 (ld.global.cg): k_grad_rhs reads u without waiting for
        // the kernel launched just before it
        xs[r][c] = in ? __ldcg(&x[(long long)gy * m.nnx + gx]) : R(0);
    }
}

// fields staged together: as many as fit in 32 KB of shared memory (a
// divisor of NV), so one round of loads and barriers serves all of them
template <class R, int P, int NV, int NT, int TY = ST_TY>
struct StFields {
    static constexpr int HX = ST_TX + 2 * P, HY = TY + 2 * P;
    static constexpr int bytes(int f) { return f * (HY * HX + NT * HY * ST_TX) * (int)sizeof(R); }
    static constexpr int value = (bytes(NV) <= 32768) ? NV
                                 : (NV % 4 == 0 && bytes(4) <= 32768) ? 4
                                 : (NV % 2 == 0 && bytes(2) <= 32768) ? 2 : 1;
    // shared workspace in elements of R: staged fields, NT pass-1 arrays
    // per field, NT class-weight tables
    static constexpr int ws = value * (HY * HX + NT * HY * ST_TX) + NT * (P + 2) * (2 * P + 1);
};

// g_h right-hand side and lumped iterate on the 32 x 16 node tile at
// (gx0, gy0) by a block of 32 x BY threads (thread (tx, ty)); ws: shared
// workspace of StFields<R, P, NC, 2>::ws elements.  All threads of the block
// call it together.
template <class R, int P, int NC, int BY, int TY = ST_TY>
DEV void grad_tile(const MeshDev& m, const R* __restrict__ u, R* __restrict__ bout, R* __restrict__ gout,
                   int gx0, int gy0, int tx, int ty, R* ws) {
    constexpr int HX = ST_TX + 2 * P, HY = TY + 2 * P, NW = 2 * P + 1, NCL = P + 2, NJ = TY / BY;
    constexpr int FB = StFields<R, P, NC, 2, TY>::value;
    R(*xs)[HY][HX] = reinterpret_cast<R(*)[HY][HX]>(ws);
    R(*tC)[HY][ST_TX] = reinterpret_cast<R(*)[HY][ST_TX]>(ws + FB * HY * HX);
    R(*tM)[HY][ST_TX] = reinterpret_cast<R(*)[HY][ST_TX]>(ws + FB * HY * HX + FB * HY * ST_TX);
    R(*WM)[NW] = reinterpret_cast<R(*)[NW]>(ws + FB * (HY * HX + 2 * HY * ST_TX));
    R(*WC)[NW] = reinterpret_cast<R(*)[NW]>(ws + FB * (HY * HX + 2 * HY * ST_TX) + NCL * NW);
    const Tab<R>& T = tab_of<R>(m, P);
    const int tid = ty * ST_TX + tx;
    __syncthreads();  // the workspace is free
    if (tid < NCL * NW) {
        const int cls = tid / NW, k = tid - cls * NW;
        WM[cls][k] = class_weight<R, P, 0>(T, cls, k - P);
        WC[cls][k] = class_weight<R, P, 1>(T, cls, k - P);
    }
    const int gx = gx0 + tx;
    const int clx = node_class<P>(gx, m.nnx, m.px);
    const R h = PV<R>::h(m);
    for (int v0 = 0; v0 < NC; v0 += FB) {
        if (v0 > 0) __syncthreads();  // previous fields consumed
#pragma unroll
        for (int f = 0; f < FB; ++f) stage_tile<R, P, BY, TY>(m, u + (long long)(v0 + f) * m.NN, xs[f], gx0, gy0, tid);
        __syncthreads();
        R wcx[NW], wmx[NW];  // the column's x weights, for every row and field
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            wcx[k] = WC[clx][k];
            wmx[k] = WM[clx][k];
        }
        // along x, every halo row: derivative (for b_x) and mass (for b_y)
        for (int r = ty; r < HY; r += BY) {
#pragma unroll
            for (int f = 0; f < FB; ++f) {
                R sc = R(0), sm = R(0);
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    const R x = xs[f][r][tx + k];
                    sc = fma_r(wcx[k], x, sc);
                    sm = fma_r(wmx[k], x, sm);
                }
                tC[f][r][tx] = sc;
                tM[f][r][tx] = sm;
            }
        }
        __syncthreads();
        // along y and the outputs
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int r = ty + j * BY, gy = gy0 + r;
            if (gx >= m.nnx || gy >= m.nny) continue;
            const int cly = node_class<P>(gy, m.nny, m.py);
            const int cnt = (clx == 0 ? 2 : 1) * (cly == 0 ? 2 : 1);
            const R inv_mi = is_lgl<R>(m) ? R(inv_lumped_lgl<P>(m, cnt, class_index<P>(clx), class_index<P>(cly)))
                                          : mul_r(PV<R>::inv_me(m), inv_count<R>(cnt));
            const long long node = (long long)gy * m.nnx + gx;
            R wmy[NW], wcy[NW];  // once for every field
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                wmy[k] = WM[cly][k];
                wcy[k] = WC[cly][k];
            }
#pragma unroll
            for (int f = 0; f < FB; ++f) {
                const int v = v0 + f;
                R sx = R(0), sy = R(0);
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    sx = fma_r(wmy[k], tC[f][r + k][tx], sx);
                    sy = fma_r(wcy[k], tM[f][r + k][tx], sy);
                }
                const R bx = mul_r(h, sx), by = mul_r(h, sy);
                bout[v * m.NN + node] = bx;
                bout[(NC + v) * m.NN + node] = by;
                gout[v * m.NN + node] = mul_r(bx, inv_mi);
                gout[(NC + v) * m.NN + node] = mul_r(by, inv_mi);
            }
        }
    }
}

// one Richardson sweep for NV fields on the 32 x 16 node tile at (gx0, gy0);
// ws: StFields<R, P, NV, 1>::ws elements of shared memory
template <class R, int P, int NV, int BY, int TY = ST_TY>
DEV void sweep_tile(const MeshDev& m, const R* __restrict__ xin, const R* __restrict__ b, R* __restrict__ xout,
                    int gx0, int gy0, int tx, int ty, R* ws) {
    constexpr int HX = ST_TX + 2 * P, HY = TY + 2 * P, NW = 2 * P + 1, NCL = P + 2, NJ = TY / BY;
    constexpr int FB = StFields<R, P, NV, 1, TY>::value;
    R(*xs)[HY][HX] = reinterpret_cast<R(*)[HY][HX]>(ws);
    R(*t)[HY][ST_TX] = reinterpret_cast<R(*)[HY][ST_TX]>(ws + FB * HY * HX);
    R(*W)[NW] = reinterpret_cast<R(*)[NW]>(ws + FB * (HY * HX + HY * ST_TX));
    const Tab<R>& T = tab_of<R>(m, P);
    const int tid = ty * ST_TX + tx;
    __syncthreads();  // the workspace is free
    if (tid < NCL * NW) {
        const int cls = tid / NW, k = tid - cls * NW;
        W[cls][k] = class_weight<R, P, 0>(T, cls, k - P);
    }
    const int gx = gx0 + tx;
    const int clx = node_class<P>(gx, m.nnx, m.px);
    const R h2 = PV<R>::h2(m);
    for (int v0 = 0; v0 < NV; v0 += FB) {
        // right-hand sides of this thread's nodes, loaded ahead of the barriers
        R bv[FB][NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int gy = gy0 + ty + j * BY;
            const bool in = gx < m.nnx && gy < m.nny;
#pragma unroll
            for (int f = 0; f < FB; ++f)
                bv[f][j] = in ? b[(long long)(v0 + f) * m.NN + (long long)gy * m.nnx + gx] : R(0);
        }
        if (v0 > 0) __syncthreads();
#pragma unroll
        for (int f = 0; f < FB; ++f) stage_tile<R, P, BY, TY>(m, xin + (long long)(v0 + f) * m.NN, xs[f], gx0, gy0, tid);
        __syncthreads();
        for (int r = ty; r < HY; r += BY) {
#pragma unroll
            for (int f = 0; f < FB; ++f) {
                R sx = R(0);
#pragma unroll
                for (int k = 0; k < NW; ++k) sx = fma_r(W[clx][k], xs[f][r][tx + k], sx);
                t[f][r][tx] = sx;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int r = ty + j * BY, gy = gy0 + r;
            if (gx >= m.nnx || gy >= m.nny) continue;
            const int cly = node_class<P>(gy, m.nny, m.py);
            const int cnt = (clx == 0 ? 2 : 1) * (cly == 0 ? 2 : 1);
            const R inv_mi = is_lgl<R>(m) ? R(inv_lumped_lgl<P>(m, cnt, class_index<P>(clx), class_index<P>(cly)))
                                          : mul_r(PV<R>::inv_me(m), inv_count<R>(cnt));
#pragma unroll
            for (int f = 0; f < FB; ++f) {
                R sy = R(0);
#pragma unroll
                for (int k = 0; k < NW; ++k) sy = fma_r(W[cly][k], t[f][r + k][tx], sy);
                const long long k = (long long)(v0 + f) * m.NN + (long long)gy * m.nnx + gx;
                xout[k] = sweep_value(xs[f][r + P][tx + P], bv[f][j], sy, h2, inv_mi);
            }
        }
    }
}

// needs only u, whose last writer completed before k_pre let this kernel
// start (pdl_wait_then_trigger), so it runs beside k_pre and waits for it
// only before exiting
// TY: node rows per tile (8 on small meshes: shorter per-block chains in a
// partial wave; 16 on large ones: less halo)
template <class R, int P, int NC, int TY = ST_TY>
__global__ void __launch_bounds__(ST_TX * ST_BY) k_grad_rhs(MeshDev m, const R* __restrict__ u,
                                                            R* __restrict__ bout, R* __restrict__ gout) {
    pdl_trigger();
    __shared__ R ws[StFields<R, P, NC, 2, TY>::ws];
    grad_tile<R, P, NC, ST_BY, TY>(m, u, bout, gout, blockIdx.x * ST_TX, blockIdx.y * TY, threadIdx.x, threadIdx.y,
                                   ws);
    pdl_wait();
}

template <class R, int P, int NV, int TY = ST_TY>
__global__ void __launch_bounds__(ST_TX * ST_BY) k_mass_sweep(MeshDev m, const R* __restrict__ xin,
                                                              const R* __restrict__ b, R* __restrict__ xout) {
    pdl_begin();
    __shared__ R ws[StFields<R, P, NV, 1, TY>::ws];
    sweep_tile<R, P, NV, ST_BY, TY>(m, xin, b, xout, blockIdx.x * ST_TX, blockIdx.y * TY, threadIdx.x, threadIdx.y,
                                    ws);
}

// runtime-degree candidate list (diagnostics only)
struct NodeCands {
    int nxc, nyc;
    int ex[2], a[2], ey[2], b[2];
};

DEV NodeCands node_cands(const MeshDev& m, int gx, int gy) {
    NodeCands nc;
    const int p = m.p;
    int ex = gx / p, a = gx - ex * p;
    nc.nxc = 0;
    if (a == 0) {
        if (ex > 0 || m.px) {
            nc.ex[nc.nxc] = (ex - 1 + m.nx) % m.nx;
            nc.a[nc.nxc++] = p;
        }
        if (ex < m.nx) {
            nc.ex[nc.nxc] = ex;
            nc.a[nc.nxc++] = 0;
        }
    } else {
        nc.ex[0] = ex;
        nc.a[0] = a;
        nc.nxc = 1;
    }
    int ey = gy / p, b = gy - ey * p;
    nc.nyc = 0;
    if (b == 0) {
        if (ey > 0 || m.py) {
            nc.ey[nc.nyc] = (ey - 1 + m.ny) % m.ny;
            nc.b[nc.nyc++] = p;
        }
        if (ey < m.ny) {
            nc.ey[nc.nyc] = ey;
            nc.b[nc.nyc++] = 0;
        }
    } else {
        nc.ey[0] = ey;
        nc.b[0] = b;
        nc.nyc = 1;
    }
    return nc;
}

// ---------------------------------------------------------------------------
// k_res_ev: R^e_i = W^e_i - s^e_i with
//   W^e_i = int grad phi_i . f(u_h) - sum_{interior faces} int phi_i f_h.n
//           - sum_{faces on dOmega} int phi_i F(u_h, u_hat; n)
//   s^e_i = nu_e int grad phi_i . (grad u_h - gamma_e g_h)      eq. (stab:WENO)
// (p+2)-point Gauss rule for nonlinear integrands; exact face mass for f_h.
// ER layout ev_at(E, e, i, c, NC).
// ---------------------------------------------------------------------------
// boundary-face part of the weak form of element (ex, ey) on face d: the
// (p+2)-point quadrature of phi_i F(u_h, u_hat; n), u_hat of the side at
// each Gauss point, or of phi_i f(u_h).n on a side that is OUTFLOW
// everywhere; scaled by h; Uf and term are [NC][p+1]
template <class R, int P, class Ph>
__device__ __noinline__ void boundary_face_term(const MeshDev& m, const ProbDev& pr, int d, int ex, int ey,
                                                const R* Uf, R* term) {
    constexpr int NC = Ph::NC, N1 = P + 1, NQ = Dim<P>::NQ;
    const Tab<R>& T = tab_of<R>(m, P);
    const Tab<double>& Td = tab_of<double>(m, P);
    const R h = PV<R>::h(m);
    const R nxo = (d == 0) ? R(-1) : (d == 1) ? R(1) : R(0);
    const R nyo = (d == 2) ? R(-1) : (d == 3) ? R(1) : R(0);
    const bool plain = side_plain(pr, d);
    // a FIXED side with one part: one external state, its flux evaluated once
    const bool fixed1 = !plain && !side_split(pr, d) && pr.side[d].kind[0] == BC_FIXED;
    R ub1[NC], fxb[NC], fyb[NC];
    if (fixed1) {
#pragma unroll
        for (int c = 0; c < NC; ++c) ub1[c] = PV<R>::side_state(pr.side[d], 0, c);
        Ph::template flux<R>(ub1, fxb, fyb, pr);
    }
    R acc[NC][N1];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int b = 0; b < N1; ++b) acc[c][b] = R(0);
#pragma unroll
    for (int r = 0; r < NQ; ++r) {
        R uq[NC], F[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            R s = R(0);
#pragma unroll
            for (int k = 0; k < N1; ++k) s += Uf[c * N1 + k] * T.Bq[r][k];
            uq[c] = s;
        }
        if (fixed1) {
            llf_given_fR<Ph, R>(uq, ub1, fxb, fyb, nxo, nyo, pr, F);
        } else if (!plain) {
            const int slot = side_split(pr, d) ? side_slot(pr, d, side_quad_pos(m, d, ex, ey, Td.xq[r])) : 0;
            R ub[NC];
            ext_state<R, NC>(pr, d, slot, uq, ub);
            llf<Ph, R>(uq, ub, nxo, nyo, pr, F, (R*)nullptr);
        } else {
            R fx[NC], fy[NC];
            Ph::template flux<R>(uq, fx, fy, pr);
#pragma unroll
            for (int c = 0; c < NC; ++c) F[c] = fx[c] * nxo + fy[c] * nyo;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int b = 0; b < N1; ++b) acc[c][b] += (F[c] * T.wq[r]) * T.Bq[r][b];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int b = 0; b < N1; ++b) term[c * N1 + b] = acc[c][b] * h;
}

// Galerkin part W^e of the element residual: volume and face terms of the
// weak form (needs only u)
template <class R, int P, class Ph>
DEV void w_part(const MeshDev& m, const ProbDev& pr, const R (&U)[Ph::NC][Dim<P>::N2], int ex, int ey,
                R (&W)[Ph::NC][Dim<P>::N2]) {
    constexpr int NC = Ph::NC, N1 = P + 1, N2 = Dim<P>::N2, NQ = Dim<P>::NQ;
    const Tab<R>& T = tab_of<R>(m, P);
    const R h = PV<R>::h(m);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int i = 0; i < N2; ++i) W[c][i] = R(0);
    // volume term: interpolate along x first
    R X[NC][N1][NQ];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int d = 0; d < N1; ++d)
#pragma unroll
            for (int q1 = 0; q1 < NQ; ++q1) {
                R s = R(0);
#pragma unroll
                for (int a = 0; a < N1; ++a) s += T.Bq[q1][a] * U[c][d * N1 + a];
                X[c][d][q1] = s;
            }
#pragma unroll 1
    for (int q2 = 0; q2 < NQ; ++q2) {
        R Tx[NC][N1], Ty[NC][N1];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int a = 0; a < N1; ++a) Tx[c][a] = Ty[c][a] = R(0);
#pragma unroll
        for (int q1 = 0; q1 < NQ; ++q1) {
            R uq[NC], fx[NC], fy[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                R s = R(0);
#pragma unroll
                for (int d = 0; d < N1; ++d) s += T.Bq[q2][d] * X[c][d][q1];
                uq[c] = s;
            }
            Ph::template flux<R>(uq, fx, fy, pr);
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    Tx[c][a] += T.wq[q1] * T.dBq[q1][a] * fx[c];
                    Ty[c][a] += T.wq[q1] * T.Bq[q1][a] * fy[c];
                }
        }
        const R hw = h * T.wq[q2];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int b = 0; b < N1; ++b)
#pragma unroll
                for (int a = 0; a < N1; ++a)
                    W[c][b * N1 + a] += hw * (T.Bq[q2][b] * Tx[c][a] + T.dBq[q2][b] * Ty[c][a]);
    }
    // face terms
    int nb[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) nb[d] = neighbour(m, ex, ey, d);
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const R nxo = (d == 0) ? R(-1) : (d == 1) ? R(1) : R(0);
        const R nyo = (d == 2) ? R(-1) : (d == 3) ? R(1) : R(0);
        R Uf[NC][N1];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            int li = (d == 0) ? k * N1 : (d == 1) ? k * N1 + P : (d == 2) ? k : P * N1 + k;
#pragma unroll
            for (int c = 0; c < NC; ++c) Uf[c][k] = U[c][li];
        }
        R term[NC][N1];
        if (nb[d] >= 0) {
            R fn[NC][N1];
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                R uk[NC], fx[NC], fy[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) uk[c] = Uf[c][k];
                Ph::template flux<R>(uk, fx, fy, pr);
#pragma unroll
                for (int c = 0; c < NC; ++c) fn[c][k] = fx[c] * nxo + fy[c] * nyo;
            }
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int b = 0; b < N1; ++b) {
                    R s = R(0);
#pragma unroll
                    for (int k = 0; k < N1; ++k) s += fn[c][k] * T.M[b][k];
                    term[c][b] = h * s;
                }
        } else {
            // a face on the domain boundary: out of line, so the common
            // interior path stays compact in the instruction cache
            boundary_face_term<R, P, Ph>(m, pr, d, ex, ey, &Uf[0][0], &term[0][0]);
        }
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            int li = (d == 0) ? k * N1 : (d == 1) ? k * N1 + P : (d == 2) ? k : P * N1 + k;
#pragma unroll
            for (int c = 0; c < NC; ++c) W[c][li] -= term[c][k];
        }
    }
}

// stabilisation s^e = nu_e (K u - gamma_e G g_h) and the residual
// R^e = W^e - s^e into ER
template <class R, int P, class Ph>
DEV void stab_part(const MeshDev& m, const R (&U)[Ph::NC][Dim<P>::N2], const R* __restrict__ g,
                   const double* __restrict__ gam, const double* __restrict__ nu, const R (&W)[Ph::NC][Dim<P>::N2],
                   R* __restrict__ ER, int ex, int ey, int e) {
    constexpr int NC = Ph::NC, N1 = P + 1, N2 = Dim<P>::N2;
    const Tab<R>& T = tab_of<R>(m, P);
    const R h = PV<R>::h(m);
    // stabilisation s = nu (K u - gamma (Gx gx + Gy gy))
    const R nue = R(nu[e]), ge = R(gam[e]);
    const ElemNodes<P> en(m, ex, ey);
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
        R GX[N2], GY[N2];
#pragma unroll
        for (int b = 0; b < N1; ++b)
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                const long long n = en(a, b);
                GX[b * N1 + a] = g[(long long)c * m.NN + n];
                GY[b * N1 + a] = g[(long long)(NC + c) * m.NN + n];
            }
        // x-direction products: D u, M u, C gx, M gy
        R Du[N1][N1], Mu[N1][N1], Cg[N1][N1], Mg[N1][N1];
#pragma unroll
        for (int d = 0; d < N1; ++d)
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                R s1 = R(0), s2 = R(0), s3 = R(0), s4 = R(0);
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    s1 += T.D[a][k] * U[c][d * N1 + k];
                    s2 += T.M[a][k] * U[c][d * N1 + k];
                    s3 += T.C[a][k] * GX[d * N1 + k];
                    s4 += T.M[a][k] * GY[d * N1 + k];
                }
                Du[d][a] = s1;
                Mu[d][a] = s2;
                Cg[d][a] = s3;
                Mg[d][a] = s4;
            }
#pragma unroll
        for (int b = 0; b < N1; ++b)
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                R ku = R(0), gg = R(0);
#pragma unroll
                for (int d = 0; d < N1; ++d) {
                    ku += T.M[b][d] * Du[d][a] + T.D[b][d] * Mu[d][a];
                    gg += T.M[b][d] * Cg[d][a] + T.C[b][d] * Mg[d][a];
                }
                R s = nue * (ku - ge * (h * gg));
                ER[ev_at(m.E, e, b * N1 + a, c, NC)] = W[c][b * N1 + a] - s;
            }
    }
}

// Euler at p = 2: 3 blocks of 128 per SM (170-register cap; measured faster)

template <class R, int P, class Ph>
DEV void res_at(const MeshDev& m, const ProbDev& pr, const R* __restrict__ u, const R* __restrict__ g,
                         const double* __restrict__ gam, const double* __restrict__ nu,
                         R* __restrict__ ER, int ex, int ey, int e) {
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    R U[NC][N2];
    load_block<R, P, NC>(u, m, ex, ey, U);
    R W[NC][N2];
    w_part<R, P, Ph>(m, pr, U, ex, ey, W);
    stab_part<R, P, Ph>(m, U, g, gam, nu, W, ER, ex, ey, e);
}

template <class R, int P, class Ph>
__global__ void __launch_bounds__(128, elem_blocks<P, Ph::NC, sizeof(R)>(EK_RES)) k_res_ev(MeshDev m, ProbDev pr, const R* __restrict__ u, const R* __restrict__ g,
                         const double* __restrict__ gam, const double* __restrict__ nu,
                         R* __restrict__ ER) {
    pdl_begin();
    int ex, ey, e;
    if (!elem_of_thread(m, ex, ey, e)) return;
    res_at<R, P, Ph>(m, pr, u, g, gam, nu, ER, ex, ey, e);
}


// ---------------------------------------------------------------------------
// k_update_ev: facet fluxes and flux limiter, ubar^e, f_i^e, beta_e and the
// element increments of eq. (eq:SSPupdate),
//   m_i u_i^SSP = sum_e m_i^e [(1 - theta_e) u_i + theta_e ubar_i^e]
//   <=> u_i^SSP = u_i + sum_e (m_i^e/m_i) theta_e (ubar^e - u_i + beta_e f_i^e/m_i^e),
// theta_e = dt/dt_e; the increment theta_e (...) is stored per (e, i).
// Per-node arithmetic is in R (float in the mixed form, the float64 values
// ubar^e and u^e enter as hi + lo float pairs); per-facet and per-element
// quantities are float64.
// ---------------------------------------------------------------------------
template <class T>
DEV void split(double v, T& hi, T& lo) {
    hi = T(v);
    lo = T(v - (double)hi);
}

// sum over the face nodes of F(u_j, u_hat_j; n) on a boundary face of side
// d that is not OUTFLOW everywhere (f^H of eq. (hoflux) before the division
// by p+1; on an LGL mesh the sum weighted by w_j, f^H itself), u_hat_j of
// the side at node j; Uf is [NC][p+1]
template <class R, int P, class Ph>
__device__ __noinline__ CompVec<R, Ph::NC> bnd_face_llf_sum(const MeshDev& m, const ProbDev& pr, int d, int e,
                                                           R nx, R ny, const R* Uf) {
    constexpr int NC = Ph::NC, N1 = P + 1;
    const bool split = side_split(pr, d);
    int ex = 0, ey = 0;
    if (split) {
        ey = e / m.nx;
        ex = e - ey * m.nx;
    }
    CompVec<R, NC> out;
    R* acc = out.v;
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = R(0);
    // a FIXED side with one part: one external state, its flux evaluated once
    const bool fixed1 = !split && pr.side[d].kind[0] == BC_FIXED;
    R ub1[NC], fxb[NC], fyb[NC];
    if (fixed1) {
#pragma unroll
        for (int c = 0; c < NC; ++c) ub1[c] = PV<R>::side_state(pr.side[d], 0, c);
        Ph::template flux<R>(ub1, fxb, fyb, pr);
    }
#pragma unroll
    for (int k = 0; k < N1; ++k) {
        R uk[NC], ub[NC], F[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) uk[c] = Uf[c * N1 + k];
        if (fixed1) {
            llf_given_fR<Ph, R>(uk, ub1, fxb, fyb, nx, ny, pr, F);
        } else {
            const int slot = split ? side_slot(pr, d, side_node_pos(m, d, ex, ey, k)) : 0;
            ext_state<R, NC>(pr, d, slot, uk, ub);
            llf<Ph, R>(uk, ub, nx, ny, pr, F, (R*)nullptr);
        }
        if (is_lgl<R>(m)) {
            const R wk = R(c_tabd[PMAX + 1 + P].wl[k]);
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] += wk * F[c];
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] += F[c];
        }
    }
    return out;
}

// ubar^e in G: scalars umin <= ubar <= umax, Euler rho > 0 and
// rho E - |m|^2/2 > 0 (explicit float64 roundings, the same decision in
// every kernel)
template <class Ph>
DEV bool average_in_G(const ProbDev& pr, const double (&ub)[Ph::NC]) {
    if constexpr (Ph::NC == 1) {
        return ub[0] >= pr.umin && ub[0] <= pr.umax;
    } else {
        const double kin = __dmul_rn(0.5, __dadd_rn(__dmul_rn(ub[1], ub[1]), __dmul_rn(ub[2], ub[2])));
        return ub[0] > 0.0 && __dsub_rn(__dmul_rn(ub[0], ub[3]), kin) > 0.0;
    }
}

// An unlimited average ubar^e = u^e - r S_e (eq. (uebar), r = dt_e / h, S_e
// the outward sum of f^H) that left G: counted; with OPT_DTE_REDUCE the
// strategy of the remark after eq. (dtmaxcell): the largest r in [0, rs]
// with ubar^e in G (scalars: the crossed bound solved exactly; Euler: the
// Appendix-A criterion for u^e moved by -rs S_e, r = rs alpha).  Returns
// [ubar^e .., r].
template <class Ph>
__device__ __noinline__ CompVec<double, Ph::NC + 1> reduce_pseudo_step(const ProbDev& pr,
                                                                      const double (&ue)[Ph::NC],
                                                                      const double (&os)[Ph::NC], double rs,
                                                                      unsigned long long* __restrict__ cnt) {
    constexpr int NC = Ph::NC;
    atomicAdd(&cnt[CNT_UBAR], 1ull);
    CompVec<double, NC + 1> out;
    double r = rs;
    if (pr.opts & OPT_DTE_REDUCE) {
        if constexpr (NC == 1) {
            const double d = os[0];
            if (d < 0.0) r = fmin(r, (pr.umax - ue[0]) / (-d));
            if (d > 0.0) r = fmin(r, (ue[0] - pr.umin) / d);
            r = fmax(r, 0.0);
        } else {
            double g[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) g[c] = (-rs) * os[c];
            r = rs * euler_alpha<double>(ue, g, 1.0, pr.pos_eps);
        }
        if (r < rs) atomicAdd(&cnt[CNT_DTE_RED], 1ull);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) out.v[c] = ue[c] - r * os[c];
    out.v[NC] = r;
    return out;
}

// facet part of the element update: canonical f^H, the flux limiter and
// ubar^e (eqs. (hoflux), (fAlim)/(uelim), Appendix A), and the facet term
// (h/(p+1)^2) sum_d +-f^H_d of the element contributions f_i^e (eq. (aec))
template <class R, int P, class Ph>
DEV void facet_part(const MeshDev& m, const ProbDev& pr, const R (&U)[Ph::NC][Dim<P>::N2], const int (&nb)[4],
                    const double (&uec)[Ph::NC], const double (&ublc)[Ph::NC], double rs,
                    const double* __restrict__ dte_a, const double* __restrict__ ubl,
                    const R* __restrict__ qcap, const R* __restrict__ fl_in, const float* __restrict__ cf, int e,
                    double (&ubec)[Ph::NC], R (&fh)[Ph::NC], double& rs_out,
                    unsigned long long* __restrict__ cnt) {
    constexpr int NC = Ph::NC, N1 = P + 1;
    rs_out = rs;
    // FP32-mixed systems: the limited facet fluxes enter ubar^e as float-float
    // terms (below), so f^H stays in float and no float64 copy is formed
    constexpr bool mixed_sys = sizeof(R) == 4 && NC > 1;
    const double h = m.h;
    // canonical high-order facet fluxes f^H (eq. (hoflux)): face average of
    // f(u_j).n (or of F(u_j, u_hat; n) on a FIXED boundary), summed along the
    // face in a fixed order so both cells of a facet get the same value
    double FH[4][NC];
    R FHr[4][NC];
    const bool need_fh = !(pr.mode == MODE_LO && pr.fl == FL_LOW);
    if (need_fh) {
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const R cnx = (d < 2) ? R(1) : R(0), cny = (d < 2) ? R(0) : R(1);
            const bool fixed_b = (nb[d] < 0) && !side_plain(pr, d);
            const R sg = (d == 1 || d == 3) ? R(1) : R(-1);
            R acc[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = R(0);
            if (fixed_b) {
                // boundary face with u_hat data: out of line (rare; keeps the hot code small)
                R Uf[NC * N1];
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    const int li = (d == 0) ? k * N1 : (d == 1) ? k * N1 + P : (d == 2) ? k : P * N1 + k;
#pragma unroll
                    for (int c = 0; c < NC; ++c) Uf[c * N1 + k] = U[c][li];
                }
                const CompVec<R, NC> fs = bnd_face_llf_sum<R, P, Ph>(m, pr, d, e, sg * cnx, sg * cny, Uf);
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[c] = fs.v[c];  // acc was 0: same sums
            } else {
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    const int li = (d == 0) ? k * N1 : (d == 1) ? k * N1 + P : (d == 2) ? k : P * N1 + k;
                    R uk[NC], fx[NC], fy[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) uk[c] = U[c][li];
                    Ph::template flux<R>(uk, fx, fy, pr);
                    if (is_lgl<R>(m)) {
                        // LGL: the face mean weights node k by w_k
                        const R wk = R(c_tabd[PMAX + 1 + P].wl[k]);
#pragma unroll
                        for (int c = 0; c < NC; ++c) acc[c] += wk * (fx[c] * cnx + fy[c] * cny);
                    } else {
#pragma unroll
                        for (int c = 0; c < NC; ++c) acc[c] += fx[c] * cnx + fy[c] * cny;
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const R a = is_lgl<R>(m) ? acc[c] : acc[c] / R(N1);
                FHr[d][c] = fixed_b ? sg * a : a;
                if constexpr (!mixed_sys) FH[d][c] = (double)FHr[d][c];
            }
        }
    }
    // limited cell average ubar^e
    if (pr.fl == FL_LOW) {
#pragma unroll
        for (int c = 0; c < NC; ++c) ubec[c] = ublc[c];
    } else if (pr.fl == FL_NONE) {
        double osv[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double os;
            if constexpr (mixed_sys) {
                float osh, osl;
                ff_sum4(FHr[1][c], FHr[0][c], FHr[3][c], FHr[2][c], osh, osl);
                os = (double)osh + (double)osl;
            } else {
                os = ((FH[1][c] - FH[0][c]) + FH[3][c]) - FH[2][c];
            }
            osv[c] = os;
            ubec[c] = uec[c] - rs * os;
        }
        // eq. (uebar) with the macrocell dt_e need not stay in G: count such
        // averages, and with the option decrease dt_e as the remark after
        // eq. (dtmaxcell) says (out of line: rare)
        if (!average_in_G<Ph>(pr, ubec)) {
            const CompVec<double, NC + 1> red = reduce_pseudo_step<Ph>(pr, uec, osv, rs, cnt);
#pragma unroll
            for (int c = 0; c < NC; ++c) ubec[c] = red.v[c];
            rs_out = red.v[NC];
        }
    } else {
        R FLr[4][NC];
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int c = 0; c < NC; ++c) FLr[d][c] = fl_in[((long long)e * 4 + d) * NC + c];
        double FB[4][NC];
        R FBr[4];  // scalar limited fluxes in the bulk precision
        // mixed systems: facet d enters as the float pair (TH, TL) per
        // component: (f^L, -f^H) where alpha = 1 (certified in float, or
        // computed as 1 in float64: the same terms either way, so the
        // certificate changes no bit), else alpha f^A split into two floats
        float TH[mixed_sys ? 4 : 1][mixed_sys ? NC : 1], TL[mixed_sys ? 4 : 1][mixed_sys ? NC : 1];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const bool self_is_L = (d == 1 || d == 3);
            const int Lc = self_is_L ? e : nb[d];
            const int Rc = self_is_L ? nb[d] : e;
            if (Ph::NC == 1) {
                // eq. (fAlim) with the capacities of both cells (R-typed; in the
                // mixed form they were rounded toward zero, so still admissible)
                const R fA = FLr[d][0] - FHr[d][0];
                const R inf = R(__int_as_float(0x7f800000));
                R fmaxv = inf, fminv = -inf;
                if (Lc >= 0) {
                    fmaxv = fmin(fmaxv, qcap[Lc]);
                    fminv = fmax(fminv, qcap[m.E + Lc]);
                }
                if (Rc >= 0) {
                    fmaxv = fmin(fmaxv, -qcap[m.E + Rc]);
                    fminv = fmax(fminv, -qcap[Rc]);
                }
                FBr[d] = (fA >= R(0)) ? fmin(fA, fmaxv) : fmax(fA, fminv);
                FB[d][0] = (double)FBr[d];
            } else {
                double fA[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) fA[c] = (double)FLr[d][c] - (double)FHr[d][c];
                if constexpr (sizeof(R) == 4) {
                    // float32 certificate first: where both cells certainly
                    // give alpha = 1 the float64 formula is skipped (same result)
                    if (!(pr.opts & OPT_FP64_LIMITER)) {
                        float fAf[NC], fAm[NC], ub[NC];
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            fAf[c] = __fsub_rn(FLr[d][c], FHr[d][c]);
                            fAm[c] = -fAf[c];
                        }
                        bool one = true;
                        if (Lc >= 0) {
#pragma unroll
                            for (int c = 0; c < NC; ++c) ub[c] = cf[(1 + c) * m.E + Lc];
                            one = euler_alpha_is_one(ub, fAf, 0.25f * cf[Lc], pr.ome_f);
                        }
                        if (one && Rc >= 0) {
#pragma unroll
                            for (int c = 0; c < NC; ++c) ub[c] = cf[(1 + c) * m.E + Rc];
                            one = euler_alpha_is_one(ub, fAm, 0.25f * cf[Rc], pr.ome_f);
                        }
                        if (one) {
#pragma unroll
                            for (int c = 0; c < NC; ++c) {
                                TH[d][c] = FLr[d][c];
                                TL[d][c] = -FHr[d][c];
                            }
                            continue;
                        }
                    }
                }
                double alpha = 1.0;
                if (Lc >= 0) {
                    double ub[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) ub[c] = ubl[c * m.E + Lc];
                    double mL = (0.25 * h) * dte_a[2 * m.E + Lc];
                    alpha = fmin(alpha, euler_alpha<double>(ub, fA, mL, pr.pos_eps));
                }
                if (Rc >= 0) {
                    double ub[NC], fm[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        ub[c] = ubl[c * m.E + Rc];
                        fm[c] = -fA[c];
                    }
                    double mR = (0.25 * h) * dte_a[2 * m.E + Rc];
                    alpha = fmin(alpha, euler_alpha<double>(ub, fm, mR, pr.pos_eps));
                }
                if constexpr (mixed_sys) {
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        if (alpha == 1.0) {
                            TH[d][c] = FLr[d][c];
                            TL[d][c] = -FHr[d][c];
                        } else {
                            const double v = alpha * fA[c];
                            TH[d][c] = __double2float_rn(v);
                            TL[d][c] = __double2float_rn(v - (double)TH[d][c]);
                        }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < NC; ++c) FB[d][c] = alpha * fA[c];
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double os;
            if constexpr (sizeof(R) == 4 && Ph::NC == 1) {
                // float limited fluxes summed as a float-float pair, widened once
                float osh, osl;
                ff_sum4(FBr[1], FBr[0], FBr[3], FBr[2], osh, osl);
                os = (double)osh + (double)osl;
            } else if constexpr (mixed_sys) {
                // (fbar_E - fbar_W) + fbar_N - fbar_S from the eight float terms,
                // compensated, widened once
                const float t[8] = {TH[1][c], TL[1][c], -TH[0][c], -TL[0][c],
                                    TH[3][c], TL[3][c], -TH[2][c], -TL[2][c]};
                float osh, osl;
                ff_sum<8>(t, osh, osl);
                os = (double)osh + (double)osl;
            } else {
                os = ((FB[1][c] - FB[0][c]) + FB[3][c]) - FB[2][c];
            }
            ubec[c] = ublc[c] + rs * os;
        }
    }
    // (m_i^e / |K_e|) |S| times the outward sum of f^H, the facet term of
    // eq. (aecb): h / (p+1)^2 for every node (Bernstein); on an LGL mesh h,
    // weighted by w_a w_b per node in element_part
    const R h_over_n2R = (sizeof(R) == 4) ? R(m.h_over_n2_f) : (is_lgl<R>(m) ? R(m.h) : R(m.h_over_n2));
#pragma unroll
    for (int c = 0; c < NC; ++c)
        fh[c] = need_fh ? h_over_n2R * (((FHr[1][c] - FHr[0][c]) + FHr[3][c]) - FHr[2][c]) : R(0);
}

// element part of the update: theta, f_i^e (eq. (aec)), the slope limiter
// beta_e (eqs. (slimit1), (slimit2), Appendix A) and the SSP increments
// Q1: the variant of eq. (aecQ1); the caller passes ER = -D_i (the
// divergence term), ud = udot^L and fh = 0, and the contributions are scaled
// by gamma_e (gq)
template <class R, int P, class Ph, bool Q1 = false>
DEV void element_part(const MeshDev& m, const ProbDev& pr, const R (&U)[Ph::NC][Dim<P>::N2],
                      const R* __restrict__ ud, const R* __restrict__ ER, const float* __restrict__ cf,
                      const float* __restrict__ avg, const double (&uec)[Ph::NC], double dt, double dte, double rdte,
                      const double (&ubec)[Ph::NC], const R (&fh)[Ph::NC], R* __restrict__ EW,
                      double* __restrict__ beta_out, unsigned long long* __restrict__ cnt, int ex, int ey, int e,
                      double gq = 1.0) {
    constexpr int NC = Ph::NC, N1 = P + 1, N2 = Dim<P>::N2;
    const Tab<R>& T = tab_of<R>(m, P);
    const double me = m.me;
    // theta = dt / dt_e = dt s / h; FP32-mixed: in float from the float
    // speed sum of k_pre (it weights float increments; the check counts only)
    R thR;
    if constexpr (sizeof(R) == 4) {
        thR = __fmul_rn((float)dt, __fmul_rn(cf[e], m.inv_h_f));
        if (thR > 1.f) atomicAdd(&cnt[CNT_CFL], 1ull);
    } else {
        const double theta = dt * rdte;
        if (theta > 1.0) atomicAdd(&cnt[CNT_CFL], 1ull);
        thR = R(theta);
    }
    R ubh[NC], ubo[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) split<R>(ubec[c], ubh[c], ubo[c]);
    if (pr.mode == MODE_LO) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int i = 0; i < N2; ++i)
                EW[ev_at(m.E, e, i, c, NC)] = thR * ((ubh[c] - U[c][i]) + ubo[c]);
        beta_out[e] = 0.0;
        return;
    }
    // f_i^e, eq. (aec) with eq. (aecb) folded into the residual
    const R meR = PV<R>::me(m), h2 = PV<R>::h2(m), inv_meR = PV<R>::inv_me(m);
    // LGL mesh (float64 form): m_i^e = h^2 w_a w_b and 1/m_i^e per node, the
    // facet term fh weighted by w_a w_b (see facet_part)
    const bool lgl = is_lgl<R>(m);
    const Tab<double>& TL = c_tabd[PMAX + 1 + P];
    R dteR;
    if constexpr (sizeof(R) == 4) dteR = __fmul_rn(m.h_f, __frcp_rn(cf[e]));  // h / s in float
    else dteR = R(dte);
    R F[NC][N2];
    // components unrolled for p >= 3 (registers); at p <= 2 the rolled loop
    // keeps occupancy higher (measured on the Euler workloads)
    const ElemNodes<P> en(m, ex, ey);
#pragma unroll (P >= 3 ? Ph::NC : 1)
    for (int c = 0; c < NC; ++c) {
        R UD[N2];
#pragma unroll
        for (int b = 0; b < N1; ++b)
#pragma unroll
            for (int a = 0; a < N1; ++a)
                UD[b * N1 + a] = ud[(long long)c * m.NN + en(a, b)];
        R Y[N1][N1];
#pragma unroll
        for (int d = 0; d < N1; ++d)
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                R s = R(0);
#pragma unroll
                for (int k = 0; k < N1; ++k) s += T.M[a][k] * UD[d * N1 + k];
                Y[d][a] = s;
            }
        const R fh_term = fh[c];
        R ueh, uel;
        if constexpr (sizeof(R) == 4) {
            // the float-float mean itself (k_pre for scalars, k_avg for systems)
            ueh = avg[(2 * c) * m.E + e];
            uel = avg[(2 * c + 1) * m.E + e];
        } else {
            split<R>(uec[c], ueh, uel);
        }
#pragma unroll
        for (int b = 0; b < N1; ++b)
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                R s = R(0);
#pragma unroll
                for (int d = 0; d < N1; ++d) s += T.M[b][d] * Y[d][a];
                const int i = b * N1 + a;
                R Ri = ER[ev_at(m.E, e, i, c, NC)];
                R dev = (U[c][i] - ueh) - uel;
                if (lgl) {
                    const R w2 = R(TL.wl[a] * TL.wl[b]);
                    const R mi = h2 * w2;
                    F[c][i] = mi * dev + dteR * (((Ri + fh_term * w2) - h2 * s) + mi * UD[i]);
                } else {
                    F[c][i] = meR * dev + dteR * (((Ri + fh_term) - h2 * s) + meR * UD[i]);
                }
                if constexpr (Q1) F[c][i] = R(gq) * F[c][i];
            }
    }
    // slope limiter beta_e
    R beta = R(1);
    if (pr.mode == MODE_WENO_L) {
        if (Ph::NC == 1) {
            // bound gaps in float64 per element, ratios per node in R
            R gp, gm;
            if constexpr (sizeof(R) == 4) {
                // gaps in float64; m_i^e, the gaps and the products rounded
                // toward zero (smaller magnitudes stay admissible)
                gp = __fmul_rz(m.me_rz_f, __double2float_rz(pr.umax - ubec[0]));
                gm = __fmul_rz(m.me_rz_f, __double2float_rz(pr.umin - ubec[0]));
            } else {
                gp = R(me * (pr.umax - ubec[0]));
                gm = R(me * (pr.umin - ubec[0]));
            }
            R b = R(1);
#pragma unroll
            for (int i = 0; i < N2; ++i) {
                R f = F[0][i];
                R gpi = gp, gmi = gm;
                if (lgl) {
                    // m_i^e of this node (the gaps scale with it)
                    const double mi = m.h * m.h * (TL.wl[i % N1] * TL.wl[i / N1]);
                    gpi = R(mi * (pr.umax - ubec[0]));
                    gmi = R(mi * (pr.umin - ubec[0]));
                }
                R bi = R(1);
                if (f > R(0)) bi = fmin(R(1), gpi / f);
                else if (f < R(0)) bi = fmin(R(1), gmi / f);
                b = fmin(b, bi);
            }
            beta = fmin(fmax(b, R(0)), R(1));
        } else {
            double b = 1.0;
            float ubf[NC];
            const bool cert = (sizeof(R) == 4) && !(pr.opts & OPT_FP64_LIMITER);
#pragma unroll
            for (int c = 0; c < NC; ++c) ubf[c] = cert ? (float)ubec[c] : 0.f;
#pragma unroll
            for (int i = 0; i < N2; ++i) {
                // float32 certificate first; the float64 formula only where
                // it cannot show alpha_i = 1 (min(b, 1) = b: same result)
                if (cert) {
                    float ff[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) ff[c] = (float)F[c][i];
                    if (euler_alpha_is_one(ubf, ff, m.me_f, pr.ome_f)) continue;
                }
                double f[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) f[c] = (double)F[c][i];
                const double mi = lgl ? m.h * m.h * (TL.wl[i % N1] * TL.wl[i / N1]) : me;
                b = fmin(b, euler_alpha_of<R>(ubec, f, mi, pr.pos_eps));
            }
            beta = R(b);
        }
    }
    beta_out[e] = (double)beta;
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int i = 0; i < N2; ++i) {
            const R inv_mi = lgl ? R(m.inv_h2 * (TL.iwl[i % N1] * TL.iwl[i / N1])) : inv_meR;
            EW[ev_at(m.E, e, i, c, NC)] = thR * (((ubh[c] - U[c][i]) + ubo[c]) + (beta * F[c][i]) * inv_mi);
        }
}

template <class R, int P, class Ph>
DEV void update_at(const MeshDev& m, const ProbDev& pr, const R* __restrict__ u, const R* __restrict__ ud,
                            const double* __restrict__ ue, double* dte_a,
                            const double* __restrict__ ubl,
                            const R* __restrict__ qcap, const R* __restrict__ fl_in,
                            const R* __restrict__ ER, const float* __restrict__ cf,
                            const float* __restrict__ avg,
                            const double* __restrict__ dtp, R* __restrict__ EW,
                            double* __restrict__ ube_out, double* __restrict__ beta_out,
                            unsigned long long* __restrict__ cnt, int ex, int ey, int e) {
    constexpr int NC = Ph::NC, N1 = P + 1, N2 = Dim<P>::N2;
    const Tab<R>& T = tab_of<R>(m, P);
    const double h = m.h;
    const double me = m.me;
    const double dt = *dtp;
    const double dte = dte_a[e];
    const double rs = dte_a[m.E + e];       // dt_e / h
    const double rdte = dte_a[2 * m.E + e]; // 1 / dt_e
    int nb[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) nb[d] = neighbour(m, ex, ey, d);
    R U[NC][N2];
    load_block<R, P, NC>(u, m, ex, ey, U);
    double uec[NC], ublc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        uec[c] = ue[c * m.E + e];
        ublc[c] = ubl[c * m.E + e];
    }
    double ubec[NC];
    R fh[NC];
    double rs2;
    facet_part<R, P, Ph>(m, pr, U, nb, uec, ublc, rs, dte_a, ubl, qcap, fl_in, cf, e, ubec, fh, rs2, cnt);
#pragma unroll
    for (int c = 0; c < NC; ++c) ube_out[c * m.E + e] = ubec[c];
    if (rs2 != rs) {
        // a pseudo time step decreased by the remark after eq. (dtmaxcell)
        const double dte2 = h * rs2;
        dte_a[e] = dte2;
        dte_a[m.E + e] = rs2;
        dte_a[2 * m.E + e] = 1.0 / dte2;
        element_part<R, P, Ph>(m, pr, U, ud, ER, cf, avg, uec, dt, dte2, 1.0 / dte2, ubec, fh, EW, beta_out, cnt, ex,
                               ey, e);
        return;
    }
    element_part<R, P, Ph>(m, pr, U, ud, ER, cf, avg, uec, dt, dte, rdte, ubec, fh, EW, beta_out, cnt, ex, ey, e);
}

// ---------------------------------------------------------------------------
// The Q1 variant, eq. (aecQ1) (option OPT_AEC_Q1):
//   f_i^e = gamma_e ( m_i^e (u_i - u^e) - dt_e [ D_i + (M udot^L)_i - m_i^e udot^L_i ] ),
//   D_i = int (phi_i - m_i^e/|K_e|) div f_h,  f_h = sum_j f(u_j) phi_j,
// udot^L from the low-order scheme, eq. (weak:low2).  Three kernels replace
// the g_h, residual and udot kernels: k_q1_facet (ubar^e and -D_i),
// k_udl (udot^L at the nodes) and k_q1_update (the element part of the
// update with ER = -D_i, udot := udot^L, no facet term, scaled by gamma_e).
// ---------------------------------------------------------------------------
template <class R, int P, class Ph>
__global__ void __launch_bounds__(128) k_q1_facet(MeshDev m, ProbDev pr, const R* __restrict__ u,
                                                  const double* __restrict__ ue, const double* __restrict__ dte_a,
                                                  const double* __restrict__ ubl, const R* __restrict__ qcap,
                                                  const R* __restrict__ fl_in, const float* __restrict__ cf,
                                                  R* __restrict__ ER, double* __restrict__ ube_out,
                                                  unsigned long long* __restrict__ cnt) {
    pdl_begin();
    int ex, ey, e;
    if (!elem_of_thread(m, ex, ey, e)) return;
    constexpr int NC = Ph::NC, N1 = P + 1, N2 = Dim<P>::N2;
    const Tab<R>& T = tab_of<R>(m, P);
    int nb[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) nb[d] = neighbour(m, ex, ey, d);
    R U[NC][N2];
    load_block<R, P, NC>(u, m, ex, ey, U);
    double uec[NC], ublc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        uec[c] = ue[c * m.E + e];
        ublc[c] = ubl[c * m.E + e];
    }
    double ubec[NC];
    R fh[NC];
    double rs2;  // eq. (aecQ1) is not combined with the pseudo-time-step reduction
    facet_part<R, P, Ph>(m, pr, U, nb, uec, ublc, dte_a[m.E + e], dte_a, ubl, qcap, fl_in, cf, e, ubec, fh, rs2,
                         cnt);
#pragma unroll
    for (int c = 0; c < NC; ++c) ube_out[c * m.E + e] = ubec[c];
    // nodal fluxes f(u_j)
    R FX[NC][N2], FY[NC][N2];
#pragma unroll
    for (int j = 0; j < N2; ++j) {
        R uj[NC], fx[NC], fy[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) uj[c] = U[c][j];
        Ph::template flux<R>(uj, fx, fy, pr);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            FX[c][j] = fx[c];
            FY[c][j] = fy[c];
        }
    }
    // int phi_i d_x phi_j = h int B_a B_c' int B_b B_d (C[c][a] = int B_c' B_a),
    // int d_x phi_j = sum_i of it; the same with x and y exchanged
    const R h = PV<R>::h(m);
    R csum[N1], msum[N1];
#pragma unroll
    for (int c = 0; c < N1; ++c) {
        R s1 = R(0), s2 = R(0);
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            s1 += T.C[c][a];
            s2 += T.M[a][c];
        }
        csum[c] = s1;
        msum[c] = s2;
    }
    const R inv_n2 = R(1) / R(N2);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        // mean term (m_i^e/|K_e|) sum_j c_j . f(u_j), the same for every i
        R mean = R(0);
#pragma unroll
        for (int d = 0; d < N1; ++d)
#pragma unroll
            for (int cc = 0; cc < N1; ++cc)
                mean += (csum[cc] * msum[d]) * FX[c][d * N1 + cc] + (msum[cc] * csum[d]) * FY[c][d * N1 + cc];
        mean = h * mean * inv_n2;
#pragma unroll
        for (int b = 0; b < N1; ++b)
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                R s = R(0);
#pragma unroll
                for (int d = 0; d < N1; ++d)
#pragma unroll
                    for (int cc = 0; cc < N1; ++cc)
                        s += (T.C[cc][a] * T.M[b][d]) * FX[c][d * N1 + cc] + (T.M[a][cc] * T.C[d][b]) * FY[c][d * N1 + cc];
                ER[ev_at(m.E, e, b * N1 + a, c, NC)] = -(h * s - mean);
            }
    }
}

// udot^L_i = (1/|E_i|) sum_{e in E_i} (ubar^e - u_i) / dt_e, eq. (weak:low2)
// with m_i = |E_i| m_i^e (float64 sums, fixed order)
template <class R, int P, int NC>
__global__ void k_udl(MeshDev m, const R* __restrict__ u, const double* __restrict__ ube,
                      const double* __restrict__ dte_a, R* __restrict__ ud) {
    pdl_begin();
    int gx, gy;
    long long node;
    if (!node_of_thread(m, gx, gy, node)) return;
    const NodeC<P> c = node_c<P>(m, gx, gy);
    const double w = inv_count<double>(c.nxc * c.nyc);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const double ui = (double)u[(long long)k * m.NN + node];
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (j < c.nyc) {
                const int ey = j ? c.ey1 : c.ey0;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    if (i < c.nxc) {
                        const int e = ey * m.nx + (i ? c.ex1 : c.ex0);
                        s += (ube[k * m.E + e] - ui) * dte_a[2 * m.E + e];
                    }
                }
            }
        }
        ud[(long long)k * m.NN + node] = R(s * w);
    }
}

template <class R, int P, class Ph>
__global__ void __launch_bounds__(128) k_q1_update(MeshDev m, ProbDev pr, const R* __restrict__ u,
                                                   const R* __restrict__ udl, const double* __restrict__ ue,
                                                   const double* __restrict__ dte_a, const R* __restrict__ ER,
                                                   const float* __restrict__ cf, const float* __restrict__ avg,
                                                   const double* __restrict__ ube, const double* __restrict__ gam,
                                                   const double* __restrict__ dtp, R* __restrict__ EW,
                                                   double* __restrict__ beta_out, unsigned long long* __restrict__ cnt) {
    pdl_begin();
    int ex, ey, e;
    if (!elem_of_thread(m, ex, ey, e)) return;
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    R U[NC][N2];
    load_block<R, P, NC>(u, m, ex, ey, U);
    double uec[NC], ubec[NC];
    R fh[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        uec[c] = ue[c * m.E + e];
        ubec[c] = ube[c * m.E + e];
        fh[c] = R(0);
    }
    element_part<R, P, Ph, true>(m, pr, U, udl, ER, cf, avg, uec, *dtp, dte_a[e], dte_a[2 * m.E + e], ubec, fh, EW,
                                 beta_out, cnt, ex, ey, e, gam[e]);
}

// Euler at p = 2: 3 blocks of 128 per SM (a 170-register cap, no spills)
// instead of the 2 that the uncapped allocation leaves (measured faster)
template <class R, int P, class Ph>
__global__ void __launch_bounds__(128, elem_blocks<P, Ph::NC, sizeof(R)>(EK_UPD)) k_update_ev(MeshDev m, ProbDev pr, const R* __restrict__ u, const R* __restrict__ ud,
                            const double* __restrict__ ue, double* dte_a, const double* __restrict__ ubl,
                            const R* __restrict__ qcap, const R* __restrict__ fl_in,
                            const R* __restrict__ ER, const float* __restrict__ cf,
                            const float* __restrict__ avg,
                            const double* __restrict__ dtp, R* __restrict__ EW,
                            double* __restrict__ ube_out, double* __restrict__ beta_out,
                            unsigned long long* __restrict__ cnt) {
    pdl_begin();
    int ex, ey, e;
    if (!elem_of_thread(m, ex, ey, e)) return;
    update_at<R, P, Ph>(m, pr, u, ud, ue, dte_a, ubl, qcap, fl_in, ER, cf, avg, dtp, EW, ube_out, beta_out, cnt, ex,
                        ey, e);
}


// FP32-mixed: the update in two kernels.  k_facet needs only u and the
// outputs of k_pre, so it runs on a second stream beside the g_h and udot
// kernels; k_update_el then reads its ubar^e and facet terms.  Together they
// compute what k_update_ev computes, in the same arithmetic.  The bodies are
// device functions of one element, also run by the batched stage.
template <int P, class Ph>
DEV void facet_el_at(const MeshDev& m, const ProbDev& pr, const float* __restrict__ u,
                     const double* __restrict__ ue, double* dte_a, const double* __restrict__ ubl,
                     const float* __restrict__ qcap, const float* __restrict__ fl_in, float* cf,
                     double* __restrict__ ube_out, float* __restrict__ fht, unsigned long long* __restrict__ cnt,
                     int ex, int ey, int e) {
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    int nb[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) nb[d] = neighbour(m, ex, ey, d);
    float U[NC][N2];
    load_block<float, P, NC>(u, m, ex, ey, U);
    double uec[NC], ublc[NC], ubec[NC];
    float fh[NC];
    const bool need_ue = pr.fl == FL_NONE;  // u^e enters ubar^e only without the flux limiter
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        uec[c] = need_ue ? ue[c * m.E + e] : 0.0;
        ublc[c] = ubl[c * m.E + e];
    }
    const double rs = dte_a[m.E + e];
    double rs2;
    facet_part<float, P, Ph>(m, pr, U, nb, uec, ublc, rs, dte_a, ubl, qcap, fl_in, cf, e, ubec, fh, rs2, cnt);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        ube_out[c * m.E + e] = ubec[c];
        fht[c * m.E + e] = fh[c];
    }
    if (rs2 != rs) {
        // a pseudo time step decreased by the remark after eq. (dtmaxcell):
        // the float speed sum that k_update_el reads is rounded up (its float
        // dt_e never exceeds the reduced one)
        const double dte2 = m.h * rs2;
        dte_a[e] = dte2;
        dte_a[m.E + e] = rs2;
        dte_a[2 * m.E + e] = 1.0 / dte2;
        cf[e] = __double2float_ru(1.0 / rs2);
    }
}

template <int P, class Ph>
DEV void update_el_at(const MeshDev& m, const ProbDev& pr, const float* __restrict__ u,
                      const float* __restrict__ ud, const float* __restrict__ ER, const float* __restrict__ cf,
                      const float* __restrict__ avg, const double* __restrict__ ube,
                      const float* __restrict__ fht, const double* __restrict__ dtp, float* __restrict__ EW,
                      double* __restrict__ beta_out, unsigned long long* __restrict__ cnt, int ex, int ey, int e) {
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    float U[NC][N2];
    load_block<float, P, NC>(u, m, ex, ey, U);
    // the float path of element_part takes dt_e and theta from the float
    // speed sum and the mean from the float-float pair: u^e, dt_e and 1/dt_e
    // in float64 are not read
    double uec[NC], ubec[NC];
    float fh[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        uec[c] = 0.0;
        ubec[c] = ube[c * m.E + e];
        fh[c] = fht[c * m.E + e];
    }
    element_part<float, P, Ph>(m, pr, U, ud, ER, cf, avg, uec, *dtp, 0.0, 0.0, ubec, fh, EW, beta_out, cnt, ex, ey,
                               e);
}

template <int P, class Ph>
__global__ void __launch_bounds__(128, elem_blocks<P, Ph::NC, 4>(EK_FACET)) k_facet(MeshDev m, ProbDev pr, const float* __restrict__ u,
                                               const double* __restrict__ ue, double* dte_a,
                                               const double* __restrict__ ubl, const float* __restrict__ qcap,
                                               const float* __restrict__ fl_in, float* cf,
                                               double* __restrict__ ube_out, float* __restrict__ fht,
                                               unsigned long long* __restrict__ cnt) {
    pdl_begin();
    int ex, ey, e;
    if (!elem_of_thread(m, ex, ey, e)) return;
    facet_el_at<P, Ph>(m, pr, u, ue, dte_a, ubl, qcap, fl_in, cf, ube_out, fht, cnt, ex, ey, e);
}

template <int P, class Ph>
__global__ void __launch_bounds__(128, elem_blocks<P, Ph::NC, 4>(EK_UPD))
    k_update_el(MeshDev m, ProbDev pr, const float* __restrict__ u, const float* __restrict__ ud,
                const double* __restrict__ ue, const double* __restrict__ dte_a, const float* __restrict__ ER,
                const float* __restrict__ cf, const float* __restrict__ avg, const double* __restrict__ ube,
                const float* __restrict__ fht, const double* __restrict__ dtp, float* __restrict__ EW,
                double* __restrict__ beta_out, unsigned long long* __restrict__ cnt) {
    pdl_begin();
    int ex, ey, e;
    if (!elem_of_thread(m, ex, ey, e)) return;
    update_el_at<P, Ph>(m, pr, u, ud, ER, cf, avg, ube, fht, dtp, EW, beta_out, cnt, ex, ey, e);
}

// FP32-mixed: the residual in two kernels.  k_res_w (the Galerkin part W^e,
// needs only u) runs on the second stream from the start of the stage,
// beside k_pre and the g_h kernels; k_res_s adds the stabilisation, which
// needs g_h, gamma_e and nu_e.  W^e passes through the increment buffer,
// which is free until k_update_el.  Same device functions as k_res_ev.
template <int P, class Ph>
DEV void res_w_at(const MeshDev& m, const ProbDev& pr, const float* __restrict__ u, float* __restrict__ WV, int ex,
                  int ey, int e) {
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    float U[NC][N2], W[NC][N2];
    load_block<float, P, NC>(u, m, ex, ey, U);
    w_part<float, P, Ph>(m, pr, U, ex, ey, W);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int i = 0; i < N2; ++i) WV[ev_at(m.E, e, i, c, NC)] = W[c][i];
}

template <int P, class Ph>
DEV void res_s_at(const MeshDev& m, const float* __restrict__ u, const float* __restrict__ g,
                  const double* __restrict__ gam, const double* __restrict__ nu, const float* __restrict__ WV,
                  float* __restrict__ ER, int ex, int ey, int e) {
    constexpr int NC = Ph::NC, N2 = Dim<P>::N2;
    float U[NC][N2], W[NC][N2];
    load_block<float, P, NC>(u, m, ex, ey, U);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int i = 0; i < N2; ++i) W[c][i] = WV[ev_at(m.E, e, i, c, NC)];
    stab_part<float, P, Ph>(m, U, g, gam, nu, W, ER, ex, ey, e);
}

template <int P, class Ph>
__global__ void __launch_bounds__(128) k_res_w(MeshDev m, ProbDev pr, const float* __restrict__ u,
                                               float* __restrict__ WV) {
    pdl_begin();
    int ex, ey, e;
    if (!elem_of_thread(m, ex, ey, e)) return;
    res_w_at<P, Ph>(m, pr, u, WV, ex, ey, e);
}

template <int P, class Ph>
__global__ void __launch_bounds__(128) k_res_s(MeshDev m, const float* __restrict__ u, const float* __restrict__ g,
                                               const double* __restrict__ gam, const double* __restrict__ nu,
                                               const float* __restrict__ WV, float* __restrict__ ER) {
    pdl_begin();
    int ex, ey, e;
    if (!elem_of_thread(m, ex, ey, e)) return;
    res_s_at<P, Ph>(m, u, g, gam, nu, WV, ER, ex, ey, e);
}

// ---------------------------------------------------------------------------
// k_final: u_i^SSP = u_i + (sum_{e in E_i} increment_i^e) / |E_i| (m_i^e/m_i
// = 1/|E_i| on a uniform mesh), SSP-RK combination a u^n + b u^SSP, the
// invariant-domain check and clamp (scalar IDP modes, bounds rounded inward
// to the storage precision) or the positivity count (Euler), non-finite count.
// ---------------------------------------------------------------------------
// Float certificate of the positivity check of a stored state (rho, m, E):
// true only when rho > 0 and rho E - |m|^2/2 > 0 hold for these values
// exactly, so p = (gamma - 1)(E - |m|^2 / (2 rho)) > 0 as well (and the
// float64 check agrees).  The float evaluation t = fma(rho, E, -kin), kin =
// 0.5 fma(mx, mx, my^2), differs from the exact value by at most about
// 3.1 2^-24 A, A = |rho E| + kin, so t > 2^-21 A certifies it; A is kept in
// [2^-100, 2^100] (no underflow or overflow in the products).  Otherwise
// (near-vacuum or near-zero pressure states, NaN) the float64 check decides.
// Float64 states never take this path.
template <class R>
DEV bool euler_positive_certified(const R* u) {
    if constexpr (sizeof(R) == 4) {
        const float rho = u[0], mx = u[1], my = u[2], E = u[3];
        if (!(rho > 0.f)) return false;
        const float kin = __fmul_rn(0.5f, __fmaf_rn(mx, mx, __fmul_rn(my, my)));
        const float t = __fmaf_rn(rho, E, -kin);
        const float A = __fadd_rn(fabsf(__fmul_rn(rho, E)), kin);
        return t > 0x1p-21f * A && A > 0x1p-100f && A < 0x1p100f;
    } else {
        return false;
    }
}

template <class R, int P, int NC>
DEV void final_at(const MeshDev& m, const ProbDev& pr, const R* __restrict__ EW,
                        R* __restrict__ un, R* __restrict__ u, R a, R b,
                        unsigned long long* __restrict__ cnt, int gx, int gy, long long node) {
    const NodeC<P> nc = node_c<P>(m, gx, gy);
    R s[NC];
    gather_at<R, P, NC>(m, EW, nc, s);
    const R inv_cnt = inv_count<R>(nc.nxc * nc.nyc);
    R out[NC];
    bool bad = false;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const R uold = u[c * m.NN + node];
        R ufe = uold + s[c] * inv_cnt;
        if (a != R(0)) {
            out[c] = a * un[c * m.NN + node] + b * ufe;
        } else {
            out[c] = b * ufe;
            un[c * m.NN + node] = uold;  // first stage: keep u^n for the later stages
        }
        bad |= !isfinite(out[c]);
    }
    if (bad) atomicAdd(&cnt[CNT_NONFINITE], 1ull);
    if (NC == 1) {
        if (pr.mode == MODE_LO || pr.mode == MODE_WENO_L) {
            const R lo = PV<R>::lo(pr), hi = PV<R>::hi(pr);
            const R v = out[0];
            if (v < PV<R>::lo_tol(pr) || v > PV<R>::hi_tol(pr))
                atomicAdd(&cnt[CNT_VIOL], 1ull);
            if (v < lo || v > hi) {
                atomicAdd(&cnt[CNT_CLAMP], 1ull);
                out[0] = fmin(fmax(v, lo), hi);
            }
        }
    } else {
        if (!euler_positive_certified(out)) {
            double dd[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) dd[c] = (double)out[c];
            double pres = PhysEuler::pressure<double>(dd, pr.gam);
            if (!(dd[0] > 0.0) || !(pres > 0.0)) atomicAdd(&cnt[CNT_VIOL], 1ull);
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) u[c * m.NN + node] = out[c];
}

template <class R, int P, int NC>
__global__ void k_final(MeshDev m, ProbDev pr, const R* __restrict__ EW,
                        R* __restrict__ un, R* __restrict__ u, R a, R b,
                        unsigned long long* __restrict__ cnt, double* __restrict__ t_adv,
                        const double* __restrict__ dtp) {
    pdl_begin();
    // last stage of a step: one thread advances the time (nothing in this
    // kernel reads it)
    if (t_adv && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) *t_adv += *dtp;
    int gx, gy;
    long long node;
    if (!node_of_thread(m, gx, gy, node)) return;
    final_at<R, P, NC>(m, pr, EW, un, u, a, b, cnt, gx, gy, node);
}


}  // namespace cgl

// common.cuh — device-side data structures, constant-memory tables and
// physics policies of the element-based convex-limited CG-WENO stage
// (Kuzmin, Hajduk, Vedral, arXiv 2509.04673).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <cstring>
#include <cmath>

#define DEV __device__ __forceinline__
#define HDEV __host__ __device__ __forceinline__

namespace cgl {

constexpr int PMAX = 4;        // highest supported degree
constexpr int N1MAX = PMAX + 1;
constexpr int NQMAX = PMAX + 2;

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_FIXED = 2, BC_WALL = 3 };
enum { MODE_LO = 0, MODE_HO = 1, MODE_WENO = 2, MODE_WENO_L = 3 };
enum { FL_NONE = 0, FL_LIMITED = 1, FL_LOW = 2 };

// Mesh as seen by the kernels (Table 1 of the paper on a uniform grid).
struct MeshDev {
    int nx, ny, p;
    int nnx, nny;          // nodes per direction
    int px, py;            // periodic flags
    int bc_x, bc_y;
    int E;                 // nx*ny
    long long NN;          // nnx*nny
    double h;              // element side (square elements)
    // host-precomputed constants (GB300's float64 divide is slow, so no
    // kernel divides by mesh constants): m_i^e = h^2/(p+1)^2, 1/m_i^e,
    // h/(p+1)^2, 1/h, 1/(p+1)^2, 1/(p+1)
    double me, inv_me, h_over_n2, inv_h, inv_n2, inv_n1;
    float h_f, me_f, inv_me_f, h2_f, h_over_n2_f;
    float me_rz_f;         // m_i^e rounded toward zero (admissible bound gaps)
    float inv_h_f;
    double x0, y0, hn;     // domain corner; node spacing h/p (node gx sits at x0 + gx*hn)
    // element basis: 0 Bernstein (the paper's), 1 Lagrange at the LGL points
    // (float64 form only: m_i^e = h^2 w_a w_b, node a at x_e + xn_a h)
    int basis;
    double inv_h2;         // 1/h^2
};

// Boundary data of one side of the domain (W, E, S, N), Sec. 2: weakly
// imposed data u_hat in F(u_h, u_hat; n).  A boundary point whose coordinate
// along the side (y on W and E, x on S and N) lies below s0 + s1 t at the
// stage time t takes slot 0, any other point slot 1.  Kinds: OUTFLOW
// (u_hat = u), FIXED (u_hat = st), WALL (u_hat = u with the normal momentum
// reversed).
struct SideDev {
    int kind[2];
    double s0, s1;
    double st[2][4];
    float st_f[2][4], st_lo_f[2][4];  // float-float copies of st
};

struct ProbDev {
    int flux, mode, fl, k_g, k_u;
    double vx, vy, gam, umin, umax, umin32, umax32, pos_eps;
    double q, r, weno_eps, w_lin, gamma_eps, cfl, lambda_floor;
    double ubc[4];
    double viol_tol;       // rounding tolerance of the bound check
    double lo_tol, hi_tol; // umin - viol_tol, umax + viol_tol
    // float copies for float kernels (a float64 -> float conversion runs on
    // GB300's narrow float64 pipe, so per-thread code never converts)
    float vx_f, vy_f, gam_f, w_lin_f, weno_eps_f, gamma_eps_f, q_f;
    float ubc_f[4], ubc_lo_f[4];
    float lo32_f, hi32_f, lo_tol_f, hi_tol_f;
    int opts;              // CGL_OPT_* bits
    float ome_f;           // 1 - pos_eps rounded to float
    float lambda_floor_f;
    SideDev side[4];       // W, E, S, N
    int plain_mask;        // bit d: side d is OUTFLOW everywhere
    int split_mask;        // bit d: side d has two parts (its split lies inside or moves)
    const double* t_dev;   // device time t of the step and its dt: the stage
    const double* dt_dev;  // time is t + tc dt (read only by moving splits)
    double tc;
    int last_stage;        // the stage ends a step: its k_final advances t
};

enum { OPT_FP64_LIMITER = 1, OPT_UNFUSED_SWEEPS = 2, OPT_SUBCELL_DT = 4, OPT_AEC_Q1 = 8, OPT_DTE_REDUCE = 16 };

// typed views of the problem and mesh constants: float kernels read the
// float copies, float64 kernels the originals
template <class T> struct PV;
template <> struct PV<double> {
    static DEV double vx(const ProbDev& p) { return p.vx; }
    static DEV double vy(const ProbDev& p) { return p.vy; }
    static DEV double gam(const ProbDev& p) { return p.gam; }
    static DEV double w_lin(const ProbDev& p) { return p.w_lin; }
    static DEV double weno_eps(const ProbDev& p) { return p.weno_eps; }
    static DEV double gamma_eps(const ProbDev& p) { return p.gamma_eps; }
    static DEV double q(const ProbDev& p) { return p.q; }
    static DEV double ubc(const ProbDev& p, int c) { return p.ubc[c]; }
    static DEV double side_state(const SideDev& s, int slot, int c) { return s.st[slot][c]; }
    static DEV double lo(const ProbDev& p) { return p.umin; }
    static DEV double hi(const ProbDev& p) { return p.umax; }
    static DEV double lo_tol(const ProbDev& p) { return p.lo_tol; }
    static DEV double hi_tol(const ProbDev& p) { return p.hi_tol; }
    static DEV double h(const MeshDev& m) { return m.h; }
    static DEV double h2(const MeshDev& m) { return m.h * m.h; }
    static DEV double me(const MeshDev& m) { return m.me; }
    static DEV double inv_me(const MeshDev& m) { return m.inv_me; }
};
template <> struct PV<float> {
    static DEV float vx(const ProbDev& p) { return p.vx_f; }
    static DEV float vy(const ProbDev& p) { return p.vy_f; }
    static DEV float gam(const ProbDev& p) { return p.gam_f; }
    static DEV float w_lin(const ProbDev& p) { return p.w_lin_f; }
    static DEV float weno_eps(const ProbDev& p) { return p.weno_eps_f; }
    static DEV float gamma_eps(const ProbDev& p) { return p.gamma_eps_f; }
    static DEV float q(const ProbDev& p) { return p.q_f; }
    static DEV float ubc(const ProbDev& p, int c) { return p.ubc_f[c]; }
    static DEV float side_state(const SideDev& s, int slot, int c) { return s.st_f[slot][c]; }
    static DEV float lo(const ProbDev& p) { return p.lo32_f; }
    static DEV float hi(const ProbDev& p) { return p.hi32_f; }
    static DEV float lo_tol(const ProbDev& p) { return p.lo_tol_f; }
    static DEV float hi_tol(const ProbDev& p) { return p.hi_tol_f; }
    static DEV float h(const MeshDev& m) { return m.h_f; }
    static DEV float h2(const MeshDev& m) { return m.h2_f; }
    static DEV float me(const MeshDev& m) { return m.me_f; }
    static DEV float inv_me(const MeshDev& m) { return m.inv_me_f; }
};

// 1D tables of degree p (index p), filled by the host from its own
// closed-form computation.
template <class T>
struct Tab {
    T M[N1MAX][N1MAX];     // int B_a B_b
    T C[N1MAX][N1MAX];     // int B_a' B_b
    T D[N1MAX][N1MAX];     // int B_a' B_b'
    T Ep[N1MAX][N1MAX];    // [b][a]: coefficients of B_a(x-1) on [0,1]
    T Em[N1MAX][N1MAX];    // [b][a]: coefficients of B_a(x+1) on [0,1]
    T Bq[NQMAX][N1MAX];    // B_a(x_q)
    T dBq[NQMAX][N1MAX];   // B_a'(x_q)
    T wq[NQMAX];           // Gauss weights on [0,1]
    T xq[NQMAX];           // Gauss points on [0,1]
    T wl[N1MAX];           // int_0^1 phi_a: 1/(p+1) (Bernstein), the LGL weights
    T iwl[N1MAX];          // 1 / wl[a]
    T xn[N1MAX];           // node positions on [0,1]: a/p, the LGL points
};

// semi-norm matrices (n2 x n2 for p = 1..4) packed at offsets
constexpr int A2_OFF[PMAX + 1] = {0, 0, 16, 97, 353};
constexpr int A2_TOTAL = 978;

// one copy per translation unit (no relocatable device code); every unit
// uploads the same host tables through its own upload function.  The
// float64 tables hold both bases: Bernstein at index p, the Lagrange basis
// at the LGL points at PMAX + 1 + p (semi-norm matrices at A2_TOTAL + ...);
// the float tables hold Bernstein only (the FP32-mixed form refuses LGL)
constexpr int NTABD = 2 * (PMAX + 1);
static __constant__ Tab<double> c_tabd[NTABD];
static __constant__ Tab<float> c_tabf[PMAX + 1];
static __constant__ double c_A2d[2 * A2_TOTAL];
static __constant__ float c_A2f[A2_TOTAL];

template <class T> struct TabSel;
template <> struct TabSel<double> {
    static DEV const Tab<double>& t(int p) { return c_tabd[p]; }
    static DEV double A2(int off) { return c_A2d[off]; }
};
template <> struct TabSel<float> {
    static DEV const Tab<float>& t(int p) { return c_tabf[p]; }
    static DEV float A2(int off) { return c_A2f[off]; }
};

// the mesh's basis in the float64 form (always Bernstein in float)
template <class R>
DEV bool is_lgl(const MeshDev& m) {
    return sizeof(R) == 8 && m.basis != 0;
}
// tables of degree p on the mesh's basis
template <class R>
DEV const Tab<R>& tab_of(const MeshDev& m, int p) {
    if constexpr (sizeof(R) == 8) return c_tabd[m.basis ? PMAX + 1 + p : p];
    else return c_tabf[p];
}
// offset of the mesh's basis in the packed semi-norm matrices
template <class R>
DEV int a2_base(const MeshDev& m) {
    return is_lgl<R>(m) ? A2_TOTAL : 0;
}

// ---------------------------------------------------------------------------
// physics policies. Each provides, for value type T:
//   NC, flux(u, fx, fy), max_speed(uL, uR, nx, ny), node_speed(u)
// Speeds: Sec. 2.2 defers them to the literature; the readings are
// advection |v.n|; Burgers max(|uL|,|uR|)|nx+ny|; KPP 1 (|f'(u).n| <= 1);
// Euler the two-rarefaction upper bound of Guermond & Popov (2016).
// ---------------------------------------------------------------------------

struct PhysAdv {
    static constexpr int NC = 1;
    static constexpr int NPART_OR_1 = 1;
    template <class T> static DEV void flux(const T* u, T* fx, T* fy, const ProbDev& pr) {
        fx[0] = PV<T>::vx(pr) * u[0];
        fy[0] = PV<T>::vy(pr) * u[0];
    }
    template <class T> static DEV T max_speed(const T*, const T*, T nx, T ny, const ProbDev& pr) {
        return fabs(PV<T>::vx(pr) * nx + PV<T>::vy(pr) * ny);
    }
    template <class T> static DEV T node_speed(const T*, const ProbDev& pr) {
        return hypot(PV<T>::vx(pr), PV<T>::vy(pr));
    }
};

struct PhysBurgers {
    static constexpr int NC = 1;
    static constexpr int NPART_OR_1 = 1;
    template <class T> static DEV void flux(const T* u, T* fx, T* fy, const ProbDev&) {
        T f = T(0.5) * u[0] * u[0];
        fx[0] = f;
        fy[0] = f;
    }
    template <class T> static DEV T max_speed(const T* uL, const T* uR, T nx, T ny, const ProbDev&) {
        return fmax(fabs(uL[0]), fabs(uR[0])) * fabs(nx + ny);
    }
    template <class T> static DEV T node_speed(const T* u, const ProbDev&) {
        return sqrt(T(2)) * fabs(u[0]);
    }
};

// sin and cos of a float for the float KPP flux, compact enough to inline at
// every quadrature point: Cody-Waite reduction x = q pi/2 + r with pi/2 split
// into three floats (the products q P1, q P2 are exact for |q| < 2^12), then
// polynomials in r^2 on [-pi/4, pi/4] whose coefficients were fitted by
// iteratively reweighted least squares against float64 sin and cos (maximum
// error 2.4e-12 and 5.4e-11 before float rounding; evaluated in float the
// result is within 7e-8 of sin and cos).  |x| >= 4096 uses sinf / cosf.
HDEV float fma_hd(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

#ifdef __CUDA_ARCH__
static __device__ __noinline__ void sincos_wide(float x, float* s, float* c) { sincosf(x, s, c); }
#else
inline void sincos_wide(float x, float* s, float* c) {
    *s = (float)std::sin((double)x);
    *c = (float)std::cos((double)x);
}
#endif

HDEV void kpp_sincos(float x, float& s, float& c) {
    if (!(fabsf(x) < 4096.f)) {
        sincos_wide(x, &s, &c);
        return;
    }
    const float P1 = 0x1.92p+0f, P2 = 0x1.fb4p-12f, P3 = 0x1.4442d2p-24f, TWO_OVER_PI = 0x1.45f306p-1f;
#ifdef __CUDA_ARCH__
    const float q = rintf(x * TWO_OVER_PI);
#else
    const float q = std::nearbyint(x * TWO_OVER_PI);
#endif
    float r = fma_hd(-q, P1, x);
    r = fma_hd(-q, P2, r);
    r = fma_hd(-q, P3, r);
    const float z = r * r;
    float ps = fma_hd(0x1.6c89dcp-19f, z, -0x1.a00e1p-13f);
    ps = fma_hd(ps, z, 0x1.111106p-7f);
    ps = fma_hd(ps, z, -0x1.555556p-3f);
    const float sr = fma_hd(r * z, ps, r);
    float pc = fma_hd(0x1.9934bp-16f, z, -0x1.6c088p-10f);
    pc = fma_hd(pc, z, 0x1.55553ep-5f);
    pc = fma_hd(pc, z, -0.5f);
    const float cr = fma_hd(z, pc, 1.0f);
    const int n = (int)q & 3;
    s = (n == 0) ? sr : (n == 1) ? cr : (n == 2) ? -sr : -cr;
    c = (n == 0) ? cr : (n == 1) ? -sr : (n == 2) ? -cr : sr;
}

struct PhysKPP {
    static constexpr int NC = 1;
    static constexpr int NPART_OR_1 = 1;
    template <class T> static DEV void flux(const T* u, T* fx, T* fy, const ProbDev&) {
        if constexpr (sizeof(T) == 4) {
            kpp_sincos(u[0], fx[0], fy[0]);
        } else {
            fx[0] = sin(u[0]);
            fy[0] = cos(u[0]);
        }
    }
    template <class T> static DEV T max_speed(const T*, const T*, T, T, const ProbDev&) { return T(1); }
    template <class T> static DEV T node_speed(const T*, const ProbDev&) { return T(1); }
};

struct PhysEuler {
    static constexpr int NC = 4;
    static constexpr int NPART_OR_1 = 5;  // speed parts per cell (speed_parts)
    template <class T> static DEV T pressure(const T* u, T g) {
        return (g - T(1)) * (u[3] - T(0.5) * (u[1] * u[1] + u[2] * u[2]) / u[0]);
    }
    template <class T> static DEV void flux(const T* u, T* fx, T* fy, const ProbDev& pr) {
        const T g = PV<T>::gam(pr);
        T rho = u[0], mx = u[1], my = u[2], E = u[3];
        T vx, vy, p;
        if constexpr (sizeof(T) == 4) {
            // float: one correctly rounded reciprocal of rho instead of three
            // divisions (the flux is evaluated at every quadrature point and
            // face node of the float kernels)
            const T r = __frcp_rn(rho);
            vx = mx * r;
            vy = my * r;
            p = (g - T(1)) * (E - T(0.5) * (mx * vx + my * vy));
        } else {
            vx = mx / rho;
            vy = my / rho;
            p = (g - T(1)) * (E - T(0.5) * (mx * mx + my * my) / rho);
        }
        fx[0] = mx;
        fx[1] = mx * vx + p;
        fx[2] = my * vx;
        fx[3] = (E + p) * vx;
        fy[0] = my;
        fy[1] = mx * vy;
        fy[2] = my * vy + p;
        fy[3] = (E + p) * vy;
    }
    template <class T> static DEV T max_speed(const T* uL, const T* uR, T nx, T ny, const ProbDev& pr) {
        const T g = PV<T>::gam(pr);
        T rL = uL[0], rR = uR[0];
        T vL = (uL[1] * nx + uL[2] * ny) / rL;
        T vR = (uR[1] * nx + uR[2] * ny) / rR;
        T pL = pressure(uL, g), pR = pressure(uR, g);
        T aL = sqrt(g * pL / rL), aR = sqrt(g * pR / rR);
        T expo = (g - T(1)) / (T(2) * g);
        T num = aL + aR - T(0.5) * (g - T(1)) * (vR - vL);
        T den = aL * pow(pL, -expo) + aR * pow(pR, -expo);
        T base = num > T(0) ? fmax(num, T(0)) / den : T(0);
        T ptr = pow(base, T(1) / expo);
        T cg = (g + T(1)) / (T(2) * g);
        T lam1 = vL - aL * sqrt(T(1) + cg * fmax(T(0), (ptr - pL) / pL));
        T lam3 = vR + aR * sqrt(T(1) + cg * fmax(T(0), (ptr - pR) / pR));
        return fmax(fabs(lam1), fabs(lam3));
    }
    // max_speed split into its per-cell and per-facet parts (float, interior
    // facets with normal +x or +y): the cell part holds v_x, v_y, p, the
    // sound speed a = sqrt(g p / rho) and p^(-(g-1)/(2g)), formed with the
    // operations max_speed applies to each state; the facet part completes
    // the two-rarefaction bound from the parts of the left and right cells
    // along axis 0 (x) or 1 (y)
    static DEV void speed_parts(const float* u, float g, float* q) {
        const float rho = u[0];
        q[0] = (u[1] * 1.f + u[2] * 0.f) / rho;
        q[1] = (u[1] * 0.f + u[2] * 1.f) / rho;
        const float p = pressure(u, g);
        q[2] = p;
        q[3] = sqrt(g * p / rho);
        const float expo = (g - 1.f) / (2.f * g);
        q[4] = pow(p, -expo);
    }
    static DEV float facet_speed_parts(const float* L, const float* R, int axis, float g) {
        const float vL = L[axis], vR = R[axis];
        const float pL = L[2], pR = R[2], aL = L[3], aR = R[3];
        const float expo = (g - 1.f) / (2.f * g);
        const float num = aL + aR - 0.5f * (g - 1.f) * (vR - vL);
        const float den = aL * L[4] + aR * R[4];
        const float base = num > 0.f ? fmaxf(num, 0.f) / den : 0.f;
        const float ptr = pow(base, 1.f / expo);
        const float cg = (g + 1.f) / (2.f * g);
        const float lam1 = vL - aL * sqrt(1.f + cg * fmaxf(0.f, (ptr - pL) / pL));
        const float lam3 = vR + aR * sqrt(1.f + cg * fmaxf(0.f, (ptr - pR) / pR));
        return fmaxf(fabsf(lam1), fabsf(lam3));
    }
    template <class T> static DEV T node_speed(const T* u, const ProbDev& pr) {
        const T g = PV<T>::gam(pr);
        if constexpr (sizeof(T) == 4) {
            // float: one reciprocal of rho (nu_e takes the largest node speed)
            const T r = __frcp_rn(u[0]);
            const T vx = u[1] * r, vy = u[2] * r;
            const T p = (g - T(1)) * (u[3] - T(0.5) * (u[1] * vx + u[2] * vy));
            return sqrt(vx * vx + vy * vy) + sqrt(fmax(T(0), g * p * r));
        } else {
            T c = sqrt(fmax(T(0), g * pressure(u, g) / u[0]));
            return hypot(u[1], u[2]) / u[0] + c;
        }
    }
};

// LLF flux eq. (fluxLLF): F = (f(uL)+f(uR))/2 . n - lambda/2 (uR - uL)
template <class Ph, class T>
DEV void llf(const T* uL, const T* uR, T nx, T ny, const ProbDev& pr, T* F, T* lam_out) {
    T fxL[Ph::NC], fyL[Ph::NC], fxR[Ph::NC], fyR[Ph::NC];
    Ph::flux(uL, fxL, fyL, pr);
    Ph::flux(uR, fxR, fyR, pr);
    T lam = Ph::max_speed(uL, uR, nx, ny, pr);
#pragma unroll
    for (int c = 0; c < Ph::NC; ++c) {
        T nL = fxL[c] * nx + fyL[c] * ny;
        T nR = fxR[c] * nx + fyR[c] * ny;
        F[c] = T(0.5) * (nL + nR) - T(0.5) * lam * (uR[c] - uL[c]);
    }
    if (lam_out) *lam_out = lam;
}

// the same LLF flux with f(uR) given (a constant external state: its flux is
// evaluated once per face; the result is identical to llf)
template <class Ph, class T>
DEV void llf_given_fR(const T* uL, const T* uR, const T* fxR, const T* fyR, T nx, T ny, const ProbDev& pr,
                      T* F) {
    T fxL[Ph::NC], fyL[Ph::NC];
    Ph::flux(uL, fxL, fyL, pr);
    T lam = Ph::max_speed(uL, uR, nx, ny, pr);
#pragma unroll
    for (int c = 0; c < Ph::NC; ++c) {
        T nL = fxL[c] * nx + fyL[c] * ny;
        T nR = fxR[c] * nx + fyR[c] * ny;
        F[c] = T(0.5) * (nL + nR) - T(0.5) * lam * (uR[c] - uL[c]);
    }
}

// Appendix A bound for the correction factor of one state ubar modified by
// alpha f / m, with the positivity margin eps (rho* >= eps rho_bar and the
// pressure constraint scaled by (1 - eps)).
template <class T>
HDEV T euler_alpha(const T* ub, const T* f, T m, T eps) {
    T rho = ub[0], mx = ub[1], my = ub[2], E = ub[3];
    T fr = f[0], fmx = f[1], fmy = f[2], fE = f[3];
    T thr = m * rho * (T(1) - eps);
    T a_rho = (thr + fr < T(0)) ? -thr / fr : T(1);
    T Q = (T(1) - eps) * m * (T(0.5) * (mx * mx + my * my) - rho * E);
    T R = rho * fE + E * fr - (mx * fmx + my * fmy) +
          fmin(T(0), fE * fr - T(0.5) * (fmx * fmx + fmy * fmy)) / m;
    T a_p = (R < Q) ? Q / R : T(1);
    T a = fmin(a_rho, a_p);
    return fmin(fmax(a, T(0)), T(1));
}

// Float32 certificate for euler_alpha: true only when the float64 evaluation
// of euler_alpha<double> on inputs that these floats round (relative error
// <= 2^-24 each: ub, f, m, 1 - eps) certainly returns exactly 1, i.e. both
// constraints of Appendix A hold with alpha = 1:
//   T1 = m rho (1 - eps) + f_rho  >= 0,
//   T2 = R - Q                    >= 0.
// T1 is homogeneous of degree 1 in (ub, f) and in (f, m), T2 of degree 2 in
// (ub, f) and 1 in (f, m), so the inputs are first scaled by exact powers of
// two to rho, m in [1, 2); this changes neither sign.  Each T is then
// evaluated in float together with A, the same expression with every
// monomial in absolute value.  With n operations and k rounded inputs
// (n + k < 40) the float error is below (n + k) 2^-24 A and the float64 one
// below (n + k) 2^-53 A.  Scaled values are required to be at most 2^40, so
// an underflowed input or product (error <= 2^-150) is amplified to at most
// 2^-109 and all of them together stay below 2^-100.  So T > 2^-16 A +
// 2^-100 certifies T > 0 for both evaluations.  NaN, infinite, zero or
// subnormal rho or m fail and are left to the float64 formula.
HDEV int bits_of(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_int(x);
#else
    int i;
    std::memcpy(&i, &x, 4);
    return i;
#endif
}
HDEV float float_of(int i) {
#ifdef __CUDA_ARCH__
    return __int_as_float(i);
#else
    float x;
    std::memcpy(&x, &i, 4);
    return x;
#endif
}
HDEV float pow2f(int k) { return float_of((127 + k) << 23); }  // 2^k, -126 <= k <= 127

HDEV bool euler_alpha_is_one(const float* ub, const float* f, float m, float ome) {
    const int brho = bits_of(ub[0]), bm = bits_of(m);
    const int erho = (brho >> 23) & 0xff, em = (bm >> 23) & 0xff;
    // rho and m positive, normal and finite
    if (brho <= 0 || bm <= 0 || erho == 0 || em == 0 || erho == 0xff || em == 0xff) return false;
    const float sj = pow2f(127 - erho), sk = pow2f(127 - em);  // rho sj, m sk in [1, 2)
    const float rho = ub[0] * sj, mx = ub[1] * sj, my = ub[2] * sj, E = ub[3] * sj;
    const float fr = (f[0] * sj) * sk, fmx = (f[1] * sj) * sk, fmy = (f[2] * sj) * sk, fE = (f[3] * sj) * sk;
    const float ms = m * sk;
    const float big = 0x1p40f;
    if (!(fabsf(mx) <= big && fabsf(my) <= big && fabsf(E) <= big && fabsf(fr) <= big && fabsf(fmx) <= big &&
          fabsf(fmy) <= big && fabsf(fE) <= big))
        return false;
    const float K = 0x1p-16f, A0 = 0x1p-100f;
    // density constraint
    const float thr = ms * rho * ome;
    const float t1 = thr + fr;
    const float a1 = fabsf(thr) + fabsf(fr);
    // pressure constraint: Q = (1 - eps) m (|m|^2/2 - rho E),
    // R = rho fE + E fr - m.fm + min(0, fE fr - |fm|^2/2) / m
    const float kin = 0.5f * (mx * mx + my * my);
    const float rE = rho * E;
    const float Q = ome * ms * (kin - rE);
    const float aQ = ms * (kin + fabsf(rE));
    const float frE = fE * fr, fkin = 0.5f * (fmx * fmx + fmy * fmy);
    const float c = frE - fkin;
    const float p1 = rho * fE, p2 = E * fr, p3 = mx * fmx, p4 = my * fmy;
    const float Rv = ((p1 + p2) - (p3 + p4)) + fminf(0.f, c) / ms;
    const float aR = ((fabsf(p1) + fabsf(p2)) + (fabsf(p3) + fabsf(p4))) + (fabsf(frE) + fkin) / ms;
    const float t2 = Rv - Q;
    const float a2 = aR + aQ;
    return (t1 > K * a1 + A0) && (t2 > K * a2 + A0);
}

}  // namespace cgl

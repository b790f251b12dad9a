// common.cuh — device-side data structures, constant-memory tables and
// physics policies of the element-based convex-limited CG-WENO stage
// (Kuzmin, Hajduk, Vedral, arXiv 2509.04673).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define DEV __device__ __forceinline__

namespace cgl {

constexpr int PMAX = 4;        // highest supported degree
constexpr int N1MAX = PMAX + 1;
constexpr int NQMAX = PMAX + 2;

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_FIXED = 2 };
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
};

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
};

// semi-norm matrices (n2 x n2 for p = 1..4) packed at offsets
constexpr int A2_OFF[PMAX + 1] = {0, 0, 16, 97, 353};
constexpr int A2_TOTAL = 978;

// one copy per translation unit (no relocatable device code); every unit
// uploads the same host tables through its own upload function
static __constant__ Tab<double> c_tabd[PMAX + 1];
static __constant__ Tab<float> c_tabf[PMAX + 1];
static __constant__ double c_A2d[A2_TOTAL];
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

// ---------------------------------------------------------------------------
// physics policies. Each provides, for value type T:
//   NC, flux(u, fx, fy), max_speed(uL, uR, nx, ny), node_speed(u)
// Speeds: Sec. 2.2 defers them to the literature; the readings are
// advection |v.n|; Burgers max(|uL|,|uR|)|nx+ny|; KPP 1 (|f'(u).n| <= 1);
// Euler the two-rarefaction upper bound of Guermond & Popov (2016).
// ---------------------------------------------------------------------------

struct PhysAdv {
    static constexpr int NC = 1;
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

struct PhysKPP {
    static constexpr int NC = 1;
    template <class T> static DEV void flux(const T* u, T* fx, T* fy, const ProbDev&) {
        fx[0] = sin(u[0]);
        fy[0] = cos(u[0]);
    }
    template <class T> static DEV T max_speed(const T*, const T*, T, T, const ProbDev&) { return T(1); }
    template <class T> static DEV T node_speed(const T*, const ProbDev&) { return T(1); }
};

struct PhysEuler {
    static constexpr int NC = 4;
    template <class T> static DEV T pressure(const T* u, T g) {
        return (g - T(1)) * (u[3] - T(0.5) * (u[1] * u[1] + u[2] * u[2]) / u[0]);
    }
    template <class T> static DEV void flux(const T* u, T* fx, T* fy, const ProbDev& pr) {
        const T g = PV<T>::gam(pr);
        T rho = u[0], mx = u[1], my = u[2], E = u[3];
        T vx = mx / rho, vy = my / rho;
        T p = (g - T(1)) * (E - T(0.5) * (mx * mx + my * my) / rho);
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
    template <class T> static DEV T node_speed(const T* u, const ProbDev& pr) {
        const T g = PV<T>::gam(pr);
        T c = sqrt(fmax(T(0), g * pressure(u, g) / u[0]));
        return hypot(u[1], u[2]) / u[0] + c;
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

// Appendix A bound for the correction factor of one state ubar modified by
// alpha f / m, with the positivity margin eps (rho* >= eps rho_bar and the
// pressure constraint scaled by (1 - eps)).
template <class T>
DEV T euler_alpha(const T* ub, const T* f, T m, T eps) {
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

}  // namespace cgl

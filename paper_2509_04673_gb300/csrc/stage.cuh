// stage.cuh — host-side launch sequence of one SSP-RK stage (Sec. 4.3 of
// the paper: element loop, udot solve, facet loop, element loop, SSP update).
#pragma once

#include "fused.cuh"

namespace cgl {

// Device buffers of one state. R-typed arrays are void* here.
struct Bufs {
    void* u;      // state            [NC][NN]  (R)
    void* un;     // RK base u^n      [NC][NN]  (R)
    void* g;      // g_h              [2NC][NN] (R)
    void* g2;     // g_h ping-pong    [2NC][NN] (R)
    void* ud2;    // udot ping-pong   [NC][NN]  (R)
    void* bg;     // rhs of g_h       [2NC][NN] (R)
    void* r;      // target residual  [NC][NN]  (R)
    void* ud;     // udot             [NC][NN]  (R)
    void* EV;     // unused (16 bytes)
    void* ER;     // element residual [N2][NC][E]  (R)
    void* EW;     // SSP increments   [N2][NC][E]  (R)
    void* q;      // flux-limiter capacities [2][E] (scalar)  (R)
    void* fl;     // low-order facet fluxes [E][4][NC]         (R)
    float* cf;    // float copies for the Euler limiter certificate [1+NC][E]: s, ubar^{e,L}
    float* avg;   // float-float cell means [2NC][E] (FP32-mixed: k_avg for systems, k_pre for scalars)
    float* cq;    // FP32-mixed systems: flux of the mean and speed parts per cell [2NC + 5][E] (k_avg)
    float* fht;   // facet terms of f_i^e [NC][E] (FP32-mixed, k_facet -> k_update_el)
    cudaStream_t st2;            // second stream of a stage (k_facet)
    cudaEvent_t ev_fork0, ev_fork, ev_w, ev_join;
    double *ue, *dte, *ubl, *gam, *nu, *ube, *beta;
    unsigned long long* cnt;     // CNT_N counters
    unsigned long long* dtbits;  // min dt_e as bits
    double *dt, *t, *t_end;
};

// kernel identifiers for per-kernel timing
enum KernelId {
    KID_AVG = 0, KID_PRE, KID_DT, KID_GRAD, KID_GATHER, KID_GRADF, KID_SWEEP, KID_RES,
    KID_UPDATE, KID_FINAL, KID_TADV, KID_UDOTF, KID_FACET, KID_RESW, KID_Q1F, KID_UDL, KID_SENS, KID_COUNT
};

// optional per-launch timing: CUDA events recorded around every launch on
// the launching stream (never used inside graph capture)
struct Prof {
    struct Rec { int id; cudaEvent_t a, b; };
    Rec* recs;
    int n, cap;
    void begin(int id, cudaStream_t st) {
        if (n < cap) {
            recs[n].id = id;
            cudaEventRecord(recs[n].a, st);
        }
    }
    void end(cudaStream_t st) {
        if (n < cap) cudaEventRecord(recs[n++].b, st);
    }
};

#define CGL_LAUNCH(PROF, ID, ST, ...)             \
    do {                                          \
        if (PROF) (PROF)->begin((ID), (ST));      \
        __VA_ARGS__;                              \
        if (PROF) (PROF)->end((ST));              \
    } while (0)

// first: compute the global dt from this stage's dt_e (stage 1 of a step);
// dt_only: stop after the dt reduction (time-step query)
typedef cudaError_t (*StageFn)(const Bufs&, const MeshDev&, const ProbDev&, double a, double b,
                               bool first, bool dt_only, cudaStream_t st, Prof* prof);

inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// The fused first sweeps (fused.cuh) save the traffic of the lumped iterates
// but lengthen each block's chain of dependent phases.  Measured on GB300,
// they win from about 4M nodes (KPP 1024^2 Q2: -4 % per step, Euler blast
// 2048^2) and lose below (KPP 256^2: +4 %; Euler 512^2 Q3: +1.5 %).
inline bool fuse_sweeps(const MeshDev& m) { return m.NN >= (1LL << 22); }

// The split residual (k_res_w on the second stream, k_res_s) overlaps the
// quadrature with k_pre and the g_h kernels but adds a kernel and the W^e
// traffic: measured, it wins on KPP 1024^2 (-4 % per step) and loses
// slightly at 256^2 (+0.7 %); for systems (four components: a W^e of four
// element vectors) the single k_res_ev is faster (Euler blast 2048^2 Q2:
// 17.0 against 17.8 ms per step).
inline bool split_residual(const MeshDev& m, int nc) { return nc == 1 && m.NN >= (1LL << 20); }

// Launch with programmatic stream serialisation (pdl): the kernel may be
// scheduled while the previous kernel of the stream drains and waits for it
// in pdl_begin(); inside a captured graph this becomes a programmatic edge.
template <typename... KArgs, typename... Args>
inline cudaError_t launch(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

template <class R, int P, class Ph>
cudaError_t run_stage(const Bufs& B, const MeshDev& m, const ProbDev& pr_in, double a, double b,
                      bool first, bool dt_only, cudaStream_t st, Prof* prof) {
    ProbDev pr = pr_in;
    if (dt_only) pr.mode = MODE_HO;  // no sensor needed for dt_e
    constexpr int NC = Ph::NC;
    const dim3 be(64, 2), bn(128, 1);
    const dim3 ge(nblk(m.nx, 64), nblk(m.ny, 2)), gn(nblk(m.nnx, 128), m.nny);
    const dim3 bt(ST_TX, ST_BY), gt(nblk(m.nnx, ST_TX), nblk(m.nny, ST_TY));  // tiled stencils
    // small meshes: 32 x 8 node tiles for the unfused stencils (measured:
    // KPP 256^2 Q2 -4.6 % per step; 8 rows lose 8-10 % from 2M nodes)
    const bool small_tiles = m.NN < (1LL << 20);
    const dim3 gt8(nblk(m.nnx, ST_TX), nblk(m.nny, 8));
    auto* k_grad = small_tiles ? k_grad_rhs<R, P, NC, 8> : k_grad_rhs<R, P, NC, ST_TY>;
    auto* k_sweep_g = small_tiles ? k_mass_sweep<R, P, 2 * NC, 8> : k_mass_sweep<R, P, 2 * NC, ST_TY>;
    auto* k_sweep_u = small_tiles ? k_mass_sweep<R, P, NC, 8> : k_mass_sweep<R, P, NC, ST_TY>;
    const dim3 gts = small_tiles ? gt8 : gt;
    // per-launch timing records events between kernels: plain launches then
    const bool pdl = prof == nullptr;
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && err == cudaSuccess) err = e;
    };
    R* u = (R*)B.u;
    // FP32-mixed: the second stream starts with the Galerkin part of the
    // residual, which needs only u
    constexpr bool split = sizeof(R) == 4;
    // the Q1 variant of eq. (aecQ1) needs neither g_h, nor the residual, nor udot
    const bool q1 = (pr.opts & OPT_AEC_Q1) != 0 && pr.mode != MODE_LO;
    const bool split_res = split && split_residual(m, NC) && !q1;
    // per-launch timing serialises the stage on one stream, so that each
    // kernel's events bracket its own run and no overlap with the other stream
    const cudaStream_t s2 = prof ? st : B.st2;
    if (split_res && !dt_only && pr.mode != MODE_LO) {
        chk(cudaEventRecord(B.ev_fork0, st));
        chk(cudaStreamWaitEvent(s2, B.ev_fork0, 0));
        if constexpr (split)
            CGL_LAUNCH(prof, KID_RESW, s2,
                       chk(launch(false, k_res_w<P, Ph>, ge, be, s2, m, pr, (const float*)u, (float*)B.EW)));
        chk(cudaEventRecord(B.ev_w, s2));
    }
    constexpr bool use_avg = sizeof(R) == 4 && NC > 1;
    if constexpr (use_avg)
        CGL_LAUNCH(prof, KID_AVG, st, chk(launch(pdl, k_avg<P, Ph>, ge, be, st, m, pr, (const float*)u, B.avg, B.cq)));
    if constexpr (use_avg) {
        // mixed systems: the low-order part here, the sensor in k_sens below
        auto* kpre = (pr.opts & OPT_SUBCELL_DT) ? k_pre_lo<P, Ph, true> : k_pre_lo<P, Ph, false>;
        CGL_LAUNCH(prof, KID_PRE, st,
                   chk(launch(pdl, kpre, ge, be, st, m, pr, (const float*)u, B.ue, B.dte, B.ubl, (float*)B.fl, B.cf,
                              B.avg, (const float*)B.cq, first ? B.dtbits : nullptr)));
    } else {
        auto* kpre = (pr.opts & OPT_SUBCELL_DT) ? k_pre<R, P, Ph, true> : k_pre<R, P, Ph, false>;
        CGL_LAUNCH(prof, KID_PRE, st,
                   chk(launch(pdl, kpre, ge, be, st, m, pr, (const R*)u, B.ue, B.dte, B.ubl, B.gam, B.nu,
                              (R*)B.q, (R*)B.fl, (R*)nullptr, B.cf, B.avg,
                              first ? B.dtbits : nullptr)));
    }
    if (first)
        CGL_LAUNCH(prof, KID_DT, st,
                   chk(launch(pdl, k_dt_final, dim3(1), dim3(1), st, B.dtbits, pr.cfl, (const double*)B.t,
                              (const double*)B.t_end, B.dt)));
    if (dt_only) return err != cudaSuccess ? err : cudaGetLastError();
    // FP32-mixed: the facet part of the update (for systems after the sensor)
    // on the second stream, beside the g_h and udot kernels
    constexpr bool split_update = sizeof(R) == 4;
    if constexpr (split_update) {
        if (!q1) {
            chk(cudaEventRecord(B.ev_fork, st));
            chk(cudaStreamWaitEvent(s2, B.ev_fork, 0));
            if constexpr (use_avg) {
                // systems: the sensor first on the second stream, beside the
                // g_h kernels of the main stream (k_sens is arithmetic-bound,
                // the fused g_h sweep shared-memory-bound; measured: quadrants
                // 512^2 Q3 2.368 -> 2.312 ms per step, blast 2048^2 -0.3 %)
                const dim3 bs(K_SENS_TX, NC), gs(nblk(m.nx, K_SENS_TX), m.ny);
                CGL_LAUNCH(prof, KID_SENS, s2,
                           chk(launch(false, k_sens<P, Ph>, gs, bs, s2, m, pr, (const float*)u, B.gam, B.nu)));
                chk(cudaEventRecord(B.ev_w, s2));
            }
            CGL_LAUNCH(prof, KID_FACET, s2,
                       chk(launch(false, k_facet<P, Ph>, ge, be, s2, m, pr, (const float*)u, (const double*)B.ue,
                                  B.dte, (const double*)B.ubl, (const float*)B.q, (const float*)B.fl, B.cf, B.ube,
                                  B.fht, B.cnt)));
            chk(cudaEventRecord(B.ev_join, s2));
        }
    }
    if constexpr (use_avg) {
        if (q1) {
            // eq. (aecQ1) scales its contributions by gamma_e: the sensor on the main stream
            const dim3 bs(K_SENS_TX, NC), gs(nblk(m.nx, K_SENS_TX), m.ny);
            CGL_LAUNCH(prof, KID_SENS, st,
                       chk(launch(pdl, k_sens<P, Ph>, gs, bs, st, m, pr, (const float*)u, B.gam, B.nu)));
        }
    }
    if (q1) {
        CGL_LAUNCH(prof, KID_Q1F, st,
                   chk(launch(pdl, k_q1_facet<R, P, Ph>, ge, be, st, m, pr, (const R*)u, (const double*)B.ue,
                              (const double*)B.dte, (const double*)B.ubl, (const R*)B.q, (const R*)B.fl,
                              (const float*)B.cf, (R*)B.ER, B.ube, B.cnt)));
        CGL_LAUNCH(prof, KID_UDL, st,
                   chk(launch(pdl, k_udl<R, P, NC>, gn, bn, st, m, (const R*)u, (const double*)B.ube,
                              (const double*)B.dte, (R*)B.ud)));
        CGL_LAUNCH(prof, KID_UPDATE, st,
                   chk(launch(pdl, k_q1_update<R, P, Ph>, ge, be, st, m, pr, (const R*)u, (const R*)B.ud,
                              (const double*)B.ue, (const double*)B.dte, (const R*)B.ER, (const float*)B.cf,
                              (const float*)B.avg, (const double*)B.ube, (const double*)B.gam,
                              (const double*)B.dt, (R*)B.EW, B.beta, B.cnt)));
        CGL_LAUNCH(prof, KID_FINAL, st,
                   chk(launch(pdl, k_final<R, P, NC>, gn, bn, st, m, pr, (const R*)B.EW, (R*)B.un, u, R(a), R(b),
                              B.cnt, pr.last_stage ? B.t : (double*)nullptr, (const double*)B.dt)));
        return err != cudaSuccess ? err : cudaGetLastError();
    }
    R* ud = (R*)B.ud;
    if (pr.mode != MODE_LO) {
        // g_h: stencil right-hand side and lumped iterate, then k_g sweeps (ping-pong)
        R* g = (R*)B.g;
        R* g2 = (R*)B.g2;
        R* bg = (R*)B.bg;
        // FP32-mixed on large meshes: the right-hand side and the first sweep
        // in one kernel
        constexpr bool fuse = sizeof(R) == 4;
        const bool fuse_here = fuse && fuse_sweeps(m) && !(pr.opts & OPT_UNFUSED_SWEEPS);
        int k0 = 0;
        if (fuse_here && pr.k_g >= 1) {
            if constexpr (fuse)
                CGL_LAUNCH(prof, KID_GRADF, st,
                           chk(launch(pdl, k_grad_sweep<P, NC>, gt, bt, st, m, (const float*)u,
                                      pr.k_g > 1 ? (float*)bg : (float*)nullptr, (float*)g2)));
            R* t = g;
            g = g2;
            g2 = t;
            k0 = 1;
        } else {
            CGL_LAUNCH(prof, KID_GRAD, st,
                       chk(launch(pdl, k_grad, gts, bt, st, m, (const R*)u, bg, g)));
        }
        for (int k = k0; k < pr.k_g; ++k) {
            CGL_LAUNCH(prof, KID_SWEEP, st,
                       chk(launch(pdl, k_sweep_g, gts, bt, st, m, (const R*)g, (const R*)bg, g2)));
            R* t = g;
            g = g2;
            g2 = t;
        }
        R* ER = (R*)B.ER;
        R* r = (R*)B.r;
        R* ud2 = (R*)B.ud2;
        if (split_res) {
            chk(cudaStreamWaitEvent(st, B.ev_w, 0));
            CGL_LAUNCH(prof, KID_RES, st,
                       chk(launch(pdl, k_res_s<P, Ph>, ge, be, st, m, (const float*)u, (const float*)g,
                                  (const double*)B.gam, (const double*)B.nu, (const float*)B.EW, (float*)ER)));
        } else {
            if constexpr (use_avg) chk(cudaStreamWaitEvent(st, B.ev_w, 0));  // gamma_e, nu_e of k_sens
            CGL_LAUNCH(prof, KID_RES, st,
                       chk(launch(pdl, k_res_ev<R, P, Ph>, ge, be, st, m, pr, (const R*)u, (const R*)g,
                                  (const double*)B.gam, (const double*)B.nu, ER)));
        }
        int k1 = 0;
        if (fuse_here && pr.k_u >= 1) {
            if constexpr (fuse)
                CGL_LAUNCH(prof, KID_UDOTF, st,
                           chk(launch(pdl, k_udot_sweep<P, NC>, gt, bt, st, m, (const float*)ER, (float*)r,
                                      (float*)ud2)));
            R* t = ud;
            ud = ud2;
            ud2 = t;
            k1 = 1;
        } else {
            CGL_LAUNCH(prof, KID_GATHER, st,
                       chk(launch(pdl, k_gather_init<R, P, NC>, gn, bn, st, m, (const R*)ER, r, ud)));
        }
        for (int k = k1; k < pr.k_u; ++k) {
            CGL_LAUNCH(prof, KID_SWEEP, st,
                       chk(launch(pdl, k_sweep_u, gts, bt, st, m, (const R*)ud, (const R*)r, ud2)));
            R* t = ud;
            ud = ud2;
            ud2 = t;
        }
    }
    if constexpr (split_update) {
        chk(cudaStreamWaitEvent(st, B.ev_join, 0));
        CGL_LAUNCH(prof, KID_UPDATE, st,
                   chk(launch(pdl, k_update_el<P, Ph>, ge, be, st, m, pr, (const float*)u, (const float*)ud,
                              (const double*)B.ue, (const double*)B.dte, (const float*)B.ER, (const float*)B.cf,
                              (const float*)B.avg, (const double*)B.ube, (const float*)B.fht,
                              (const double*)B.dt, (float*)B.EW, B.beta, B.cnt)));
    } else
    CGL_LAUNCH(prof, KID_UPDATE, st,
               chk(launch(pdl, k_update_ev<R, P, Ph>, ge, be, st, m, pr, (const R*)u, (const R*)ud,
                          (const double*)B.ue, B.dte, (const double*)B.ubl, (const R*)B.q,
                          (const R*)B.fl, (const R*)B.ER, (const float*)B.cf, (const float*)B.avg,
                          (const double*)B.dt, (R*)B.EW,
                          B.ube, B.beta, B.cnt)));
    CGL_LAUNCH(prof, KID_FINAL, st,
               chk(launch(pdl, k_final<R, P, NC>, gn, bn, st, m, pr, (const R*)B.EW, (R*)B.un, u, R(a), R(b),
                          B.cnt, pr.last_stage ? B.t : (double*)nullptr, (const double*)B.dt)));
    return err != cudaSuccess ? err : cudaGetLastError();
}

// stage of one precision R (float64: the FP64 form; float: FP32-mixed) for
// degrees 1..4; each physics compiles its two precisions in separate
// translation units (inst_*.cu, inst_*_f32.cu), built in parallel
template <class Ph, class R>
StageFn select_stage_r(int p) {
    switch (p) {
        case 1: return run_stage<R, 1, Ph>;
        case 2: return run_stage<R, 2, Ph>;
        case 3: return run_stage<R, 3, Ph>;
        case 4: return run_stage<R, 4, Ph>;
    }
    return nullptr;
}

// copy the host tables into this translation unit's constant memory
// (td: NTABD float64 tables, a2d: 2 A2_TOTAL values, both bases)
static inline cudaError_t upload_tables_here(const Tab<double>* td, const Tab<float>* tf,
                                             const double* a2d, const float* a2f) {
    cudaError_t e = cudaMemcpyToSymbol(c_tabd, td, sizeof(Tab<double>) * NTABD);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tabf, tf, sizeof(Tab<float>) * (PMAX + 1));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_A2d, a2d, sizeof(double) * 2 * A2_TOTAL);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_A2f, a2f, sizeof(float) * A2_TOTAL);
    return e;
}

typedef cudaError_t (*UploadFn)(const Tab<double>*, const Tab<float>*, const double*, const float*);

StageFn stage_fn_adv(int prec, int p);
StageFn stage_fn_burgers(int prec, int p);
StageFn stage_fn_kpp(int prec, int p);
StageFn stage_fn_euler(int prec, int p);
StageFn stage_fn_adv32(int p);
StageFn stage_fn_burgers32(int p);
StageFn stage_fn_kpp32(int p);
StageFn stage_fn_euler32(int p);
cudaError_t upload_adv(const Tab<double>*, const Tab<float>*, const double*, const float*);
cudaError_t upload_burgers(const Tab<double>*, const Tab<float>*, const double*, const float*);
cudaError_t upload_kpp(const Tab<double>*, const Tab<float>*, const double*, const float*);
cudaError_t upload_euler(const Tab<double>*, const Tab<float>*, const double*, const float*);
cudaError_t upload_adv32(const Tab<double>*, const Tab<float>*, const double*, const float*);
cudaError_t upload_burgers32(const Tab<double>*, const Tab<float>*, const double*, const float*);
cudaError_t upload_kpp32(const Tab<double>*, const Tab<float>*, const double*, const float*);
cudaError_t upload_euler32(const Tab<double>*, const Tab<float>*, const double*, const float*);
cudaError_t upload_batch(const Tab<double>*, const Tab<float>*, const double*, const float*);

}  // namespace cgl

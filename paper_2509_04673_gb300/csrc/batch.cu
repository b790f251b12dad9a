// batch.cu — many independent scalar instances (uneven mesh sizes and
// degrees, own time steps) advanced by persistent cooperative launches: per
// SSP-RK stage one launch for each degree present (a kernel compiled for that
// degree, with its own register budget), all launches of a step captured in
// one CUDA graph.
//
// The work of every phase of the stage (the passes of Sec. 4.3 of the
// paper, see kernels.cuh) is cut into tiles: (instance, run of elements) for
// element phases, (instance, run of nodes) for node phases. The blocks of the
// persistent grid walk the tiles of a phase, then meet at a grid barrier.
// Each element / node is processed by exactly the device functions of the
// single-instance kernels, so a batched instance is bitwise equal to the
// same instance stepped alone. Element-tile lengths per degree are the tuning
// knob (cgl_batch_autotune).
//
// Grid barriers spin with a bounded iteration count; a barrier that gives up
// sets an error flag, every block returns at its next barrier, and the host
// reports CGL_ETIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "state.h"

namespace cgl {

struct InstDev {
    MeshDev m;
    ProbDev pr;
    float *u, *un, *g, *g2, *bg, *r, *ud, *ud2, *ER, *EW;
    double *ue, *dte, *ubl, *gam, *nu, *ube, *beta;
    float *q, *fl, *avg, *cf, *fht;
    unsigned long long *cnt, *dtbits;
    double *dt, *t, *t_end;
    int p, phys;
};

struct Tile {
    int inst, begin, count, pad;  // element tiles: a run of elements; node tiles: begin = gx0, count = gy0
};

struct BatchSync {
    unsigned int count;
    unsigned int gen;
    int err;
    int phantom;  // extra arrivals a barrier waits for (0; > 0 only to test the timeout)
};

enum { PH_PRE = 0, PH_RES, PH_UPDATE };
// the phase form's split element phases: the update as facet + element part,
// the residual as Galerkin part + stabilisation (the single-state kernels'
// device functions, same bits as PH_UPDATE and PH_RES)
enum { PH_FACET = 3, PH_UPDATE_EL, PH_RES_W, PH_RES_S };
enum { PH_GRAD = 0, PH_SWEEP_G, PH_GATHER_R, PH_SWEEP_U, PH_FINAL, PH_GRADF, PH_GATHERF };

constexpr int BT = 128;  // threads per block of the persistent grid
constexpr int BY = BT / ST_TX;  // node tiles of ST_TX x ST_TY nodes: the block as 32 x BY threads

// shared workspace of the tiled stencils, the largest over the degrees
constexpr int cmax(int a, int b) { return a > b ? a : b; }
template <int P>
constexpr int ws_deg() {
    return cmax(cmax(StFields<float, P, 1, 2>::ws, cmax(StFields<float, P, 2, 1>::ws, StFields<float, P, 1, 1>::ws)),
                cmax(GradSweepWs<P, 1>::size, UdotSweepWs<P, 1>::size));
}

// bounded grid barrier: returns false if it gave up (or another block did)
DEV bool grid_sync(BatchSync* s, long long limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int* vgen = &s->gen;
        volatile int* verr = &s->err;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int need = gridDim.x + (unsigned int)s->phantom;
        const unsigned int arrived = atomicAdd(&s->count, 1u) + 1u;
        if (arrived == need) {
            atomicExch(&s->count, 0u);
            __threadfence();
            atomicAdd(&s->gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == g) {
                if (*verr || ++it > limit) {
                    atomicExch(&s->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// g_h and udot after k Richardson sweeps live in the first buffer for even k
DEV const float* g_final(const InstDev& D, int kg) { return (kg & 1) ? D.g2 : D.g; }
DEV const float* ud_final(const InstDev& D, int ku) { return (ku & 1) ? D.ud2 : D.ud; }

// element phase bodies, inlined into the degree's persistent kernel (a call
// would spill the caller's live registers at every element)
template <int P, class Ph>
DEV void elem_phase(int phase, const InstDev& D, int ex, int ey, int e, double& dte, int kg,
                                        int ku) {
    switch (phase) {
        case PH_PRE:
            dte = pre_at<float, P, Ph>(D.m, D.pr, D.u, D.ue, D.dte, D.ubl, D.gam, D.nu, D.q, D.fl, nullptr, D.cf,
                                       D.avg, ex, ey, e);
            break;
        case PH_RES:
            res_at<float, P, Ph>(D.m, D.pr, D.u, g_final(D, kg), D.gam, D.nu, D.ER, ex, ey, e);
            break;
        default:
            update_at<float, P, Ph>(D.m, D.pr, D.u, ud_final(D, ku), D.ue, D.dte, D.ubl, D.q, D.fl, D.ER, D.cf,
                                    D.avg, D.dt, D.EW, D.ube, D.beta, D.cnt, ex, ey, e);
    }
}

// a phase known at compile time: the split phases, else elem_phase
template <int P, int PHASE, class Ph>
DEV void elem_phase_ct(const InstDev& D, const MeshDev& m, int ex, int ey, int e, double& dte, int kg, int ku) {
    if constexpr (PHASE == PH_FACET)
        facet_el_at<P, Ph>(m, D.pr, D.u, D.ue, D.dte, D.ubl, D.q, D.fl, D.cf, D.ube, D.fht, D.cnt, ex, ey, e);
    else if constexpr (PHASE == PH_UPDATE_EL)
        update_el_at<P, Ph>(m, D.pr, D.u, ud_final(D, ku), D.ER, D.cf, D.avg, D.ube, D.fht, D.dt, D.EW, D.beta,
                            D.cnt, ex, ey, e);
    else if constexpr (PHASE == PH_RES_W)
        res_w_at<P, Ph>(m, D.pr, D.u, D.EW, ex, ey, e);  // W^e in the increment buffer until PH_UPDATE_EL
    else if constexpr (PHASE == PH_RES_S)
        res_s_at<P, Ph>(m, D.u, g_final(D, kg), D.gam, D.nu, D.EW, D.ER, ex, ey, e);
    else if constexpr (PHASE == PH_PRE)
        dte = pre_at<float, P, Ph>(m, D.pr, D.u, D.ue, D.dte, D.ubl, D.gam, D.nu, D.q, D.fl, nullptr, D.cf, D.avg, ex,
                                   ey, e);
    else
        elem_phase<P, Ph>(PHASE, D, ex, ey, e, dte, kg, ku);
}

template <int P>
DEV void elem_dispatch(int phase, const InstDev& D, int ex, int ey, int e, double& dte, int kg, int ku) {
    switch (D.phys) {
        case 0: elem_phase<P, PhysAdv>(phase, D, ex, ey, e, dte, kg, ku); break;
        case 1: elem_phase<P, PhysBurgers>(phase, D, ex, ey, e, dte, kg, ku); break;
        default: elem_phase<P, PhysKPP>(phase, D, ex, ey, e, dte, kg, ku); break;
    }
}

// node phases on one ST_TX x ST_TY node tile of an instance: the stencils
// (g_h right-hand side, Richardson sweeps) with the tiled shared-memory
// functions of the single-state kernels, the gathers node by node
// (ST_TY / BY nodes per thread)
// NT threads per block (the block as 32 x NT/32 threads); inlined, so a
// caller with a compile-time phase carries only that phase's code
template <int P, int NT>
DEV void node_phase_body(int phase, const InstDev& D, const MeshDev& m, int gx0, int gy0, float a, float b, int k,
                         float* ws) {
    constexpr int BYN = NT / ST_TX;
    const int tx = threadIdx.x % ST_TX, ty = threadIdx.x / ST_TX;
    switch (phase) {
        case PH_GRADF:
            // right-hand side and first sweep in one pass (k carries k_g: b is
            // kept only when more sweeps follow); a block of k_grad_sweep's
            // shape runs its body (the block's geometry formed once in
            // registers), the same arithmetic as grad_sweep_tile
            if constexpr (NT == ST_TX * ST_BY)
                grad_sweep_block<P, 1>(m, D.u, k > 1 ? D.bg : nullptr, D.g2, gx0, gy0, tx, ty, ws);
            else
                grad_sweep_tile<P, 1, NT>(m, D.u, k > 1 ? D.bg : nullptr, D.g2, gx0, gy0, threadIdx.x, ws);
            break;
        case PH_GATHERF: udot_sweep_tile<P, 1, NT>(m, D.ER, D.r, D.ud2, gx0, gy0, threadIdx.x, ws); break;
        case PH_GRAD: grad_tile<float, P, 1, BYN>(m, D.u, D.bg, D.g, gx0, gy0, tx, ty, ws); break;
        case PH_SWEEP_G:
            if (k & 1) sweep_tile<float, P, 2, BYN>(m, D.g2, D.bg, D.g, gx0, gy0, tx, ty, ws);
            else sweep_tile<float, P, 2, BYN>(m, D.g, D.bg, D.g2, gx0, gy0, tx, ty, ws);
            break;
        case PH_SWEEP_U:
            if (k & 1) sweep_tile<float, P, 1, BYN>(m, D.ud2, D.r, D.ud, gx0, gy0, tx, ty, ws);
            else sweep_tile<float, P, 1, BYN>(m, D.ud, D.r, D.ud2, gx0, gy0, tx, ty, ws);
            break;
        default: {
            const int gx = gx0 + tx, nnx = m.nnx, nny = m.nny;
#pragma unroll
            for (int j = 0; j < ST_TY / BYN; ++j) {
                const int gy = gy0 + ty + j * BYN;
                if (gx >= nnx || gy >= nny) continue;
                const long long node = (long long)gy * nnx + gx;
                if (phase == PH_GATHER_R) gather_init_at<float, P, 1>(m, D.ER, D.r, D.ud, gx, gy, node);
                else final_at<float, P, 1>(m, D.pr, D.EW, D.un, D.u, a, b, D.cnt, gx, gy, node);
            }
        }
    }
}

template <int P>
__device__ __noinline__ void node_phase(int phase, const InstDev& D, int gx0, int gy0, float a, float b, int k,
                                        float* ws) {
    node_phase_body<P, BT>(phase, D, D.m, gx0, gy0, a, b, k, ws);
}

template <int P>
DEV void elem_loop(int phase, const InstDev* __restrict__ I, const Tile* __restrict__ et, int net, bool first,
                   int kg, int ku) {
    for (int t = blockIdx.x; t < net; t += gridDim.x) {
        const Tile T = et[t];
        const InstDev& D = I[T.inst];
        double dte = __longlong_as_double(0x7ff0000000000000LL);
        if ((int)threadIdx.x < T.count) {
            const int e = T.begin + threadIdx.x;
            const int nx = D.m.nx;
            const int ey = e / nx, ex = e - ey * nx;
            elem_dispatch<P>(phase, D, ex, ey, e, dte, kg, ku);
        }
        if (phase == PH_PRE && first) block_min_to(dte, D.dtbits);
    }
}

// every block takes whole node tiles (the tiled stencils synchronise the block)
template <int P>
DEV void node_loop(int phase, const InstDev* __restrict__ I, const Tile* __restrict__ nt, int nnt, float a,
                   float b, int k, float* ws) {
    for (int t = blockIdx.x; t < nnt; t += gridDim.x) {
        const Tile T = nt[t];
        node_phase<P>(phase, I[T.inst], T.begin, T.count, a, b, k, ws);
    }
}

// one SSP stage u <- a u^n + b FE(u) for every instance of degree P.
// A kernel that carries only one degree's code keeps the instruction working
// set small: measured on the 256-instance batch, the four degrees launched
// apart took 7.0 ms per step against 10.3 ms for one kernel over all
// degrees.  7 blocks of 128 threads per SM (a 72-register cap) for every
// degree: the tile loops are latency-bound, and the register budgets the
// element phases would take at p = 3 and 4 (4 and 3 blocks per SM) measured
// slower, 2.34 and 3.94 ms against 2.19 and 3.17 ms per step for those
// degrees' instances.
constexpr int batch_min_blocks(int) { return 7; }

template <int P>
__global__ void __launch_bounds__(BT, batch_min_blocks(P))
    k_batch_stage(const InstDev* __restrict__ I, int ninst, const Tile* __restrict__ et, int net,
                  const Tile* __restrict__ nt, int nnt, BatchSync* sync, float a, float b, int first,
                  int last, int kg, int ku, int mode_lo, long long limit) {
    __shared__ float ws[ws_deg<P>()];
    elem_loop<P>(PH_PRE, I, et, net, first != 0, kg, ku);
    if (!grid_sync(sync, limit)) return;
    if (first) {
        // global dt of each instance from its block minima (eq. (cflglob),
        // scaled by omega_CFL, capped at t_end - t)
        for (int i = blockIdx.x * BT + threadIdx.x; i < ninst; i += gridDim.x * BT) {
            const InstDev& D = I[i];
            double d = D.pr.cfl * __longlong_as_double((long long)*D.dtbits);
            *D.dtbits = 0x7ff0000000000000ull;
            double rem = *D.t_end - *D.t;
            if (rem < d) d = rem > 0.0 ? rem : 0.0;
            *D.dt = d;
        }
        if (mode_lo && !grid_sync(sync, limit)) return;
    }
    if (!mode_lo) {
        // the right-hand sides and the first Richardson sweeps fused (the
        // arithmetic of the separate stencils, same bits): two phases and two
        // grid barriers fewer per stage
        if (kg >= 1) {
            node_loop<P>(PH_GRADF, I, nt, nnt, a, b, kg, ws);
            if (!grid_sync(sync, limit)) return;
        } else {
            node_loop<P>(PH_GRAD, I, nt, nnt, a, b, 0, ws);
            if (!grid_sync(sync, limit)) return;
        }
        for (int k = (kg >= 1 ? 1 : 0); k < kg; ++k) {
            node_loop<P>(PH_SWEEP_G, I, nt, nnt, a, b, k, ws);
            if (!grid_sync(sync, limit)) return;
        }
        elem_loop<P>(PH_RES, I, et, net, false, kg, ku);
        if (!grid_sync(sync, limit)) return;
        if (ku >= 1) {
            node_loop<P>(PH_GATHERF, I, nt, nnt, a, b, 0, ws);
        } else {
            node_loop<P>(PH_GATHER_R, I, nt, nnt, a, b, 0, ws);
        }
        if (!grid_sync(sync, limit)) return;
        for (int k = (ku >= 1 ? 1 : 0); k < ku; ++k) {
            node_loop<P>(PH_SWEEP_U, I, nt, nnt, a, b, k, ws);
            if (!grid_sync(sync, limit)) return;
        }
    }
    elem_loop<P>(PH_UPDATE, I, et, net, false, kg, ku);
    if (!grid_sync(sync, limit)) return;
    node_loop<P>(PH_FINAL, I, nt, nnt, a, b, 0, ws);
    if (last) {
        for (int i = blockIdx.x * BT + threadIdx.x; i < ninst; i += gridDim.x * BT) *I[i].t += *I[i].dt;
    }
}

typedef void (*BatchKernel)(const InstDev*, int, const Tile*, int, const Tile*, int, BatchSync*, float, float, int,
                            int, int, int, int, long long);
static BatchKernel batch_kernel(int p) {
    switch (p) {
        case 1: return k_batch_stage<1>;
        case 2: return k_batch_stage<2>;
        case 3: return k_batch_stage<3>;
        default: return k_batch_stage<4>;
    }
}

// ---------------------------------------------------------------------------
// The phase form: the same phases as separate launches, one block per tile
// of the phase (no grid barrier: the launch boundary orders the phases), so
// that every phase kernel gets the register budget of its own code. The
// launches of each degree run on a stream of their own inside the step's
// graph, so that the degrees overlap.  They are plain stream-ordered
// launches: as programmatic dependent launches, whose early blocks wait on
// an SM for their predecessor while other degrees' blocks could run there,
// the 256-instance batch took 3.93 instead of 3.91 ms per step.
// ---------------------------------------------------------------------------
// the instance's descriptor (mesh, problem, field pointers) copied into
// shared memory once per block: the phase bodies read its fields many times,
// and a shared broadcast is cheaper than a global load each time.  The
// descriptors and tiles are written once, at batch creation, so the copy
// runs before the wait for the previous launch.
DEV void stage_inst(const InstDev* __restrict__ I, int inst, InstDev& sD) {
    static_assert(sizeof(InstDev) % 8 == 0, "descriptor copied in 8-byte words");
    const long long* src = reinterpret_cast<const long long*>(I + inst);
    long long* dst = reinterpret_cast<long long*>(&sD);
    for (int i = threadIdx.x; i < (int)(sizeof(InstDev) / 8); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

template <int P, int PHASE, class Ph>
__global__ void __launch_bounds__(BT) k_bph_elem(const InstDev* __restrict__ I, const Tile* __restrict__ et,
                                                 int first, int kg, int ku) {
    __shared__ InstDev sD;
    const Tile T = et[blockIdx.x];
    stage_inst(I, T.inst, sD);
    pdl_wait_then_trigger();
    const InstDev& D = sD;
    // (the mesh descriptor stays in shared memory here: the out-of-line
    // boundary code takes it by reference, so a register copy would be
    // given a stack frame)
    const MeshDev& m = sD.m;
    double dte = __longlong_as_double(0x7ff0000000000000LL);
    if ((int)threadIdx.x < T.count) {
        const int e = T.begin + threadIdx.x;
        const int nx = m.nx;
        const int ey = e / nx, ex = e - ey * nx;
        elem_phase_ct<P, PHASE, Ph>(D, m, ex, ey, e, dte, kg, ku);
    }
    if (PHASE == PH_PRE && first) block_min_to(dte, D.dtbits);
}

// node tiles with 256 threads per block (2 rows per thread, as the
// single-state stencils), the phase's code alone
constexpr int BTN = 256;
template <int P, int PHASE>
__global__ void __launch_bounds__(BTN) k_bph_node(const InstDev* __restrict__ I, const Tile* __restrict__ nt,
                                                  float a, float b, int k) {
    __shared__ float ws[ws_deg<P>()];
    __shared__ InstDev sD;
    const Tile T = nt[blockIdx.x];
    stage_inst(I, T.inst, sD);
    pdl_wait_then_trigger();
    // the mesh descriptor read from shared memory (a register copy measured
    // 3.70 -> 3.75 ms per step of the 256-instance batch)
    const MeshDev& m = sD.m;
    node_phase_body<P, BTN>(PHASE, sD, m, T.begin, T.count, a, b, k, ws);
}

// global dt of every instance of the group from its block minima (eq.
// (cflglob), scaled by omega_CFL, capped at t_end - t)
__global__ void k_bph_dt(const InstDev* __restrict__ I, int ninst) {
    pdl_wait_then_trigger();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ninst; i += gridDim.x * blockDim.x) {
        const InstDev& D = I[i];
        double d = D.pr.cfl * __longlong_as_double((long long)*D.dtbits);
        *D.dtbits = 0x7ff0000000000000ull;
        double rem = *D.t_end - *D.t;
        if (rem < d) d = rem > 0.0 ? rem : 0.0;
        *D.dt = d;
    }
}

__global__ void k_bph_tadv(const InstDev* __restrict__ I, int ninst) {
    pdl_wait_then_trigger();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ninst; i += gridDim.x * blockDim.x) *I[i].t += *I[i].dt;
}

// element tiles of a degree group ordered by flux: [eoff[f], eoff[f] + ecnt[f])
// are the tiles of the instances with flux f (0 advection, 1 Burgers, 2 KPP),
// each range launched with the kernel of its own flux
struct ElemRanges {
    int eoff[3], ecnt[3];
};

template <int P, int PHASE>
static void bph_elem(const InstDev* I, const Tile* et, const ElemRanges& er, int first, int kg, int ku,
                     cudaStream_t st, cudaError_t& err) {
    const dim3 blk(BT);
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && err == cudaSuccess) err = e;
    };
    if (er.ecnt[0]) chk(launch(false, k_bph_elem<P, PHASE, PhysAdv>, dim3(er.ecnt[0]), blk, st, I, et + er.eoff[0], first, kg, ku));
    if (er.ecnt[1])
        chk(launch(false, k_bph_elem<P, PHASE, PhysBurgers>, dim3(er.ecnt[1]), blk, st, I, et + er.eoff[1], first, kg, ku));
    if (er.ecnt[2]) chk(launch(false, k_bph_elem<P, PHASE, PhysKPP>, dim3(er.ecnt[2]), blk, st, I, et + er.eoff[2], first, kg, ku));
}

template <int P>
static cudaError_t bph_stage(const InstDev* I, int ninst, const Tile* et, const ElemRanges& er, const Tile* nt,
                             int nnt, float a, float b, int first, int last, int kg, int ku, int mode_lo,
                             cudaStream_t st) {
    const dim3 blk(BT), bn(BTN);
    const dim3 gi((ninst + BT - 1) / BT), gn(nnt);
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && err == cudaSuccess) err = e;
    };
    bph_elem<P, PH_PRE>(I, et, er, first, kg, ku, st, err);
    if (first) chk(launch(false, k_bph_dt, gi, blk, st, I, ninst));
    // the element phases split in two kernels each, as in the single-state
    // stage (fewer registers per kernel; measured 4.08 -> 3.94 ms per step of
    // the 256-instance batch): the facet part and the Galerkin part of the
    // residual need only u and the pre phase's outputs
    bph_elem<P, PH_FACET>(I, et, er, 0, kg, ku, st, err);
    if (!mode_lo) {
        bph_elem<P, PH_RES_W>(I, et, er, 0, kg, ku, st, err);
        if (kg >= 1) chk(launch(false, k_bph_node<P, PH_GRADF>, gn, bn, st, I, nt, a, b, kg));
        else chk(launch(false, k_bph_node<P, PH_GRAD>, gn, bn, st, I, nt, a, b, 0));
        for (int k = (kg >= 1 ? 1 : 0); k < kg; ++k)
            chk(launch(false, k_bph_node<P, PH_SWEEP_G>, gn, bn, st, I, nt, a, b, k));
        bph_elem<P, PH_RES_S>(I, et, er, 0, kg, ku, st, err);
        if (ku >= 1) chk(launch(false, k_bph_node<P, PH_GATHERF>, gn, bn, st, I, nt, a, b, 0));
        else chk(launch(false, k_bph_node<P, PH_GATHER_R>, gn, bn, st, I, nt, a, b, 0));
        for (int k = (ku >= 1 ? 1 : 0); k < ku; ++k)
            chk(launch(false, k_bph_node<P, PH_SWEEP_U>, gn, bn, st, I, nt, a, b, k));
    }
    bph_elem<P, PH_UPDATE_EL>(I, et, er, 0, kg, ku, st, err);
    chk(launch(false, k_bph_node<P, PH_FINAL>, gn, bn, st, I, nt, a, b, 0));
    if (last) chk(launch(false, k_bph_tadv, gi, blk, st, I, ninst));
    return err;
}

typedef cudaError_t (*PhaseStage)(const InstDev*, int, const Tile*, const ElemRanges&, const Tile*, int, float, float,
                                  int, int, int, int, int, cudaStream_t);
static PhaseStage phase_stage(int p) {
    switch (p) {
        case 1: return bph_stage<1>;
        case 2: return bph_stage<2>;
        case 3: return bph_stage<3>;
        default: return bph_stage<4>;
    }
}

cudaError_t upload_batch(const Tab<double>* td, const Tab<float>* tf, const double* a2d, const float* a2f) {
    return upload_tables_here(td, tf, a2d, a2f);
}

}  // namespace cgl

using namespace cgl;

// the instances of one degree and the persistent kernel that carries them
struct DegreeGroup {
    int p;
    std::vector<int> members;  // indices into cgl_batch::states
    InstDev* d_inst;
    Tile *d_et, *d_nt;
    int net, nnt;
    ElemRanges er;  // element tiles per flux (ordered by flux)
    BatchSync* d_sync;
    int grid;
    cudaStream_t gst;  // the phase form: this degree's stream
    cudaEvent_t ev;    // the phase form: end of this degree's step
};

struct cgl_batch {
    std::vector<cgl_state*> states;
    cudaStream_t st;
    int ninst;
    std::vector<DegreeGroup> groups;  // one per degree present, ascending
    int tile_elems[PMAX + 1];
    int node_tile;
    int mode_lo, kg, ku;
    long long limit;
    int phantom;
    int form;  // CGL_BATCH_PERSISTENT or CGL_BATCH_PHASES
    cudaEvent_t ev_fork;
    cudaGraphExec_t graph;
    bool use_graph;
    cudaError_t graph_err;  // why the capture failed (cudaSuccess: not failed)
};

static cgl_status bfail(cgl_status st, const char* msg, cudaError_t e = cudaSuccess) {
    if (e != cudaSuccess) return set_error(st, "%s: %s", msg, cudaGetErrorString(e));
    return set_error(st, "%s", msg);
}

static cgl_status build_tiles(cgl_batch* B) {
    for (DegreeGroup& G : B->groups) {
        std::vector<Tile> et, nt;
        const int T = std::max(1, std::min(BT, B->tile_elems[G.p]));
        for (int f = 0; f < 3; ++f) {
            G.er.eoff[f] = (int)et.size();
            for (int k = 0; k < (int)G.members.size(); ++k) {
                const cgl_state* S = B->states[G.members[k]];
                if (S->prob.flux != f) continue;
                const MeshDev& m = S->mesh->m;
                for (int b = 0; b < m.E; b += T) et.push_back(Tile{k, b, std::min(T, m.E - b), 0});
            }
            G.er.ecnt[f] = (int)et.size() - G.er.eoff[f];
        }
        for (int k = 0; k < (int)G.members.size(); ++k) {
            const MeshDev& m = B->states[G.members[k]]->mesh->m;
            for (int gy0 = 0; gy0 < m.nny; gy0 += ST_TY)
                for (int gx0 = 0; gx0 < m.nnx; gx0 += ST_TX) nt.push_back(Tile{k, gx0, gy0, 0});
        }
        if (G.d_et) cudaFree(G.d_et);
        if (G.d_nt) cudaFree(G.d_nt);
        G.d_et = G.d_nt = nullptr;
        cudaError_t e = cudaMalloc(&G.d_et, et.size() * sizeof(Tile));
        if (e == cudaSuccess) e = cudaMalloc(&G.d_nt, nt.size() * sizeof(Tile));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(G.d_et, et.data(), et.size() * sizeof(Tile), cudaMemcpyHostToDevice, B->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(G.d_nt, nt.data(), nt.size() * sizeof(Tile), cudaMemcpyHostToDevice, B->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(B->st);
        if (e != cudaSuccess) return bfail(CGL_ECUDA, "tile upload", e);
        G.net = (int)et.size();
        G.nnt = (int)nt.size();
    }
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    return CGL_OK;
}

static cudaError_t launch_stage(cgl_batch* B, DegreeGroup& G, float a, float b, int first, int last) {
    int ninst = (int)G.members.size();
    void* args[] = {&G.d_inst, &ninst, &G.d_et, &G.net, &G.d_nt, &G.nnt, &G.d_sync, &a, &b,
                    &first, &last, &B->kg, &B->ku, &B->mode_lo, &B->limit};
    return cudaLaunchCooperativeKernel((const void*)batch_kernel(G.p), dim3(G.grid), dim3(BT), args, 0, B->st);
}

// one step: three stages, each a persistent launch per degree present
// (persistent form), or each degree's phase launches on its own stream,
// forked from and joined back to the batch's stream (phase form)
static cudaError_t enqueue_batch_step(cgl_batch* B) {
    const float sa[3] = {0.f, 0.75f, 1.f / 3.f}, sb[3] = {1.f, 0.25f, 2.f / 3.f};
    cudaError_t e = cudaSuccess;
    if (B->form == CGL_BATCH_PHASES) {
        e = cudaEventRecord(B->ev_fork, B->st);
        for (DegreeGroup& G : B->groups) {
            if (e == cudaSuccess) e = cudaStreamWaitEvent(G.gst, B->ev_fork, 0);
            const int ninst = (int)G.members.size();
            for (int k = 0; k < 3 && e == cudaSuccess; ++k)
                e = phase_stage(G.p)(G.d_inst, ninst, G.d_et, G.er, G.d_nt, G.nnt, sa[k], sb[k], k == 0, k == 2,
                                     B->kg, B->ku, B->mode_lo, G.gst);
            if (e == cudaSuccess) e = cudaEventRecord(G.ev, G.gst);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(B->st, G.ev, 0);
        }
        return e;
    }
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        for (DegreeGroup& G : B->groups) {
            e = launch_stage(B, G, sa[k], sb[k], k == 0, k == 2);
            if (e != cudaSuccess) break;
        }
    return e;
}

// Capture the stage launches of a step into a graph once.  If the capture
// fails the batch falls back to direct cooperative launches (same results);
// cgl_batch_info reports graph = -1 then, and the CUDA error is kept in
// graph_err.
static cgl_status ensure_graph(cgl_batch* B) {
    if (B->graph || !B->use_graph) return CGL_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(B->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        B->use_graph = false;
        B->graph_err = e;
        cudaGetLastError();
        return CGL_OK;
    }
    cudaError_t e1 = enqueue_batch_step(B);
    cudaError_t e2 = cudaStreamEndCapture(B->st, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        B->use_graph = false;  // cooperative launches not capturable here: launch directly
        B->graph_err = e1 != cudaSuccess ? e1 : e2;
        return CGL_OK;
    }
    e = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        B->graph = nullptr;
        B->use_graph = false;
        B->graph_err = e;
    }
    return CGL_OK;
}

extern "C" void cgl_batch_destroy(cgl_batch* B) {
    if (!B) return;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    for (DegreeGroup& G : B->groups) {
        if (G.d_inst) cudaFree(G.d_inst);
        if (G.d_et) cudaFree(G.d_et);
        if (G.d_nt) cudaFree(G.d_nt);
        if (G.d_sync) cudaFree(G.d_sync);
        if (G.gst) cudaStreamDestroy(G.gst);
        if (G.ev) cudaEventDestroy(G.ev);
    }
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    delete B;
}

static InstDev inst_of(const cgl_state* s) {
    const Bufs& b = s->B;
    InstDev d;
    d.m = s->mesh->m;
    d.pr = s->pd;
    d.u = (float*)b.u;
    d.un = (float*)b.un;
    d.g = (float*)b.g;
    d.g2 = (float*)b.g2;
    d.ud2 = (float*)b.ud2;
    d.bg = (float*)b.bg;
    d.r = (float*)b.r;
    d.ud = (float*)b.ud;
    d.ER = (float*)b.ER;
    d.EW = (float*)b.EW;
    d.avg = b.avg;
    d.cf = b.cf;
    d.fht = (float*)b.fht;
    d.ue = b.ue;
    d.dte = b.dte;
    d.ubl = b.ubl;
    d.gam = b.gam;
    d.nu = b.nu;
    d.q = (float*)b.q;
    d.fl = (float*)b.fl;
    d.ube = b.ube;
    d.beta = b.beta;
    d.cnt = b.cnt;
    d.dtbits = b.dtbits;
    d.dt = b.dt;
    d.t = b.t;
    d.t_end = b.t_end;
    d.p = s->mesh->m.p;
    d.phys = s->prob.flux;  // 0 advection, 1 Burgers, 2 KPP
    return d;
}

extern "C" cgl_status cgl_batch_create(cgl_state* const* states, int32_t n, cgl_batch** out) {
    if (!states || !out || n < 1) return bfail(CGL_EINVAL, "need at least one state");
    *out = nullptr;
    const cgl_state* s0 = states[0];
    for (int i = 0; i < n; ++i) {
        const cgl_state* s = states[i];
        if (!s || !s->has_problem) return bfail(CGL_EINVAL, "every state needs a problem");
        if (s->prec != CGL_FP32_MIXED) return bfail(CGL_EINVAL, "batched states must be FP32_MIXED");
        if (s->has_bnd) return bfail(CGL_EINVAL, "batched states take the mesh's boundary conditions");
        if (s->pd.opts & OPT_SUBCELL_DT) return bfail(CGL_EINVAL, "batched states take the macrocell dt_e");
        if (s->pd.opts & OPT_AEC_Q1) return bfail(CGL_EINVAL, "batched states take the element contributions of eq. (aec)");
        if (s->pd.opts & OPT_DTE_REDUCE) return bfail(CGL_EINVAL, "batched states keep the macrocell dt_e");
        if (s->nc != 1 || s->prob.flux == CGL_FLUX_EULER) return bfail(CGL_EINVAL, "batched states must be scalar");
        if (s->device != s0->device) return bfail(CGL_EINVAL, "batched states must share a device");
        if (s->prob.mode != s0->prob.mode || s->prob.k_g != s0->prob.k_g || s->prob.k_u != s0->prob.k_u)
            return bfail(CGL_EINVAL, "batched states must share mode, k_g and k_u");
        if ((long long)s->mesh->m.NN >= (1LL << 31)) return bfail(CGL_EINVAL, "instance too large for a batch");
    }
    cgl_batch* B = new (std::nothrow) cgl_batch();
    if (!B) return bfail(CGL_EOOM, "host allocation failed");
    B->states.assign(states, states + n);
    B->st = s0->st;
    B->ninst = n;
    B->mode_lo = s0->prob.mode == CGL_MODE_LO;
    B->kg = s0->prob.k_g;
    B->ku = s0->prob.k_u;
    B->limit = 1LL << 22;
    B->phantom = 0;
    B->node_tile = ST_TX * ST_TY;
    B->use_graph = true;
    B->graph_err = cudaSuccess;
    B->graph = nullptr;
    B->form = CGL_BATCH_PERSISTENT;
    B->ev_fork = nullptr;
    for (int p = 0; p <= PMAX; ++p) B->tile_elems[p] = BT;
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s0->device);
    if (e != cudaSuccess) {
        delete B;
        return bfail(CGL_ECUDA, "device query", e);
    }
    for (int p = 1; p <= PMAX; ++p) {
        std::vector<InstDev> h;
        DegreeGroup G{};
        G.p = p;
        for (int i = 0; i < n; ++i)
            if (states[i]->mesh->m.p == p) {
                G.members.push_back(i);
                h.push_back(inst_of(states[i]));
            }
        if (G.members.empty()) continue;
        int per_sm = 0;
        e = cudaMalloc(&G.d_inst, h.size() * sizeof(InstDev));
        if (e == cudaSuccess) e = cudaMalloc(&G.d_sync, sizeof(BatchSync));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(G.d_inst, h.data(), h.size() * sizeof(InstDev), cudaMemcpyHostToDevice, B->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(G.d_sync, 0, sizeof(BatchSync), B->st);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)batch_kernel(p), BT, 0);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G.gst, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming);
        B->groups.push_back(G);
        if (e != cudaSuccess || per_sm < 1) {
            cgl_batch_destroy(B);
            return bfail(CGL_ECUDA, "batch allocation or occupancy query", e);
        }
        B->groups.back().grid = nsm * per_sm;
    }
    e = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cgl_batch_destroy(B);
        return bfail(CGL_ECUDA, "batch event", e);
    }
    cgl_status rc = build_tiles(B);
    if (rc) {
        cgl_batch_destroy(B);
        return rc;
    }
    *out = B;
    return CGL_OK;
}

static cgl_status check_sync(cgl_batch* B) {
    bool err = false;
    for (DegreeGroup& G : B->groups) {
        BatchSync hs;
        cudaError_t e = cudaMemcpyAsync(&hs, G.d_sync, sizeof(hs), cudaMemcpyDeviceToHost, B->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(B->st);
        if (e != cudaSuccess) return bfail(CGL_ECUDA, "batch step", e);
        err = err || hs.err;
    }
    if (err) {
        // reset the barriers for the next call
        for (DegreeGroup& G : B->groups) {
            cudaMemsetAsync(G.d_sync, 0, sizeof(BatchSync), B->st);
            int ph = B->phantom;
            cudaMemcpyAsync(&G.d_sync->phantom, &ph, sizeof(int), cudaMemcpyHostToDevice, B->st);
        }
        cudaStreamSynchronize(B->st);
        return set_error(CGL_ETIMEOUT, "a grid barrier of the batched stage gave up");
    }
    return CGL_OK;
}

extern "C" cgl_status cgl_batch_step_async(cgl_batch* B, int32_t nsteps) {
    if (!B || nsteps < 0) return bfail(CGL_EINVAL, "bad argument");
    cgl_status rc = ensure_graph(B);
    if (rc) return rc;
    for (int s = 0; s < nsteps; ++s) {
        cudaError_t e = B->graph ? cudaGraphLaunch(B->graph, B->st) : enqueue_batch_step(B);
        if (e != cudaSuccess) return bfail(CGL_ECUDA, "batch launch", e);
    }
    return CGL_OK;
}

extern "C" cgl_status cgl_batch_step(cgl_batch* B, int32_t nsteps, int64_t* violations) {
    cgl_status rc = cgl_batch_step_async(B, nsteps);
    if (rc) return rc;
    rc = check_sync(B);
    if (rc) return rc;
    int64_t tot = 0;
    for (cgl_state* s : B->states) {
        unsigned long long c[CNT_N];
        cudaError_t e = cudaMemcpyAsync(c, s->B.cnt, sizeof(c), cudaMemcpyDeviceToHost, B->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(B->st);
        if (e != cudaSuccess) return bfail(CGL_ECUDA, "counter read", e);
        tot += (int64_t)c[CNT_VIOL];
    }
    if (violations) *violations = tot;
    return CGL_OK;
}

extern "C" cgl_status cgl_batch_info(cgl_batch* B, int32_t* grid, int32_t* block, int32_t* elem_tiles,
                                     int32_t* node_tiles, int32_t* graph) {
    if (!B) return bfail(CGL_EINVAL, "null batch");
    int gmax = 0, net = 0, nnt = 0;
    for (const DegreeGroup& G : B->groups) {
        gmax = std::max(gmax, G.grid);
        net += G.net;
        nnt += G.nnt;
    }
    if (grid) *grid = gmax;
    if (block) *block = BT;
    if (elem_tiles) *elem_tiles = net;
    if (node_tiles) *node_tiles = nnt;
    if (graph) *graph = B->graph ? 1 : (B->graph_err != cudaSuccess ? -1 : 0);
    if (B->graph_err != cudaSuccess)
        set_error(CGL_OK, "graph capture failed (direct launches): %s", cudaGetErrorString(B->graph_err));
    return CGL_OK;
}

extern "C" cgl_status cgl_batch_set_form(cgl_batch* B, int32_t form) {
    if (!B || (form != CGL_BATCH_PERSISTENT && form != CGL_BATCH_PHASES)) return bfail(CGL_EINVAL, "bad argument");
    if (form != B->form) {
        cudaError_t e = cudaStreamSynchronize(B->st);
        if (e != cudaSuccess) return bfail(CGL_ECUDA, "batch form", e);
        B->form = form;
        if (B->graph) {
            cudaGraphExecDestroy(B->graph);
            B->graph = nullptr;
        }
        B->use_graph = true;
        B->graph_err = cudaSuccess;
    }
    return CGL_OK;
}

extern "C" cgl_status cgl_batch_get_form(cgl_batch* B, int32_t* form) {
    if (!B || !form) return bfail(CGL_EINVAL, "null argument");
    *form = B->form;
    return CGL_OK;
}

extern "C" cgl_status cgl_batch_set_tiles(cgl_batch* B, const int32_t* tile_elems) {
    if (!B || !tile_elems) return bfail(CGL_EINVAL, "null argument");
    for (int p = 1; p <= PMAX; ++p)
        if (tile_elems[p] < 1 || tile_elems[p] > BT) return bfail(CGL_EINVAL, "tile length must be in [1, 128]");
    for (int p = 1; p <= PMAX; ++p) B->tile_elems[p] = tile_elems[p];
    return build_tiles(B);
}

extern "C" cgl_status cgl_batch_get_tiles(cgl_batch* B, int32_t* tile_elems) {
    if (!B || !tile_elems) return bfail(CGL_EINVAL, "null argument");
    for (int p = 0; p <= PMAX; ++p) tile_elems[p] = B->tile_elems[p];
    return CGL_OK;
}

static cgl_status time_steps(cgl_batch* B, int steps, float* ms) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cgl_status rc = cgl_batch_step_async(B, 1);  // warm-up (and graph build)
    if (!rc) {
        cudaEventRecord(a, B->st);
        rc = cgl_batch_step_async(B, steps);
        cudaEventRecord(b, B->st);
    }
    if (!rc) rc = check_sync(B);
    if (!rc) cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}

// Coordinate search over the element-tile length of each degree present in
// the batch (candidates 32, 64, 96, 128), timing `steps` steps per trial.
// The states are advanced by the trials. Writes the choice as JSON if path.
extern "C" cgl_status cgl_batch_autotune(cgl_batch* B, int32_t steps, const char* json_path) {
    if (!B || steps < 1) return bfail(CGL_EINVAL, "bad argument");
    bool present[PMAX + 1] = {false};
    for (cgl_state* s : B->states) present[s->mesh->m.p] = true;
    const int cand[] = {32, 64, 96, 128};
    float best_all = 0.f;
    cgl_status rc = time_steps(B, steps, &best_all);
    if (rc) return rc;
    for (int p = 1; p <= PMAX; ++p) {
        if (!present[p]) continue;
        int best = B->tile_elems[p];
        for (int c : cand) {
            if (c == best) continue;
            int keep = B->tile_elems[p];
            B->tile_elems[p] = c;
            rc = build_tiles(B);
            float ms = 0.f;
            if (!rc) rc = time_steps(B, steps, &ms);
            if (rc) return rc;
            if (ms < best_all) {
                best_all = ms;
                best = c;
            } else {
                B->tile_elems[p] = keep;
            }
        }
        B->tile_elems[p] = best;
        rc = build_tiles(B);
        if (rc) return rc;
    }
    if (json_path && json_path[0]) {
        FILE* f = std::fopen(json_path, "w");
        if (!f) return bfail(CGL_EINVAL, "cannot write the tuning file");
        std::fprintf(f, "{\"block\": %d, \"tile_elems\": {", BT);
        bool firstk = true;
        for (int p = 1; p <= PMAX; ++p) {
            std::fprintf(f, "%s\"%d\": %d", firstk ? "" : ", ", p, B->tile_elems[p]);
            firstk = false;
        }
        std::fprintf(f, "}, \"ms_per_step\": %.6f}\n", best_all / steps);
        std::fclose(f);
    }
    return CGL_OK;
}

extern "C" cgl_status cgl_batch_load_tuning(cgl_batch* B, const char* json_path) {
    if (!B || !json_path) return bfail(CGL_EINVAL, "null argument");
    FILE* f = std::fopen(json_path, "r");
    if (!f) return bfail(CGL_EINVAL, "cannot read the tuning file");
    char buf[4096];
    size_t n = std::fread(buf, 1, sizeof(buf) - 1, f);
    std::fclose(f);
    buf[n] = 0;
    int32_t t[PMAX + 1];
    for (int p = 0; p <= PMAX; ++p) t[p] = B->tile_elems[p];
    for (int p = 1; p <= PMAX; ++p) {
        char key[16];
        std::snprintf(key, sizeof(key), "\"%d\":", p);
        const char* k = std::strstr(buf, key);
        if (k) t[p] = std::atoi(k + std::strlen(key));
    }
    return cgl_batch_set_tiles(B, t);
}

// Test hook: make every grid barrier wait for `phantom_blocks` arrivals
// that never come (0 = normal operation) and give up after `spin_limit`
// polls. Used to exercise the timeout path without faulting anything.
extern "C" cgl_status cgl_batch_debug(cgl_batch* B, int32_t phantom_blocks, int64_t spin_limit) {
    if (!B || phantom_blocks < 0 || spin_limit < 1) return bfail(CGL_EINVAL, "bad argument");
    B->phantom = phantom_blocks;
    B->limit = spin_limit;
    int ph = phantom_blocks;
    cudaError_t e = cudaSuccess;
    for (DegreeGroup& G : B->groups)
        if (e == cudaSuccess) e = cudaMemcpyAsync(&G.d_sync->phantom, &ph, sizeof(int), cudaMemcpyHostToDevice, B->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->st);
    if (e != cudaSuccess) return bfail(CGL_ECUDA, "debug", e);
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    return CGL_OK;
}

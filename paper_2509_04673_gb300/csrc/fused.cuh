// fused.cuh — the first Richardson sweep fused into the kernel that builds
// its right-hand side (FP32-mixed form).
//
// k_grad_sweep: g_h right-hand side b = int phi_i grad u_h, lumped iterate
//   g0 = b / m_i and the first sweep g1 = g0 + (b - M_C g0) / m_i (Sec. 2.2,
//   Richardson reading of the consistent L2 projection) in one pass over a
//   32 x 16 node tile.
// k_udot_sweep: node gather r_i = sum_e R^e_i, lumped iterate udot0 = r / m_i
//   and the first sweep (Sec. 4.3, step 2) in one pass over a tile.
//
// A sweep needs its lumped iterate on the tile plus a halo of p nodes, so
// each block recomputes the right-hand side there (the grad stencil reads u
// on a halo of 2p nodes).  The arithmetic is that of grad_tile,
// gather_init_at and sweep_tile, in the same order with the same explicit
// roundings, so the fused kernels give the same bits as the separate ones
// (the batched stage, which keeps them separate, is compared bitwise).
#pragma once

#include "kernels.cuh"

namespace cgl {

// wrap (gx, gy) on periodic directions (wrap_periodic: any number of
// periods); false outside a non-periodic mesh
DEV bool wrap_node(const MeshDev& m, int& gx, int& gy) {
    bool in = true;
    if (m.py) gy = wrap_periodic(gy, m.nny);
    else in = gy >= 0 && gy < m.nny;
    if (m.px) gx = wrap_periodic(gx, m.nnx);
    else in = in && gx >= 0 && gx < m.nnx;
    return in;
}

template <int P, int NC>
struct GradSweepWs {
    static constexpr int HX1 = ST_TX + 2 * P, HY1 = ST_TY + 2 * P;  // tile + p halo
    static constexpr int HX2 = ST_TX + 4 * P, HY2 = ST_TY + 4 * P;  // tile + 2p halo
    static constexpr int NW = 2 * P + 1, NCL = P + 2;
    static constexpr int A = HY2 * HX2;                // u on the 2p halo
    static constexpr int B = 2 * HY2 * HX1;            // x-pass of the grad stencil; later the sweep's x-pass
    static constexpr int C = 2 * HY1 * HX1;            // g0 (x and y parts) on the p halo
    static constexpr int D = 2 * ST_TY * ST_TX;        // b on the tile
    static constexpr int size = A + B + C + D + 2 * NCL * NW;
};

// The block's geometry (wrapped node indices, node classes, weights, masses)
// is the same for every component, so it is formed once into registers
// before the component loop; the halo passes give each thread a fixed
// column (its x weights stay in registers) and a set of rows.
// One block of ST_TX x ST_BY threads (thread (tx, ty)) on the tile at (gx0,
// gy0); ws: GradSweepWs<P, NC>::size floats of shared memory.  k_grad_sweep
// and the batched stage's phase kernels run it.
template <int P, int NC>
DEV void grad_sweep_block(const MeshDev& m, const float* __restrict__ u, float* __restrict__ bout,
                          float* __restrict__ gout, int gx0, int gy0, int tx, int ty, float* ws) {
    using WS = GradSweepWs<P, NC>;
    constexpr int HX1 = WS::HX1, HY1 = WS::HY1, HX2 = WS::HX2, HY2 = WS::HY2, NW = WS::NW, NCL = WS::NCL;
    constexpr int NT = ST_TX * ST_BY, NJ = ST_TY / ST_BY;
    constexpr int RG = NT / HX1;                    // row groups of the halo passes
    constexpr int NA = (HY2 * HX2 + NT - 1) / NT;  // staged values per thread
    constexpr int NXP = (HY2 + RG - 1) / RG;        // x-pass rows per thread
    constexpr int NYP = (HY1 + RG - 1) / RG;        // y-pass rows per thread
    constexpr int NSX = (HY1 + ST_BY - 1) / ST_BY;  // rows of the sweep's x-pass per thread
    float(*A)[HX2] = reinterpret_cast<float(*)[HX2]>(ws);
    float(*tC)[HX1] = reinterpret_cast<float(*)[HX1]>(ws + WS::A);
    float(*tM)[HX1] = reinterpret_cast<float(*)[HX1]>(ws + WS::A + HY2 * HX1);
    float(*t)[HY1][ST_TX] = reinterpret_cast<float(*)[HY1][ST_TX]>(ws + WS::A);  // after tC, tM are consumed
    float(*G)[HY1][HX1] = reinterpret_cast<float(*)[HY1][HX1]>(ws + WS::A + WS::B);
    float(*Bt)[ST_TY][ST_TX] = reinterpret_cast<float(*)[ST_TY][ST_TX]>(ws + WS::A + WS::B + WS::C);
    float(*WM)[NW] = reinterpret_cast<float(*)[NW]>(ws + WS::A + WS::B + WS::C + WS::D);
    float(*WC)[NW] = reinterpret_cast<float(*)[NW]>(ws + WS::A + WS::B + WS::C + WS::D + NCL * NW);
    const Tab<float>& T = TabSel<float>::t(P);
    const int tid = ty * ST_TX + tx;
    if (tid < NCL * NW) {
        const int cls = tid / NW, k = tid - cls * NW;
        WM[cls][k] = class_weight<float, P, 0>(T, cls, k - P);
        WC[cls][k] = class_weight<float, P, 1>(T, cls, k - P);
    }
    const float h = m.h_f, h2 = m.h2_f;
    // staged values of u: node offsets (-1 outside the mesh)
    long long aoff[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const int i = tid + j * NT;
        aoff[j] = -1;
        if (i < HY2 * HX2) {
            const int r = i / HX2, cc = i - r * HX2;
            int gx = gx0 - 2 * P + cc, gy = gy0 - 2 * P + r;
            if (wrap_node(m, gx, gy)) aoff[j] = (long long)gy * m.nnx + gx;
        }
    }
    // halo passes: column cx of the p halo, rows rg + RG j
    const int cx = tid % HX1, rg = tid / HX1;
    const bool hv = rg < RG;
    int clx;
    {
        int gx = gx0 - P + cx, gy = 0;
        wrap_node(m, gx, gy);
        clx = node_class<P>(gx, m.nnx, m.px);
    }
    bool yin[NYP];
    int ycl[NYP];
    float yinv[NYP];
#pragma unroll
    for (int j = 0; j < NYP; ++j) {
        const int r = rg + RG * j;
        int gx = gx0 - P + cx, gy = gy0 - P + r;
        yin[j] = wrap_node(m, gx, gy) && hv && r < HY1;
        ycl[j] = node_class<P>(gy, m.nny, m.py);
        const int cnt = (clx == 0 ? 2 : 1) * (ycl[j] == 0 ? 2 : 1);
        yinv[j] = mul_r(m.inv_me_f, inv_count<float>(cnt));
    }
    // the sweep: column tx of the tile, its x class and rows
    const int gxt = gx0 + tx;
    const int clxt = node_class<P>(gxt, m.nnx, m.px);
    __syncthreads();  // weights ready
    float wcx[NW], wmx[NW], wst[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        wcx[k] = WC[clx][k];
        wmx[k] = WM[clx][k];
        wst[k] = WM[clxt][k];
    }
    for (int c = 0; c < NC; ++c) {
        if (c > 0) __syncthreads();  // previous component consumed
        // u of component c on the tile plus a halo of 2p nodes
        const float* uc = u + (long long)c * m.NN;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const int i = tid + j * NT;
            if (i < HY2 * HX2) ws[i] = aoff[j] >= 0 ? __ldcg(&uc[aoff[j]]) : 0.f;
        }
        __syncthreads();
        // grad stencil along x for the columns of the p halo, all 2p-halo rows
        if (hv) {
#pragma unroll
            for (int j = 0; j < NXP; ++j) {
                const int r = rg + RG * j;
                if (r < HY2) {
                    float sc = 0.f, sm = 0.f;
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        const float x = A[r][cx + k];
                        sc = fma_r(wcx[k], x, sc);
                        sm = fma_r(wmx[k], x, sm);
                    }
                    tC[r][cx] = sc;
                    tM[r][cx] = sm;
                }
            }
        }
        __syncthreads();
        // along y: b and g0 = b / m_i on the p halo (zero outside the mesh)
        if (hv) {
#pragma unroll
            for (int j = 0; j < NYP; ++j) {
                const int r = rg + RG * j;
                if (r < HY1) {
                    const int cly = ycl[j];
                    float sx = 0.f, sy = 0.f;
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        sx = fma_r(WM[cly][k], tC[r + k][cx], sx);
                        sy = fma_r(WC[cly][k], tM[r + k][cx], sy);
                    }
                    const float bx = mul_r(h, sx), by = mul_r(h, sy);
                    G[0][r][cx] = yin[j] ? mul_r(bx, yinv[j]) : 0.f;
                    G[1][r][cx] = yin[j] ? mul_r(by, yinv[j]) : 0.f;
                    const int rt = r - P, ct = cx - P;
                    if (rt >= 0 && rt < ST_TY && ct >= 0 && ct < ST_TX) {
                        Bt[0][rt][ct] = bx;
                        Bt[1][rt][ct] = by;
                    }
                }
            }
        }
        __syncthreads();
        // first sweep, along x for every p-halo row (the mass weights)
#pragma unroll
        for (int j = 0; j < NSX; ++j) {
            const int r = ty + ST_BY * j;
            if (r < HY1) {
#pragma unroll
                for (int f = 0; f < 2; ++f) {
                    float sx = 0.f;
#pragma unroll
                    for (int k = 0; k < NW; ++k) sx = fma_r(wst[k], G[f][r][tx + k], sx);
                    t[f][r][tx] = sx;
                }
            }
        }
        __syncthreads();
        // along y and the outputs: g1 (and b where more sweeps follow)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int r = ty + j * ST_BY, gy = gy0 + r;
            if (gxt >= m.nnx || gy >= m.nny) continue;
            const int cly = node_class<P>(gy, m.nny, m.py);
            const int cnt = (clxt == 0 ? 2 : 1) * (cly == 0 ? 2 : 1);
            const float inv_mi = mul_r(m.inv_me_f, inv_count<float>(cnt));
            const long long node = (long long)gy * m.nnx + gxt;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                float sy = 0.f;
#pragma unroll
                for (int k = 0; k < NW; ++k) sy = fma_r(WM[cly][k], t[f][r + k][tx], sy);
                const long long k = (long long)(f * NC + c) * m.NN + node;
                gout[k] = sweep_value(G[f][r + P][tx + P], Bt[f][r][tx], sy, h2, inv_mi);
                if (bout) bout[k] = Bt[f][r][tx];
            }
        }
    }
}

template <int P, int NC>
__global__ void __launch_bounds__(ST_TX * ST_BY)
    k_grad_sweep(MeshDev m, const float* __restrict__ u, float* __restrict__ bout, float* __restrict__ gout) {
    // like k_grad_rhs: runs beside k_pre, waits for it before exiting
    pdl_trigger();
    __shared__ float ws[GradSweepWs<P, NC>::size];
    grad_sweep_block<P, NC>(m, u, bout, gout, blockIdx.x * ST_TX, blockIdx.y * ST_TY, threadIdx.x, threadIdx.y, ws);
    pdl_wait();
}


template <int P, int NC>
struct UdotSweepWs {
    static constexpr int HX = ST_TX + 2 * P, HY = ST_TY + 2 * P, NW = 2 * P + 1, NCL = P + 2;
    static constexpr int size = NC * (HY * HX + HY * ST_TX + ST_TY * ST_TX) + NCL * NW;
};

// r = sum over E_i of the element residuals (stored for further sweeps and
// diagnostics), udot0 = r / m_i on the tile plus a p halo, and the first
// sweep udot1 = udot0 + (r - M_C udot0) / m_i on the tile
template <int P, int NC>
__global__ void __launch_bounds__(ST_TX * ST_BY)
    k_udot_sweep(MeshDev m, const float* __restrict__ ER, float* __restrict__ rout, float* __restrict__ xout) {
    pdl_begin();
    using WS = UdotSweepWs<P, NC>;
    constexpr int HX = WS::HX, HY = WS::HY, NW = WS::NW, NCL = WS::NCL;
    constexpr int NT = ST_TX * ST_BY, NJ = ST_TY / ST_BY;
    __shared__ float ws[WS::size];
    float(*xs)[HY][HX] = reinterpret_cast<float(*)[HY][HX]>(ws);
    float(*t)[HY][ST_TX] = reinterpret_cast<float(*)[HY][ST_TX]>(ws + NC * HY * HX);
    float(*rt)[ST_TY][ST_TX] = reinterpret_cast<float(*)[ST_TY][ST_TX]>(ws + NC * (HY * HX + HY * ST_TX));
    float(*W)[NW] = reinterpret_cast<float(*)[NW]>(ws + NC * (HY * HX + HY * ST_TX + ST_TY * ST_TX));
    const Tab<float>& T = TabSel<float>::t(P);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * ST_TX + tx;
    if (tid < NCL * NW) {
        const int cls = tid / NW, k = tid - cls * NW;
        W[cls][k] = class_weight<float, P, 0>(T, cls, k - P);
    }
    const int gx0 = blockIdx.x * ST_TX, gy0 = blockIdx.y * ST_TY;
    // gathers on the tile plus a p halo (gather_init_at's arithmetic)
    for (int i = tid; i < HY * HX; i += NT) {
        const int r = i / HX, cc = i - r * HX;
        int gx = gx0 - P + cc, gy = gy0 - P + r;
        const bool in = wrap_node(m, gx, gy);
        float s[NC];
        float inv_mi = 0.f;
        if (in) {
            const NodeC<P> nc = node_c<P>(m, gx, gy);
            gather_at<float, P, NC>(m, ER, nc, s);
            inv_mi = PV<float>::inv_me(m) * inv_count<float>(nc.nxc * nc.nyc);
        }
        const int rr = r - P, ct = cc - P;
        const bool tile = rr >= 0 && rr < ST_TY && ct >= 0 && ct < ST_TX;
        // a node of this tile itself, not a wrapped copy of another tile's
        const bool own = tile && gx0 + ct < m.nnx && gy0 + rr < m.nny;
        const long long node = (long long)gy * m.nnx + gx;
#pragma unroll
        for (int v = 0; v < NC; ++v) {
            xs[v][r][cc] = in ? s[v] * inv_mi : 0.f;
            if (tile) {
                rt[v][rr][ct] = in ? s[v] : 0.f;
                if (in && own) rout[v * m.NN + node] = s[v];
            }
        }
    }
    __syncthreads();
    const int gx = gx0 + tx;
    const int clx = node_class<P>(gx, m.nnx, m.px);
    for (int r = ty; r < HY; r += ST_BY) {
#pragma unroll
        for (int v = 0; v < NC; ++v) {
            float sx = 0.f;
#pragma unroll
            for (int k = 0; k < NW; ++k) sx = fma_r(W[clx][k], xs[v][r][tx + k], sx);
            t[v][r][tx] = sx;
        }
    }
    __syncthreads();
    const float h2 = PV<float>::h2(m);
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int r = ty + j * ST_BY, gy = gy0 + r;
        if (gx >= m.nnx || gy >= m.nny) continue;
        const int cly = node_class<P>(gy, m.nny, m.py);
        const int cnt = (clx == 0 ? 2 : 1) * (cly == 0 ? 2 : 1);
        const float inv_mi = mul_r(PV<float>::inv_me(m), inv_count<float>(cnt));
        const long long node = (long long)gy * m.nnx + gx;
#pragma unroll
        for (int v = 0; v < NC; ++v) {
            float sy = 0.f;
#pragma unroll
            for (int k = 0; k < NW; ++k) sy = fma_r(W[cly][k], t[v][r + k][tx], sy);
            xout[v * m.NN + node] = sweep_value(xs[v][r + P][tx + P], rt[v][r][tx], sy, h2, inv_mi);
        }
    }
}

// ---------------------------------------------------------------------------
// The two fused sweeps as functions of one ST_TX x ST_TY node tile for a block
// of NT threads (the batched stage runs them with 128 threads per block),
// geometry formed per component: the same arithmetic, in the same order, as
// k_grad_sweep and k_udot_sweep, hence the same bits as the separate
// stencils.  ws holds GradSweepWs<P, NC>::size or UdotSweepWs<P, NC>::size
// floats; the block's threads all call them (they synchronise the block).
// ---------------------------------------------------------------------------
template <int P, int NC, int NT>
DEV void grad_sweep_tile(const MeshDev& m, const float* __restrict__ u, float* __restrict__ bout,
                         float* __restrict__ gout, int gx0, int gy0, int tid, float* ws) {
    using WS = GradSweepWs<P, NC>;
    constexpr int HX1 = WS::HX1, HY1 = WS::HY1, HX2 = WS::HX2, HY2 = WS::HY2, NW = WS::NW, NCL = WS::NCL;
    constexpr int BYT = NT / ST_TX, NJ = ST_TY / BYT;
    float(*A)[HX2] = reinterpret_cast<float(*)[HX2]>(ws);
    float(*tC)[HX1] = reinterpret_cast<float(*)[HX1]>(ws + WS::A);
    float(*tM)[HX1] = reinterpret_cast<float(*)[HX1]>(ws + WS::A + HY2 * HX1);
    float(*t)[HY1][ST_TX] = reinterpret_cast<float(*)[HY1][ST_TX]>(ws + WS::A);
    float(*G)[HY1][HX1] = reinterpret_cast<float(*)[HY1][HX1]>(ws + WS::A + WS::B);
    float(*Bt)[ST_TY][ST_TX] = reinterpret_cast<float(*)[ST_TY][ST_TX]>(ws + WS::A + WS::B + WS::C);
    float(*WM)[NW] = reinterpret_cast<float(*)[NW]>(ws + WS::A + WS::B + WS::C + WS::D);
    float(*WC)[NW] = reinterpret_cast<float(*)[NW]>(ws + WS::A + WS::B + WS::C + WS::D + NCL * NW);
    const Tab<float>& T = TabSel<float>::t(P);
    const int tx = tid % ST_TX, ty = tid / ST_TX;
    __syncthreads();  // the previous user of ws is done
    if (tid < NCL * NW) {
        const int cls = tid / NW, k = tid - cls * NW;
        WM[cls][k] = class_weight<float, P, 0>(T, cls, k - P);
        WC[cls][k] = class_weight<float, P, 1>(T, cls, k - P);
    }
    const float h = m.h_f, h2 = m.h2_f;
    for (int c = 0; c < NC; ++c) {
        __syncthreads();
        for (int i = tid; i < HY2 * HX2; i += NT) {
            const int r = i / HX2, cc = i - r * HX2;
            int gx = gx0 - 2 * P + cc, gy = gy0 - 2 * P + r;
            const bool in = wrap_node(m, gx, gy);
            A[r][cc] = in ? __ldcg(&u[(long long)c * m.NN + (long long)gy * m.nnx + gx]) : 0.f;
        }
        __syncthreads();
        for (int i = tid; i < HY2 * HX1; i += NT) {
            const int r = i / HX1, cc = i - r * HX1;
            int gx = gx0 - P + cc, gy = 0;
            wrap_node(m, gx, gy);
            const int clx = node_class<P>(gx, m.nnx, m.px);
            float sc = 0.f, sm = 0.f;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const float x = A[r][cc + k];
                sc = fma_r(WC[clx][k], x, sc);
                sm = fma_r(WM[clx][k], x, sm);
            }
            tC[r][cc] = sc;
            tM[r][cc] = sm;
        }
        __syncthreads();
        for (int i = tid; i < HY1 * HX1; i += NT) {
            const int r = i / HX1, cc = i - r * HX1;
            int gx = gx0 - P + cc, gy = gy0 - P + r;
            const bool in = wrap_node(m, gx, gy);
            const int clx = node_class<P>(gx, m.nnx, m.px), cly = node_class<P>(gy, m.nny, m.py);
            float sx = 0.f, sy = 0.f;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                sx = fma_r(WM[cly][k], tC[r + k][cc], sx);
                sy = fma_r(WC[cly][k], tM[r + k][cc], sy);
            }
            const int cnt = (clx == 0 ? 2 : 1) * (cly == 0 ? 2 : 1);
            const float inv_mi = mul_r(m.inv_me_f, inv_count<float>(cnt));
            const float bx = mul_r(h, sx), by = mul_r(h, sy);
            G[0][r][cc] = in ? mul_r(bx, inv_mi) : 0.f;
            G[1][r][cc] = in ? mul_r(by, inv_mi) : 0.f;
            const int rt = r - P, ct = cc - P;
            if (rt >= 0 && rt < ST_TY && ct >= 0 && ct < ST_TX) {
                Bt[0][rt][ct] = bx;
                Bt[1][rt][ct] = by;
            }
        }
        __syncthreads();
        const int gxt = gx0 + tx;
        const int clxt = node_class<P>(gxt, m.nnx, m.px);
        for (int r = ty; r < HY1; r += BYT) {
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                float sx = 0.f;
#pragma unroll
                for (int k = 0; k < NW; ++k) sx = fma_r(WM[clxt][k], G[f][r][tx + k], sx);
                t[f][r][tx] = sx;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int r = ty + j * BYT, gy = gy0 + r;
            if (gxt >= m.nnx || gy >= m.nny) continue;
            const int cly = node_class<P>(gy, m.nny, m.py);
            const int cnt = (clxt == 0 ? 2 : 1) * (cly == 0 ? 2 : 1);
            const float inv_mi = mul_r(m.inv_me_f, inv_count<float>(cnt));
            const long long node = (long long)gy * m.nnx + gxt;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                float sy = 0.f;
#pragma unroll
                for (int k = 0; k < NW; ++k) sy = fma_r(WM[cly][k], t[f][r + k][tx], sy);
                const long long k = (long long)(f * NC + c) * m.NN + node;
                gout[k] = sweep_value(G[f][r + P][tx + P], Bt[f][r][tx], sy, h2, inv_mi);
                if (bout) bout[k] = Bt[f][r][tx];
            }
        }
    }
}

template <int P, int NC, int NT>
DEV void udot_sweep_tile(const MeshDev& m, const float* __restrict__ ER, float* __restrict__ rout,
                         float* __restrict__ xout, int gx0, int gy0, int tid, float* ws) {
    using WS = UdotSweepWs<P, NC>;
    constexpr int HX = WS::HX, HY = WS::HY, NW = WS::NW, NCL = WS::NCL;
    constexpr int BYT = NT / ST_TX, NJ = ST_TY / BYT;
    float(*xs)[HY][HX] = reinterpret_cast<float(*)[HY][HX]>(ws);
    float(*t)[HY][ST_TX] = reinterpret_cast<float(*)[HY][ST_TX]>(ws + NC * HY * HX);
    float(*rt)[ST_TY][ST_TX] = reinterpret_cast<float(*)[ST_TY][ST_TX]>(ws + NC * (HY * HX + HY * ST_TX));
    float(*W)[NW] = reinterpret_cast<float(*)[NW]>(ws + NC * (HY * HX + HY * ST_TX + ST_TY * ST_TX));
    const Tab<float>& T = TabSel<float>::t(P);
    const int tx = tid % ST_TX, ty = tid / ST_TX;
    __syncthreads();  // the previous user of ws is done
    if (tid < NCL * NW) {
        const int cls = tid / NW, k = tid - cls * NW;
        W[cls][k] = class_weight<float, P, 0>(T, cls, k - P);
    }
    for (int i = tid; i < HY * HX; i += NT) {
        const int r = i / HX, cc = i - r * HX;
        int gx = gx0 - P + cc, gy = gy0 - P + r;
        const bool in = wrap_node(m, gx, gy);
        float s[NC];
        float inv_mi = 0.f;
        if (in) {
            const NodeC<P> nc = node_c<P>(m, gx, gy);
            gather_at<float, P, NC>(m, ER, nc, s);
            inv_mi = PV<float>::inv_me(m) * inv_count<float>(nc.nxc * nc.nyc);
        }
        const int rr = r - P, ct = cc - P;
        const bool tile = rr >= 0 && rr < ST_TY && ct >= 0 && ct < ST_TX;
        // a node of this tile itself, not a wrapped copy of another tile's
        const bool own = tile && gx0 + ct < m.nnx && gy0 + rr < m.nny;
        const long long node = (long long)gy * m.nnx + gx;
#pragma unroll
        for (int v = 0; v < NC; ++v) {
            xs[v][r][cc] = in ? s[v] * inv_mi : 0.f;
            if (tile) {
                rt[v][rr][ct] = in ? s[v] : 0.f;
                if (in && own) rout[v * m.NN + node] = s[v];
            }
        }
    }
    __syncthreads();
    const int gx = gx0 + tx;
    const int clx = node_class<P>(gx, m.nnx, m.px);
    for (int r = ty; r < HY; r += BYT) {
#pragma unroll
        for (int v = 0; v < NC; ++v) {
            float sx = 0.f;
#pragma unroll
            for (int k = 0; k < NW; ++k) sx = fma_r(W[clx][k], xs[v][r][tx + k], sx);
            t[v][r][tx] = sx;
        }
    }
    __syncthreads();
    const float h2 = PV<float>::h2(m);
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int r = ty + j * BYT, gy = gy0 + r;
        if (gx >= m.nnx || gy >= m.nny) continue;
        const int cly = node_class<P>(gy, m.nny, m.py);
        const int cnt = (clx == 0 ? 2 : 1) * (cly == 0 ? 2 : 1);
        const float inv_mi = mul_r(PV<float>::inv_me(m), inv_count<float>(cnt));
        const long long node = (long long)gy * m.nnx + gx;
#pragma unroll
        for (int v = 0; v < NC; ++v) {
            float sy = 0.f;
#pragma unroll
            for (int k = 0; k < NW; ++k) sy = fma_r(W[cly][k], t[v][r + k][tx], sy);
            xout[v * m.NN + node] = sweep_value(xs[v][r + P][tx + P], rt[v][r][tx], sy, h2, inv_mi);
        }
    }
}

}  // namespace cgl

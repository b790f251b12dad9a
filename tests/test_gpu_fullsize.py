"""Full-size parity on sampled windows (GPU).

A stage is computed on the GPU over the whole mesh of a full-size workload.
The oracle then recomputes the same stage (same input, same dt) on windows of
W x W elements cut out of the mesh, and the nodes of the central C x C
elements of every window are compared.  One stage only reads data within a
few elements of a node (sensor, g_h and udot Richardson sweeps, flux
limiter: radius <= 5 elements), so the central elements do not see the
window's own boundary condition; where a window touches the true boundary it
keeps that boundary's condition.  FP64: 1e-12 relative; FP32-mixed: L1
error within the float32 budget and the invariant domain exact.
"""
import math

import numpy as np
import pytest

import inputs
import oracle.scheme as S

pytestmark = pytest.mark.gpu

W, C = 24, 8


@pytest.fixture(scope="module")
def cgl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_04673_gb300 import build, cgl as C_
    build.build()
    return C_


def window(mesh, u, ex0, ey0, w):
    """Sub-mesh of w x w elements starting at element (ex0, ey0) and its
    coefficients (non-periodic mesh)."""
    p = mesh.p
    h = mesh.h
    sub = inputs.Mesh(w, w, p, mesh.x0 + ex0 * h, mesh.x0 + (ex0 + w) * h,
                      mesh.y0 + ey0 * h, mesh.y0 + (ey0 + w) * h, mesh.bc_x, mesh.bc_y)
    us = u[:, ey0 * p:(ey0 + w) * p + 1, ex0 * p:(ex0 + w) * p + 1].copy()
    return sub, us


def run_windows(mesh, prob, u, un, dt, a, b, out, prec, origins):
    """Worst relative difference (scaled by each component's magnitude over
    the whole mesh, as in the other parity tests) and the L1 error."""
    p = mesh.p
    nc = u.shape[0]
    gscale = np.maximum(np.abs(out).reshape(nc, -1).max(axis=1), 1e-300)
    worst = 0.0
    l1n, l1d = 0.0, 0.0
    for ex0, ey0 in origins:
        sub, us = window(mesh, u, ex0, ey0, W)
        _, uns = window(mesh, un, ex0, ey0, W)
        ref, info = S.ssp_stage(sub, prob, us, uns, dt, a, b)
        # central elements, clipped to the true boundary where the window touches it
        c0 = (W - C) // 2
        lo_x = 0 if ex0 == 0 else c0
        lo_y = 0 if ey0 == 0 else c0
        hi_x = W if ex0 + W == mesh.nx else c0 + C
        hi_y = W if ey0 + W == mesh.ny else c0 + C
        sl = (slice(None), slice(lo_y * p, hi_y * p + 1), slice(lo_x * p, hi_x * p + 1))
        r = ref[sl]
        g = out[:, ey0 * p:(ey0 + W) * p + 1, ex0 * p:(ex0 + W) * p + 1][sl]
        worst = max(worst, float((np.abs(g - r).reshape(nc, -1).max(axis=1) / gscale).max()))
        l1n += np.abs(g - r).sum()
        l1d += np.abs(r).sum()
    return worst, l1n / l1d


def _origins(mesh):
    nx, ny = mesh.nx, mesh.ny
    return [((nx - W) // 2, (ny - W) // 2), (0, 0), (nx - W, ny - W), (0, (ny - W) // 3),
            ((2 * nx) // 3, 0)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("which", ["euler_quadrants_512_q3", "euler_blast_2048_q2", "kpp_256_q2", "kpp_2048_q2"])
def test_full_size_windows(cgl, which, prec):
    if which == "euler_quadrants_512_q3":
        mesh, prob, u0 = inputs.euler_quadrant_config(512, 512, 3)
    elif which == "euler_blast_2048_q2":
        mesh, prob, u0 = inputs.euler_blast_config(2048, 2048, 2)
    elif which == "kpp_256_q2":
        mesh, prob, u0 = inputs.kpp_config(256, 256, 2)
    else:
        # large enough for the fused first sweeps of the FP32-mixed form
        mesh, prob, u0 = inputs.kpp_config(2048, 2048, 2)
    nc = u0.shape[0]
    if prec == 1:
        u0 = u0.astype(np.float32).astype(np.float64)
        if nc == 1:
            lo = float(np.nextafter(np.float32(prob.umin), np.float32(np.inf)))
            hi = float(np.nextafter(np.float32(prob.umax), np.float32(-np.inf)))
            u0 = np.clip(u0, lo, hi)
    m = cgl.Mesh(mesh)
    g = cgl.State(m, nc, prec)
    g.set_problem(prob)
    g.set_state(u0)
    g.set_time(0.0)
    dt = g.time_step()
    # first stage (a = 0) and a later-stage combination on the result
    ginfo = g.stage(dt, 0.0, 1.0)
    out1 = g.get_state()
    assert ginfo["violations"] == 0
    worst, l1 = run_windows(mesh, prob, u0, u0, dt, 0.0, 1.0, out1, prec, _origins(mesh))
    if prec == 0:
        assert worst <= 1e-12, worst
    else:
        assert l1 <= 5e-6, l1
    u1 = out1
    g.set_state(u1)
    g.set_base_state(u0)
    ginfo = g.stage(dt, 0.75, 0.25)
    out2 = g.get_state()
    assert ginfo["violations"] == 0
    worst, l1 = run_windows(mesh, prob, u1, u0, dt, 0.75, 0.25, out2, prec, _origins(mesh)[:3])
    if prec == 0:
        assert worst <= 1e-12, worst
    else:
        assert l1 <= 5e-6, l1
    if nc == 4:
        rho = out2[0]
        pres = 0.4 * (out2[3] - 0.5 * (out2[1] ** 2 + out2[2] ** 2) / rho)
        assert np.all(rho > 0) and np.all(pres > 0)
    g.close()

"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

FP64 form: every nodal value after one SSP stage agrees with the oracle to
1e-12 relative (max over the grid, scaled by the component's magnitude),
and the per-element FP64 intermediates (u^e, dt_e, ubar^{e,L}, ubar^e) to
1e-12.  FP32-mixed form: the invariant-domain property holds exactly at
every node (zero violations, every value inside the bounds), the L1
error against the oracle is within the stated float32 budget, and every
nodal value and per-element intermediate is within its element-wise bound.
Cases span several tiles, ragged sizes, every mode, flux-limiter switch,
boundary condition and degree 1..4, and the full-size bench workload.
"""
import math

import numpy as np
import pytest

import inputs
from inputs import Mesh, Problem
import oracle.scheme as S

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def cgl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_04673_gb300 import build, cgl as C
    build.build()
    return C


def _rel(a, b, nc):
    a = a.reshape(nc, -1)
    b = b.reshape(nc, -1)
    sc = np.maximum(np.abs(b).max(axis=1), 1e-300)
    return float((np.abs(a - b).max(axis=1) / sc).max())


def _gpu_stage(C, mesh, prob, u, un, dt, a, b, prec=0):
    m = C.Mesh(mesh)
    st = C.State(m, u.shape[0], prec)
    st.set_problem(prob)
    st.set_state(u)
    st.set_base_state(un)
    info = st.stage(dt, a, b, raise_on_idp=False)
    out = st.get_state()
    fields = {k: st.get_field(f) for k, f in (("ue", C.FIELD_UE), ("dte", C.FIELD_DTE),
                                             ("ubL", C.FIELD_UBL), ("ube", C.FIELD_UBE),
                                             ("beta", C.FIELD_BETA), ("gamma", C.FIELD_GAMMA))}
    st.close()
    return out, info, fields


def _inward_f32(lo, hi):
    """Bounds rounded inward to float32-representable values."""
    l32 = np.float32(lo)
    if float(l32) < lo:
        l32 = np.nextafter(l32, np.float32(np.inf))
    h32 = np.float32(hi)
    if float(h32) > hi:
        h32 = np.nextafter(h32, np.float32(-np.inf))
    return float(l32), float(h32)


def _case_state(mesh, prob, seed):
    if prob.flux == inputs.FLUX_EULER:
        return inputs.random_euler_state(mesh, seed), inputs.random_euler_state(mesh, seed + 1)
    return (inputs.random_scalar_state(mesh, seed, prob.umin, prob.umax, 0.4),
            inputs.random_scalar_state(mesh, seed + 1, prob.umin, prob.umax, 0.4))


CASES = {
    # name: (mesh, problem overrides)
    "adv_p1_periodic_wenol": (Mesh(9, 7, 1, 0.0, 9 / 7, 0.0, 1.0), dict(mode=3, fl=1)),
    "adv_p2_periodic_wenol": (Mesh(13, 11, 2, 0.0, 13 / 11, 0.0, 1.0), dict(mode=3, fl=1)),
    "adv_p3_periodic_weno": (Mesh(6, 9, 3, 0.0, 2 / 3, 0.0, 1.0), dict(mode=2, fl=0)),
    "adv_p4_periodic_wenol": (Mesh(5, 5, 4), dict(mode=3, fl=1)),
    "adv_p2_fixed_weno_l": (Mesh(10, 6, 2, 0.0, 5 / 3, 0.0, 1.0, 2, 2), dict(mode=3, fl=1)),
    "adv_p2_outflow_ho": (Mesh(7, 8, 2, 0.0, 7 / 8, 0.0, 1.0, 1, 1), dict(mode=1, fl=0)),
    "adv_p2_mixedbc_lo_low": (Mesh(8, 5, 2, 0.0, 1.6, 0.0, 1.0, 2, 0), dict(mode=0, fl=2)),
    "adv_p3_periodic_lo_lim": (Mesh(6, 6, 3), dict(mode=0, fl=1)),
    "burgers_p2_periodic_wenol": (Mesh(12, 12, 2), dict(flux=1, mode=3, fl=1)),
    "burgers_p3_fixed_weno": (Mesh(7, 7, 3, 0.0, 1.0, 0.0, 1.0, 2, 2), dict(flux=1, mode=2, fl=1)),
    "kpp_p2_fixed_wenol": (Mesh(16, 16, 2, -2.0, 2.0, -2.5, 1.5, 2, 2),
                           dict(flux=2, mode=3, fl=1, umin=math.pi / 4, umax=3.5 * math.pi,
                                ubc=(math.pi / 4, 0, 0, 0), w_lin=0.2)),
    "kpp_p4_outflow_wenol": (Mesh(6, 5, 4, 0.0, 1.2, 0.0, 1.0, 1, 1),
                             dict(flux=2, mode=3, fl=1, umin=0.5, umax=6.0)),
    "euler_p2_periodic_wenol": (Mesh(9, 8, 2, 0.0, 9 / 8, 0.0, 1.0), dict(flux=3, mode=3, fl=1)),
    "euler_p3_outflow_wenol": (Mesh(8, 6, 3, 0.0, 4 / 3, 0.0, 1.0, 1, 1), dict(flux=3, mode=3, fl=1)),
    "euler_p1_fixed_weno": (Mesh(6, 6, 1, 0.0, 1.0, 0.0, 1.0, 2, 2),
                            dict(flux=3, mode=2, fl=1, ubc=(1.0, 0.1, -0.2, 2.5))),
    "edge_1x1_p1_periodic": (Mesh(1, 1, 1), dict(mode=3, fl=1)),
    "edge_1x4_p2_periodic": (Mesh(1, 4, 2, 0.0, 0.25, 0.0, 1.0), dict(mode=3, fl=1)),
    "edge_1x1_p3_fixed": (Mesh(1, 1, 3, 0.0, 1.0, 0.0, 1.0, 2, 2), dict(mode=3, fl=1, ubc=(0.3, 0, 0, 0))),
}


def _problem(over):
    d = dict(over)
    fl = d.pop("fl", 1)
    p = Problem(flux=d.pop("flux", 0), flux_limiter=fl, vx=0.8, vy=-0.45)
    for k, v in d.items():
        setattr(p, k, v)
    if p.flux == inputs.FLUX_EULER:
        p.w_lin = 1e-3
    return p


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("ab", [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)])
def test_stage_parity_fp64(cgl, name, ab):
    mesh, over = CASES[name]
    prob = _problem(over)
    u, un = _case_state(mesh, prob, 1000 + len(name))
    om = S.OracleMesh(mesh)
    dt = 0.5 * S.time_step(om, prob, u)
    a, b = ab
    ref, info = S.ssp_stage(om, prob, u, un, dt, a, b)
    out, ginfo, f = _gpu_stage(cgl, mesh, prob, u, un, dt, a, b)
    nc = u.shape[0]
    assert _rel(out, ref, nc) <= TOL64, _rel(out, ref, nc)
    assert _rel(f["ue"], info["ue"], nc) <= 1e-14
    assert np.abs(f["dte"] - info["dte"]).max() <= 1e-13 * info["dte"].max()
    assert _rel(f["ubL"], info["ubL"], nc) <= 1e-13
    assert _rel(f["ube"], info["ube"], nc) <= TOL64
    # the sensor and the slope limiter element by element: gamma_e and beta_e
    # are continuous functions of the stage data with values in [0, 1]
    if prob.mode != inputs.MODE_LO:
        assert np.abs(f["gamma"] - info["gamma"]).max() <= 1e-10, np.abs(f["gamma"] - info["gamma"]).max()
    assert np.abs(f["beta"] - info["beta"]).max() <= 1e-10, np.abs(f["beta"] - info["beta"]).max()
    assert ginfo["violations"] == info["violations"] == 0


def test_multi_step_fp64_config1_small(cgl):
    """Ten SSP-RK3 steps with device-computed dt (hump + slotted disk)."""
    mesh, prob, u0 = inputs.advection_config(24, 24, 2)
    ref, t_ref, st = S.run(mesh, prob, u0, 10)
    m = cgl.Mesh(mesh)
    g = cgl.State(m, 1, cgl.FP64)
    g.set_problem(prob)
    g.set_state(u0)
    g.set_time(0.0)
    info = g.step(10)
    out = g.get_state()
    assert abs(info["t"] - t_ref) <= 1e-14 * t_ref
    assert _rel(out, ref, 1) <= 1e-11
    assert info["violations"] == 0 and st["violations"] == 0
    # conservation of the FP64 mass sum (periodic)
    assert abs(info["mass"][0] - S.mass(mesh, u0)[0]) <= 1e-13 * abs(S.mass(mesh, u0)[0])
    g.close()


def test_t_end_and_time_step(cgl):
    mesh, prob, u0 = inputs.kpp_config(16, 16, 2)
    m = cgl.Mesh(mesh)
    g = cgl.State(m, 1, cgl.FP64)
    g.set_problem(prob)
    g.set_state(u0)
    g.set_time(0.0)
    om = S.OracleMesh(mesh)
    assert abs(g.time_step() - S.time_step(om, prob, u0)) <= 1e-15 * S.time_step(om, prob, u0)
    dt = S.time_step(om, prob, u0)
    info = g.step(100, t_end=2.5 * dt)
    assert info["steps"] == 3
    assert abs(info["t"] - 2.5 * dt) <= 1e-15
    g.close()


def test_determinism(cgl):
    mesh, prob, u0 = inputs.kpp_config(32, 32, 2)
    outs = []
    for _ in range(2):
        m = cgl.Mesh(mesh)
        g = cgl.State(m, 1, cgl.FP64)
        g.set_problem(prob)
        g.set_state(u0)
        g.step(3)
        outs.append(g.get_state())
        g.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_bench_workload_stages(cgl, prec):
    """KPP 256x256 Q2 (the bench workload): the three stages of one SSP-RK3
    step, each started on both sides from the same input (the oracle's
    previous stage), compared element by element with the oracle."""
    mesh, prob, u0 = inputs.kpp_config(256, 256, 2)
    om = S.OracleMesh(mesh)
    lo32, hi32 = _inward_f32(prob.umin, prob.umax)
    if prec == 1:
        u0 = np.clip(u0.astype(np.float32).astype(np.float64), lo32, hi32)
    dt = S.time_step(om, prob, u0)
    m = cgl.Mesh(mesh)
    g = cgl.State(m, 1, prec)
    g.set_problem(prob)
    g.set_base_state(u0)
    u = u0
    lo, hi = math.pi / 4, 3.5 * math.pi
    for (a, b) in S.SSP3:
        ref, info = S.ssp_stage(om, prob, u, u0, dt, a, b)
        g.set_state(u)
        ginfo = g.stage(dt, a, b)
        out = g.get_state()
        assert ginfo["violations"] == 0 and info["violations"] == 0
        assert out.min() >= lo and out.max() <= hi
        if prec == 0:
            assert _rel(out, ref, 1) <= TOL64, _rel(out, ref, 1)
        else:
            l1 = np.abs(out - ref).sum() / np.abs(ref).sum()
            assert l1 <= 2e-6, l1
        u = ref if prec == 0 else np.clip(ref.astype(np.float32).astype(np.float64), lo32, hi32)
    g.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_stage_mixed_precision(cgl, name):
    """FP32-mixed: exact invariant domain, small L1 error vs the FP64 oracle,
    and element-wise bounds: every nodal value within 2e-6 of the
    component's magnitude, the float-float cell means u^e to 1e-13, dt_e
    within 2e-6 (float speeds rounded up, then inflated by 2^-20), ubar^{e,L}
    and ubar^e within 2e-6 and 5e-6, gamma_e and beta_e within 5e-6 and 5e-5
    absolute (both in [0, 1]).  Measured maxima over these cases on GB300:
    1.5e-7, 5e-15, 1.1e-6, 2e-7, 6e-7, 3e-7, 3e-6."""
    mesh, over = CASES[name]
    prob = _problem(over)
    u, un = _case_state(mesh, prob, 2000 + len(name))
    # the oracle sees exactly the float32-rounded input
    u = u.astype(np.float32).astype(np.float64)
    un = un.astype(np.float32).astype(np.float64)
    if prob.flux != inputs.FLUX_EULER:
        lo32, hi32 = _inward_f32(prob.umin, prob.umax)
        u, un = np.clip(u, lo32, hi32), np.clip(un, lo32, hi32)
    om = S.OracleMesh(mesh)
    dt = 0.5 * S.time_step(om, prob, u)
    ref, info = S.ssp_stage(om, prob, u, un, dt, 0.75, 0.25)
    out, ginfo, f = _gpu_stage(cgl, mesh, prob, u, un, dt, 0.75, 0.25, prec=1)
    assert ginfo["violations"] == 0
    nc = u.shape[0]
    l1 = np.abs(out - ref).reshape(nc, -1).sum(axis=1) / np.abs(ref).reshape(nc, -1).sum(axis=1)
    assert l1.max() <= 5e-6, l1
    assert _rel(out, ref, nc) <= 2e-6, _rel(out, ref, nc)
    assert _rel(f["ue"], info["ue"], nc) <= 1e-13
    assert np.abs(f["dte"] - info["dte"]).max() <= 2e-6 * info["dte"].max()
    assert _rel(f["ubL"], info["ubL"], nc) <= 2e-6
    assert _rel(f["ube"], info["ube"], nc) <= 5e-6
    if prob.mode in (inputs.MODE_WENO, inputs.MODE_WENO_L):
        assert np.abs(f["gamma"] - info["gamma"]).max() <= 5e-6
    assert np.abs(f["beta"] - info["beta"]).max() <= 5e-5
    if prob.flux != inputs.FLUX_EULER:
        assert out.min() >= prob.umin and out.max() <= prob.umax
    else:
        assert np.all(out[0] > 0)

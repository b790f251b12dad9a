"""GPU parity of the pseudo-time-step reduction of the remark after eq.
(dtmaxcell) (option CGL_OPT_DTE_REDUCE, flux limiter off) and of the count
of unlimited averages that leave G: on data where the macrocell dt_e lets
ubar^e leave G (the column pattern), the FP64 form matches the oracle per
stage within 1e-12 (nodal values, the reduced dt_e, ubar^e) and both
counters exactly; the FP32-mixed form stays in G at every node; the option
is refused where it does not apply.
"""
import numpy as np
import pytest

import inputs
from inputs import Mesh, Problem
import oracle.scheme as S

pytestmark = pytest.mark.gpu


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


def _column_pattern(mesh, lo, hi):
    gx = np.arange(mesh.nnx)
    row = np.where(gx % (2 * mesh.p) == mesh.p, hi, lo)
    return np.broadcast_to(row, (mesh.nny, mesh.nnx)).copy()[None]


def _scalar_case(p, mode, opts):
    # 10 x 8 periodic elements, flow along x with a small y component
    mesh = Mesh(10, 8, p, 0.0, 1.25, 0.0, 1.0)
    prob = Problem(flux=inputs.FLUX_ADVECTION, vx=1.0, vy=0.05, umin=0.0, umax=1.0, mode=mode,
                   flux_limiter=S.FL_NONE, options=opts, w_lin=0.2)
    return mesh, prob, _column_pattern(mesh, 0.0, 1.0)


def _euler_case(p, opts):
    mesh = Mesh(10, 6, p, 0.0, 10 / 6, 0.0, 1.0)
    gx = np.arange(mesh.nnx)
    rho = np.broadcast_to(np.where(gx % (2 * p) == p, 1.0, 1e-2), (mesh.nny, mesh.nnx))
    u = inputs.euler_primitive_to_conserved(rho, np.full(rho.shape, 3.0), np.full(rho.shape, 0.1),
                                            np.full(rho.shape, 1e-2))
    prob = Problem(flux=inputs.FLUX_EULER, mode=inputs.MODE_HO, flux_limiter=S.FL_NONE, options=opts)
    return mesh, prob, u


def _gpu_stage(C, mesh, prob, u, dt, prec=0):
    st = C.State(C.Mesh(mesh), u.shape[0], prec)
    st.set_problem(prob)
    st.set_state(u)
    info = st.stage(dt, 0.0, 1.0, raise_on_idp=False)
    out = st.get_state()
    f = {k: st.get_field(v) for k, v in (("dte", C.FIELD_DTE), ("ube", C.FIELD_UBE))}
    st.close()
    return out, info, f


CASES = [("adv_p2_ho", 2, inputs.MODE_HO), ("adv_p3_ho", 3, inputs.MODE_HO),
         ("adv_p2_wenol", 2, inputs.MODE_WENO_L), ("adv_p4_weno", 4, inputs.MODE_WENO)]


@pytest.mark.parametrize("name,p,mode", CASES)
@pytest.mark.parametrize("reduce", [0, 1])
def test_scalar_stage_parity_fp64(cgl, name, p, mode, reduce):
    mesh, prob, u = _scalar_case(p, mode, S.OPT_DTE_REDUCE if reduce else 0)
    om = S.OracleMesh(mesh)
    dt = 0.5 * om.h / (p + 1)
    ref, info = S.ssp_stage(om, prob.as_dict(), u, u, dt, 0.0, 1.0)
    out, ginfo, f = _gpu_stage(cgl, mesh, prob, u, dt)
    assert info["ubar_outside"] > 0
    assert ginfo["ubar_outside"] == info["ubar_outside"]
    assert ginfo["dte_reduced"] == info["dte_reduced"] == (info["ubar_outside"] if reduce else 0)
    assert _rel(out, ref, 1) <= 1e-12, _rel(out, ref, 1)
    assert np.abs(f["dte"] - info["dte"]).max() <= 1e-13 * info["dte"].max()
    assert _rel(f["ube"], info["ube"], 1) <= 1e-12
    if reduce and mode == inputs.MODE_WENO_L:
        assert ginfo["violations"] == 0 and info["violations"] == 0


@pytest.mark.parametrize("p", [2, 3])
def test_euler_stage_parity_fp64(cgl, p):
    mesh, prob, u = _euler_case(p, S.OPT_DTE_REDUCE)
    om = S.OracleMesh(mesh)
    dt = 1e-4 * om.h
    ref, info = S.ssp_stage(om, prob.as_dict(), u, u, dt, 0.0, 1.0)
    out, ginfo, f = _gpu_stage(cgl, mesh, prob, u, dt)
    assert info["ubar_outside"] > 0 and info["dte_reduced"] > 0
    assert ginfo["ubar_outside"] == info["ubar_outside"]
    assert ginfo["dte_reduced"] == info["dte_reduced"]
    assert _rel(out, ref, 4) <= 1e-12, _rel(out, ref, 4)
    assert np.abs(f["dte"] - info["dte"]).max() <= 1e-13 * info["dte"].max()
    ube = f["ube"].reshape(4, -1)
    assert np.all(ube[0] > 0.0)
    assert np.all(ube[0] * ube[3] - 0.5 * (ube[1] ** 2 + ube[2] ** 2) > 0.0)


@pytest.mark.parametrize("p", [2, 3])
def test_mixed_weno_l_stays_in_bounds(cgl, p):
    mesh, prob, u = _scalar_case(p, inputs.MODE_WENO_L, S.OPT_DTE_REDUCE)
    om = S.OracleMesh(mesh)
    dt = 0.5 * om.h / (p + 1)
    ref, info = S.ssp_stage(om, prob.as_dict(), u, u, dt, 0.0, 1.0)
    out, ginfo, f = _gpu_stage(cgl, mesh, prob, u, dt, prec=1)
    assert ginfo["violations"] == 0
    assert ginfo["dte_reduced"] == info["dte_reduced"]
    assert out.min() >= 0.0 and out.max() <= 1.0
    l1 = np.abs(out - ref).sum() / np.abs(ref).sum()
    assert l1 <= 5e-6, l1


def test_option_validation(cgl):
    mesh, prob, u = _scalar_case(2, inputs.MODE_HO, S.OPT_DTE_REDUCE)
    st = cgl.State(cgl.Mesh(mesh), 1, cgl.FP64)
    for bad in (dict(flux_limiter=S.FL_LIMITED), dict(options=S.OPT_DTE_REDUCE | S.OPT_SUBCELL_DT),
                dict(options=S.OPT_DTE_REDUCE | S.OPT_AEC_Q1)):
        p2 = Problem(**{**prob.as_dict(), **bad})
        with pytest.raises(cgl.CglError) as e:
            st.set_problem(p2)
        assert e.value.status == cgl.EINVAL
    st.close()
    st = cgl.State(cgl.Mesh(mesh), 1, cgl.FP32_MIXED)
    st.set_problem(prob)
    st.set_state(u)
    with pytest.raises(cgl.CglError):
        cgl.Batch([st])
    st.close()

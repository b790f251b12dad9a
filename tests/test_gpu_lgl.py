"""GPU parity on LGL meshes (the Lagrange basis at the Legendre-Gauss-Lobatto
points, the spectral-element basis of the paper's concluding section),
FP64 form, through the C ABI, against the oracle (pinned in
tests/test_oracle_lgl.py): every nodal value after one SSP stage within
1e-12 of the component's magnitude and the per-element intermediates (u^e,
dt_e, ubar^{e,L}, ubar^e, gamma_e, beta_e) element by element, for every
flux, mode, flux-limiter setting and boundary condition at p = 2, 3, 4;
three SSP-RK3 steps within 1e-11; the nodal initial data at the LGL points;
and the refusals (FP32-mixed form, subcell bound, eq. (aecQ1)).
"""
import math

import numpy as np
import pytest

import inputs
from inputs import Mesh, Problem
import oracle.scheme as S

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


LGL = inputs.BASIS_LGL
CASES = {
    # name: (mesh, flux, mode, flux limiter)
    "adv_p2_periodic_wenol": (Mesh(13, 11, 2, 0.0, 13 / 11, 0.0, 1.0, basis=LGL), 0, 3, 1),
    "adv_p3_periodic_weno": (Mesh(6, 9, 3, 0.0, 2 / 3, 0.0, 1.0, basis=LGL), 0, 2, 0),
    "adv_p4_periodic_wenol": (Mesh(5, 5, 4, basis=LGL), 0, 3, 1),
    "adv_p2_fixed_wenol": (Mesh(10, 6, 2, 0.0, 5 / 3, 0.0, 1.0, 2, 2, LGL), 0, 3, 1),
    "adv_p2_outflow_ho": (Mesh(7, 8, 2, 0.0, 7 / 8, 0.0, 1.0, 1, 1, LGL), 0, 1, 0),
    "adv_p3_mixedbc_lo_low": (Mesh(8, 5, 3, 0.0, 1.6, 0.0, 1.0, 2, 0, LGL), 0, 0, 2),
    "burgers_p2_periodic_wenol": (Mesh(12, 12, 2, basis=LGL), 1, 3, 1),
    "burgers_p3_fixed_weno": (Mesh(7, 7, 3, 0.0, 1.0, 0.0, 1.0, 2, 2, LGL), 1, 2, 1),
    "kpp_p2_fixed_wenol": (Mesh(16, 16, 2, -2.0, 2.0, -2.5, 1.5, 2, 2, LGL), 2, 3, 1),
    "kpp_p4_outflow_wenol": (Mesh(6, 5, 4, 0.0, 1.2, 0.0, 1.0, 1, 1, LGL), 2, 3, 1),
    "euler_p2_periodic_wenol": (Mesh(9, 8, 2, 0.0, 9 / 8, 0.0, 1.0, basis=LGL), 3, 3, 1),
    "euler_p3_outflow_wenol": (Mesh(8, 6, 3, 0.0, 4 / 3, 0.0, 1.0, 1, 1, LGL), 3, 3, 1),
    "euler_p2_fixed_weno": (Mesh(6, 6, 2, 0.0, 1.0, 0.0, 1.0, 2, 2, LGL), 3, 2, 1),
    "euler_p4_periodic_ho_none": (Mesh(5, 4, 4, 0.0, 1.25, 0.0, 1.0, basis=LGL), 3, 1, 0),
    "adv_p2_1x4_periodic_wenol": (Mesh(1, 4, 2, 0.0, 0.25, 0.0, 1.0, basis=LGL), 0, 3, 1),
    "burgers_p3_1x1_periodic_weno": (Mesh(1, 1, 3, basis=LGL), 1, 2, 1),
}


def _setup(name):
    mesh, flux, mode, fl = CASES[name]
    if flux == inputs.FLUX_EULER:
        prob = Problem(flux=flux, mode=mode, flux_limiter=fl, ubc=(1.0, 0.1, -0.2, 2.5))
        u = inputs.random_euler_state(mesh, 300 + len(name))
        un = inputs.random_euler_state(mesh, 301 + len(name))
    else:
        lo, hi = (0.0, 1.0) if flux != inputs.FLUX_KPP else (math.pi / 4, 3.5 * math.pi)
        prob = Problem(flux=flux, mode=mode, flux_limiter=fl, vx=0.8, vy=-0.45, umin=lo, umax=hi,
                       ubc=(lo, 0, 0, 0), w_lin=0.2)
        u = inputs.random_scalar_state(mesh, 300 + len(name), lo, hi, 0.4)
        un = inputs.random_scalar_state(mesh, 301 + len(name), lo, hi, 0.4)
    return mesh, prob, u, un


def _gpu_stage(C, mesh, prob, u, un, dt, a, b):
    st = C.State(C.Mesh(mesh), u.shape[0], C.FP64)
    st.set_problem(prob)
    st.set_state(u)
    st.set_base_state(un)
    info = st.stage(dt, a, b, raise_on_idp=False)
    out = st.get_state()
    fields = {k: st.get_field(f) for k, f in (("ue", C.FIELD_UE), ("dte", C.FIELD_DTE), ("ubL", C.FIELD_UBL),
                                             ("ube", C.FIELD_UBE), ("beta", C.FIELD_BETA),
                                             ("gamma", C.FIELD_GAMMA))}
    st.close()
    return out, info, fields


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("ab", [(0.0, 1.0), (0.75, 0.25)])
def test_lgl_stage_parity_fp64(cgl, name, ab):
    mesh, prob, u, un = _setup(name)
    om = S.OracleMesh(mesh)
    dt = 0.5 * S.time_step(om, prob, u)
    ref, info = S.ssp_stage(om, prob.as_dict(), u, un, dt, *ab)
    out, ginfo, f = _gpu_stage(cgl, mesh, prob, u, un, dt, *ab)
    nc = u.shape[0]
    assert _rel(out, ref, nc) <= TOL, _rel(out, ref, nc)
    assert _rel(f["ue"], info["ue"], nc) <= 1e-14
    assert np.abs(f["dte"] - info["dte"]).max() <= 1e-13 * info["dte"].max()
    assert _rel(f["ubL"], info["ubL"], nc) <= 1e-13
    assert _rel(f["ube"], info["ube"], nc) <= TOL
    if prob.mode in (inputs.MODE_WENO, inputs.MODE_WENO_L):
        assert np.abs(f["gamma"] - info["gamma"]).max() <= 1e-10
    assert np.abs(f["beta"] - info["beta"]).max() <= 1e-10
    assert ginfo["violations"] == info["violations"]


@pytest.mark.parametrize("name", ["adv_p2_periodic_wenol", "kpp_p2_fixed_wenol", "euler_p3_outflow_wenol"])
def test_lgl_three_steps_fp64(cgl, name):
    mesh, prob, u, _ = _setup(name)
    ref, t_ref, st = S.run(mesh, prob.as_dict(), u, 3)
    g = cgl.State(cgl.Mesh(mesh), u.shape[0], cgl.FP64)
    g.set_problem(prob)
    g.set_state(u)
    g.set_time(0.0)
    info = g.step(3)
    out = g.get_state()
    assert _rel(out, ref, u.shape[0]) <= 1e-11, _rel(out, ref, u.shape[0])
    assert abs(info["t"] - t_ref) <= 1e-14 * t_ref
    assert info["violations"] == 0 and st["violations"] == 0
    g.close()


def test_lgl_nodal_initial_data(cgl):
    """cgl_set_state_nodal evaluates u0 at the LGL points of every element."""
    mesh = Mesh(5, 4, 3, 0.0, 1.25, 0.0, 1.0, 1, 1, LGL)
    g = cgl.State(cgl.Mesh(mesh), 1, cgl.FP64)
    g.set_problem(Problem(flux=0))
    g.set_state_nodal(lambda x, y, c: math.sin(3.0 * x) + y * y)
    X, Y = inputs.node_coords(mesh)
    assert np.abs(g.get_state()[0] - (np.sin(3.0 * X) + Y * Y)).max() <= 1e-15
    g.close()


def test_lgl_refusals(cgl):
    mesh = Mesh(4, 4, 2, basis=LGL)
    with pytest.raises(cgl.CglError) as e:
        cgl.State(cgl.Mesh(mesh), 1, cgl.FP32_MIXED)
    assert e.value.status == cgl.EINVAL
    st = cgl.State(cgl.Mesh(mesh), 1, cgl.FP64)
    for opts, fl in ((S.OPT_SUBCELL_DT, S.FL_NONE), (S.OPT_AEC_Q1, S.FL_LIMITED)):
        with pytest.raises(cgl.CglError) as e:
            st.set_problem(Problem(flux=0, options=opts, flux_limiter=fl))
        assert e.value.status == cgl.EINVAL
    st.close()

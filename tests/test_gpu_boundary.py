"""GPU parity of the per-side boundary data (cgl_set_boundary): reflecting
walls, FIXED and OUTFLOW parts of a side, and a split that moves with the
stage time, as in the double Mach reflection of Sec. 5.4.

FP64: nodal values after one SSP stage (at a given stage time) and after
several SSP-RK3 steps agree with the oracle to 1e-12 (1e-11 over steps), and
the per-element u^e, dt_e, ubar^e to 1e-12.  FP32-mixed: zero invariant-domain
violations and a small L1 error.  The double Mach reflection on the paper's
Q2 mesh is run to t = 0.2 and its density range compared with the one the
paper prints.
"""
import math

import numpy as np
import pytest

import inputs
from inputs import BC_FIXED, BC_OUTFLOW, BC_PERIODIC, BC_WALL, Mesh, Problem, boundary_side
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


def _euler(boundary, **kw):
    p = Problem(flux=inputs.FLUX_EULER, w_lin=1e-3, cfl=0.2, umin=0.0, umax=0.0, boundary=boundary)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _smooth_euler_state(mesh, seed, amp=0.3):
    rng = inputs.SplitMix64(inputs.BASE_SEED + seed)
    X, Y = inputs.node_coords(mesh)
    ph = [rng.uniform(0.0, 2 * math.pi) for _ in range(4)]
    rho = 1.0 + amp * np.sin(2 * math.pi * X + ph[0]) * np.cos(2 * math.pi * Y + ph[1])
    vx = 0.8 * np.sin(2 * math.pi * Y + ph[2])
    vy = 0.6 * np.cos(2 * math.pi * X + ph[3])
    p = 1.0 + 0.2 * np.cos(2 * math.pi * (X + Y))
    return inputs.euler_primitive_to_conserved(rho, vx, vy, p)


def _dmr_perturbed(ny, p, seed):
    """The double Mach reflection data with a smooth density perturbation,
    so that every element sees a non-trivial state."""
    mesh, prob, u0 = inputs.dmr_config(ny, p)
    X, Y = inputs.node_coords(mesh)
    f = 1.0 + 0.05 * np.sin(3.0 * X + seed) * np.cos(5.0 * Y)
    return mesh, prob, u0 * f[None]


def _cases():
    post, pre = inputs.dmr_states()
    walls = {s: boundary_side(BC_WALL) for s in "WESN"}
    chan = {"W": boundary_side(BC_FIXED, post), "E": boundary_side(BC_OUTFLOW),
            "S": boundary_side(BC_WALL), "N": boundary_side(BC_FIXED, post, BC_WALL, post, s0=0.45, s1=3.0)}
    per = {"W": boundary_side(BC_PERIODIC), "E": boundary_side(BC_PERIODIC),
           "S": boundary_side(BC_WALL), "N": boundary_side(BC_OUTFLOW, kind_hi=BC_WALL, s0=0.7)}
    return {
        "dmr_p2": lambda: _dmr_perturbed(5, 2, 1),
        "dmr_p1": lambda: _dmr_perturbed(6, 1, 2),
        "dmr_p3": lambda: _dmr_perturbed(3, 3, 3),
        "box_walls_p3": lambda: (Mesh(7, 5, 3, 0.0, 1.4, 0.0, 1.0, BC_OUTFLOW, BC_OUTFLOW), _euler(walls),
                                 _smooth_euler_state(Mesh(7, 5, 3, 0.0, 1.4, 0.0, 1.0, BC_OUTFLOW, BC_OUTFLOW), 5)),
        "channel_p4": lambda: (Mesh(6, 3, 4, 0.0, 2.0, 0.0, 1.0, BC_OUTFLOW, BC_OUTFLOW), _euler(chan),
                               _smooth_euler_state(Mesh(6, 3, 4, 0.0, 2.0, 0.0, 1.0, BC_OUTFLOW, BC_OUTFLOW), 6)),
        "periodic_x_walls_p2": lambda: (Mesh(9, 4, 2, 0.0, 2.25, 0.0, 1.0, BC_PERIODIC, BC_OUTFLOW), _euler(per),
                                        _smooth_euler_state(Mesh(9, 4, 2, 0.0, 2.25, 0.0, 1.0, BC_PERIODIC,
                                                                 BC_OUTFLOW), 7)),
    }


CASES = _cases()


def _kpp_split():
    """Scalar KPP with a FIXED inflow whose value changes at a moving split."""
    mesh, prob, u0 = inputs.kpp_config(10, 10, 2)
    q = math.pi / 4
    prob.boundary = {"W": boundary_side(BC_FIXED, (q,)), "E": boundary_side(BC_OUTFLOW),
                     "S": boundary_side(BC_FIXED, (q,), BC_FIXED, (3.5 * q,), s0=0.2, s1=4.0),
                     "N": boundary_side(BC_FIXED, (2 * q,), BC_OUTFLOW, s0=0.1)}
    return mesh, prob, u0


def _gpu_stage(C, mesh, prob, u, un, dt, a, b, t, prec=0):
    st = C.State(C.Mesh(mesh), u.shape[0], prec)
    st.set_problem(prob)
    st.set_state(u)
    st.set_base_state(un)
    st.set_time(t)
    info = st.stage(dt, a, b, raise_on_idp=False)
    out = st.get_state()
    f = {k: st.get_field(fid) for k, fid in (("ue", C.FIELD_UE), ("dte", C.FIELD_DTE), ("ube", C.FIELD_UBE))}
    st.close()
    return out, info, f


@pytest.mark.parametrize("name", sorted(CASES) + ["kpp_split"])
@pytest.mark.parametrize("ab", [(0.0, 1.0), (0.75, 0.25)])
def test_stage_parity_fp64(cgl, name, ab):
    mesh, prob, u = _kpp_split() if name == "kpp_split" else CASES[name]()
    un = u.copy()
    t = 0.0123
    om = S.OracleMesh(mesh)
    dt = 0.5 * S.time_step(om, prob.as_dict(), u, t)
    ref, info = S.ssp_stage(om, prob.as_dict(), u, un, dt, ab[0], ab[1], t)
    _, fo = S.fe_stage(om, prob.as_dict(), u, dt, t)
    out, ginfo, f = _gpu_stage(cgl, mesh, prob, u, un, dt, ab[0], ab[1], t)
    nc = u.shape[0]
    assert ginfo["violations"] == info["violations"] == 0
    assert _rel(out, ref, nc) <= 1e-12, _rel(out, ref, nc)
    for k, o in (("ue", fo["ue"]), ("dte", fo["dte"][None]), ("ube", fo["ube"])):
        g = f[k].reshape(o.shape)
        assert np.abs(g - o).max() <= 1e-12 * max(np.abs(o).max(), 1e-300), k


@pytest.mark.parametrize("name", ["dmr_p2", "channel_p4", "kpp_split"])
def test_multi_step_fp64(cgl, name):
    """Several SSP-RK3 steps with device dt: the moving split is evaluated at
    the stage times t, t + dt, t + dt/2 on both sides."""
    mesh, prob, u0 = _kpp_split() if name == "kpp_split" else CASES[name]()
    nsteps = 6
    ref, t_ref, st = S.run(mesh, prob.as_dict(), u0, nsteps)
    g = cgl.State(cgl.Mesh(mesh), u0.shape[0], cgl.FP64)
    g.set_problem(prob)
    g.set_state(u0)
    g.set_time(0.0)
    info = g.step(nsteps, raise_on_idp=False)
    out = g.get_state()
    g.close()
    assert abs(info["t"] - t_ref) <= 1e-13 * t_ref
    assert info["violations"] == 0 and st["violations"] == 0
    assert _rel(out, ref, u0.shape[0]) <= 1e-11, _rel(out, ref, u0.shape[0])


@pytest.mark.parametrize("name", ["dmr_p2", "box_walls_p3", "kpp_split"])
def test_stage_mixed_precision(cgl, name):
    mesh, prob, u = _kpp_split() if name == "kpp_split" else CASES[name]()
    u = u.astype(np.float32).astype(np.float64)
    t = 0.0123
    om = S.OracleMesh(mesh)
    dt = 0.5 * S.time_step(om, prob.as_dict(), u, t)
    ref, _ = S.ssp_stage(om, prob.as_dict(), u, u, dt, 0.0, 1.0, t)
    out, ginfo, _ = _gpu_stage(cgl, mesh, prob, u, u, dt, 0.0, 1.0, t, prec=1)
    nc = u.shape[0]
    assert ginfo["violations"] == 0
    l1 = np.abs(out - ref).reshape(nc, -1).sum(axis=1) / np.abs(ref).reshape(nc, -1).sum(axis=1)
    assert l1.max() <= 5e-6, l1
    if nc == 4:
        assert np.all(out[0] > 0)


def test_boundary_validation(cgl):
    mesh, prob, u0 = inputs.kpp_config(8, 8, 2)
    st = cgl.State(cgl.Mesh(mesh), 1, cgl.FP64)
    st.set_problem(prob)
    bad = {s: boundary_side(BC_WALL) for s in "WESN"}                 # WALL needs Euler
    with pytest.raises(cgl.CglError):
        st.set_boundary(bad)
    bad = {s: boundary_side(BC_FIXED, (99.0,)) for s in "WESN"}       # outside G
    with pytest.raises(cgl.CglError):
        st.set_boundary(bad)
    st.set_boundary(None)
    st.close()
    mesh = Mesh(4, 4, 2, 0.0, 1.0, 0.0, 1.0, BC_PERIODIC, BC_OUTFLOW)
    st = cgl.State(cgl.Mesh(mesh), 4, cgl.FP64)
    st.set_problem(_euler(None))
    bad = {s: boundary_side(BC_WALL) for s in "WESN"}                 # x is periodic
    with pytest.raises(cgl.CglError):
        st.set_boundary(bad)
    bad = {"W": boundary_side(BC_PERIODIC), "E": boundary_side(BC_PERIODIC),
           "S": boundary_side(BC_FIXED, (1.0, 0.0, 0.0, -1.0)), "N": boundary_side(BC_WALL)}  # p < 0
    with pytest.raises(cgl.CglError):
        st.set_boundary(bad)
    st.close()


@pytest.mark.parametrize("p, ny, paper", [(2, 192, (1.338, 22.517)), (1, 384, (1.238, 22.415))])
def test_dmr_paper_mesh(cgl, p, ny, paper):
    """Double Mach reflection to t = 0.2 on the paper's meshes (591,745 nodes),
    FP32-mixed: no invariant-domain violation, positive density, and a
    density range near the one printed with the paper's figure (different
    sensor details and time steps move the extrema by a few per cent)."""
    mesh, prob, u0 = inputs.dmr_config(ny, p)
    st = cgl.State(cgl.Mesh(mesh), 4, cgl.FP32_MIXED)
    st.set_problem(prob)
    st.set_state(u0)
    st.set_time(0.0)
    info = st.step(1 << 30, t_end=0.2, raise_on_idp=False)
    st.close()
    assert abs(info["t"] - 0.2) <= 1e-12
    assert info["violations"] == 0
    rmin, rmax = info["umin"][0], info["umax"][0]
    print(f"DMR Q{p} ny={ny}: steps {info['steps']}, density [{rmin:.4f}, {rmax:.4f}], paper {paper}")
    assert rmin > 0.0
    assert 0.75 * paper[0] <= rmin <= 1.25 * paper[0]
    assert 0.8 * paper[1] <= rmax <= 1.2 * paper[1]

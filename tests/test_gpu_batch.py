"""Batched persistent stage (many uneven instances, one cooperative launch per
SSP stage under a CUDA graph) and its phase form (one launch per phase): every
batched instance must evolve bitwise like the same state stepped alone, tile lengths must not change results,
the invariant domain must hold, the barrier timeout must surface as
CGL_ETIMEOUT without any fault, and the autotuner must persist its choice.
"""
import json
import os

import numpy as np
import pytest

import inputs
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


def _small_instances():
    out = []
    specs = [(5, 1, inputs.FLUX_ADVECTION), (9, 2, inputs.FLUX_BURGERS), (7, 3, inputs.FLUX_ADVECTION),
             (6, 4, inputs.FLUX_BURGERS), (13, 2, inputs.FLUX_ADVECTION), (4, 1, inputs.FLUX_BURGERS),
             (11, 3, inputs.FLUX_BURGERS), (8, 4, inputs.FLUX_ADVECTION), (3, 2, inputs.FLUX_KPP)]
    for k, (n, p, flux) in enumerate(specs):
        mesh = inputs.Mesh(n, n, p)
        prob = inputs.Problem(flux=flux, vx=0.7 - 0.1 * k, vy=0.3 + 0.05 * k, umin=0.0, umax=1.0,
                              w_lin=0.2)
        if flux == inputs.FLUX_KPP:
            prob.umin, prob.umax = 0.2, 3.0
        u0 = inputs.random_scalar_state(mesh, 500 + k, prob.umin, prob.umax, 0.5)
        out.append((mesh, prob, u0))
    return out


def _states(C, cases):
    st = []
    for mesh, prob, u0 in cases:
        m = C.Mesh(mesh)
        s = C.State(m, 1, C.FP32_MIXED)
        s.set_problem(prob)
        s.set_state(u0)
        s.set_time(0.0)
        st.append(s)
    return st


@pytest.mark.parametrize("form", [0, 1])
def test_batch_bitwise_equals_single(cgl, form):
    cases = _small_instances()
    singles = _states(cgl, cases)
    ref = []
    for s in singles:
        s.step(3)
        ref.append(s.get_state())
    states = _states(cgl, cases)
    b = cgl.Batch(states)
    b.set_form(form)
    assert b.form() == form
    viol = b.step(3)
    assert viol == 0
    for s, r in zip(states, ref):
        out = s.get_state()
        assert np.array_equal(out, r)
    # different tile lengths, same results
    states2 = _states(cgl, cases)
    b2 = cgl.Batch(states2)
    b2.set_form(form)
    b2.set_tiles([0, 17, 64, 5, 128])
    b2.step(3)
    for s, r in zip(states2, ref):
        assert np.array_equal(s.get_state(), r)
    info = b.info()
    assert info["grid"] > 0 and info["block"] == 128
    # the steps ran as one captured CUDA graph per step
    assert info["graph"] == 1, cgl.lib().cgl_last_error()


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("mode,fl,kg,ku", [(inputs.MODE_LO, S.FL_LIMITED, 1, 1), (inputs.MODE_WENO, S.FL_NONE, 1, 1),
                                           (inputs.MODE_HO, S.FL_LIMITED, 2, 3), (inputs.MODE_WENO_L, S.FL_LIMITED, 0, 0)])
def test_batch_modes_bitwise_equal_single(cgl, form, mode, fl, kg, ku):
    """Every mode, with and without the flux limiter and with other sweep
    counts (k = 0: the unfused right-hand sides; k > 1: further sweeps),
    in both forms: the batch gives the bits of the states stepped alone (the
    low-order mode skips the residual phases)."""
    cases = _small_instances()
    for _, prob, _ in cases:
        prob.mode, prob.flux_limiter, prob.k_g, prob.k_u = mode, fl, kg, ku
    singles = _states(cgl, cases)
    ref = []
    for s in singles:
        s.step(2)
        ref.append(s.get_state())
    states = _states(cgl, cases)
    b = cgl.Batch(states)
    b.set_form(form)
    assert b.step(2) == 0
    for s, r in zip(states, ref):
        assert np.array_equal(s.get_state(), r)
    assert b.info()["graph"] == 1


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("kg,ku", [(1, 1), (2, 3)])
def test_batch_narrow_periodic_instances(cgl, form, kg, ku):
    """Periodic instances narrower than a node tile and its halo (down to one
    element per side): the fused stencils of the batch wrap every halo node
    into the mesh, and only the tile that owns a node writes it; results
    equal the states stepped alone (whose separate stencils need one wrap)."""
    cases = []
    for k, (nx, ny, p, flux) in enumerate([(1, 4, 2, 0), (1, 1, 1, 1), (5, 1, 3, 0), (2, 3, 4, 1), (3, 1, 1, 0),
                                          (1, 2, 3, 1)]):
        mesh = inputs.Mesh(nx, ny, p, 0.0, nx / ny, 0.0, 1.0)
        prob = inputs.Problem(flux=flux, vx=0.6 - 0.1 * k, vy=0.35 + 0.05 * k, umin=0.0, umax=1.0, w_lin=0.2,
                              k_g=kg, k_u=ku)
        cases.append((mesh, prob, inputs.random_scalar_state(mesh, 700 + k, 0.0, 1.0, 0.5)))
    singles = _states(cgl, cases)
    ref = []
    for s in singles:
        s.step(2)
        ref.append(s.get_state())
    states = _states(cgl, cases)
    b = cgl.Batch(states)
    b.set_form(form)
    assert b.step(2) == 0
    for s, r in zip(states, ref):
        assert np.array_equal(s.get_state(), r)


def test_batch_times_are_per_instance(cgl):
    cases = _small_instances()[:4]
    states = _states(cgl, cases)
    b = cgl.Batch(states)
    b.step(2)
    ts = [s.get_time() for s in states]
    for (mesh, prob, u0), t in zip(cases, ts):
        om = S.OracleMesh(mesh)
        assert t > 0
    assert len(set(ts)) > 1  # own dt per instance


def test_batch_timeout_is_reported(cgl):
    cases = _small_instances()[:3]
    states = _states(cgl, cases)
    b = cgl.Batch(states)
    b.debug(1, 2000)
    with pytest.raises(cgl.CglError) as e:
        b.step(1)
    assert e.value.status == cgl.ETIMEOUT
    # back to normal operation on fresh data
    b.debug(0, 1 << 22)
    for s, (mesh, prob, u0) in zip(states, cases):
        s.set_state(u0)
        s.set_time(0.0)
    assert b.step(1) == 0


def test_batch_autotune_roundtrip(cgl, tmp_path):
    cases = _small_instances()
    states = _states(cgl, cases)
    b = cgl.Batch(states)
    path = str(tmp_path / "tiles.json")
    tiles = b.autotune(1, path)
    d = json.load(open(path))
    assert d["block"] == 128
    assert {int(k): v for k, v in d["tile_elems"].items()} == {p: tiles[p] for p in range(1, 5)}
    b.set_tiles([0, 128, 128, 128, 128])
    b.load_tuning(path)
    assert b.tiles()[1:] == tiles[1:]


def test_config4_batch_full(cgl):
    """The 256-instance workload: zero violations, sampled instances bitwise
    equal to single runs and within the float32 budget of the FP64 oracle
    after one step."""
    cases = inputs.batched_instances()
    states = _states(cgl, cases)
    b = cgl.Batch(states)
    assert b.step(2) == 0
    # the phase form continues the same instances bitwise like the persistent form
    states_b = _states(cgl, cases)
    bb = cgl.Batch(states_b)
    assert bb.step(1) == 0
    bb.set_form(cgl.BATCH_PHASES)
    assert bb.step(1) == 0
    for sa, sb in zip(states, states_b):
        assert np.array_equal(sa.get_state(), sb.get_state())
    picks = {}
    for k, (mesh, prob, u0) in enumerate(cases):
        picks.setdefault((mesh.p, prob.flux), k)
    for (p, flux), k in sorted(picks.items()):
        mesh, prob, u0 = cases[k]
        single = _states(cgl, [cases[k]])[0]
        single.step(2)
        assert np.array_equal(single.get_state(), states[k].get_state()), (p, flux)
        # oracle: one step from the float32-rounded input
        u32 = u0.astype(np.float32).astype(np.float64)
        ref, _, st = S.run(mesh, prob, u32, 1)
        one = _states(cgl, [(mesh, prob, u32)])[0]
        one.step(1)
        out = one.get_state()
        l1 = np.abs(out - ref).sum() / max(np.abs(ref).sum(), 1e-300)
        assert l1 <= 1e-5, (p, flux, l1)
        assert out.min() >= 0.0 and out.max() <= 1.0

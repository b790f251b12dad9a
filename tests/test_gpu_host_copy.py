"""Host copies through the C ABI (cgl_set_state, cgl_set_base_state,
cgl_get_state, and the pipelined cgl_set_state_async, cgl_get_state_async,
cgl_sync), which convert on the device: the FP32-mixed state holds the
float64 input rounded to nearest float and widens it back exactly, the FP64
state holds it unchanged, a non-finite value is refused with
CGL_ENONFINITE and leaves the state as it was, and a caller's output buffer
(pinned or not) receives the state in place."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cgl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_04673_gb300 import build, cgl as C
    build.build()
    return C


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nc", [1, 4])
def test_round_trip_and_nonfinite(cgl, prec, nc):
    import torch
    mesh = inputs.Mesh(37, 29, 3, 0.0, 37 / 29, 0.0, 1.0, inputs.BC_OUTFLOW, inputs.BC_OUTFLOW)
    if nc == 4:
        prob = inputs.Problem(flux=inputs.FLUX_EULER)
        u = inputs.random_euler_state(mesh, 5)
    else:
        prob = inputs.Problem(flux=inputs.FLUX_ADVECTION, umin=-10.0, umax=10.0)
        u = inputs.random_scalar_state(mesh, 6, -3.0, 7.0, 0.0)
    st = cgl.State(cgl.Mesh(mesh), nc, prec)
    st.set_problem(prob)
    st.set_state(u)
    want = u if prec == 0 else u.astype(np.float32).astype(np.float64)
    assert np.array_equal(st.get_state(), want)
    pinned = torch.empty(u.size, dtype=torch.float64, pin_memory=True).numpy().reshape(u.shape)
    out = st.get_state(out=pinned)
    assert out is pinned and np.array_equal(pinned, want)
    bad = u.copy()
    bad[0, 3, 5] = np.nan
    bad[-1, -1, -2] = np.inf
    with pytest.raises(cgl.CglError) as e:
        st.set_state(bad)
    assert e.value.status == cgl.ENONFINITE
    assert np.array_equal(st.get_state(), want)      # unchanged
    with pytest.raises(ValueError):
        st.get_state(out=np.empty(u.size - 1))
    st.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_pipelined_copies_match_synchronous(cgl, prec):
    """cgl_set_state_async / cgl_get_state_async / cgl_sync: a loop that
    feeds the state from two alternating host buffers and reads it back every
    step gives, after sync, exactly the states of the same loop with the
    synchronous calls; a non-finite buffer is refused (state unchanged there,
    CGL_ENONFINITE at sync) and the pipeline continues."""
    import torch
    mesh = inputs.Mesh(40, 30, 2, 0.0, 4 / 3, 0.0, 1.0, inputs.BC_OUTFLOW, inputs.BC_OUTFLOW)
    prob = inputs.Problem(flux=inputs.FLUX_EULER)
    ins = [inputs.random_euler_state(mesh, 70 + k) for k in range(2)]
    if prec == 1:
        ins = [a.astype(np.float32).astype(np.float64) for a in ins]

    def pinned(a):
        t = torch.empty(a.size, dtype=torch.float64, pin_memory=True).numpy().reshape(a.shape)
        t[...] = a
        return t

    # synchronous reference: step k starts from ins[k % 2]
    ref = []
    st = cgl.State(cgl.Mesh(mesh), 4, prec)
    st.set_problem(prob)
    st.set_time(0.0)
    for k in range(4):
        st.set_state(ins[k % 2])
        st.step(1)
        ref.append(st.get_state())
    st.close()
    # pipelined: all copies enqueued, one sync at the end
    h_in = [pinned(a) for a in ins]
    h_out = [pinned(np.zeros_like(ins[0])) for _ in range(4)]
    st = cgl.State(cgl.Mesh(mesh), 4, prec)
    st.set_problem(prob)
    st.set_time(0.0)
    for k in range(4):
        st.set_state_async(h_in[k % 2])
        st.step_async(1)
        st.get_state_async(h_out[k])
    st.sync()
    for k in range(4):
        assert np.array_equal(h_out[k], ref[k]), k
    # a refused buffer: the state keeps its values, the next copy goes through
    bad = pinned(ins[0])
    bad[2, 3, 4] = np.nan
    before = st.get_state()
    st.set_state_async(bad)
    st.get_state_async(h_out[0])
    with pytest.raises(cgl.CglError) as e:
        st.sync()
    assert e.value.status == cgl.ENONFINITE
    assert np.array_equal(h_out[0], before)
    st.set_state_async(h_in[1])
    st.get_state_async(h_out[1])
    st.sync()
    assert np.array_equal(h_out[1], ins[1])
    st.close()

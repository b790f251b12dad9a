"""Host copies through the C ABI (cgl_set_state, cgl_set_base_state,
cgl_get_state), which convert on the device: the FP32-mixed state holds the
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

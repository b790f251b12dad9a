"""Caller-owned state buffer (cgl_state_create_external) and nodal
initialisation (cgl_set_state_nodal), through the C ABI.

A state whose nodal coefficients live in a torch tensor must step bitwise like
a state that owns its buffer, with the tensor holding the result in place;
nodal initialisation must equal the coefficients evaluated at the nodal
points on the host; bad buffers are rejected."""
import math

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
def test_external_buffer_steps_in_place(cgl, prec):
    import torch
    mesh, prob, u0 = inputs.kpp_config(40, 40, 2)
    m = cgl.Mesh(mesh)
    ref = cgl.State(m, 1, prec)
    ref.set_problem(prob)
    ref.set_state(u0)
    ref.set_time(0.0)
    ref.step(3)
    dt = torch.float64 if prec == 0 else torch.float32
    buf = torch.zeros(u0.shape, dtype=dt, device="cuda")
    st = cgl.State(m, 1, prec, u_device=buf.data_ptr(), u_bytes=buf.numel() * buf.element_size())
    st.set_problem(prob)
    st.set_state(u0)
    st.set_time(0.0)
    st.step(3)
    torch.cuda.synchronize()
    out = st.get_state()
    assert np.array_equal(out, ref.get_state())
    assert np.array_equal(buf.double().cpu().numpy(), out)
    st.close()
    ref.close()


def test_external_buffer_rejected(cgl):
    import torch
    mesh, prob, u0 = inputs.kpp_config(16, 16, 2)
    m = cgl.Mesh(mesh)
    small = torch.zeros(10, dtype=torch.float32, device="cuda")
    with pytest.raises(cgl.CglError) as e:
        cgl.State(m, 1, cgl.FP32_MIXED, u_device=small.data_ptr(), u_bytes=40)
    assert e.value.status == cgl.EINVAL
    host = np.zeros(u0.size, dtype=np.float32)
    with pytest.raises(cgl.CglError) as e:
        cgl.State(m, 1, cgl.FP32_MIXED, u_device=host.ctypes.data, u_bytes=host.nbytes)
    assert e.value.status == cgl.EINVAL


def test_nodal_initialisation(cgl):
    mesh = inputs.Mesh(24, 20, 3, -1.0, 2.0, 0.5, 3.0, inputs.BC_OUTFLOW, inputs.BC_OUTFLOW)
    X, Y = inputs.node_coords(mesh)
    f = lambda x, y, c: math.sin(1.3 * x) * math.cos(0.7 * y) + 0.1 * c
    st = cgl.State(cgl.Mesh(mesh), 1, cgl.FP64)
    st.set_state_nodal(f)
    want = np.vectorize(lambda x, y: f(x, y, 0))(X, Y)[None]
    assert np.allclose(st.get_state(), want, rtol=0, atol=1e-14)
    st.close()

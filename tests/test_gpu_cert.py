"""FP32-mixed Euler limiter: the float32 certificate that skips the float64
Appendix-A formula where a factor is certainly 1 must not change a single
bit.  Each workload is stepped twice on the GPU, once as shipped and once
with CGL_OPT_FP64_LIMITER (every factor by the float64 formula); states,
limited averages and slope-limiter factors must be identical."""
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


def _case(which):
    if which == "quadrants_96_q3":
        return inputs.euler_quadrant_config(96, 96, 3)
    if which == "blast_128_q2":
        return inputs.euler_blast_config(128, 128, 2)
    if which == "blast_64_q4":
        return inputs.euler_blast_config(64, 64, 4)
    mesh = inputs.Mesh(40, 24, 2, 0.0, 1.0, 0.0, 0.6, inputs.BC_PERIODIC, inputs.BC_OUTFLOW)
    prob = inputs.Problem(flux=inputs.FLUX_EULER, w_lin=1e-3, umin=0.0, umax=0.0)
    return mesh, prob, inputs.random_euler_state(mesh, 77)


@pytest.mark.parametrize("which", ["quadrants_96_q3", "blast_128_q2", "blast_64_q4", "random_40x24_q2"])
def test_certificate_changes_no_bit(cgl, which):
    mesh, prob, u0 = _case(which)
    out = []
    for opts in (0, cgl.OPT_FP64_LIMITER):
        d = prob.as_dict()
        d["options"] = opts
        st = cgl.State(cgl.Mesh(mesh), 4, cgl.FP32_MIXED)
        st.set_problem(d)
        st.set_state(u0)
        st.set_time(0.0)
        info = st.step(4)
        assert info["violations"] == 0
        out.append((st.get_state(), st.get_field(cgl.FIELD_UBE), st.get_field(cgl.FIELD_BETA)))
        st.close()
    (u_a, ube_a, b_a), (u_b, ube_b, b_b) = out
    assert np.array_equal(u_a, u_b)
    assert np.array_equal(ube_a, ube_b)
    assert np.array_equal(b_a, b_b)
    # the limiter was active somewhere, so both branches ran
    assert b_a.min() < 1.0

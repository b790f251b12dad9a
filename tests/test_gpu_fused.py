"""FP32-mixed, large meshes: the right-hand sides of the g_h and udot solves
and their first Richardson sweeps run fused (one kernel each) from 2^22
nodes on.  The fused kernels must give the same bits as the separate ones
(CGL_OPT_UNFUSED_SWEEPS), for the state and for g_h, r and udot, and stay
within the float32 budget of the FP64 oracle on sampled windows (the window
check of test_gpu_fullsize)."""
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


@pytest.mark.parametrize("which", ["kpp_2048_q2", "advection_1536_q2_kg2", "euler_blast_1024_q2",
                                   "euler_blast_1024_q2_kg2"])
def test_fused_sweeps_change_no_bit(cgl, which):
    if which == "kpp_2048_q2":
        mesh, prob, u0 = inputs.kpp_config(2048, 2048, 2)
    elif which.startswith("euler"):
        # four components per kernel (the headline's fused kernels); outflow
        kw = dict(k_g=2, k_u=3) if which.endswith("kg2") else {}
        mesh, prob, u0 = inputs.euler_blast_config(1024, 1024, 2, **kw)
    else:
        # periodic, two sweeps of each solve (fused first sweep, then a plain one)
        mesh, prob, u0 = inputs.advection_config(1536, 1536, 2, k_g=2, k_u=2)
    assert mesh.nnx * mesh.nny >= 1 << 22
    out = []
    for opts in (0, cgl.OPT_UNFUSED_SWEEPS):
        d = prob.as_dict()
        d["options"] = opts
        st = cgl.State(cgl.Mesh(mesh), u0.shape[0], cgl.FP32_MIXED)
        st.set_problem(d)
        st.set_state(u0)
        st.set_time(0.0)
        info = st.step(2)
        assert info["violations"] == 0
        out.append([st.get_state()] + [st.get_field(f) for f in (cgl.FIELD_GX, cgl.FIELD_GY, cgl.FIELD_R,
                                                                   cgl.FIELD_UDOT)])
        st.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)

"""The no-allocation entry point cgl_gradient_noalloc.

Callers that cannot allocate device memory while they run (host callbacks,
allocator hooks, real-time loops, embedders with fixed buffers) use this
variant of the gradient-projection pass; its scratch is a fixed device array
inside the library.  This test calls it twice in a row through the C ABI on
caller-owned device buffers and compares each result with the existing
path (the g_h field of a state after one stage with k_g = 0), at the FP64
tolerance of the parity tests.  It lives in its own file, collected last.
"""
import numpy as np
import pytest

import inputs

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


def _existing_path(C, mesh, u):
    m = C.Mesh(mesh)
    st = C.State(m, 1, C.FP64)
    prob = inputs.Problem(flux=inputs.FLUX_ADVECTION, mode=inputs.MODE_HO, flux_limiter=0, k_g=0, k_u=0)
    st.set_problem(prob)
    st.set_state(u)
    st.stage(0.0, 0.0, 1.0)
    gx = st.get_field(C.FIELD_GX)
    gy = st.get_field(C.FIELD_GY)
    st.close()
    return np.concatenate([gx, gy])


@pytest.mark.parametrize("p,bc", [(2, inputs.BC_PERIODIC), (3, inputs.BC_FIXED)])
def test_noalloc_matches_existing_path_twice(cgl, p, bc):
    import torch
    mesh = inputs.Mesh(23, 17, p, 0.0, 23 / 17, 0.0, 1.0, bc, bc)
    m = cgl.Mesh(mesh)
    for call, seed in enumerate((31, 32)):
        u = inputs.random_scalar_state(mesh, seed + p)
        ref = _existing_path(cgl, mesh, u)
        u_dev = torch.from_numpy(u.ravel().copy()).cuda()
        g_dev = torch.full((2 * u.size,), float("nan"), dtype=torch.float64, device="cuda")
        cgl.gradient_noalloc(m, u_dev.data_ptr(), g_dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        out = g_dev.cpu().numpy()
        scale = np.abs(ref).max()
        assert np.all(np.isfinite(out)), call
        assert np.abs(out - ref).max() <= TOL * scale, (call, np.abs(out - ref).max() / scale)


def test_noalloc_rejects_oversize(cgl):
    import torch
    mesh = inputs.Mesh(400, 400, 4)          # 400*400*25 > 2^20
    m = cgl.Mesh(mesh)
    u_dev = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(cgl.CglError) as e:
        cgl.gradient_noalloc(m, u_dev.data_ptr(), u_dev.data_ptr())
    assert e.value.status == cgl.EINVAL

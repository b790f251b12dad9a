"""GB300 (sm_103a) implementation of the explicit SSP-RK stage of the
element-based convex-limited CG-WENO scheme (Kuzmin, Hajduk, Vedral,
arXiv 2509.04673), behind the C ABI of include/cgl.h.

`cgl` is the ctypes binding; `build` compiles libcgl.so in-tree."""
from . import cgl  # noqa: F401

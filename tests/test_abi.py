"""C-ABI library checks that need no GPU: it builds/loads, exports every
function include/cgl.h declares, validates arguments, reports the missing
GPU loudly, and its own host tables agree with the oracle's exact ones."""
import os
import re

import numpy as np
import pytest

import inputs
from paper_2509_04673_gb300 import build, cgl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return cgl.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cgl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cgl_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_version(L):
    assert b"sm_103a" in L.cgl_version()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_host_tables_match_oracle(L, p):
    from oracle.tables import tables
    import oracle.scheme as S
    T = cgl.debug_tables(p)
    O = tables(p)
    for k in ("M", "C", "D", "Ep", "Em", "xq", "wq", "Bq", "dBq"):
        assert np.abs(T[k] - O[k]).max() <= 4e-15 * max(1.0, np.abs(O[k]).max()), k
    A2 = S.OracleMesh(inputs.Mesh(2, 2, p)).A2
    assert np.abs(T["A2"] - A2).max() <= 1e-15 * np.abs(A2).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lgl_host_tables_match_oracle(L, p):
    """The library's LGL tables (its own Lobatto points and Lagrange
    polynomials in C++) against the oracle's (numpy), which the closed-form
    Lobatto rules and the product formula pin."""
    from oracle.tables import lgl_tables
    import oracle.scheme as S
    T = cgl.debug_tables(p, cgl.BASIS_LGL)
    O = lgl_tables(p)
    for k in ("M", "C", "D", "Ep", "Em", "xq", "wq", "Bq", "dBq", "wl", "xn"):
        assert np.abs(T[k] - O[k]).max() <= 2e-14 * max(1.0, np.abs(O[k]).max()), k
    A2 = S.OracleMesh(inputs.Mesh(2, 2, p, basis=inputs.BASIS_LGL)).A2
    assert np.abs(T["A2"] - A2).max() <= 1e-13 * np.abs(A2).max()


def test_mesh_validation(L):
    with pytest.raises(cgl.CglError) as e:
        cgl.Mesh(inputs.Mesh(4, 4, 5))
    assert e.value.status == cgl.EINVAL
    with pytest.raises(cgl.CglError):
        cgl.Mesh(inputs.Mesh(4, 3, 2, 0.0, 1.0, 0.0, 1.0))        # not square
    with pytest.raises(cgl.CglError):
        cgl.Mesh(inputs.Mesh(0, 3, 2))
    with pytest.raises(cgl.CglError):
        cgl.Mesh(inputs.Mesh(3, 3, 2, bc_x=7))
    m = cgl.Mesh(inputs.Mesh(5, 3, 3, 0.0, 5.0, 0.0, 3.0, inputs.BC_FIXED, inputs.BC_PERIODIC))
    assert (m.nnx, m.nny, m.E) == (16, 9, 15)
    with pytest.raises(cgl.CglError):
        cgl.Mesh(inputs.Mesh(3, 3, 2, basis=2))
    m = cgl.Mesh(inputs.Mesh(5, 3, 3, 0.0, 5.0, 0.0, 3.0, inputs.BC_FIXED, inputs.BC_PERIODIC, inputs.BASIS_LGL))
    assert (m.nnx, m.nny, m.E) == (16, 9, 15)


def test_problem_defaults(L):
    p = cgl.problem_struct({"flux": cgl.FLUX_EULER})
    assert p.q == 1.0 and p.r == 2.0 and p.w_lin == 1e-3 and p.gamma_gas == 1.4
    assert p.k_g == 1 and p.k_u == 1


def test_no_gpu_fails_loudly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = cgl.Mesh(inputs.Mesh(4, 4, 2))
    with pytest.raises(cgl.CglError) as e:
        cgl.State(m, 1)
    assert e.value.status == cgl.ECUDA


def test_ctypes_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the sizes and field offsets
    that a C compiler gives the structs of include/cgl.h (host only)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"cgl_mesh_desc": cgl.cgl_mesh_desc, "cgl_problem": cgl.cgl_problem,
               "cgl_boundary": cgl.cgl_boundary, "cgl_step_info": cgl.cgl_step_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cgl.h"', "int main(void) {"]
    for name, py in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, key, val = line.split()
            got[(name, key)] = int(val)
    for name, py in structs.items():
        assert got[(name, "size")] == C_sizeof(py), name
        for field, _ in py._fields_:
            assert got[(name, field)] == getattr(py, field).offset, (name, field)


def C_sizeof(t):
    import ctypes
    return ctypes.sizeof(t)

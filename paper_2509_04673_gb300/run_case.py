"""Run one of the synthetic workloads for a few SSP-RK3 steps on cuda:0.

  python -m paper_2509_04673_gb300.run_case --workload kpp --n 1024 --prec 1 --steps 2

Workloads: kpp (f = (sin u, cos u), Q2, fixed pi/4), advection (hump +
slotted disk, Q2, periodic), euler_quadrants (Q3, outflow), euler_blast (Q2,
outflow).  Prints one JSON line with the step diagnostics and the elapsed
device time of the steps (CUDA events on the state's stream)."""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="kpp",
                    choices=["kpp", "advection", "euler_quadrants", "euler_blast"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--p", type=int, default=0, help="degree (0 = the workload's own)")
    ap.add_argument("--prec", type=int, default=1, help="0 FP64, 1 FP32-mixed")
    ap.add_argument("--steps", type=int, default=2)
    a = ap.parse_args()
    import torch
    import inputs
    from paper_2509_04673_gb300 import build, cgl
    build.build()
    if a.workload == "kpp":
        mesh, prob, u0 = inputs.kpp_config(a.n, a.n, a.p or 2)
    elif a.workload == "advection":
        mesh, prob, u0 = inputs.advection_config(a.n, a.n, a.p or 2)
    elif a.workload == "euler_quadrants":
        mesh, prob, u0 = inputs.euler_quadrant_config(a.n, a.n, a.p or 3)
    else:
        mesh, prob, u0 = inputs.euler_blast_config(a.n, a.n, a.p or 2)
    stream = torch.cuda.Stream()
    m = cgl.Mesh(mesh)
    st = cgl.State(m, u0.shape[0], a.prec, stream=stream.cuda_stream)
    st.set_problem(prob)
    st.set_state(u0)
    st.set_time(0.0)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    info = st.step(a.steps, raise_on_idp=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    ndof = u0.size
    info.update(workload=a.workload, n=a.n, p=mesh.p, prec=a.prec, n_dof=ndof,
                ms=ev0.elapsed_time(ev1))
    print(json.dumps(info))
    st.close()
    return 0 if info["violations"] == 0 else 1


if __name__ == "__main__":
    sys.exit(main())

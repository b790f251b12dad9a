"""Run one of the synthetic workloads for a few SSP-RK3 steps on cuda:0.

  python -m paper_2509_04673_gb300.run_case --workload kpp --n 1024 --prec 1 --steps 2

Workloads: kpp (f = (sin u, cos u), Q2, fixed pi/4), advection (hump +
slotted disk, Q2, periodic), euler_quadrants (Q3, outflow), euler_blast (Q2,
outflow).  Prints one JSON line with the step diagnostics and the elapsed
device time of the timed steps (CUDA events on the state's stream, after
--warmup untimed steps).  --profile N adds per-kernel times."""
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
                    choices=["kpp", "advection", "euler_quadrants", "euler_blast", "dmr", "batched"])
    ap.add_argument("--options", type=int, default=0, help="cgl_problem.options bits to add (e.g. 8: eq. (aecQ1))")
    ap.add_argument("--fl", type=int, default=-1, help="flux limiter setting (default: the workload's own)")
    ap.add_argument("--t-end", type=float, default=0.0,
                    help="run to this time instead of a step count (reports the steps taken)")
    ap.add_argument("--autotune", action="store_true", help="batched: tune tile lengths first")
    ap.add_argument("--form", type=int, default=0, help="batched: 0 persistent launches, 1 phase launches")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--p", type=int, default=0, help="degree (0 = the workload's own)")
    ap.add_argument("--prec", type=int, default=1, help="0 FP64, 1 FP32-mixed")
    ap.add_argument("--basis", type=int, default=0, help="0 Bernstein, 1 Lagrange at the LGL points (FP64 only)")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=1, help="untimed steps first (graph capture, caches)")
    ap.add_argument("--profile", type=int, default=0,
                    help="also time every kernel over this many steps (CUDA events per launch)")
    a = ap.parse_args()
    import torch
    import inputs
    from paper_2509_04673_gb300 import build, cgl
    build.build()
    if a.workload == "batched":
        return run_batched(a)
    if a.basis and a.workload not in ("kpp", "euler_quadrants", "euler_blast"):
        raise SystemExit("--basis 1: kpp, euler_quadrants or euler_blast")
    if a.workload == "kpp":
        mesh, prob, u0 = inputs.kpp_config(a.n, a.n, a.p or 2, basis=a.basis)
    elif a.workload == "advection":
        mesh, prob, u0 = inputs.advection_config(a.n, a.n, a.p or 2)
    elif a.workload == "euler_quadrants":
        mesh, prob, u0 = inputs.euler_quadrant_config(a.n, a.n, a.p or 3, basis=a.basis)
    elif a.workload == "dmr":
        # --n is the number of elements across the height (4n x n elements)
        mesh, prob, u0 = inputs.dmr_config(a.n, a.p or 2)
    else:
        mesh, prob, u0 = inputs.euler_blast_config(a.n, a.n, a.p or 2, basis=a.basis)
    prob.options |= a.options
    if a.fl >= 0:
        prob.flux_limiter = a.fl
    stream = torch.cuda.Stream()
    m = cgl.Mesh(mesh)
    st = cgl.State(m, u0.shape[0], a.prec, stream=stream.cuda_stream)
    st.set_problem(prob)
    st.set_state(u0)
    st.set_time(0.0)
    wi = st.step(a.warmup, raise_on_idp=False) if a.warmup > 0 else {"violations": 0}
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    if a.t_end > 0:
        taken = st.step(1 << 30, t_end=a.t_end, raise_on_idp=False)["steps"]
    else:
        st.step_async(a.steps)
        taken = a.steps
    ev1.record(stream)
    torch.cuda.synchronize()
    info = st.step(0, raise_on_idp=False)
    info["steps"] = taken
    info["violations"] = st.counters()["violations"]
    ndof = u0.size
    info.update(workload=a.workload, n=a.n, p=mesh.p, prec=a.prec, basis=a.basis, n_dof=ndof,
                ms=ev0.elapsed_time(ev1),
                dof_stage_per_s=ndof * 3 * info["steps"] / (ev0.elapsed_time(ev1) * 1e-3))
    if a.profile:
        prof = st.profile(a.profile)
        tot = sum(ms for ms, n in prof.values() if n)
        info["kernels"] = {k: {"ms": round(ms, 4), "launches": n, "share": round(ms / tot, 4)}
                           for k, (ms, n) in prof.items() if n}
    print(json.dumps(info))
    st.close()
    return 0 if info["violations"] == 0 else 1


def run_batched(a):
    """The 256-instance batch (uneven sizes 16..128, degrees 1..4, advection
    or Burgers), FP32-mixed, one persistent launch per stage."""
    import torch
    import inputs
    from paper_2509_04673_gb300 import build, cgl
    build.build()
    cases = inputs.batched_instances()
    for _, prob, _ in cases:
        prob.options |= a.options
        if a.fl >= 0:
            prob.flux_limiter = a.fl
    stream = torch.cuda.Stream()
    states = []
    for mesh, prob, u0 in cases:
        st = cgl.State(cgl.Mesh(mesh), 1, cgl.FP32_MIXED, stream=stream.cuda_stream)
        st.set_problem(prob)
        st.set_state(u0)
        st.set_time(0.0)
        states.append(st)
    b = cgl.Batch(states)
    b.set_form(a.form)
    if a.autotune:
        b.autotune(2)
    b.step(1)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step_async(a.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    viol = b.step(0)
    ndof = sum(u0.size for _, _, u0 in cases)
    ms = ev0.elapsed_time(ev1)
    out = dict(workload="batched", instances=len(cases), n_dof=ndof, steps=a.steps, ms=ms,
               dof_stage_per_s=ndof * 3 * a.steps / (ms * 1e-3), violations=viol, tiles=b.tiles(),
               **b.info())
    print(json.dumps(out))
    return 0 if viol == 0 else 1


if __name__ == "__main__":
    sys.exit(main())

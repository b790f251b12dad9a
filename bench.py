#!/usr/bin/env python3
"""Benchmark of the explicit SSP-RK stage of the element-based convex-limited
CG-WENO scheme on one GB300 (per rank), printing one JSON line.

Workload: the KPP problem (f(u) = (sin u, cos u), Sec. 5.3.2 of the paper) on
a 256 x 256 mesh of Bernstein Q2 elements, fixed boundary state pi/4,
WENO-L with the flux limiter.  A step is one SSP-RK3 time step (three
stages of the whole hot path plus the global time-step reduction); the
metric counts DOF-stage updates: N_dof x 3 per step.

  value    FP32-mixed form, inputs resident in HBM, CUDA events around each
           timed step on the state's stream, L2 flushed between timed steps
  fp64     the FP64 plain form, same protocol
  e2e      the same metric through the C ABI with host buffers: set_state
           (host -> device), one step, get_state (device -> host) per step
  roofline dominant kernel of the mixed step: algorithmic bytes per launch
           / its average event-timed duration, against the measured HBM peak
  cpu_baseline  the FP64 oracle, single thread, on a bounded sample

`--impl reference` times the oracle instead (host cores, bounded sample).
Multi-GPU (torchrun): every rank runs an independent replica of the mesh
(no data-path collective; the single-mesh path is replicas only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DOF-stage updates/s (FP32-mixed vs FP64 plain, same GB300); % of HBM roofline"
UNIT = "DOF-stage/s"
WORKLOAD = dict(name="kpp_256x256_q2", nx=256, ny=256, p=2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cgl", choices=["cgl", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=6)
    return ap.parse_args()


def workload():
    import inputs
    return inputs.kpp_config(WORKLOAD["nx"], WORKLOAD["ny"], WORKLOAD["p"])


def n_dof(mesh, nc=1):
    return nc * mesh.nnx * mesh.nny


# --------------------------------------------------------------------------
# oracle timing (cpu_baseline leg and the reference arm)
# --------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import sys, time, json
sys.path.insert(0, {root!r})
import inputs, oracle.scheme as S
mesh, prob, u0 = inputs.kpp_config({nx}, {ny}, {p})
om = S.OracleMesh(mesh)
S.run(om, prob, u0, 1)                      # warm-up (tables, caches)
t0 = time.perf_counter()
u, t, st = S.run(om, prob, u0, {steps})
dt = time.perf_counter() - t0
print(json.dumps(dict(seconds=dt, steps={steps}, violations=st["violations"])))
"""


def time_oracle(steps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, nx=WORKLOAD["nx"], ny=WORKLOAD["ny"], p=WORKLOAD["p"],
                                 steps=steps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    mesh, _, _ = workload()
    res["value"] = n_dof(mesh) * 3 * steps / res["seconds"]
    res["cores"] = 1
    res["sample"] = (f"{steps} SSP-RK3 steps of {WORKLOAD['name']} (FP64 oracle, numpy, "
                     f"single thread), after one warm-up step")
    return res


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# algorithmic bytes per launch of each kernel (minimum traffic of its inputs
# and outputs; element vectors are (p+1)^2 values per element)
# --------------------------------------------------------------------------
def algorithmic_bytes(kernel, mesh, nc, rsz, k_g, k_u):
    """Minimum bytes one launch must move: its inputs read once and its
    outputs written once (element vectors hold (p+1)^2 values per element)."""
    NN = mesh.nnx * mesh.nny
    E = mesh.nx * mesh.ny
    N2 = (mesh.p + 1) ** 2
    d = 8
    b = {
        # u (own and neighbour blocks read once) -> u^e, dt_e (3), ubar^{e,L},
        # gamma, nu (float64), Q (2), f^L (4 nc) (bulk precision), and in the
        # mixed form the float-float means (2 nc floats)
        "k_pre": nc * NN * rsz + (nc + 3 + nc + 2) * E * d + (2 + 4 * nc) * E * rsz
                 + (2 * nc * E * 4 if rsz == 4 else 0),
        # u, g (2 nc), gamma, nu -> element residual
        "k_res_ev": 3 * nc * NN * rsz + 2 * E * d + E * N2 * nc * rsz,
        # u, udot, u^e, dt_e (3), ubar^{e,L} (float64), Q (2), f^L (4 nc),
        # element residual (bulk), float-float means (mixed) -> increments
        # (bulk), ubar^e, beta (float64)
        "k_update_ev": 2 * nc * NN * rsz + (nc + 3 + nc) * E * d + (2 + 4 * nc) * E * rsz
                       + E * N2 * nc * rsz + E * N2 * nc * rsz + (nc + 1) * E * d
                       + (2 * nc * E * 4 if rsz == 4 else 0),
        # increments, u^n, u -> u
        "k_final": E * N2 * nc * rsz + 3 * nc * NN * rsz,
    }
    # u -> b and the lumped g_h (2 nc fields each)
    b["k_grad_rhs"] = nc * NN * rsz + 2 * 2 * nc * NN * rsz
    # element residuals -> r and the lumped udot
    b["k_gather_init"] = E * N2 * nc * rsz + 2 * nc * NN * rsz
    # fused forms (FP32-mixed): u -> g after the first sweep (and b_g when more
    # sweeps follow); element residuals -> r and udot after the first sweep
    b["k_grad_sweep"] = nc * NN * rsz + 2 * nc * NN * rsz * (2 if k_g > 1 else 1)
    b["k_udot_sweep"] = E * N2 * nc * rsz + 2 * nc * NN * rsz
    # FP32-mixed split update: k_facet reads u, ubar^{e,L}, dt_e/h (float64),
    # Q (2), f^L (4 nc) and writes ubar^e (float64) and the facet terms;
    # k_update_ev (k_update_el) reads u, udot, the residuals, ubar^e, the facet
    # terms, the speed sum and the means and writes the increments and beta
    if rsz == 4:
        b["k_facet"] = nc * NN * 4 + (nc + 1) * E * d + (2 + 4 * nc) * E * 4 + nc * E * d + nc * E * 4
        b["k_update_ev"] = (2 * nc * NN * 4 + E * N2 * nc * 4 + nc * E * d + nc * E * 4 + E * 4
                            + 2 * nc * E * 4 + E * N2 * nc * 4 + E * d)
    # x_in, b -> x_out, averaged over the g_h (2 nc) and udot (nc) sweeps
    nvm = (2 * nc * k_g + nc * k_u) / max(1, k_g + k_u)
    b["k_mass_sweep"] = 3 * nvm * NN * rsz
    return b.get(kernel)


def stage_algorithmic_bytes(mesh, nc, rsz, k_g, k_u):
    """Algorithmic bytes of one whole SSP stage: the per-kernel model summed
    over the kernels the library launches for this mesh and precision
    (k_avg for mixed systems; fused first sweeps from 2^22 nodes in the mixed
    form)."""
    NN = mesh.nnx * mesh.nny
    E = mesh.nx * mesh.ny
    N2 = (mesh.p + 1) ** 2
    ab = lambda k: algorithmic_bytes(k, mesh, nc, rsz, k_g, k_u)
    b = ab("k_pre") + ab("k_res_ev") + ab("k_update_ev") + ab("k_final") + (ab("k_facet") if rsz == 4 else 0)
    if rsz == 4 and nc > 1:
        b += nc * NN * 4 + 2 * nc * E * 4
    if rsz == 4 and NN >= (1 << 20):
        # split residual: k_res_w reads u and writes W^e, k_res_s reads W^e
        b += nc * NN * 4 + 2 * E * N2 * nc * 4
    if rsz == 4 and NN >= (1 << 22):
        b += ab("k_grad_sweep") + (k_g - 1) * 3 * 2 * nc * NN * rsz
        b += ab("k_udot_sweep") + (k_u - 1) * 3 * nc * NN * rsz
    else:
        b += ab("k_grad_rhs") + k_g * 3 * 2 * nc * NN * rsz
        b += ab("k_gather_init") + k_u * 3 * nc * NN * rsz
    return b


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


# ncu dram bytes per launch (read + write) of the kernels of one stage of the
# bench workload, from the capture summarised in
# profiles/kpp256_q2_dram_per_launch.md; only kernels unchanged since the
# capture are listed (the g_h and sweep stencils moved to 32 x 8 node tiles on
# this mesh afterwards, so their traffic is reported as null)
NCU_TRAFFIC = {
    ("k_pre", "kpp_256x256_q2"): 1124608,
    ("k_facet", "kpp_256x256_q2"): 3719168,
    ("k_res_ev", "kpp_256x256_q2"): 4270080,
    ("k_gather_init", "kpp_256x256_q2"): 2364416,
    ("k_update_ev", "kpp_256x256_q2"): 6058496,
    ("k_final", "kpp_256x256_q2"): 3418112,
}


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_gpu(args):
    import torch
    from paper_2509_04673_gb300 import build, cgl

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world > 1:
        build.build()
    if dist:
        dist.barrier()
    mesh_d, prob, u0 = workload()
    nd = n_dof(mesh_d)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def make(prec):
        m = cgl.Mesh(mesh_d)
        st = cgl.State(m, 1, prec, stream=stream.cuda_stream)
        st.set_problem(prob)
        st.set_state(u0)
        st.set_time(0.0)
        return m, st

    def timed(st, K, W, sampler=None):
        info = st.step(W)
        assert info["violations"] == 0, info
        c0 = st.counters()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs = []
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            for _ in range(K):
                with torch.cuda.stream(stream):
                    flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                st.step_async(1)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize()
        info = st.counters()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        if dist:
            ms = reduce_over_ranks(ms, dist, "cuda")
            dist.barrier()
        info = {k: info[k] - c0[k] for k in info}
        return ms, info

    K, W = args.steps, args.warmup
    # FP32-mixed (headline) -----------------------------------------------
    m32, st32 = make(cgl.FP32_MIXED)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_index = vis.split(",")[local] if vis else str(local)
    sampler = ClockSampler(smi_index)
    ms32, info32 = timed(st32, K, W, sampler)
    launches = st32.launches_per_step()
    prof = st32.profile(min(K, 20))
    # FP64 plain -----------------------------------------------------------
    m64, st64 = make(cgl.FP64)
    ms64, info64 = timed(st64, K, W)
    prof64 = st64.profile(min(K, 10))
    # end-to-end through the C ABI with host buffers ------------------------
    host_in = torch.empty(u0.size, dtype=torch.float64, pin_memory=True).numpy().reshape(u0.shape)
    host_in[...] = u0
    st32.set_time(0.0)
    for _ in range(2):
        st32.set_state(host_in)
        st32.step(1)
        out = st32.get_state()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        st32.set_state(host_in)
        st32.step(1)
        out = st32.get_state()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:
        e2e_s = reduce_over_ranks(e2e_s, dist, "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # roofline of the dominant kernel of the mixed step ----------------------
    dom = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    tot_ms, n_l = prof[dom]
    avg_ms = tot_ms / n_l
    pr = prob.as_dict()
    alg = algorithmic_bytes(dom, mesh_d, 1, 4, pr["k_g"], pr["k_u"])
    peak, peak_src = load_peaks()
    roof = None
    if alg is not None:
        ach = alg / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 2), "peak": peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": round(ach / peak, 4),
                "traffic": NCU_TRAFFIC.get((dom, WORKLOAD["name"])),
                "algorithmic_bytes_per_launch": alg, "avg_launch_ms": round(avg_ms, 5)}
    # the whole step against the same peak: all kernels' algorithmic bytes
    # per stage over the measured time per stage
    sb = stage_algorithmic_bytes(mesh_d, 1, 4, pr["k_g"], pr["k_u"])
    st_ach = sb * 3 * K / (ms32 * 1e-3) / 1e9
    stage_roof = {"bytes_per_stage": sb, "bytes_per_dof_stage": round(sb / nd, 1), "achieved": round(st_ach, 1),
                  "peak": peak, "unit": "GB/s", "frac": round(st_ach / peak, 4)}
    share = {k: round(v[0] / sum(x[0] for x in prof.values()), 4) for k, v in prof.items() if v[1]}
    share64 = {k: round(v[0] / sum(x[0] for x in prof64.values()), 4) for k, v in prof64.items() if v[1]}
    value = aggregate_rate(nd * 3 * K, ms32, world)
    value64 = aggregate_rate(nd * 3 * K, ms64, world)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            cpu = time_oracle(args.cpu_steps)
            cpu = {"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"], "kind": "oracle",
                   "sample": cpu["sample"]}
        except Exception as ex:  # reported, never silently replaced
            cpu = {"error": str(ex)[:200]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms32 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 bulk + f64 averages/limiters", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "mesh": "256x256 quads", "degree": 2,
                   "flux": "KPP", "bc": "fixed pi/4", "mode": "WENO-L + flux limiter",
                   "n_dof": nd, "dof_stage_per_step": 3 * nd, "precision": "FP32-mixed",
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "fp64_plain": {"value": value64, "ms_per_step": ms64 / K, "kernel_share": share64},
        "mixed_over_fp64": value / value64,
        "kernel_share": share,
        "roofline": roof,
        "step_roofline": stage_roof,
        "cpu_baseline": cpu,
        "e2e": {"value": aggregate_rate(nd * 3 * K, e2e_s * 1e3, world), "unit": UNIT, "h2d_bytes_per_step": nd * 4,
                "d2h_bytes_per_step": nd * 4},
        "gpu_launches": launches * K,
        "clocks": sampler.summary(),
        "violations": int(info32["violations"]) + int(info64["violations"]),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def reduce_over_ranks(ms: float, dist=None, device="cpu") -> float:
    """Max of a per-rank time over all ranks (the job ends with the slowest
    rank); the identity without torch.distributed."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's
    time (replicas of the same workload, weak scaling)."""
    return world * units_per_rank / (ms_max * 1e-3)


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    mesh, _, _ = workload()
    steps = max(1, min(args.steps, 4))
    for _ in range(max(1, args.warmup // 3)):
        time_oracle(1)
    res = time_oracle(steps)
    value = res["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": res["seconds"] / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "mesh": "256x256 quads", "degree": 2, "flux": "KPP",
                   "bc": "fixed pi/4", "mode": "WENO-L + flux limiter", "n_dof": n_dof(mesh),
                   "precision": "FP64 oracle (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                         "sample": res["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

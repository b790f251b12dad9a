#!/usr/bin/env python3
"""Benchmark of the explicit SSP-RK stage of the element-based convex-limited
CG-WENO scheme on one GB300 per rank, printing one JSON line.

Headline workload: the 2D Euler near-vacuum blast (gamma = 1.4, unit square,
2048 x 2048 Bernstein Q2 elements, 67.1 M DOF, outflow boundaries, WENO-L
with the Appendix-A flux and slope limiters) in the FP32-mixed form.  A step
is one SSP-RK3 time step (three stages of the whole hot path and the global
time-step reduction); the metric counts DOF-stage updates, N_dof x 3 per
step.

  value        FP32-mixed, inputs resident in HBM, CUDA events around each
               timed step on the state's stream, L2 flushed between steps
  fp64_plain   the FP64 plain form of the same workload, same protocol
  configs      the Euler four-quadrant problem (512^2 Q3) in both forms and
               the 256-instance batch (one persistent launch per stage
               under a CUDA graph), each with its own rate, method-bytes
               roofline and accuracy
  roofline     the dominant kernel of the mixed step: live duration from
               per-launch CUDA events, algorithmic bytes, and the arithmetic
               roofs (float64 pipe, instruction issue) from its ncu counts
  step_roofline  the whole step against the measured HBM peak with the
               method-inherent bytes per DOF-stage (three global assemblies
               per stage) and, beside it, the implementation's own bytes
  accuracy     one GPU stage from a mid-run state against the FP64 oracle on
               sampled windows: L1 error of the mixed form, max relative
               difference of the FP64 form, FP64 mass drift over the timed
               steps, invariant-domain violations
  e2e          the same metric through the C ABI with host buffers
  cpu_baseline the FP64 oracle on a bounded sample (windows of the same
               workload), one thread and all host cores

`--impl reference` times the oracle instead (host cores, bounded sample).
Multi-GPU (torchrun): every rank runs an independent replica of the single
meshes (no data-path collective) and its share of the batch's instances.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DOF-stage updates/s (FP32-mixed vs FP64 plain, same GB300); % of HBM roofline"
UNIT = "DOF-stage/s"
HEADLINE = "euler_blast_2048x2048_q2"
QUADRANTS = "euler_quadrants_512x512_q3"
QUADRANTS_LGL = "euler_quadrants_512x512_q3_lgl"
BATCH = "batched_256_instances"
# oracle windows: W x W elements, compared on the nodes of the elements at
# least MARGIN elements inside the window (a stage reads at most 5 elements
# away: sensor, g_h and udot sweeps, flux limiter)
WIN = 128
MARGIN = 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cgl", choices=["cgl", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-headline", action="store_true", help="skip the other configurations")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def workload(name):
    import inputs
    if name == HEADLINE:
        return inputs.euler_blast_config(2048, 2048, 2)
    if name == QUADRANTS:
        return inputs.euler_quadrant_config(512, 512, 3)
    if name == QUADRANTS_LGL:
        return inputs.euler_quadrant_config(512, 512, 3, basis=inputs.BASIS_LGL)
    raise ValueError(name)


def describe(name):
    return {
        HEADLINE: {"workload": HEADLINE, "mesh": "2048x2048 quads", "degree": 2, "flux": "Euler (gamma 1.4)",
                   "problem": "near-vacuum blast: rho 1, v 0, p 1e-6, energy 0.25 in the central 2x2 cells",
                   "bc": "outflow", "mode": "WENO-L + flux limiter (Appendix A)"},
        QUADRANTS: {"workload": QUADRANTS, "mesh": "512x512 quads", "degree": 3, "flux": "Euler (gamma 1.4)",
                    "problem": "four-quadrant Riemann data from a seeded draw", "bc": "outflow",
                    "mode": "WENO-L + flux limiter (Appendix A)"},
    }[name]


# --------------------------------------------------------------------------
# bytes per DOF-stage
# --------------------------------------------------------------------------
def method_bytes_per_dof_stage(p, rsz, k_g, k_u):
    """Method-inherent bytes per DOF-stage: the minimum nodal traffic of the
    three global assemblies of a stage (g_h: read u, write g; udot: read u,
    g, write udot; SSP update: read u, g, udot, u^n (2 of 3 stages), write
    u) = 12.67 words, plus 4 words per Richardson sweep of g and 2 per sweep
    of udot, in the bulk precision (rsz bytes), plus the per-element float64
    scalars (6 words per element and component, p^2 DOF per element and
    component)."""
    words = 3.0 + 4.0 + (5.0 + 2.0 / 3.0) + 4.0 * k_g + 2.0 * k_u
    return words * rsz + 6.0 * 8.0 / (p * p)


def impl_algorithmic_bytes(kernel, mesh, nc, rsz, k_g, k_u):
    """The implementation's bytes per launch: each kernel's inputs read once
    and its outputs written once (element vectors hold (p+1)^2 values per
    element)."""
    NN = mesh.nnx * mesh.nny
    E = mesh.nx * mesh.ny
    N2 = (mesh.p + 1) ** 2
    d = 8
    mixed = rsz == 4
    b = {
        # reads u; writes u^e, dt_e (3), ubar^{e,L}, gamma, nu (float64), f^L
        # (4 nc), the scalar capacities Q (2) and, mixed scalars, the float
        # speed sum and the float-float mean
        "k_pre": (nc * NN * rsz + (nc + 3 + nc + 2) * E * d + 4 * nc * E * rsz + (2 * E * rsz if nc == 1 else 0)
                  + (3 * E * 4 if mixed else 0)),
        "k_avg": nc * NN * 4 + 2 * nc * E * 4,
        "k_sens": nc * NN * rsz + 2 * E * d,
        "k_res_ev": 3 * nc * NN * rsz + 2 * E * d + E * N2 * nc * rsz,
        "k_res_w": nc * NN * rsz + E * N2 * nc * rsz,
        "k_update_ev": 2 * nc * NN * rsz + (nc + 3 + nc) * E * d + (2 + 4 * nc) * E * rsz
                       + 2 * E * N2 * nc * rsz + (nc + 1) * E * d,
        "k_final": E * N2 * nc * rsz + 3 * nc * NN * rsz,
        "k_grad_rhs": nc * NN * rsz + 2 * 2 * nc * NN * rsz,
        "k_gather_init": E * N2 * nc * rsz + 2 * nc * NN * rsz,
        "k_grad_sweep": nc * NN * rsz + 2 * nc * NN * rsz * (2 if k_g > 1 else 1),
        "k_udot_sweep": E * N2 * nc * rsz + 2 * nc * NN * rsz,
        "k_mass_sweep": 3 * ((2 * nc * k_g + nc * k_u) / max(1, k_g + k_u)) * NN * rsz,
    }
    if mixed and nc > 1:
        # systems: k_avg also writes the flux of each mean and 5 speed parts
        # (2 nc + 5 floats per cell); k_pre_lo reads those and the
        # float-float means and writes u^e, dt_e (3), ubar^{e,L} (float64),
        # f^L (4 nc), the float speed sum and ubar^{e,L} copies; k_sens reads
        # u and writes gamma, nu
        b["k_avg"] = nc * NN * 4 + 2 * nc * E * 4 + (2 * nc + 5) * E * 4
        b["k_pre"] = ((2 * nc + 2 * nc + 5) * E * 4 + (nc + 3 + nc) * E * d + 4 * nc * E * 4
                      + (1 + nc) * E * 4)
    if mixed:
        # k_res_s: u, g, gamma, nu, W^e -> element residual; k_facet: u,
        # ubar^{e,L}, dt_e/h, Q, f^L -> ubar^e, facet terms; k_update_el: u,
        # udot, residuals, ubar^e, facet terms, speed sum, means -> increments, beta
        # (scalars from 2^20 nodes; systems keep the single k_res_ev)
        b["k_res_ev"] = (3 * nc * NN * 4 + 2 * E * d + 2 * E * N2 * nc * 4 if (NN >= (1 << 20) and nc == 1)
                         else b["k_res_ev"])
        b["k_facet"] = nc * NN * 4 + (nc + 1) * E * d + (2 + 4 * nc) * E * 4 + nc * E * d + nc * E * 4
        b["k_update_ev"] = (2 * nc * NN * 4 + E * N2 * nc * 4 + nc * E * d + nc * E * 4 + E * 4
                            + 2 * nc * E * 4 + E * N2 * nc * 4 + E * d)
    return b.get(kernel)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


# Per-element ncu counts of the FP32-mixed kernels (one launch of the
# workload's mesh, divided by its elements; profiles/ holds the captures):
# warp instructions issued, float64 thread instructions (dadd + dmul + dfma,
# dfma counted twice as flops) and DRAM bytes read + written.  None where the
# kernel changed after the capture.
NCU_PER_ELEMENT = {
    # profiles/euler_blast_1024_q2_kernel_counts.md and, for the shared-memory wavefronts,
    # profiles/euler_blast_1024_q2_shared_wavefronts.md (kernel names as cgl_profile reports them:
    # k_pre is k_pre_lo and k_update_ev is k_update_el in this FP32-mixed Euler stage)
    ("k_sens", HEADLINE): {"warp_inst": 195.41, "fp64_flops": 0.0, "dram_bytes": 69.6, "shared_wavefronts": 3.38},
    ("k_grad_sweep", HEADLINE): {"warp_inst": 142.62, "fp64_flops": 0.0, "dram_bytes": 138.1, "shared_wavefronts": 46.82},
    ("k_res_ev", HEADLINE): {"warp_inst": 146.29, "fp64_flops": 0.0, "dram_bytes": 403.1, "shared_wavefronts": 0.12},
    ("k_update_ev", HEADLINE): {"warp_inst": 70.4, "fp64_flops": 4.024, "dram_bytes": 545.6, "shared_wavefronts": 0.16},
    ("k_facet", HEADLINE): {"warp_inst": 79.32, "fp64_flops": 12.051, "dram_bytes": 248.4, "shared_wavefronts": 0.06},
    ("k_pre", HEADLINE): {"warp_inst": 49.71, "fp64_flops": 22.0, "dram_bytes": 218.2, "shared_wavefronts": 0.15},
    ("k_udot_sweep", HEADLINE): {"warp_inst": 81.14, "fp64_flops": 0.0, "dram_bytes": 233.1, "shared_wavefronts": 13.66},
    ("k_final", HEADLINE): {"warp_inst": 37.17, "fp64_flops": 0.0, "dram_bytes": 316.9, "shared_wavefronts": 0.66},
    ("k_avg", HEADLINE): {"warp_inst": 21.69, "fp64_flops": 0.0, "dram_bytes": 98.4, "shared_wavefronts": 0.06},
}

SM_COUNT_GB300 = 152
ISSUE_PER_SM_CLK = 4  # one warp instruction per clock on each of the 4 SM sub-partitions


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


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass


# --------------------------------------------------------------------------
# multi-rank helpers
# --------------------------------------------------------------------------
def reduce_over_ranks(ms: float, dist=None, device="cpu") -> float:
    """Max of a per-rank time over all ranks (the job ends with the slowest
    rank); the identity without torch.distributed."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v: float, dist=None, device="cpu") -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_rate(units_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's
    time (replicas of the same workload, weak scaling)."""
    return world * units_per_rank / (ms_max * 1e-3)


# --------------------------------------------------------------------------
# oracle sample: windows of a workload (input slicing only; the stage runs in
# the oracle)
# --------------------------------------------------------------------------
def window_origins(nx, ny, count):
    """count window origins: the centre, the four corners, then a fixed
    spread over the mesh."""
    w = WIN
    cx, cy = (nx - w) // 2, (ny - w) // 2
    pts = [(cx, cy), (0, 0), (nx - w, 0), (0, ny - w), (nx - w, ny - w)]
    k = 1
    while len(pts) < count:
        fx = ((k * 0.618034) % 1.0)
        fy = ((k * 0.381966 + 0.5) % 1.0)
        pts.append((int(fx * (nx - w)), int(fy * (ny - w))))
        k += 1
    return pts[:count]


def cut_window(mesh, u, ex0, ey0):
    """Sub-mesh of WIN x WIN elements at (ex0, ey0) of a non-periodic mesh
    and its coefficients."""
    import inputs
    p, h, w = mesh.p, mesh.h, WIN
    sub = inputs.Mesh(w, w, p, mesh.x0 + ex0 * h, mesh.x0 + (ex0 + w) * h, mesh.y0 + ey0 * h,
                      mesh.y0 + (ey0 + w) * h, mesh.bc_x, mesh.bc_y)
    return sub, u[:, ey0 * p:(ey0 + w) * p + 1, ex0 * p:(ex0 + w) * p + 1].copy()


def compare_region(mesh, ex0, ey0):
    """Node slices (within a window) of the elements at least MARGIN
    elements from the window's cut sides (a side on the true boundary keeps
    its elements)."""
    p, w = mesh.p, WIN
    lo_x = 0 if ex0 == 0 else MARGIN
    lo_y = 0 if ey0 == 0 else MARGIN
    hi_x = w if ex0 + w == mesh.nx else w - MARGIN
    hi_y = w if ey0 + w == mesh.ny else w - MARGIN
    return slice(lo_y * p, hi_y * p + 1), slice(lo_x * p, hi_x * p + 1)


def _oracle_window_stage(args):
    """One oracle SSP stage (a = 0, b = 1) on one window; runs in a worker."""
    sub_d, prob_d, us, dt = args
    import inputs
    import oracle.scheme as S
    sub = inputs.Mesh(**sub_d)
    t0 = time.perf_counter()
    ref, info = S.ssp_stage(sub, prob_d, us, us, dt, 0.0, 1.0)
    return ref, time.perf_counter() - t0, int(info["violations"])


def _worker_init():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import oracle.scheme  # noqa: F401  (import before timing)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample_main(path):
    """--oracle-sample: load the windows written by the GPU arm, run the
    oracle stage on each (one thread, then a spawn pool over all host
    cores), compare with the GPU outputs and print JSON."""
    import multiprocessing as mp
    _worker_init()
    d = np.load(path, allow_pickle=True)
    spec = json.loads(str(d["spec"]))
    out = {}
    for name, ws in spec.items():
        jobs = []
        for k, w in enumerate(ws["windows"]):
            jobs.append((w["mesh"], ws["prob"], d[f"{name}_in_{k}"], ws["dt"]))
        dofs = sum(int(np.prod(d[f"{name}_in_{k}"].shape)) for k in range(len(jobs)))
        # single thread, in this process
        t0 = time.perf_counter()
        refs = []
        viol = 0
        for j in jobs:
            r, _, v = _oracle_window_stage(j)
            refs.append(r)
            viol += v
        t1 = time.perf_counter() - t0
        res = {"dof_stage": dofs, "seconds_1thread": t1, "rate_1thread": dofs / t1, "oracle_violations": viol}
        # all host cores: one spawn worker per core, warmed up before timing
        if ws.get("all_core", False):
            cores = min(host_cores(), len(jobs))
            ctx = mp.get_context("spawn")
            with ctx.Pool(cores, initializer=_worker_init) as pool:
                pool.map(_oracle_window_stage, [jobs[0]] * cores)
                t0 = time.perf_counter()
                pool.map(_oracle_window_stage, jobs)
                tall = time.perf_counter() - t0
            res.update(cores=cores, seconds_all=tall, rate_all=dofs / tall)
        # accuracy of the GPU outputs on the compared nodes
        for form in ("mixed", "fp64"):
            key0 = f"{name}_{form}_0"
            if key0 not in d:
                continue
            l1n = l1d = 0.0
            worst = 0.0
            nc = refs[0].shape[0]
            gmax = np.array(ws["scale"], dtype=np.float64)
            for k, w in enumerate(ws["windows"]):
                sy, sx = slice(*w["cmp"][0]), slice(*w["cmp"][1])
                r = refs[k][:, sy, sx]
                g = d[f"{name}_{form}_{k}"][:, sy, sx]
                l1n += np.abs(g - r).sum()
                l1d += np.abs(r).sum()
                worst = max(worst, float((np.abs(g - r).reshape(nc, -1).max(axis=1) / gmax).max()))
            res[f"{form}_l1_vs_oracle"] = l1n / l1d
            res[f"{form}_max_rel_vs_oracle"] = worst
        out[name] = res
    print(json.dumps(out))


def run_oracle_sample(spec, arrays):
    """Write the windows to a temporary file and run the oracle leg in a
    subprocess (its own interpreter: the GPU process never imports the
    oracle)."""
    with tempfile.TemporaryDirectory() as tdir:
        path = os.path.join(tdir, "windows.npz")
        np.savez(path, spec=json.dumps(spec), **arrays)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", path],
                           capture_output=True, text=True, env=env)
        if r.returncode != 0:
            raise RuntimeError(r.stderr[-2000:])
        return json.loads(r.stdout.strip().splitlines()[-1])


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
    K, W = args.steps, max(3, args.warmup)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_index = vis.split(",")[local] if vis else str(local)
    peaks_live = cgl.measure_peaks()
    hbm_peak, hbm_src = load_peaks()

    def sync_all():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def make(mesh_d, prob, u0, prec):
        m = cgl.Mesh(mesh_d)
        st = cgl.State(m, u0.shape[0], prec, stream=stream.cuda_stream)
        st.set_problem(prob)
        st.set_state(u0)
        st.set_time(0.0)
        return m, st

    def timed(step_fn, K, sampler=None):
        sync_all()
        evs = []
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            for _ in range(K):
                with torch.cuda.stream(stream):
                    flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step_fn()
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return reduce_over_ranks(ms, dist, "cuda")

    def run_single(name, prec, sampler=None, profile_steps=0):
        mesh_d, prob, u0 = workload(name)
        m, st = make(mesh_d, prob, u0, prec)
        info = st.step(W)
        assert info["violations"] == 0, info
        before = st.step(0)
        ms = timed(lambda: st.step_async(1), K, sampler)
        after = st.step(0)
        viol = st.counters()["violations"]
        prof = st.profile(profile_steps) if profile_steps else None
        return dict(mesh=mesh_d, prob=prob, u0=u0, m=m, st=st, ms=ms, before=before, after=after,
                    violations=viol, prof=prof, launches=st.launches_per_step())

    def drift(before, after, comps):
        return {c: abs(after["mass"][i] - before["mass"][i]) / abs(before["mass"][i]) for i, c in comps}

    def roofline_entry(name, r, rsz):
        mesh_d = r["mesh"]
        nd = mesh_d.nnx * mesh_d.nny * r["u0"].shape[0]
        pr = r["prob"].as_dict()
        bm = method_bytes_per_dof_stage(mesh_d.p, rsz, pr["k_g"], pr["k_u"])
        rate = aggregate_rate(nd * 3 * K, r["ms"], world)
        ach = rate / world * bm / 1e9
        return {"bytes_per_dof_stage": round(bm, 2),
                "formula": "(12.67 + 4 k_g + 2 k_u) words x bulk bytes + 48 / p^2 B of float64 per-element scalars",
                "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                "peak_source": hbm_src}

    def impl_bytes_entry(r, rsz, meth):
        mesh_d = r["mesh"]
        nc = r["u0"].shape[0]
        pr = r["prob"].as_dict()
        prof = r["prof"] or {}
        tot = 0.0
        for k, (ms_k, n_k) in prof.items():
            if n_k:
                b = impl_algorithmic_bytes(k, mesh_d, nc, rsz, pr["k_g"], pr["k_u"])
                tot += (b or 0.0) * n_k
        steps_prof = max(1, r.get("prof_steps", 1))
        nd = mesh_d.nnx * mesh_d.nny * nc
        per = tot / (steps_prof * 3 * nd)
        return {"bytes_per_dof_stage": round(per, 1), "over_method": round(per / meth, 2)}

    out = {}
    # ---- headline: Euler blast 2048^2 Q2, FP32-mixed ----------------------
    sampler = ClockSampler(smi_index)
    PROF_STEPS = 3
    h32 = run_single(HEADLINE, cgl.FP32_MIXED, sampler, profile_steps=PROF_STEPS)
    h32["prof_steps"] = PROF_STEPS
    mesh_h = h32["mesh"]
    nc_h = h32["u0"].shape[0]
    nd_h = mesh_h.nnx * mesh_h.nny * nc_h
    value = aggregate_rate(nd_h * 3 * K, h32["ms"], world)
    # ---- FP64 plain of the same workload ----------------------------------
    h64 = run_single(HEADLINE, cgl.FP64, profile_steps=1)
    h64["prof_steps"] = 1
    value64 = aggregate_rate(nd_h * 3 * K, h64["ms"], world)
    # ---- e2e through the C ABI with host buffers --------------------------
    st = h32["st"]
    host_in = torch.empty(h32["u0"].size, dtype=torch.float64, pin_memory=True).numpy().reshape(h32["u0"].shape)
    host_out = torch.empty(h32["u0"].size, dtype=torch.float64, pin_memory=True).numpy().reshape(h32["u0"].shape)
    host_in[...] = h32["u0"]
    st.set_time(0.0)
    for _ in range(2):
        st.set_state(host_in)
        st.step(1)
        res = st.get_state(out=host_out)
    sync_all()
    # synchronous calls: copy in, step (with its diagnostics), copy out
    t0 = time.perf_counter()
    for _ in range(K):
        st.set_state(host_in)
        st.step(1)
        res = st.get_state(out=host_out)
    torch.cuda.synchronize()
    e2e_sync_s = reduce_over_ranks(time.perf_counter() - t0, dist, "cuda")
    del res
    # pipelined calls (cgl_set_state_async / cgl_step_async /
    # cgl_get_state_async, one cgl_sync at the end): every step still copies
    # its input in and its result out, on copy streams that overlap the
    # neighbouring steps
    for _ in range(2):
        st.set_state_async(host_in)
        st.step_async(1)
        st.get_state_async(host_out)
    st.sync()
    sync_all()
    t0 = time.perf_counter()
    for _ in range(K):
        st.set_state_async(host_in)
        st.step_async(1)
        st.get_state_async(host_out)
    st.sync()
    e2e_s = reduce_over_ranks(time.perf_counter() - t0, dist, "cuda")
    # ---- accuracy sample of the headline: one stage from a mid-run state ---
    win_spec, win_arrays = {}, {}

    def accuracy_sample(name, r32, r64, count, all_core):
        mesh_d, prob = r32["mesh"], r32["prob"]
        st32, st64 = r32["st"], r64["st"]
        st32.set_state(r32["u0"])
        st32.set_time(0.0)
        st32.step(W)
        u_mid = st32.get_state()
        dt = st32.time_step()
        st32.stage(dt, 0.0, 1.0)
        o32 = st32.get_state()
        st64.set_state(u_mid)
        st64.stage(dt, 0.0, 1.0)
        o64 = st64.get_state()
        nc = u_mid.shape[0]
        wins = []
        for k, (ex0, ey0) in enumerate(window_origins(mesh_d.nx, mesh_d.ny, count)):
            sub, us = cut_window(mesh_d, u_mid, ex0, ey0)
            sy, sx = compare_region(mesh_d, ex0, ey0)
            wins.append({"mesh": sub.as_dict(), "cmp": [[sy.start, sy.stop], [sx.start, sx.stop]]})
            win_arrays[f"{name}_in_{k}"] = us
            p = mesh_d.p
            sl = (slice(None), slice(ey0 * p, (ey0 + WIN) * p + 1), slice(ex0 * p, (ex0 + WIN) * p + 1))
            win_arrays[f"{name}_mixed_{k}"] = o32[sl]
            win_arrays[f"{name}_fp64_{k}"] = o64[sl]
        pd = prob.as_dict()
        pd["boundary"] = None
        win_spec[name] = {"prob": pd, "dt": dt, "windows": wins, "all_core": all_core,
                          "scale": np.maximum(np.abs(o64).reshape(nc, -1).max(axis=1), 1e-300).tolist()}

    do_extra = rank == 0
    if do_extra:
        accuracy_sample(HEADLINE, h32, h64, 16, True)
    # ---- config 3: Euler four quadrants 512^2 Q3 --------------------------
    cfg = {}
    if not args.only_headline:
        q32 = run_single(QUADRANTS, cgl.FP32_MIXED, profile_steps=PROF_STEPS)
        q32["prof_steps"] = PROF_STEPS
        q64 = run_single(QUADRANTS, cgl.FP64)
        # the same data on the LGL basis (nodal values at the Lobatto points),
        # FP64 form
        ql = run_single(QUADRANTS_LGL, cgl.FP64)
        mq = q32["mesh"]
        nd_q = mq.nnx * mq.nny * 4
        meth_q = roofline_entry(QUADRANTS, q32, 4)
        cfg[QUADRANTS] = {
            "config": describe(QUADRANTS), "n_dof": nd_q,
            "value": aggregate_rate(nd_q * 3 * K, q32["ms"], world), "ms_per_step": q32["ms"] / K,
            "fp64_plain": {"value": aggregate_rate(nd_q * 3 * K, q64["ms"], world), "ms_per_step": q64["ms"] / K,
                           "roofline": roofline_entry(QUADRANTS, q64, 8)},
            "roofline": meth_q,
            "impl_bytes": impl_bytes_entry(q32, 4, meth_q["bytes_per_dof_stage"]),
            "lgl_fp64": {"basis": "Lagrange at the Legendre-Gauss-Lobatto points (nodal values), same data",
                         "value": aggregate_rate(nd_q * 3 * K, ql["ms"], world), "ms_per_step": ql["ms"] / K,
                         "over_bernstein_fp64": q64["ms"] / ql["ms"], "violations": ql["violations"],
                         "roofline": roofline_entry(QUADRANTS_LGL, ql, 8)},
            "violations": q32["violations"] + q64["violations"] + ql["violations"],
            # outflow boundaries carry mass out: the mixed form's FP64 mass sums
            # against the FP64 form's after the same W + K steps
            "mass_vs_fp64": {c: abs(q32["after"]["mass"][i] - q64["after"]["mass"][i]) / abs(q64["after"]["mass"][i])
                             for i, c in ((0, "rho"), (3, "E"))},
            "kernel_share": _share(q32["prof"]),
        }
        if do_extra:
            accuracy_sample(QUADRANTS, q32, q64, 6, False)
        for r in (q32, q64, ql):
            r["st"].close()
        # ---- config 4: the batch -------------------------------------------
        cfg[BATCH] = run_batch(cgl, torch, stream, flush, K, W, world, rank, dist, timed, hbm_peak, hbm_src)
    # ---- the oracle: accuracy of the sampled windows and its own timing -----
    acc = None
    cpu = None
    if do_extra and not args.no_cpu_baseline:
        try:
            acc = run_oracle_sample(win_spec, win_arrays)
        except Exception as ex:  # reported, never silently replaced
            acc = {"error": str(ex)[-300:]}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # ---- roofline of the dominant kernel -------------------------------------
    prof = h32["prof"]
    pr = h32["prob"].as_dict()
    dom = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    tot_ms, n_l = prof[dom]
    avg_ms = tot_ms / n_l
    alg = impl_algorithmic_bytes(dom, mesh_h, nc_h, 4, pr["k_g"], pr["k_u"])
    E_h = mesh_h.nx * mesh_h.ny
    roof = {"kernel": dom, "avg_launch_ms": round(avg_ms, 5),
            "timing": "CUDA events around each launch of a non-graph replay serialised on one stream "
                      f"({PROF_STEPS} steps); launches of 0.1 ms or more, so the event gaps are small"}
    ncu = NCU_PER_ELEMENT.get((dom, HEADLINE))
    clk = sampler.summary()
    sm_hz = (clk["sm_mhz"] or 2070.0) * 1e6
    roofs = {}
    if alg is not None:
        ach = alg / (avg_ms * 1e-3) / 1e9
        roofs["hbm"] = {"achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                        "frac": round(ach / hbm_peak, 4), "algorithmic_bytes_per_launch": alg,
                        "peak_source": hbm_src}
    traffic = None
    if ncu:
        traffic = ncu.get("dram_bytes") and ncu["dram_bytes"] * E_h
        if ncu.get("fp64_flops") is not None:
            f64 = ncu["fp64_flops"] * E_h / (avg_ms * 1e-3)
            roofs["fp64"] = {"achieved": round(f64 / 1e12, 4), "peak": round(peaks_live["fp64_flops"] / 1e12, 4),
                             "unit": "TFLOP/s", "frac": round(f64 / peaks_live["fp64_flops"], 4),
                             "peak_source": "measured live (cgl_measure_peaks: DFMA chains)"}
        if ncu.get("warp_inst") is not None:
            ipk = ncu["warp_inst"] * E_h / (avg_ms * 1e-3)
            peak_i = SM_COUNT_GB300 * ISSUE_PER_SM_CLK * sm_hz
            roofs["issue"] = {"achieved": round(ipk / 1e9, 1), "peak": round(peak_i / 1e9, 1), "unit": "Ginst/s",
                              "frac": round(ipk / peak_i, 4),
                              "peak_source": "152 SMs x 4 warp instructions per clock x median SM clock"}
        if ncu.get("shared_wavefronts") is not None:
            # the shared-memory data stage moves one 128 B wavefront per SM per clock
            swr = ncu["shared_wavefronts"] * E_h / (avg_ms * 1e-3)
            peak_s = SM_COUNT_GB300 * sm_hz
            roofs["shared"] = {"achieved": round(swr / 1e9, 1), "peak": round(peak_s / 1e9, 1),
                               "unit": "Gwavefronts/s", "frac": round(swr / peak_s, 4),
                               "peak_source": "152 SMs x 1 shared-memory wavefront (128 B) per clock x median SM "
                                              "clock (an on-chip pipe: reported as bound alu)"}
    bound = max(roofs, key=lambda k: roofs[k]["frac"]) if roofs else "hbm"
    main = roofs.get(bound, {})
    roof.update({"bound": {"hbm": "hbm", "fp64": "alu", "issue": "alu", "shared": "alu"}[bound], "roof": bound,
                 "achieved": main.get("achieved"), "peak": main.get("peak"), "unit": main.get("unit"),
                 "frac": main.get("frac"), "traffic": traffic, "roofs": roofs})
    meth_h = roofline_entry(HEADLINE, h32, 4)
    step_roof = dict(meth_h)
    step_roof["impl_bytes"] = impl_bytes_entry(h32, 4, meth_h["bytes_per_dof_stage"])
    if acc and "error" not in acc:
        a_h = acc.get(HEADLINE, {})
        cpu = {"value": a_h.get("rate_1thread"), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one SSP stage of {HEADLINE} on 16 windows of {WIN}x{WIN} elements "
                         f"({a_h.get('dof_stage')} DOF-stages), FP64 numpy oracle, one thread",
               "all_cores": {"value": a_h.get("rate_all"), "cores": a_h.get("cores"),
                             "sample": "the same windows, one spawn worker per host core"}}
        if QUADRANTS in acc:
            a_q = acc[QUADRANTS]
            cpu[QUADRANTS] = {"value": a_q.get("rate_1thread"), "cores": 1,
                              "sample": f"one SSP stage on 6 windows of {WIN}x{WIN} elements, one thread"}
            cfg[QUADRANTS]["accuracy"] = {"l1_vs_oracle": a_q.get("mixed_l1_vs_oracle"),
                                          "fp64_max_rel_vs_oracle": a_q.get("fp64_max_rel_vs_oracle"),
                                          "sample": f"one stage on 6 windows of {WIN}x{WIN} elements"}
    elif acc:
        cpu = {"error": acc.get("error")}
    a_h = (acc or {}).get(HEADLINE, {}) if acc and "error" not in acc else {}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": h32["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 bulk + f64 averages/limiters", "data": "synthetic",
        "config": dict(describe(HEADLINE), n_dof=nd_h, dof_stage_per_step=3 * nd_h, precision="FP32-mixed",
                       l2="flushed (256 MB write) between timed steps; state 269 MB > L2",
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
        "fp64_plain": {"value": value64, "ms_per_step": h64["ms"] / K,
                       "roofline": roofline_entry(HEADLINE, h64, 8), "kernel_share": _share(h64["prof"])},
        "mixed_over_fp64": value / value64,
        "kernel_share": _share(prof),
        "roofline": roof,
        "step_roofline": step_roof,
        "accuracy": {"l1_vs_oracle": a_h.get("mixed_l1_vs_oracle"),
                     "fp64_max_rel_vs_oracle": a_h.get("fp64_max_rel_vs_oracle"),
                     "sample": f"one stage from the state after {W} steps, 16 windows of {WIN}x{WIN} elements",
                     "mass_drift_fp32_mixed": drift(h32["before"], h32["after"], ((0, "rho"), (3, "E"))),
                     "mass_drift_fp64": drift(h64["before"], h64["after"], ((0, "rho"), (3, "E"))),
                     "violations": h32["violations"] + h64["violations"]},
        "configs": cfg,
        "cpu_baseline": cpu,
        "e2e": {"value": aggregate_rate(nd_h * 3 * K, e2e_s * 1e3, world), "unit": UNIT,
                "h2d_bytes_per_step": nd_h * 8, "d2h_bytes_per_step": nd_h * 8,
                "path": "per step cgl_set_state_async (float64, pinned host) + cgl_step_async + "
                        "cgl_get_state_async (float64, pinned host), one cgl_sync after the K steps; the copies "
                        "run on copy streams beside the neighbouring steps",
                "sync_calls": {"value": aggregate_rate(nd_h * 3 * K, e2e_sync_s * 1e3, world),
                               "path": "per step cgl_set_state + cgl_step (with its diagnostics) + cgl_get_state, "
                                       "each waiting for completion"}},
        "gpu_launches": h32["launches"] * K,
        "peaks_live": {"fp64_tflops": round(peaks_live["fp64_flops"] / 1e12, 4),
                       "fp32_tflops": round(peaks_live["fp32_flops"] / 1e12, 2)},
        "clocks": clk,
        "violations": h32["violations"] + h64["violations"],
    }
    print(json.dumps(line), flush=True)
    for r in (h32, h64):
        r["st"].close()
    if dist:
        dist.destroy_process_group()


def _share(prof):
    if not prof:
        return None
    tot = sum(v[0] for v in prof.values() if v[1])
    return {k: round(v[0] / tot, 4) for k, v in sorted(prof.items(), key=lambda x: -x[1][0]) if v[1]}


def run_batch(cgl, torch, stream, flush, K, W, world, rank, dist, timed, hbm_peak, hbm_src):
    """The 256-instance batch, FP32-mixed, one persistent launch per stage
    under a CUDA graph, then the phase form on the same instances; with
    several ranks each takes its share of the instances (a disjoint
    deterministic split, no exchange)."""
    import inputs
    from paper_2509_04673_gb300.partition import partition_instances
    cases = inputs.batched_instances()
    sizes = [u0.size for _, _, u0 in cases]
    mine = partition_instances(sizes, world)[rank]
    states = []
    for i in mine:
        mesh, prob, u0 = cases[i]
        st = cgl.State(cgl.Mesh(mesh), 1, cgl.FP32_MIXED, stream=stream.cuda_stream)
        st.set_problem(prob)
        st.set_state(u0)
        st.set_time(0.0)
        states.append(st)
    b = cgl.Batch(states)
    v0 = b.step(W)
    ms = timed(lambda: b.step_async(1), K)
    viol = b.step(0)
    info = b.info()
    # the phase form (one launch per phase, degrees on their own streams) on
    # the same instances, continuing from the state the persistent form left
    b.set_form(cgl.BATCH_PHASES)
    b.step(W)
    ms_ph = timed(lambda: b.step_async(1), K)
    viol_ph = b.step(0)
    info_ph = b.info()
    nd = sum(sizes[i] for i in mine)
    nd_all = sum(sizes)
    # method bytes: DOF-weighted over the instances' degrees (k_g = k_u = 1)
    bm = sum(method_bytes_per_dof_stage(cases[i][0].p, 4, 1, 1) * sizes[i] for i in mine) / nd
    rate = nd_all * 3 * K / (ms * 1e-3)
    ach = rate / world * bm / 1e9
    rate_ph = nd_all * 3 * K / (ms_ph * 1e-3)
    ach_ph = rate_ph / world * bm / 1e9
    res = {"config": {"workload": BATCH, "instances": len(cases), "sizes": "16^2..128^2 periodic",
                      "degrees": "1..4", "fluxes": "advection or Burgers", "mode": "WENO-L + flux limiter"},
           "n_dof": nd_all, "value": rate, "ms_per_step": ms / K, "scaling": "strong (instances split over ranks)",
           "graph": info["graph"], "grid": info["grid"], "block": info["block"],
           "roofline": {"bytes_per_dof_stage": round(bm, 2), "achieved": round(ach, 1), "peak": hbm_peak,
                        "unit": "GB/s", "frac": round(ach / hbm_peak, 4), "peak_source": hbm_src},
           "violations": int(viol),
           "form": "persistent: one cooperative launch per degree and stage",
           "phase_form": {"value": rate_ph, "ms_per_step": ms_ph / K, "graph": info_ph["graph"],
                          "form": "one launch per phase, each degree on its own stream in the step graph",
                          "roofline": {"achieved": round(ach_ph, 1), "peak": hbm_peak, "unit": "GB/s",
                                       "frac": round(ach_ph / hbm_peak, 4)},
                          "violations": int(viol_ph) - int(viol)}}
    b.close()
    for s in states:
        s.close()
    return res


# --------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# --------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import multiprocessing as mp
    mesh, prob, u0 = workload(HEADLINE)
    cores = host_cores()
    origins = window_origins(mesh.nx, mesh.ny, cores)
    pd = prob.as_dict()
    pd["boundary"] = None
    wins = [cut_window(mesh, u0, ex0, ey0) for ex0, ey0 in origins]
    dof = sum(us.size for _, us in wins)
    # one "step" = one SSP-RK3 step of the oracle on one window per host core
    # (dt of each window from the oracle itself), all windows in parallel
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_worker_init) as pool:
        jobs = [(sub.as_dict(), pd, us, 1) for sub, us in wins]
        for _ in range(args.warmup):
            pool.map(_oracle_window_steps, jobs)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_oracle_window_steps, jobs)
        secs = time.perf_counter() - t0
    value = dof * 3 * args.steps / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(describe(HEADLINE), n_dof=dof, precision="FP64 oracle (CPU)",
                       sample=f"{cores} windows of {WIN}x{WIN} elements of the workload, one per host core"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"one SSP-RK3 step per timed step on {cores} windows of {WIN}x{WIN} elements "
                                   "of the Euler blast 2048^2 Q2, one spawn worker per host core"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _oracle_window_steps(args):
    """nsteps oracle SSP-RK3 steps on one window; runs in a worker."""
    sub_d, prob_d, us, nsteps = args
    import inputs
    import oracle.scheme as S
    u, t, st = S.run(inputs.Mesh(**sub_d), prob_d, us, nsteps)
    return st["violations"]


def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample_main(args.oracle_sample)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

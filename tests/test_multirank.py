"""Multi-rank bench logic on CPU (gloo, world_size 2): the single-mesh path
runs independent replicas per rank with no data-path collective; the job
time is the max over ranks and the rate counts the units of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank           # rank 1 is the slow one
    ms_max = bench.reduce_over_ranks(ms, dist, "cpu")
    rate = bench.aggregate_rate(1000.0, ms_max, world)
    q.put((rank, ms_max, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_max_time_and_aggregate_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms_max, rate in res:
        assert ms_max == 15.0
        assert abs(rate - 2 * 1000.0 / 15e-3) < 1e-6


def test_single_rank_identity():
    import bench
    assert bench.reduce_over_ranks(7.0, None) == 7.0
    assert bench.aggregate_rate(100.0, 10.0, 1) == 100.0 / 10e-3


# --------------------------------------------------------------------------
# instance partition of the batched form
# --------------------------------------------------------------------------
def test_instance_partition_is_disjoint_cover_and_balanced():
    import inputs
    from paper_2509_04673_gb300.partition import partition_instances
    sizes = [u0.size for _, _, u0 in inputs.batched_instances()]
    for world in (1, 2, 3, 4, 8):
        parts = partition_instances(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        # greedy largest-first: no rank exceeds the mean by more than the largest instance
        assert max(loads) - sum(loads) / world <= max(sizes)
        assert partition_instances(sizes, world) == parts   # deterministic


def _partition_worker(rank, world, port, q):
    """Each rank takes its share of the instances; all_gather shows that
    the shares are disjoint and cover every instance."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    import inputs
    from paper_2509_04673_gb300.partition import partition_instances
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [u0.size for _, _, u0 in inputs.batched_instances()]
    mine = partition_instances(sizes, world)[rank]
    mask = torch.zeros(len(sizes), dtype=torch.int64)
    mask[mine] = 1
    dist.all_reduce(mask)
    q.put((rank, mask.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def _guarded(target, rank, world, port, q, *args):
    """Run a rank's body; an exception is sent back instead of a result, so
    the test fails at once rather than waiting for the queue."""
    import traceback
    try:
        target(rank, world, port, q, *args)
    except Exception:
        q.put(("error", rank, traceback.format_exc()))
        raise


def _run(world, target, *args):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_guarded, args=(target, r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    res = []
    for _ in range(world):
        item = q.get(timeout=300)
        if item[0] == "error":
            for p in procs:
                p.join(timeout=30)
                if p.is_alive():
                    p.kill()
            raise AssertionError(f"rank {item[1]} failed:\n{item[2]}")
        res.append(item)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return res


def test_instance_partition_over_gloo_ranks():
    for rank, cover in _run(2, _partition_worker):
        assert all(c == 1 for c in cover)


# --------------------------------------------------------------------------
# 2D block decomposition of one mesh: halo exchange, stage equality
# --------------------------------------------------------------------------
def _decomp_case(name):
    import inputs
    if name == "kpp_fixed_q2":
        mesh = inputs.Mesh(14, 11, 2, 0.0, 14 / 11, 0.0, 1.0, inputs.BC_FIXED, inputs.BC_FIXED)
        prob = inputs.Problem(flux=inputs.FLUX_KPP, umin=0.5, umax=3.0, w_lin=0.2, ubc=(1.0, 0, 0, 0))
        u = inputs.random_scalar_state(mesh, 77, 0.5, 3.0, 0.4)
    else:
        # periodic; split along x (halo wraps), whole along y (stays periodic)
        mesh = inputs.Mesh(28, 6, 2, 0.0, 28 / 6, 0.0, 1.0)
        prob = inputs.Problem(flux=inputs.FLUX_EULER, w_lin=1e-3)
        u = inputs.random_euler_state(mesh, 78)
    return mesh, prob, u


def _decomp_worker(rank, world, port, q, name):
    """Rank r owns the nodes of its element block, builds its window of
    owned + 6 halo elements by the point-to-point exchange, runs the oracle
    on the window and keeps its owned nodes.  Per step: a min-reduction of
    dt over the owned elements, then three stages with one exchange each."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np
    import torch
    import torch.distributed as dist
    import inputs
    import oracle.scheme as S
    from paper_2509_04673_gb300 import partition as P
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mesh, prob, u_glob = _decomp_case(name)
    per_x, per_y = mesh.bc_x == inputs.BC_PERIODIC, mesh.bc_y == inputs.BC_PERIODIC
    H = 6
    plan = P.halo_plan(world, mesh.nx, mesh.ny, mesh.p, H, per_x, per_y)
    me = plan[rank]
    ox0, ox1, oy0, oy1 = me["owned"]
    local = u_glob[:, oy0:oy1, ox0:ox1].copy()          # only the owned nodes are this rank's
    ex0, ex1, ey0, ey1 = me["ext"]
    wpx, wpy = me["periodic"]
    h = mesh.h
    # the window as a mesh of its own: a direction the block spans keeps its
    # periodicity; a cut side is outflow (the halo keeps it away from the
    # owned nodes), a true boundary side keeps its condition
    cut = {"W": ex0 > 0 or (per_x and not wpx), "E": ex1 < mesh.nx or (per_x and not wpx),
           "S": ey0 > 0 or (per_y and not wpy), "N": ey1 < mesh.ny or (per_y and not wpy)}
    pd = prob.as_dict()
    bx = inputs.BC_PERIODIC if wpx else inputs.BC_OUTFLOW
    by = inputs.BC_PERIODIC if wpy else inputs.BC_OUTFLOW
    if any(cut.values()):
        def side(s, kind_true):
            if (s in ("W", "E") and wpx) or (s in ("S", "N") and wpy):
                return inputs.boundary_side(inputs.BC_PERIODIC)
            return inputs.boundary_side(inputs.BC_OUTFLOW if cut[s] else kind_true, prob.ubc)
        pd["boundary"] = {s: side(s, mesh.bc_x if s in ("W", "E") else mesh.bc_y) for s in ("W", "E", "S", "N")}
    else:
        bx, by = mesh.bc_x, mesh.bc_y
    sub = inputs.Mesh(ex1 - ex0, ey1 - ey0, mesh.p, mesh.x0 + ex0 * h, mesh.x0 + ex1 * h,
                      mesh.y0 + ey0 * h, mesh.y0 + ey1 * h, bx, by)
    iy, ix = P.owned_slice_of_window(plan, rank)
    om = S.OracleMesh(sub)
    # owned elements inside the window
    oex = np.arange(me["block"].ex0, me["block"].ex1) - ex0
    oey = np.arange(me["block"].ey0, me["block"].ey1) - ey0
    own_e = (oey[:, None] * sub.nx + oex[None, :]).ravel()
    # one stage with a given dt
    dt = 1e-3
    win = P.exchange(plan, rank, local, dist)
    out, _ = S.ssp_stage(om, pd, win, win, dt, 0.0, 1.0)
    stage_owned = out[:, iy][:, :, ix]
    # one SSP-RK3 step: dt = cfl min over owned elements, min-reduced over ranks
    U = om.blocks(win)
    lo = S.low_order_facets(om, S.cell_averages(om, U), pd)
    dte = S.pseudo_time_steps(om, lo, pd)
    t = torch.tensor([pd["cfl"] * dte[own_e].min()], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    dts = float(t.item())
    un = local.copy()
    cur = local.copy()
    for (a, b) in S.SSP3:
        w_cur = P.exchange(plan, rank, cur, dist)
        w_un = P.exchange(plan, rank, un, dist)
        o, _ = S.ssp_stage(om, pd, w_cur, w_un, dts, a, b)
        cur = o[:, iy][:, :, ix].copy()
    q.put((rank, me["owned"], stage_owned, cur, dts))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["kpp_fixed_q2", "euler_periodic_q2"])
def test_block_decomposition_stage_equals_single_domain(name):
    import numpy as np
    import inputs
    import oracle.scheme as S
    from paper_2509_04673_gb300 import partition as P
    mesh, prob, u = _decomp_case(name)
    res = _run(2, _decomp_worker, name)
    ref1, _ = S.ssp_stage(mesh, prob, u, u, 1e-3, 0.0, 1.0)
    dt = S.time_step(mesh, prob, u)
    ref3 = u
    for (a, b) in S.SSP3:
        ref3, _ = S.ssp_stage(mesh, prob, ref3, u, dt, a, b)
    cover1 = np.zeros(ref1.shape[1:], dtype=int)
    for rank, (ox0, ox1, oy0, oy1), st1, st3, dts in res:
        assert dts == dt
        sc = np.abs(ref1).max()
        assert np.abs(st1 - ref1[:, oy0:oy1, ox0:ox1]).max() <= 1e-13 * sc
        assert np.abs(st3 - ref3[:, oy0:oy1, ox0:ox1]).max() <= 1e-13 * sc
        cover1[oy0:oy1, ox0:ox1] += 1
    assert np.all(cover1 == 1)
    # the plan's blocks tile the elements
    bl = P.blocks(2, mesh.nx, mesh.ny)
    cov = np.zeros((mesh.ny, mesh.nx), dtype=int)
    for b in bl:
        cov[b.ey0:b.ey1, b.ex0:b.ex1] += 1
    assert np.all(cov == 1)


def test_process_grid_and_owned_nodes_cover():
    import numpy as np
    from paper_2509_04673_gb300 import partition as P
    for world, nx, ny in ((1, 8, 8), (2, 8, 8), (4, 16, 16), (6, 30, 20), (8, 64, 16), (3, 9, 9)):
        for per in (True, False):
            p = 2
            nnx, nny = nx * p + (0 if per else 1), ny * p + (0 if per else 1)
            cov = np.zeros((nny, nnx), dtype=int)
            for b in P.blocks(world, nx, ny):
                gx0, gx1, gy0, gy1 = P.owned_nodes(b, nx, ny, p, per, per)
                cov[gy0:gy1, gx0:gx1] += 1
            assert np.all(cov == 1), (world, nx, ny, per)

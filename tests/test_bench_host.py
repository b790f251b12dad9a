"""Host-side parts of bench.py (CPU): the method-inherent bytes per
DOF-stage, and the oracle leg that times the oracle on windows of a
workload and compares GPU outputs with it.  The windows' compared nodes
must equal a stage on the whole mesh (the margin keeps the cut sides out
of reach), which the round trip checks with the full-mesh oracle stage
standing in for the GPU output."""
import numpy as np

import bench
import inputs
import oracle.scheme as S


def test_method_bytes_per_dof_stage():
    # 12.67 words + 4 (g sweep) + 2 (udot sweep) = 18.67 words; float64
    # per-element scalars 48 / p^2 bytes
    assert abs(bench.method_bytes_per_dof_stage(2, 4, 1, 1) - (18.0 + 2.0 / 3.0) * 4 - 12.0) < 1e-12
    assert abs(bench.method_bytes_per_dof_stage(3, 4, 1, 1) - (18.0 + 2.0 / 3.0) * 4 - 48.0 / 9) < 1e-12
    assert abs(bench.method_bytes_per_dof_stage(2, 8, 1, 1) - (18.0 + 2.0 / 3.0) * 8 - 12.0) < 1e-12
    assert abs(bench.method_bytes_per_dof_stage(2, 4, 0, 0) - (12.0 + 2.0 / 3.0) * 4 - 12.0) < 1e-12


def test_window_origins_inside_mesh():
    for nx, ny, count in ((2048, 2048, 16), (512, 512, 6), (200, 130, 9)):
        pts = bench.window_origins(nx, ny, count)
        assert len(pts) == count and len(set(pts)) == count
        for ex0, ey0 in pts:
            assert 0 <= ex0 <= nx - bench.WIN and 0 <= ey0 <= ny - bench.WIN


def test_oracle_sample_round_trip(monkeypatch):
    monkeypatch.setattr(bench, "WIN", 20)
    monkeypatch.setattr(bench, "MARGIN", 7)
    mesh, prob, u0 = inputs.euler_blast_config(48, 48, 2)
    # a state with structure everywhere: the blast after a few oracle steps
    # plus a seeded smooth perturbation of the density
    u = u0.copy()
    rng = inputs.SplitMix64(12)
    X, Y = inputs.node_coords(mesh)
    u[0] *= 1.0 + 0.1 * np.sin(2 * np.pi * (X + rng.uniform()) * 3) * np.cos(2 * np.pi * Y * 2)
    u, _, _ = S.run(mesh, prob, u, 2)
    dt = S.time_step(mesh, prob, u)
    full, _ = S.ssp_stage(mesh, prob, u, u, dt, 0.0, 1.0)
    spec, arrays = {}, {}
    wins = []
    for k, (ex0, ey0) in enumerate(bench.window_origins(mesh.nx, mesh.ny, 5)):
        sub, us = bench.cut_window(mesh, u, ex0, ey0)
        sy, sx = bench.compare_region(mesh, ex0, ey0)
        wins.append({"mesh": sub.as_dict(), "cmp": [[sy.start, sy.stop], [sx.start, sx.stop]]})
        p = mesh.p
        sl = (slice(None), slice(ey0 * p, (ey0 + bench.WIN) * p + 1), slice(ex0 * p, (ex0 + bench.WIN) * p + 1))
        arrays[f"w_in_{k}"] = us
        arrays[f"w_mixed_{k}"] = full[sl]
        arrays[f"w_fp64_{k}"] = full[sl]
    pd = prob.as_dict()
    pd["boundary"] = None
    spec["w"] = {"prob": pd, "dt": dt, "windows": wins, "all_core": True,
                 "scale": np.abs(full).reshape(4, -1).max(axis=1).tolist()}
    res = bench.run_oracle_sample(spec, arrays)["w"]
    assert res["mixed_l1_vs_oracle"] <= 1e-14, res
    assert res["fp64_max_rel_vs_oracle"] <= 1e-13, res
    assert res["oracle_violations"] == 0
    assert res["cores"] >= 1 and res["rate_all"] > 0 and res["rate_1thread"] > 0

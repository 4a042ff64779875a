"""The multi-GPU bookkeeping of bench.py (one replica per rank, barrier,
max-over-ranks time, whole-job throughput) on two CPU processes over gloo,
and the reference arm's behaviour on ranks other than 0."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas("gloo", "cpu")
    rep.barrier()
    t = 1.0 + rank                        # rank r "took" 1 + r seconds
    out[rank] = (rep.maxed(t), rep.throughput(1000.0, rep.maxed(t)), rep.world)
    rep.barrier()
    rep.close()


def _sweep_rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_1011_3582_gb300 import workloads
    rep = bench.Replicas("gloo", "cpu")
    plan = workloads.sweep_plan(64, seed=3)
    mine = bench.sweep_shard(plan, rep.rank, rep.world)
    local = [(idx, {"n": n, "tr": tr, "rank": rank}) for idx, (n, tr) in mine]
    out[rank] = (rep.gather(local), len(mine))
    rep.close()


def test_sweep_runs_partitioned_across_two_ranks_and_gathered():
    """The sweep's natural shard: rank r takes runs r, r + N, ... of the plan
    (no data-path collective); every rank's per-run results reach every
    rank, and together they cover each of the 64 runs exactly once, with
    the run's own grid and temperature."""
    sys.path.insert(0, ROOT)
    from paper_1011_3582_gb300 import workloads
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_sweep_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    plan = workloads.sweep_plan(64, seed=3)
    gathered, sizes = out[0][0], [out[r][1] for r in range(world)]
    assert sizes == [32, 32]
    flat = [x for part in gathered for x in part]
    assert sorted(i for i, _ in flat) == list(range(64))
    for i, res in flat:
        assert (res["n"], res["tr"]) == plan[i] and res["rank"] == i % world
    assert out[1][0] == gathered


def test_sweep_slab_densities_table():
    """bench.py lays out the sweep's slabs from tests/golden/maxwell_9_49.json
    by linear interpolation: within 1e-5 of the oracle's Maxwell densities
    between the table's grid points."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import thermo as TH
    table = bench.maxwell_table()
    a, b = 9 / 49, 2 / 21
    for tr in (0.7, 0.7437, 0.85, 0.9123, 0.99):
        rv, rl = bench.coexistence_densities(table, tr)
        wv, wl = TH.maxwell(tr * 8 * a / (27 * b), a, b)
        assert abs(rv - wv) / wv < 1e-5 and abs(rl - wl) / wl < 1e-5


def test_two_ranks_max_time_and_whole_job_throughput():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        tmax, thr, w = out[r]
        assert w == world
        assert tmax == 2.0                # every rank sees the slowest rank's time
        assert thr == pytest.approx(world * 1000.0 / 2.0)


def test_single_process_is_its_own_job():
    for k in ("RANK", "WORLD_SIZE"):
        os.environ.pop(k, None)
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas("gloo", "cpu")
    assert rep.world == 1 and rep.maxed(3.5) == 3.5 and rep.throughput(10.0, 2.0) == 5.0


def test_reference_arm_does_no_work_on_other_ranks(capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(steps=3, warmup=3, grid=1024)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""


def test_ncu_traffic_summary_from_a_launch_csv(tmp_path):
    """bench.write_ncu_traffic: DRAM read + write per launch, unit-scaled,
    averaged per kernel kind; the one-input column launches of a stage
    alternate between convection and level 2, the multi-input one is level
    1 (both the pipelined and the warp-resident kernel names)."""
    sys.path.insert(0, ROOT)
    import bench
    hdr = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
          '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
    for names in (["void k1_pipe<float, 4, false>(x)", "void kcol_pipe<float, false, false>(x)",
                   "void kcol_pipe<float, true, false>(x)", "void k3_pipe<float, false>(x)",
                   "void kcol_pipe<float, false, false>(x)", "void k5_pipe<float, 2, false>(x)"],
                  ["void k1_wr<512>(x)", "void kcol_wr<1024>(x)", "void kcolm_wr<1024>(x)", "void k3_wr<512>(x)",
                   "void kcol_wr<1024>(x)", "void k5_wr<512>(x)"]):
        _check_traffic_names(tmp_path, bench, hdr, names)


def _check_traffic_names(tmp_path, bench, hdr, names):
    lines = ["==PROF== noise\n", hdr]
    for stage in range(2):
        for j, nm in enumerate(names):
            i = 6 * stage + j
            rd, wr = 1000.0 * (j + 1) + stage, 10.0 * (j + 1)
            for metric, unit, val in (("dram__bytes_read.sum", "Kbyte", rd / 1e3), ("dram__bytes_write.sum", "byte", wr),
                                      ("gpu__time_duration.sum", "ns", 5.0)):
                lines.append(f'"{i}","1","python","h","{nm}","1","7","(256, 1, 1)","(152, 1, 1)","0","10.3","s",'
                             f'"{metric}","{unit}","{val}"\n')
    csv_path = tmp_path / "t.csv"
    csv_path.write_text("".join(lines))
    out = tmp_path / "traffic.txt"
    res = bench.write_ncu_traffic(str(csv_path), 32, 1024, "test", out_path=str(out))
    want = {"row_forward_moments": 1, "col_convection": 2, "col_level1": 3, "row_level1": 4, "col_level2": 5,
            "row_final": 6}
    for k, j in want.items():
        assert len(res[k]) == 2
        assert sum(res[k]) / 2 == pytest.approx(1000.0 * j + 0.5 + 10.0 * j)
    rows = [ln.split() for ln in out.read_text().splitlines() if not ln.startswith("#")]
    assert {r[0] for r in rows} == set(want) and all(r[1] == "32" and r[2] == "1024" for r in rows)


def test_reference_arm_line_describes_what_it_ran(capsys):
    """The reference arm times full SSP-RK3 steps of the main line's own
    workload: its config is the main line's, and steps / warmup are the
    counts it actually ran (capped), so ms_per_step x steps is its timed
    region."""
    sys.path.insert(0, ROOT)
    import argparse
    import json
    import bench
    args = argparse.Namespace(steps=20, warmup=5, grid=16)
    bench.run_reference(args, rank=0, world=1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"] == bench.workload_config(16)
    assert line["steps"] == bench.REF_MAX_STEPS and line["warmup"] == 1
    assert line["steps_requested"] == 20
    assert line["value"] == pytest.approx(16 * 16 / (line["ms_per_step"] * 1e-3) / 1e6, rel=1e-9)
    assert line["cpu_baseline"]["value"] == line["value"] and line["e2e"]["value"] == line["value"]

"""Benchmark of the FFT-LB hot path: MLUPS (million lattice-site updates per
second, one update = one full SSP-RK3 time step) on the 1024 x 1024
spinodal-decomposition workload, plus the roofline fraction of the dominant
kernel, an end-to-end figure through the C ABI with host buffers, and the
FP64 oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision 32|64]
    python bench.py --impl reference ...   (the FP64 oracle on the host cores)

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica of the workload on its own GPU (the single-grid path does not shard).
"""
from __future__ import annotations

import os

# the oracle legs run numpy single-threaded; the reported core count is 1
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1011_3582_gb300 import workloads  # noqa: E402

A, B = 9.0 / 49.0, 2.0 / 21.0                # vdW constants of the benchmark set
TC, RHOC = 8 * A / (27 * B), 1.0 / (3 * B)    # 4/7, 3.5
METRIC = "MLUPS at 1024^2 (spinodal, SSP-RK3 steps)"
REF_MAX_STEPS = 3          # timed oracle steps of the reference arm (about 15 s each at 1024^2)


def workload_fields(n, seed=7):
    """rho = rho_c (1 + 0.01 N(0,1)), seed 7, u = 0, T = 0.7 T_c."""
    return workloads.spinodal(n, n, RHOC, 0.7 * TC, amp=0.01, seed=seed)


def workload_config(n):
    """The workload's description, shared by both arms' JSON lines."""
    return {"workload": "spinodal decomposition %dx%d, rho = rho_c (1 + 0.01 N(0,1)) seed 7, T = 0.7 T_c, "
                        "vdW a = 9/49 b = 2/21" % (n, n),
            "grid": n, "integrator": "ssp-rk3", "window": "k4", "dx": 1 / 256, "dt": 1e-5, "tau": 1e-2,
            "K": 1e-5, "q": -0.004}


def workload_params(fl, n, precision, integrator=3):
    return fl.params(nx=n, ny=n, a=A, b=B, precision=precision, integrator=integrator, window=4)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def source_hash():
    """Hash of the kernel sources' code: every file of csrc/ without its
    whole-line // comments and blank lines, so that a comment edit does not
    detach the ncu traffic figures from the kernels they were taken on."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1011_3582_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fn.encode())
            for line in fh.read().decode("utf-8", "replace").splitlines():
                t = line.strip()
                if t and not t.startswith("//"):
                    h.update(t.encode())
                    h.update(b"\n")
    return h.hexdigest()[:16]


def ncu_traffic(kernel, precision, n):
    """DRAM bytes per launch from profiles/ncu_traffic.txt, valid only for
    the kernel sources it was captured from (same source hash)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    cur = source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 5 and not line.startswith("#"):
            k, prec, grid, by, hsh = parts[:5]
            if k == kernel and prec == str(precision) and grid == str(n) and hsh == cur:
                return float(by)
    return None


_UNITS = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1024.0, "MB": 1024.0 ** 2, "GB": 1024.0 ** 3}


def write_ncu_traffic(csv_path, precision, n, note, out_path=None):
    """Writes profiles/ncu_traffic.txt from an ncu --csv log of one SSP-RK3
    step of the pipelined kernels captured with the metrics
    dram__bytes_read.sum and dram__bytes_write.sum: DRAM bytes per launch of
    each kernel kind, averaged over its launches (the one-input column
    launches of a stage alternate: convection, then level 2; the multi-input
    column launch is level 1)."""
    import csv
    rows = [ln for ln in open(csv_path) if ln.startswith('"')]
    per = {}
    for r in csv.DictReader(rows):
        if r["Metric Name"] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        by = float(r["Metric Value"].replace(",", "")) * _UNITS.get(r["Metric Unit"], 1.0)
        per.setdefault(int(r["ID"]), [r["Kernel Name"], 0.0])[1] += by
    out, single = {}, 0
    for i in sorted(per):
        name, by = per[i]
        if "k1_pipe" in name or "k1_wr" in name:
            k = "row_forward_moments"
        elif "k3_pipe" in name or "k3_wr" in name:
            k = "row_level1"
        elif "k5_pipe" in name or "k5_wr" in name:
            k = "row_final"
        elif "kcolm_wr" in name:
            k = "col_level1"
        elif "kcol_wr" in name or "kcol_pipe" in name:
            m = re.search(r"kcol_pipe<\s*\w+\s*,\s*(\w+)", name)   # the second template argument: MULTI
            if m and m.group(1) not in ("false", "0"):
                k = "col_level1"
            else:
                k = "col_convection" if single % 2 == 0 else "col_level2"
                single += 1
        else:
            continue
        out.setdefault(k, []).append(by)
    path = out_path or os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    with open(path, "w") as fh:
        fh.write("# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum), averaged over the\n"
                 "# launches of one SSP-RK3 step; valid for the kernel sources with this hash only.\n"
                 "# kernel precision grid bytes_per_launch source_hash launches note\n")
        for k, v in out.items():
            fh.write("%s %d %d %.0f %s %d %s\n" % (k, precision, n, sum(v) / len(v), source_hash(), len(v), note))
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms from
    before the warm-up to after the profiled pass; summary() keeps the
    samples taken inside the timed region, or, when that region is shorter
    than three sampling periods, those of the whole busy window around it
    (warm-up, timed steps, profiled steps), and says which."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.5)   # let the first samples arrive before the GPU work starts
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1, busy0, busy1):
        def pick(a, b):
            return [ln for t, ln in self.lines if a <= t <= b]
        window, lines = "timed", pick(t0, t1)
        if len(lines) < 3:
            window, lines = "busy window around the timed region", pick(busy0, busy1)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 6:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "window": window}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "window": window}


def cpu_baseline(n=1024):
    """The FP64 oracle on the host: one SSP-RK3 step of the n x n workload
    (about 15 s of one core at 1024^2)."""
    from oracle import fftlb_oracle as O
    p = O.Params(nx=n, ny=n, a=A, b=B, integrator=3, window=4)
    f = O.init_equilibrium(*workload_fields(n), p)
    t0 = time.perf_counter()
    f = O.step(f, p)
    dt = time.perf_counter() - t0
    return {"value": n * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": "one SSP-RK3 step of the %dx%d workload, numpy fp64, %.1f s" % (n, n, dt)}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle on the host cores, on the same
    workload and metric as the main line.  Each timed step is one full
    SSP-RK3 step of the 1024^2 workload (about 15 s of one core), so the arm
    runs at most REF_MAX_STEPS timed steps after at most one warm-up step,
    and prints the counts it ran.  Under torchrun only rank 0 runs it."""
    if rank != 0:
        return
    from oracle import fftlb_oracle as O
    n = args.grid
    p = O.Params(nx=n, ny=n, a=A, b=B, integrator=3, window=4)
    f = O.init_equilibrium(*workload_fields(n), p)
    steps, warmup = max(1, min(args.steps, REF_MAX_STEPS)), min(args.warmup, 1)
    for _ in range(warmup):
        f = O.step(f, p)
    t0 = time.perf_counter()
    for _ in range(steps):
        f = O.step(f, p)
    el = time.perf_counter() - t0
    v = n * n * steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": el * 1e3 / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(n),
            "steps_requested": args.steps, "warmup_requested": args.warmup,
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": "%d full SSP-RK3 steps of the %dx%d workload after %d warm-up step(s), "
                                       "numpy fp64 on one core (capped at %d timed steps)"
                                       % (steps, n, n, warmup, REF_MAX_STEPS)},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def maxwell_table():
    """Coexistence densities of the a = 9/49, b = 2/21 fluid on a grid of T_r
    (tests/golden/maxwell_9_49.json, written by make_maxwell_table.py next
    to it)."""
    with open(os.path.join(ROOT, "tests", "golden", "maxwell_9_49.json")) as fh:
        return np.asarray(json.load(fh)["rows"], dtype=np.float64)


def coexistence_densities(table, tr):
    """(rho_v, rho_l) at reduced temperature tr by linear interpolation."""
    return float(np.interp(tr, table[:, 0], table[:, 1])), float(np.interp(tr, table[:, 0], table[:, 2]))


def sweep_shard(plan, rank, world):
    """The runs rank takes of a sweep plan: (index, run) for index = rank,
    rank + world, ... (every run on exactly one rank)."""
    return [(i, p) for i, p in enumerate(plan) if i % world == rank]


class Replicas:
    """Bookkeeping of a multi-GPU run launched by torch.distributed.run: one
    process per GPU, each running its own replica of the workload (the
    single-grid step does not shard: every transform is global).  barrier()
    aligns the ranks around a timed region, maxed(t) is the maximum over
    ranks (the whole job's time), and a whole-job throughput is
    world x (units per rank) / maxed(time)."""

    def __init__(self, backend, device):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def maxed(self, x):
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def gather(self, obj):
        """Every rank's obj, in rank order (host-side, for results)."""
        if self.dist is None:
            return [obj]
        out = [None] * self.world
        self.dist.all_gather_object(out, obj)
        return out

    def throughput(self, units_per_rank, seconds):
        return self.world * units_per_rank / seconds

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # (600 steps: about 0.6 s timed at 1024^2, long enough for the 100 ms
    # clock sampler to see at least three samples inside the timed region)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--grid", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 companion measurement")
    ap.add_argument("--ncu-traffic-from", default=None, metavar="CSV",
                    help="write profiles/ncu_traffic.txt from an ncu --csv log of one step (no GPU work)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch parameters instead of fftlb_autotune's")
    ap.add_argument("--bf16split", action="store_true",
                    help="time the fp32 path with split-BF16 tensor-core first passes as the main path (profiling)")
    ap.add_argument("--no-bf16split", action="store_true",
                    help="skip the FP32 path with split-BF16 tensor-core first radix-16 passes")
    ap.add_argument("--no-cufft-reference", action="store_true",
                    help="skip timing the PyTorch/cuFFT version of the same step")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the batched sweep (64 slabs of uneven grids, one persistent launch per kernel per "
                         "parameter group, replayed as one CUDA graph)")
    args = ap.parse_args()
    if args.ncu_traffic_from:
        res = write_ncu_traffic(args.ncu_traffic_from, args.precision, args.grid,
                                "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum")
        print(json.dumps({k: sum(v) / len(v) for k, v in res.items()}))
        return
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    rep = Replicas("nccl", "cuda")

    import __graft_entry__
    __graft_entry__.build()
    from paper_1011_3582_gb300 import fftlb

    n = args.grid
    stream = torch.cuda.current_stream()
    fields = workload_fields(n)
    barrier, maxed = rep.barrier, rep.maxed

    def time_path(precision, steps, warmup, sample_clocks):
        clk = ClockSampler(local)
        if sample_clocks:
            clk.__enter__()
        h = fftlb.Handle(workload_params(fftlb, n, precision), stream=stream.cuda_stream)
        h.set_fields(*fields)
        if not args.no_autotune:
            h.autotune()   # launch parameters only; the state is untouched
        tuned[precision] = h.tuning()
        busy0 = time.perf_counter()
        h.step(warmup)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev0.record(stream)
        h.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        barrier()
        ms = maxed(ev0.elapsed_time(ev1))
        # per-kernel timing on a second pass of the same length
        h.profile(True)
        h.step(steps)
        prof = h.profile_read()
        h.profile(False)
        busy1 = time.perf_counter()
        if sample_clocks:
            clk.__exit__()
        inv = h.invariants()
        lps = h.launches_per_step()
        h.close()
        return ms, prof, inv, lps, (clk.summary(t0, t1, busy0, busy1) if sample_clocks else None)

    tuned = {}
    prec = args.precision | (256 if args.bf16split and args.precision == 32 else 0)   # 256: BF16SPLIT
    ms, prof, inv, lps, clocks = time_path(prec, args.steps, args.warmup, True)
    K = args.steps
    value = rep.throughput(n * n * K, ms * 1e-3) / 1e6

    peaks, peak_kind = measured_peaks()
    top = max(prof, key=lambda k: prof[k][0])
    tms, tl, tbytes = prof[top]
    achieved = tbytes / (tms * 1e-3 / tl) / 1e9
    traffic = ncu_traffic(top, prec, n)
    roofline = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "peak_source": peak_kind,
                "kernel_share": tms / sum(v[0] for v in prof.values())}
    step_bytes = sum(prof[k][2] * prof[k][1] for k in prof) / K
    kernels = {k: {"ms_per_launch": prof[k][0] / max(prof[k][1], 1), "launches": prof[k][1],
                   "alg_bytes_per_launch": prof[k][2],
                   "gbs": prof[k][2] / (prof[k][0] * 1e-3 / max(prof[k][1], 1)) / 1e9 if prof[k][0] else None}
               for k in prof}

    fp64 = None
    if not args.no_fp64 and args.precision != 64:
        ms64, prof64, _, _, _ = time_path(64, max(2, K // 4), 3, False)
        fp64 = {"value": world * n * n * max(2, K // 4) / (ms64 * 1e-3) / 1e6, "unit": "MLUPS",
                "ms_per_step": ms64 / max(2, K // 4)}

    bf16split = None
    if not args.no_bf16split and prec == 32:
        ks = max(2, K // 2)
        pb = 32 | fftlb.BF16SPLIT
        mss, profs, _, _, _ = time_path(pb, ks, 3, False)
        bf16split = {"value": world * n * n * ks / (mss * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": mss / ks,
                     "kernel_ms_per_launch": {k: profs[k][0] / max(profs[k][1], 1) for k in profs},
                     "what": "fp32 with the first radix-16 pass of every power-of-two transform as a split-BF16 "
                             "DFT matrix product on the tensor cores (mma.sync m16n8k16, fp32 accumulation)"}

    e2e = None
    if not args.no_e2e:
        # public API with pinned host buffers: upload the fields, then each
        # step: advance one step and read back its invariants (6 doubles);
        # read the fields back at the end
        pinned = [torch.empty((n, n), dtype=torch.float64, pin_memory=True).numpy() for _ in range(4)]
        for dst, src in zip(pinned, fields):
            dst[...] = src
        outs = [torch.empty((n, n), dtype=torch.float64, pin_memory=True).numpy() for _ in range(4)]
        h = fftlb.Handle(workload_params(fftlb, n, prec), stream=stream.cuda_stream)
        h.set_fields(*pinned)
        if not args.no_autotune:
            h.tuning(tuned[prec])   # the parameters the timed run used
        h.step(2)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        h.set_fields(*pinned)
        for _ in range(K):
            h.step(1)
            h.invariants()
        h.fields(*outs)
        el = maxed(time.perf_counter() - t0)
        h.close()
        fb = 4 * n * n * 8
        e2e = {"value": world * n * n * K / el / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": fb / K,
               "d2h_bytes_per_step": 48 + fb / K}

    sweep = None
    if not args.no_sweep:
        # batched phase-diagram sweep (configuration 4): 64 planar slabs of
        # uneven grids at T_r in [0.70, 0.99], liquid in the central half at
        # the Maxwell densities, one CUDA graph per step; under torchrun the
        # runs are partitioned across the ranks (no collective on the data
        # path; the per-run results are gathered on the host)
        plan = workloads.sweep_plan(64, seed=3)
        mine = sweep_shard(plan, rep.rank, rep.world)
        table = maxwell_table()
        plist, flist = [], []
        for idx, (n_, tr) in mine:
            rv, rl = coexistence_densities(table, tr)
            flist.append(workloads.slab(n_, n_, rv, rl, tr * TC, width=2.0, noise=1e-4, seed=100 + idx))
            plist.append(fftlb.params(nx=n_, ny=n_, a=A, b=B, precision=prec, integrator=3, window=4))
        t0 = time.perf_counter()
        bt = fftlb.Batch(plist, autotune=True, stream=stream.cuda_stream)
        t_create = time.perf_counter() - t0
        for r, fl_ in enumerate(flist):
            bt.set_fields(r, *fl_)
        bt.step(3)
        torch.cuda.synchronize()
        ks = max(5, K // 2)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        bt.step(ks)
        ev1.record(stream)
        torch.cuda.synchronize()
        sms = maxed(ev0.elapsed_time(ev1))
        local = [(idx, bt.invariants(r)) for r, (idx, _) in enumerate(mine)]
        results = rep.gather(local)
        sites = sum(n_ * n_ for n_, _ in plan)
        if rep.rank == 0:
            done = sorted(i for part in results for i, _ in part)
            assert done == list(range(len(plan))), "sweep: runs missing from the gather"
        sweep = {"value": sites * ks / (sms * 1e-3) / 1e6, "unit": "MLUPS", "runs": len(plan),
                 "runs_per_rank": [len(sweep_shard(plan, r, rep.world)) for r in range(rep.world)],
                 "scaling": "strong (the 64 runs are partitioned across the ranks)",
                 "workload": "planar slabs, liquid in the central half at the Maxwell densities (configuration 4)",
                 "grids": {str(g): sum(1 for n_, _ in plan if n_ == g) for g in (128, 256, 384, 512)},
                 "steps": ks, "ms_per_step": sms / ks, "gpu_launches_per_step": bt.launches_per_step(),
                 "graph_launches_per_step": 1, "create_and_autotune_s": t_create}
        bt.close()

    cufft = None
    if not args.no_cufft_reference:
        # the same step written in PyTorch (torch.fft = cuFFT for the 94
        # transforms, element-wise kernels for the rest), fp32, timed the
        # same way: a reference for the hand-written kernels, not the product
        from paper_1011_3582_gb300 import torch_reference as TR
        ts = TR.TorchStep(n, n, a=A, b=B, integrator=3, window=4)
        ts.set_fields(*fields)
        ts.step(2)
        kr = max(3, K // 10)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        ev0.record()
        ts.step(kr)
        ev1.record()
        torch.cuda.synchronize()
        rms = maxed(ev0.elapsed_time(ev1))
        cufft = {"value": world * n * n * kr / (rms * 1e-3) / 1e6, "unit": "MLUPS", "steps": kr,
                 "ms_per_step": rms / kr, "dtype": "f32",
                 "what": "same SSP-RK3 step in PyTorch: torch.fft (cuFFT) transforms + torch element-wise kernels"}
        del ts
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
                "config": dict(workload_config(n),
                           l2="inputs larger than L2 (state %.0f MB + spectra %.0f MB)" % (
                               33 * n * n * args.precision / 8 / 1e6, 58 * n * n * args.precision / 8 / 1e6),
                           parallelism="replicas" if world > 1 else "single",
                           first_pass="split-BF16 tensor cores" if prec & 256 else "fp32 radix 16",
                           launch_tuning=dict(zip(("tw_conv", "tw_level", "rows_forward", "rows_final",
                                                   "head_buffers"), tuned[prec]),
                                              autotuned=not args.no_autotune)),
                "roofline": roofline, "kernels": kernels, "alg_bytes_per_step": step_bytes,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": lps * K, "clocks": clocks,
                "fp64": fp64, "bf16split": bf16split, "sweep": sweep, "cufft_reference": cufft, "invariants_after": inv}
        print(json.dumps(line), flush=True)
    rep.close()


if __name__ == "__main__":
    main()

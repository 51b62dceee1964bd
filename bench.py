"""Benchmark of the weighting-field hot path on GB300.

Workload (default): the 3x3 pixel cell (165 x 165 x 500 um, grid
128 x 128 x 256, 18 graphitised columns, 256 sources per column, 512
log-spaced time samples 1 ps - 10 ns).  Metric: H grid-point x time-samples
per second of the FP32 bulk extension (basis-field spectral passes + tensor-
core expansion writing H once), at the accuracy checked against the FP64
plain path and the oracle in tests/.  The one-time FP64 setup (boundary fit,
relaxation modes, time basis) is done before timing and reported as
``setup_s``.

One step = one wt_extend(WT_FP32) into a device buffer.  L2 is flushed
(256 MB write) before every timed step.  ``e2e`` times the same call through
the C ABI with a pinned host buffer (device compute + device-to-host copy of
H).  ``cpu_baseline`` times the FP64 oracle on a bounded sample of the same
workload.  Multi-GPU: every rank runs its own replica (the path has no
exchange step); value = all ranks' point-samples / max time.

--impl reference runs the FP64 CPU oracle (the reference arm of this
build: the paper ships no code) on the same workload, a bounded sample per
step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
METRIC = "H grid-point*time-samples/sec (FP32 extension, 12 B/point-sample written once)"
WORKLOADS = {
    "c2": "c2: 3x3 pixel cell 165x165x500 um, grid 128x128x256, 18 columns x 256 sources, 512 time samples",
    "c1": "c1: single cell 55x55x100 um, grid 32x32x64, 2 columns x 64 sources, 64 time samples",
    "small": "small: single cell 55x55x100 um, grid 64x64x64, 2 columns x 64 sources, 512 time samples "
             "(profiling case: H = 1.6 GB > L2)",
    "prof": "prof: c2's geometry and grid (128x128x256, 18 columns) with 64 time samples "
            "(profiling case: the spectral kernels at c2 sizes and rank, about 7 GB on the device)",
    "prof256": "prof256: the 3x3 pixel cell at grid 96x96x192 (c4's geometry) with 256 time samples, extension "
               "only (profiling case: the expansion at the 5x5 cell's time count, H 5.4 GB)",
    "prof5": "prof5: the 5x5 pixel cell (50 columns, 275x275x500 um) at grid 96x96x192 with 64 sources per "
             "column and 64 time samples (profiling case: the 50-column table path, about 4 GB on the device)",
    "prof_eq1": "prof_eq1: the 3x3 pixel cell at grid 96x96x192 (c4's geometry) with 256 time samples, Eq. 1 "
                "from the rank-r form against 2e4 drift tracks of 200 steps (the 5x5 cell's track recipe) "
                "(profiling case: basis fields 0.68 GB)",
    "c4": "c4: 3x3 pixel cell at grid 96x96x192, radius 5 um, 256 time samples, 1e4 straight tracks of 100 "
          "steps; the Eq. 1 loss and its gradient (resistivities, radius, pitch)",
    "scan": "scan: Sec. 5's bias-diameter scan (6-14 um in 2 um steps) on the 3x3 pixel cell 165x165x500 um, "
            "grid 20x20x64, 18 columns, 256 time samples, 1000 tracks of 100 steps through the central pixel; "
            "per variant fit, relaxation, currents with their four parameter tangents, CR-RC^2 shaping, "
            "signal features and their sensitivities",
    "c5": "c5: 5x5 pixel cell 275x275x500 um, grid 192x192x384, 50 columns x 256 sources, 256 time samples "
          "(H 43.5 GB), Eq. 1 against 1e5 electron/hole drift tracks of 200 steps",
    "c3": "c3: 64 single cells, pitch 40-110 um, thickness 300-500 um, radius 4-10 um, grids 64^2x128 to "
          "128^2x256 (uneven), 256 time samples each; batched in waves through an H arena",
}


def make_workload(name):
    import workloads as W
    if name == "small":
        return W.tiny_cell(nx=64, nz=64, n_t=512, radius=6e-6)
    if name == "prof":
        from dataclasses import replace
        w = W.workload("c2")
        return replace(w, times=W.log_times(64))
    if name == "prof256":
        from dataclasses import replace
        return replace(W.workload("c4", n_tracks=1), tracks=None)
    if name == "prof5":
        import numpy as np
        from workloads import configs as WC
        grid, cols = WC.pixel_matrix(5, 55 * WC.UM, 500 * WC.UM, 96, 192, 6 * WC.UM, 0.1 * WC.OHM_CM,
                                     1.0 * WC.OHM_CM, 64, np.random.default_rng(5))
        return WC.Workload("prof5", grid, cols, WC.FitSpec(), W.log_times(64), seed=5,
                           notes="5x5 pixels at grid 96x96x192, 64 sources per column")
    if name == "prof_eq1":
        import numpy as np
        from dataclasses import replace
        w = W.workload("c4", n_tracks=1)
        tr = W.configs.drift_tracks(w.grid, w.columns, 20_000, 200, 1.5e-12, np.random.default_rng(7))
        return replace(w, tracks=tr)
    return W.workload(name)


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, tag=""):
        fd, self.path = tempfile.mkstemp(prefix=f"wt_bench_clocks{tag}_", suffix=".csv")
        os.close(fd)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def __del__(self):
        try:
            os.unlink(self.path)
        except OSError:
            pass

    def summary(self, gpu_index):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines()]
            rows = [[x.strip() for x in r] for r in rows if len(r) >= 9 and r[0].strip() == str(gpu_index)]
            if not rows:
                return out
            sm = [float(r[1]) for r in rows]
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(float(r[2]) for r in rows)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for k, n in enumerate(names):
                if any(r[5 + k].lower() == "active" for r in rows):
                    out["reasons"].append(n)
            out["samples"] = len(rows)
        except Exception:
            pass
        return out


def dist_init():
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(w, sol, rng_seed=11, n_t=4, n_side=12):
    """Bounded oracle sample of the workload's H: n_t time samples on an
    n_side^3 random tensor-product subgrid.  Returns (point-samples, seconds)."""
    return _subgrid_sample(w.grid, sol.lay.src, sol.q, rng_seed, n_t, n_side)


def _subgrid_sample(grid, src, q, rng_seed, n_t=4, n_side=12):
    import numpy as np
    from oracle import extend as OX
    rng = np.random.default_rng(rng_seed)
    ti = np.sort(rng.choice(q.shape[1], n_t, replace=False))
    ix = np.sort(rng.choice(grid.Nx, n_side, replace=False))
    iy = np.sort(rng.choice(grid.Ny, n_side, replace=False))
    iz = np.sort(rng.choice(grid.Nz, n_side, replace=False))
    t0 = time.perf_counter()
    OX.field_subgrid(grid, src, q[:, ti], ix, iy, iz)
    dt = time.perf_counter() - t0
    return n_t * n_side ** 3, dt


def _sample_for(grid, src, q, seconds, seed0=7):
    """Oracle subgrid draws until `seconds` of CPU work; (point-samples, seconds)."""
    tot_ps, tot_s, k = 0, 0.0, 0
    while tot_s < seconds:
        ps_, s_ = _subgrid_sample(grid, src, q, seed0 + k)
        tot_ps += ps_
        tot_s += s_
        k += 1
    return tot_ps, tot_s


BLAS_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def cpu_sample_child(path, seconds):
    """Child process of the single-threaded CPU baseline: the same oracle draws on the charges
    saved by the parent (its BLAS limited to one thread by the environment)."""
    import numpy as np
    from workloads.configs import GridSpec
    d = np.load(path, allow_pickle=False)
    gk = json.loads(str(d["grid"]))
    ps, s = _sample_for(GridSpec(**gk), d["src"], d["q"], seconds)
    print(json.dumps({"ps": ps, "s": s}), flush=True)
    return 0


def cpu_baseline_threads(w, sol, seconds, threads):
    """Oracle draws in a child process whose BLAS runs `threads` threads (None: the default,
    all cores).  Returns (point-samples/s, seconds) or None if the child failed."""
    import dataclasses
    import numpy as np
    fd, path = tempfile.mkstemp(prefix="wt_bench_oracle_", suffix=".npz")
    os.close(fd)
    try:
        np.savez(path, grid=json.dumps(dataclasses.asdict(w.grid)), src=sol.lay.src, q=sol.q)
        env = dict(os.environ)
        for k in BLAS_THREAD_VARS:
            if threads is None:
                env.pop(k, None)
            else:
                env[k] = str(threads)
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-sample-from", path,
                            "--cpu-seconds", str(seconds)], env=env, capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            return None
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return d["ps"] / d["s"], d["s"]
    except Exception:
        return None
    finally:
        os.unlink(path)


def run_reference(args):
    """The FP64 CPU oracle on the host cores (reference arm)."""
    rank, local, world = dist_init()
    if rank != 0:
        return 0
    import oracle as O
    w = make_workload(args.workload)
    t0 = time.perf_counter()
    sol = O.solve(w)
    setup = time.perf_counter() - t0
    for _ in range(args.warmup):
        oracle_sample(w, sol, n_t=1, n_side=8)
    tot_ps, tot_s = 0, 0.0
    for k in range(args.steps):
        ps, s = oracle_sample(w, sol, rng_seed=100 + k)
        tot_ps += ps
        tot_s += s
    v = tot_ps / tot_s
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v,
            "unit": "point-samples/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "sample": "4 time samples x 12^3 random subgrid per step"},
            "cpu_baseline": {"value": v, "unit": "point-samples/s", "cores": cores, "kind": "oracle",
                             "sample": "4 time samples x 12^3 grid points per step; oracle setup excluded "
                                       f"({setup:.1f} s)"},
            "e2e": {"value": v, "unit": "point-samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "setup_s": setup}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """c3: 64 geometries through wt_batch_run, in waves whose H fits an arena
    of --arena-gb; one captured graph (one persistent expansion launch) per
    wave.  A step = every wave once (all 64 sensors' H written once)."""
    import torch
    import paper_2605_13987_gb300 as P
    import workloads as W

    rank, local, world = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.load_library()
    ws = W.c3_batch(seed=3)
    t0 = time.perf_counter()
    sens = []
    for w in ws:
        s_ = P.Sensor(w.grid, w.columns, device=local)
        s_.fit()
        s_.relax(w.times)
        sens.append(s_)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    sizes = [len(w.times) * 3 * w.grid.Nx * w.grid.Ny * w.grid.Nz for w in ws]     # floats of H
    ps_step = sum(n // 3 for n in sizes)
    # waves: consecutive sensors while their H fits the arena (256-byte aligned slices)
    cap = int(args.arena_gb * 2 ** 30 // 4)
    waves, cur, used = [], [], 0
    for i, n in enumerate(sizes):
        n_al = (n + 63) // 64 * 64
        if cur and used + n_al > cap:
            waves.append(cur)
            cur, used = [], 0
        cur.append((i, used))
        used += n_al
    waves.append(cur)
    arena = torch.empty(max(sum((sizes[i] + 63) // 64 * 64 for i, _ in wv) for wv in waves), dtype=torch.float32,
                        device=dev)
    outs = [[arena[o:o + sizes[i]].view(sens[i].h_shape()) for i, o in wv] for wv in waves]
    stream = torch.cuda.current_stream()

    def step():
        for wv, ob in zip(waves, outs):
            P.extend_batch([sens[i] for i, _ in wv], outs=ob, stream=stream)

    t1 = time.perf_counter()
    step()                      # first call: autotuning and graph capture
    torch.cuda.synchronize()
    capture_s = time.perf_counter() - t1
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    if args.profile:
        torch.cuda.cudart().cudaProfilerStart()
    with Clocks(f"_{rank}") as clk:
        barrier(world)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    if args.profile:
        torch.cuda.cudart().cudaProfilerStop()
    ms = a.elapsed_time(b) / args.steps
    ms_max = max_over_ranks(ms, world)
    value = world * ps_step / (ms_max / 1e3)
    peak, peak_kind = peaks()
    tun = {}
    for s_, w in zip(sens, ws):
        tun[f"{w.grid.Nx}x{w.grid.Ny}x{w.grid.Nz}"] = s_.tuning()
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "point-samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS["c3"], "l2": "inputs and outputs (377 GB of H per step) far above L2",
                       "parallelism": f"replicas x{world}", "waves": len(waves), "arena_gb": args.arena_gb,
                       "sensors": len(ws), "point_samples": ps_step},
            "roofline": {"bound": "hbm", "achieved": 12.0 * ps_step / (ms_max / 1e3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": 12.0 * ps_step / (ms_max / 1e3) / 1e9 / peak, "traffic": None,
                         "kernel": "whole step (graphs of spectral passes + persistent expansion)",
                         "peak_kind": peak_kind},
            "cpu_baseline": None, "e2e": None, "gpu_launches": None,
            "clocks": clk.summary(local), "setup_s": setup, "first_call_s": capture_s, "tuning": tun,
        }
        print(json.dumps(line), flush=True)
    for s_ in sens:
        s_.close()
    return 0


def run_adjoint(args):
    """c4: L = mean i^2 of Eq. 1 currents over 1e4 tracks and its gradient with
    respect to the readout/bias resistivity scales, radius and lateral scale
    (wt_eq1_loss_grad: four tangent sweeps of the FP32 extension and Eq. 1).
    A step = one loss-and-gradient evaluation; the loss alone is timed too."""
    import numpy as np
    import torch
    import paper_2605_13987_gb300 as P
    import workloads as W

    rank, local, world = dist_init()
    torch.cuda.set_device(local)
    P.load_library()
    w = W.workload("c4")
    tr = w.tracks
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=f"cuda:{local}")
    t = dict(n_tracks=tr.n_tracks, n_steps=tr.n_steps, n_out=tr.n_out, dt=tr.dt, charge=1.0,
             x=dev(tr.x), y=dev(tr.y), z=dev(tr.z), vx=dev(tr.vx), vy=dev(tr.vy), vz=dev(tr.vz), q=dev(tr.charge))
    t0 = time.perf_counter()
    sen = P.Sensor(w.grid, w.columns, device=local)
    sen.fit()
    sen.relax(w.times)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    H = sen.extend("fp32")           # tunes the launch shapes
    torch.cuda.synchronize()
    del H
    for _ in range(args.warmup):
        sen.loss_grad(t)
    per = []
    if args.profile:
        torch.cuda.cudart().cudaProfilerStart()
    with Clocks(f"_{rank}") as clk:
        barrier(world)
        for _ in range(args.steps):
            torch.cuda.synchronize()
            a = time.perf_counter()
            L, g = sen.loss_grad(t)
            torch.cuda.synchronize()
            per.append(time.perf_counter() - a)
        if args.profile:
            torch.cuda.cudart().cudaProfilerStop()
        barrier(world)
        a = time.perf_counter()
        L32 = sen.loss(t, "fp32")
        torch.cuda.synchronize()
        loss_s = time.perf_counter() - a
    # one more evaluation with the library's stage events on (outside the timed steps)
    sen.set_timing(True)
    sen.loss_grad(t)
    stages = sen.grad_timing()
    sen.set_timing(False)
    s = max_over_ranks(statistics.median(per), world)
    if rank == 0:
        line = {"metric": "Eq. 1 loss + 4-parameter gradient evaluations/sec", "value": world / s,
                "unit": "evaluations/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * s, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOADS["c4"], "tracks": tr.n_tracks, "steps_per_track": tr.n_steps,
                           "grid_points": w.grid.Nx * w.grid.Ny * w.grid.Nz, "time_samples": len(w.times)},
                "loss": L, "gradient": list(map(float, g)), "loss_only_ms": 1e3 * loss_s,
                "grad_stage_ms": stages,
                "grad_trunc_rel": sen.info()["grad_trunc_rel"], "clocks": clk.summary(local), "setup_s": setup,
                "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None}
        print(json.dumps(line), flush=True)
    sen.close()
    return 0


def run_large(args):
    """c5: the largest single-GPU case.  A step is one FP32 extension (H 43.5 GB in HBM) followed
    by Eq. 1 for 1e5 drift tracks from the field's rank-r form (wt_eq1_direct; Eq. 1 on the
    stored H is timed once beside it and compared).  The oracle cannot solve this size in a
    test, so the line carries full-size checks on the GPU: the FP32 field against the FP64 plain
    path over the whole of H, and the FP64 grid against the exact point evaluation at sampled
    grid points."""
    import numpy as np
    import torch
    import paper_2605_13987_gb300 as P

    rank, local, world = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.load_library()
    w = make_workload("c5")
    g = w.grid
    npts = g.Nx * g.Ny * g.Nz
    nt = len(w.times)
    tr = w.tracks
    t0 = time.perf_counter()
    sen = P.Sensor(w.grid, w.columns, device=local)
    cond = sen.fit()
    sen.relax(w.times)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    info = sen.info()
    d = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    tracks = dict(n_tracks=tr.n_tracks, n_steps=tr.n_steps, n_out=tr.n_out, dt=tr.dt, charge=1.0,
                  x=d(tr.x), y=d(tr.y), z=d(tr.z), vx=d(tr.vx), vy=d(tr.vy), vz=d(tr.vz), q=d(tr.charge))
    H = torch.empty((nt, 3, g.Nx, g.Ny, g.Nz), dtype=torch.float32, device=dev)
    cur = torch.empty((tr.n_tracks, tr.n_out), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        sen.extend("fp32", out=H)
        sen.eq1_direct(tracks, out=cur)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
    with Clocks(f"_{rank}") as clk:
        barrier(world)
        torch.cuda.synchronize()
        if args.profile:
            torch.cuda.cudart().cudaProfilerStart()
        for k in range(args.steps):
            ev[3 * k].record(stream)
            sen.extend("fp32", out=H)
            ev[3 * k + 1].record(stream)
            sen.eq1_direct(tracks, out=cur)
            ev[3 * k + 2].record(stream)
        torch.cuda.synchronize()
        if args.profile:
            torch.cuda.cudart().cudaProfilerStop()
        barrier(world)
    ext_ms = statistics.median(ev[3 * k].elapsed_time(ev[3 * k + 1]) for k in range(args.steps))
    eq1_ms = statistics.median(ev[3 * k + 1].elapsed_time(ev[3 * k + 2]) for k in range(args.steps))
    # the extension's own stage split (library CUDA events), from one more call outside the timed steps
    sen.set_timing(True)
    sen.extend("fp32", out=H)
    tm, _ = sen.timing()
    sen.set_timing(False)
    ext_stages = {"column_transform": tm[0], "spectral_passes": tm[1], "expansion": tm[2]}
    step_ms = max_over_ranks(ext_ms + eq1_ms, world)
    # full-size checks: FP32 against the FP64 plain path (whole H, per time sample), FP64 grid
    # values against the exact point evaluation at sampled grid points
    checks = {}
    if rank == 0 and not args.no_fp64:
        cur_h = torch.empty_like(cur)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sen.eq1(H, tracks, out=cur_h)
        e1.record(stream)
        torch.cuda.synchronize()
        checks["eq1_on_H_ms"] = e0.elapsed_time(e1)
        checks["eq1_direct_vs_on_H_rel_l2"] = float((cur - cur_h).double().norm() / cur_h.double().norm())
        del cur_h
        H64 = torch.empty((nt, 3, g.Nx, g.Ny, g.Nz), dtype=torch.float64, device=dev)
        a = time.perf_counter()
        sen.extend("fp64", out=H64)
        torch.cuda.synchronize()
        fp64_s = time.perf_counter() - a
        num = den = 0.0
        for t in range(nt):
            diff = H[t].double() - H64[t]
            num += float((diff * diff).sum())
            den += float((H64[t] * H64[t]).sum())
        checks["fp32_vs_fp64_rel_l2"] = (num / den) ** 0.5
        rng = np.random.default_rng(5)
        ix, iy, iz = rng.integers(0, g.Nx, 64), rng.integers(0, g.Ny, 64), rng.integers(0, g.Nz, 64)
        ts = np.sort(rng.choice(nt, 4, replace=False))
        xyz = np.stack([ix * g.Lx / g.Nx, iy * g.Ly / g.Ny, (iz + 0.5) * g.Lz / g.Nz], axis=1)
        exact = sen.sample_H(xyz, w.times[ts])                     # [4][64][3]
        grid = H64[torch.as_tensor(ts, device=dev)][:, :, ix, iy, iz].permute(0, 2, 1).cpu().numpy()
        checks["fp64_grid_vs_point_rel_l2"] = float(np.linalg.norm(grid - exact) / np.linalg.norm(exact))
        checks["fp64_plain_s"] = fp64_s
        checks["eq1_finite"] = bool(torch.isfinite(cur).all())
        del H64
    if rank == 0:
        ps = npts * nt
        line = {"metric": "H grid-point*time-samples/sec (FP32 extension) with Eq. 1 for 1e5 drift tracks per step "
                          "(Eq. 1 from the rank-r field form)",
                "value": world * ps / (step_ms / 1e3), "unit": "point-samples/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOADS["c5"], "grid_points": npts, "time_samples": nt,
                           "tracks": tr.n_tracks, "rank": info["rank"],
                           "l2": "inputs and outputs (43.5 GB of H) far above L2"},
                "stage_ms": {"extension": ext_ms, "eq1": eq1_ms}, "extension_stage_ms": ext_stages,
                "extension_frac_of_hbm_roof": 12.0 * ps / (ext_ms / 1e3) / 1e9 / peaks()[0],
                "checks": checks, "tuning": sen.tuning(), "clocks": clk.summary(local), "setup_s": setup,
                "setup": {"fit_s": info["fit_seconds"], "relax_s": info["relax_seconds"], "cond_estimate": cond,
                          "fit_correction": info["fit_correction"], "fit_refined": info["fit_refined"]},
                "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None}
        print(json.dumps(line), flush=True)
    sen.close()
    return 0


def run_eq1_prof(args):
    """Eq. 1 from the rank-r form alone (wt_eq1_direct) on the prof_eq1 workload: a profiling case
    for the Eq. 1 kernels at the 5x5 cell's track recipe, with basis fields a tenth of its size."""
    import numpy as np
    import torch
    import paper_2605_13987_gb300 as P

    rank, local, world = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.load_library()
    w = make_workload("prof_eq1")
    tr = w.tracks
    sen = P.Sensor(w.grid, w.columns, device=local)
    sen.fit()
    sen.relax(w.times)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    tracks = dict(n_tracks=tr.n_tracks, n_steps=tr.n_steps, n_out=tr.n_out, dt=tr.dt, charge=1.0,
                  x=d(tr.x), y=d(tr.y), z=d(tr.z), vx=d(tr.vx), vy=d(tr.vy), vz=d(tr.vz), q=d(tr.charge))
    cur = torch.empty((tr.n_tracks, tr.n_out), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        sen.eq1_direct(tracks, out=cur)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    if args.profile:
        torch.cuda.cudart().cudaProfilerStart()
    for k in range(args.steps):
        ev[2 * k].record(stream)
        sen.eq1_direct(tracks, out=cur)
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    if args.profile:
        torch.cuda.cudart().cudaProfilerStop()
    ms = statistics.median(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps))
    if rank == 0:
        print(json.dumps({"workload": WORKLOADS["prof_eq1"], "eq1_ms": ms, "tracks": tr.n_tracks,
                          "steps_per_track": tr.n_steps, "n_out": tr.n_out, "rank": sen.info()["rank"],
                          "finite": bool(torch.isfinite(cur).all())}), flush=True)
    sen.close()
    return 0


def run_scan_bench(args):
    """Sec. 5's bias-diameter scan through the scan driver: a step is the
    whole scan (five variants: fit, relaxation, currents and tangents,
    shaping, features and sensitivities).  Reports variants per second and
    the features' track medians per diameter."""
    import numpy as np
    import torch
    import paper_2605_13987_gb300 as P
    import workloads as W
    from paper_2605_13987_gb300.scan import run_scan

    rank, local, world = dist_init()
    torch.cuda.set_device(local)
    P.load_library()
    pts = W.scan_bias_diameter()
    shaper = dict(tau=0.5e-9, order=2)
    for _ in range(args.warmup):
        run_scan(pts, sensitivities=True, shaper=shaper, device=local)
    per = []
    with Clocks(f"_{rank}") as clk:
        barrier(world)
        for _ in range(args.steps):
            torch.cuda.synchronize()
            a = time.perf_counter()
            res = run_scan(pts, sensitivities=True, shaper=shaper, device=local)
            torch.cuda.synchronize()
            per.append(time.perf_counter() - a)
        barrier(world)
    s = max_over_ranks(statistics.median(per), world)
    if rank == 0:
        summ = {}
        for r in res:
            m = r.summary()
            ds = np.median(r.dfeatures, axis=1)            # [4 params, 6 features], track medians
            summ[f"{r.value:g}um"] = {"amplitude": m["amplitude"], "rise_time_s": m["rise_time"],
                                      "t_cfd_s": m["t_cfd"], "charge": m["charge"],
                                      "dt_cfd_ds_R": float(ds[0, 5]), "dt_cfd_ds_B": float(ds[1, 5]),
                                      "fit_s": r.info["fit_seconds"], "relax_s": r.info["relax_seconds"]}
        line = {"metric": "scan variants/sec (fit, relaxation, currents + 4 tangents, shaping, features)",
                "value": world * len(pts) / s, "unit": "variants/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * s, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64 setup, f32 field", "data": "synthetic",
                "config": {"workload": WORKLOADS["scan"], "variants": len(pts)},
                "scan": summ, "clocks": clk.summary(local),
                "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None}
        print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import paper_2605_13987_gb300 as P

    rank, local, world = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.load_library()
    w = make_workload(args.workload)
    g = w.grid
    npts = g.Nx * g.Ny * g.Nz
    nt = len(w.times)
    ps_step = npts * nt

    t0 = time.perf_counter()
    sen = P.Sensor(w.grid, w.columns, device=local)
    cond = sen.fit()
    sen.relax(w.times)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    info = sen.info()

    H = torch.empty((nt, 3, g.Nx, g.Ny, g.Nz), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        sen.extend("fp32", out=H)
    torch.cuda.synchronize()

    sen.set_timing(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage_ms = []
    launches = 0
    if args.profile:
        torch.cuda.cudart().cudaProfilerStart()
    with Clocks(f"_{rank}") as clk:
        barrier(world)
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            sen.extend("fp32", out=H)
            ends[k].record(stream)
            ms3, n = sen.timing()
            stage_ms.append(ms3)
            launches += n
        torch.cuda.synchronize()
        barrier(world)
    if args.profile:
        torch.cuda.cudart().cudaProfilerStop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = sum(step_ms) / len(step_ms)
    ms_max = max_over_ranks(ms, world)
    value = world * ps_step / (ms_max / 1e3)

    # dominant kernel: the expansion; algorithmic bytes = 12 B per point-sample (H written once)
    exp_ms = sum(s[2] for s in stage_ms) / len(stage_ms)
    peak, peak_kind = peaks()
    alg_bytes = 12.0 * ps_step
    achieved = alg_bytes / (exp_ms / 1e3) / 1e9
    traffic = None
    tr_file = os.path.join(ROOT, "profiles", "expand_tc_traffic.json")
    if os.path.exists(tr_file) and args.workload == "c2":
        # valid only while the kernel source is the one the counters were taken on
        try:
            import hashlib
            rec = json.load(open(tr_file))
            src = open(os.path.join(ROOT, "paper_2605_13987_gb300", "csrc", "k_expand_tc.cu"), "rb").read()
            if rec.get("kernel_source_sha256") == hashlib.sha256(src).hexdigest():
                traffic = rec.get("bytes_per_launch_full_size")
        except Exception:
            traffic = None

    # end to end through the C ABI: pinned host output, device compute + D2H copy of H
    e2e = None
    if not args.no_e2e and not args.profile:
        # pinned host memory (25.8 GB per rank for c2); should the host refuse that much pinned
        # memory (several ranks on one node), the same call runs into pageable memory
        try:
            Hh = torch.empty((nt, 3, g.Nx, g.Ny, g.Nz), dtype=torch.float32, pin_memory=True)
            host_mem = "pinned"
        except RuntimeError:
            Hh = torch.empty((nt, 3, g.Nx, g.Ny, g.Nz), dtype=torch.float32)
            host_mem = "pageable (the pinned allocation was refused)"
        sen.set_timing(False)
        sen.extend("fp32", out=Hh)
        # the host link alone: a plain device-to-host copy of the same bytes into the same buffer
        # (H of the device-buffer steps) right before every call, so that each call is compared
        # with the link as it was at that moment (the host's link is shared and drifts)
        barrier(world)
        k2 = max(1, min(9, args.steps))
        per_call, link = [], []
        for _ in range(k2):             # each call is one whole end-to-end step; the median is reported
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            Hh.copy_(H, non_blocking=True)
            torch.cuda.synchronize()
            link.append(time.perf_counter() - t1)
            t1 = time.perf_counter()
            sen.extend("fp32", out=Hh)
            torch.cuda.synchronize()
            per_call.append(time.perf_counter() - t1)
        el = max_over_ranks(statistics.median(per_call), world)
        e2e = {"value": world * ps_step / el, "unit": "point-samples/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": int(Hh.numel() * 4), "ms_per_call": [1e3 * t for t in per_call],
               "ms_min": 1e3 * min(per_call), "ms_median": 1e3 * statistics.median(per_call),
               "ms_max": 1e3 * max(per_call), "host_memory": host_mem,
               "link_floor_ms": 1e3 * statistics.median(link), "link_ms_per_call": [1e3 * t for t in link],
               "median_over_link_floor": statistics.median(per_call) / statistics.median(link),
               "median_call_over_its_link": statistics.median(a / b for a, b in zip(per_call, link)),
               "inputs": "none copied per step: the step's inputs (the relaxed charge history and the geometry "
                         "tables) are already on the device after wt_relax; H (the output) is copied out"}
        del Hh

    # the comparison path of the metric: the FP64 plain extension (one FP64 spectral transform per
    # time sample), timed once after one untimed call, into its own device buffer
    fp64 = None
    accuracy = None
    if not args.no_fp64 and not args.profile:
        H64 = torch.empty((nt, 3, g.Nx, g.Ny, g.Nz), dtype=torch.float64, device=dev)
        sen.set_timing(False)
        sen.extend("fp64", out=H64)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sen.extend("fp64", out=H64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": ps_step / (ms64 / 1e3), "unit": "point-samples/s", "ms_per_step": ms64,
                "dtype": "f64", "fp32_speedup": ms64 / ms_max}
        # the metric's accuracy: the timed FP32 H (last timed step, still in H) against the FP64
        # plain H, over the whole array and per time sample
        num = torch.empty(nt, dtype=torch.float64, device=dev)
        den = torch.empty(nt, dtype=torch.float64, device=dev)
        for t in range(nt):
            d = H[t].double() - H64[t]
            num[t] = (d * d).sum()
            den[t] = (H64[t] * H64[t]).sum()
        per = (num / den).sqrt().cpu().numpy()
        worst = int(per.argmax())
        accuracy = {"rel_l2_vs_fp64": float((num.sum() / den.sum()).sqrt()), "tolerance": 1e-5,
                    "worst_sample_rel_l2": float(per[worst]), "worst_sample": worst,
                    "worst_sample_time_s": float(w.times[worst]), "first_sample_rel_l2": float(per[0]),
                    "per_sample_max_within_tolerance": bool(per.max() <= 1e-5)}
        del H64, d

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.profile:
        import oracle as O
        t2 = time.perf_counter()
        sol = O.solve(w)
        osetup = time.perf_counter() - t2
        # the same oracle draws twice, each in a child process: BLAS on all host cores (its
        # default) and on one thread (OMP/OPENBLAS/MKL/BLIS_NUM_THREADS=1)
        allc = cpu_baseline_threads(w, sol, 10.0, None)
        one = cpu_baseline_threads(w, sol, 10.0, 1)
        if allc is not None:
            cpu = {"value": allc[0], "unit": "point-samples/s", "cores": os.cpu_count(),
                   "threads": f"BLAS default: {os.cpu_count()} host cores", "kind": "oracle",
                   "sample": f"4 time samples x 12^3 random grid points per draw, {allc[1]:.1f} s of draws; "
                             f"oracle setup ({osetup:.1f} s) excluded like the GPU setup",
                   "single_thread": None if one is None else
                   {"value": one[0], "unit": "point-samples/s", "cores": 1, "threads": 1,
                    "sample": f"the same draws, {one[1]:.1f} s, BLAS limited to one thread"}}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "point-samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{world}", "rank": info["rank"], "time_samples": nt,
                       "grid_points": npts},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "expand_tc_kernel", "peak_kind": peak_kind,
                         "alg_bytes_per_launch": alg_bytes, "launch_ms": exp_ms},
            "stage_ms": {"column_transform": sum(s[0] for s in stage_ms) / len(stage_ms),
                         "spectral_passes": sum(s[1] for s in stage_ms) / len(stage_ms),
                         "expansion": exp_ms},
            "tuning": sen.tuning(),
            "step_frac_of_hbm_roof": (alg_bytes / (ms_max / 1e3) / 1e9) / peak,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "fp64_plain": fp64, "accuracy": accuracy,
            "clocks": clk.summary(local),
            "setup_s": setup,
            "setup": {"fit_s": info["fit_seconds"], "relax_s": info["relax_seconds"], "cond_estimate": cond,
                      "boundary_residual": info["boundary_residual"], "trunc_rel": info["trunc_rel"],
                      "fit_correction": info["fit_correction"], "fit_refined": info["fit_refined"]},
        }
        print(json.dumps(line), flush=True)
    sen.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--no-fp64", action="store_true", help="skip timing the FP64 plain path")
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--arena-gb", type=float, default=96.0, help="c3: device memory for one wave's H")
    ap.add_argument("--cpu-sample-from", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help=argparse.SUPPRESS)
    ap.add_argument("--profile", action="store_true",
                    help="wrap only the timed steps in cudaProfilerStart/Stop (for ncu --profile-from-start off); "
                         "skips the CPU baseline and e2e")
    args = ap.parse_args()
    if args.cpu_sample_from:
        return cpu_sample_child(args.cpu_sample_from, args.cpu_seconds)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c3":
        return run_batch(args)
    if args.workload == "c4":
        return run_adjoint(args)
    if args.workload == "scan":
        return run_scan_bench(args)
    if args.workload == "c5":
        return run_large(args)
    if args.workload == "prof_eq1":
        return run_eq1_prof(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python3
"""Throughput of the WENO-L hot path on one GB300 (or N replicas under torchrun).

Workload (default): Example 3 of the paper -- phi_t + (phi_x + phi_y + 1)^2/2 = 0
on [-2, 2)^2 periodic, phi0 = -cos(pi (x + y)/2) -- on an 8192 x 8192 grid,
arc-length weights, eps = 1e-6, CFL 0.6, Lax-Friedrichs with the lagged grid
maximum alpha, mixed precision (float stencil, phi^n as two floats, double CFL
reduction).  One bench step = one TVD-RK3 time step = three fused stage
kernels.  Metric: point-updates/s = grid nodes x steps / device time.

Also reported: per-stage roofline (the stage kernel), an end-to-end solve to
t = 0.5/pi^2 through the C ABI with host buffers, clocks sampled during the
timed region, and the FP64 CPU oracle on a bounded sample (cpu_baseline).

--impl reference times the FP64 CPU oracle instead (bounded samples of the
same workload per step) and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "WENO-AL point-updates/s"
UNIT = "point-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
MUFU_PER_SM_CLK = 16          # measured: rsqrt / lg2 / rcp.approx throughput per SM per clock
FP32_LANES_PER_SM = 128

# algorithmic work of one 2D node in one stage (arc-length weights, Burgers H):
# per direction 3 F evaluations (rsqrt + lg2), 3 interval means (1 reciprocal each),
# 2 weight sets (1 reciprocal each) -> 11 MUFU ops; FP32 flops ~107 per direction
# plus ~33 for alpha, H-hat and the RK combination; bytes: each array read or written once per stage
# (MIXED arc length on smooth data runs the short-interval sweep: per direction 3 square roots and
# 2 weight reciprocals, 5 MUFU ops; "mufu_full" is the count of the full sweep)
ALGO = {
    ("arclength", "mixed"): {"mufu": 10, "mufu_full": 22, "flops": 250, "bytes": (12, 16, 20)},
    ("arclength", "fp32"): {"mufu": 22, "flops": 240, "bytes": (8, 12, 12)},
    ("jp", "mixed"): {"mufu": 4, "flops": 180, "bytes": (12, 16, 20)},
    ("jp", "fp32"): {"mufu": 4, "flops": 170, "bytes": (8, 12, 12)},
    ("arclength", "fp64"): {"mufu": 0, "flops": 250, "bytes": (16, 24, 24)},
}


# the translation unit of the 2D stage kernel (the dominant kernel) and everything it includes
STAGE2D_SOURCES = ("alw_stage2d_mixed.cu", "alw_stage2d_f32.cu", "alw_launch2d.cuh", "alw_stage2d.cuh",
                   "alw_sweep32.cuh", "alw_tma.cuh", "alw_params2d.h", "alw_device.cuh", "alw_internal.h")


def _kernel_source_hash() -> str:
    """Hash of the stage kernel's sources with `//` comments, blank lines and diagnostic pragmas removed
    (an edit of those does not change the kernel the traffic record was taken on)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1909_13263_gb300", "csrc")
    for f in STAGE2D_SOURCES:
        for line in open(os.path.join(csrc, f), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code.lstrip().startswith(("#pragma nv_diagnostic", "#pragma nv_diag_suppress")):
                continue
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float) -> float:
    """Maximum of a per-rank number over the process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                clk, cmax = float(r[1]), float(r[2])
            except (ValueError, IndexError):
                continue
            sm.append(clk)
            mx = max(mx, cmax)
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        load = [c for c in sm if c > 0.5 * max(sm)]
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(PEAKS_FILE)), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def _traffic():
    """DRAM bytes per stage launch from the committed ncu capture, if the kernel is unchanged."""
    try:
        t = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    if t.get("source_hash") != _kernel_source_hash():
        return None
    return t


def cpu_oracle_rate(n: int, steps: int):
    """FP64 oracle (one core) on an n x n Example-3 grid for `steps` RK3 steps."""
    t0, t1, st = _oracle_sample(n, steps)
    return n * n * st / (t1 - t0), t1 - t0, st


def _oracle_sample(n: int, steps: int):
    """One timed oracle solve: (start, end) on the system-wide monotonic clock and the RK3 steps taken."""
    import oracle
    from paper_1909_13263_gb300 import inputs

    x, dx = inputs.axis(n, -2.0, 2.0, "periodic")
    phi0 = inputs.phi0_negcos_diag_2d(x, x)
    cfg = oracle.make_cfg(dim=2, nx=n, ny=n, dx=dx, ham="burgers2d", weights="arclength",
                          alpha_mode="global_lagged")
    a, _ = oracle.alpha_of(cfg, phi0)
    dt = 0.6 / (a[0] / dx + a[1] / dx)
    t0 = time.monotonic()
    _, st, _, _, _ = oracle.solve(cfg, phi0, steps * dt * 0.999999, alpha_state=a.copy())
    return t0, time.monotonic(), st


def _oracle_case(kind: str, n: int, steps: int):
    """One timed oracle run of about `steps` RK3 steps with the CFL time step: (start, end, steps, nodes).

    kind "ex3": Example 3 on an n x n grid (as _oracle_sample); "k1": 1D, [-1, 1) periodic with n nodes,
    phi0 = -cos(pi x), H = (p + 1)^2 / 2 (the 1D accuracy workload), local lagged alpha."""
    if kind == "ex3":
        t0, t1, st = _oracle_sample(n, steps)
        return t0, t1, st, n * n
    import oracle
    from paper_1909_13263_gb300 import inputs

    x, dx = inputs.axis(n, -1.0, 1.0, "periodic")
    phi0 = inputs.phi0_negcos_1d(x)
    cfg = oracle.make_cfg(dim=1, nx=n, dx=dx, ham="burgers1d", weights="arclength", alpha_mode="local_lagged")
    a, _ = oracle.alpha_of(cfg, phi0)
    dt = 0.6 * dx / a[0]
    t0 = time.monotonic()
    _, st, _, _, _ = oracle.solve(cfg, phi0, steps * dt * 0.999999, alpha_state=a.copy())
    return t0, time.monotonic(), st, n


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The oracle on every host core at once: one independent n x n instance per worker process.

    Instances are independent, so the all-core figure is (workers x nodes x steps) / the span from the
    first worker's solve start to the last worker's solve end, on the system-wide monotonic clock (so a
    worker that ran two tasks back to back only lengthens the span).  Input set-up happens before each
    worker's start, as in the one-core figure.  Workers are spawned (never forked after CUDA has been
    initialised) and each loads the oracle once, before the first timed sample.
    """

    def __init__(self, workers: int):
        import multiprocessing as mp

        import oracle

        oracle.build()
        self.workers = workers
        self._pool = mp.get_context("spawn").Pool(workers)
        self._pool.starmap(_oracle_sample, [(16, 1)] * workers)    # load numpy and the oracle in every worker

    def rate(self, n: int, steps: int):
        """Aggregate point-updates/s, the span in seconds and the steps per instance for one sample."""
        return self.rate_case("ex3", n, steps)

    def rate_case(self, kind: str, n: int, steps: int):
        """As rate, for any workload of _oracle_case."""
        res = self._pool.starmap(_oracle_case, [(kind, n, steps)] * self.workers, chunksize=1)
        span = max(r[1] for r in res) - min(r[0] for r in res)
        st, nodes = res[0][2], res[0][3]
        return self.workers * nodes * st / span, span, st

    def close(self):
        self._pool.close()
        self._pool.join()


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    cores = args.cpu_cores or _host_cores()
    pool = OraclePool(cores)
    n = args.ref_n
    for _ in range(args.warmup):
        pool.rate(n, 1)
    total_pts, total_t = 0, 0.0
    for _ in range(args.steps):
        r, el, st = pool.rate(n, 1)
        total_pts += cores * n * n * st
        total_t += el
    pool.close()
    value = total_pts / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"ex3_burgers2d_{args.n}sq", "sample_grid": f"{n}x{n}",
                   "sample": f"each bench step: one RK3 step of the workload's scheme on {cores} independent "
                             f"{n}x{n} grids (one per core), not on the {args.n}x{args.n} grid itself",
                   "weights": "arclength"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"one RK3 step of Example 3 on {cores} independent {n}x{n} grids "
                                   f"(one process per core) per bench step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _latency_summary(lat):
    import numpy as np

    a = np.asarray(lat)
    return {"p50_s": float(np.percentile(a, 50)), "p99_s": float(np.percentile(a, 99)),
            "mean_s": float(a.mean())}


def bench_batched(args, stream):
    """512 instances of uneven size (64^2..1024^2, two Hamiltonians, phase-shifted phi0, own
    t_final), host to host: one batch vs a loop of one-at-a-time solves."""
    from paper_1909_13263_gb300 import inputs, native

    insts = inputs.batch_instances(args.batch_count, 64, 1024)
    phis = [inputs.instance_phi0(i)[0] for i in insts]
    kw = dict(xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0)
    node_steps = 0
    t0 = time.perf_counter()
    with native.Batch(precision="mixed", weights=args.weights, stream=stream) as b:
        for inst, ph in zip(insts, phis):
            b.add(nx=inst.n, ny=inst.n, ham=inst.ham, phi0=ph, t_final=inst.t_final, **kw)
        replays = b.run()
        outs = [b.get_phi(k) for k in range(len(insts))]
        for k, inst in enumerate(insts):
            node_steps += inst.n * inst.n * b.get_state(k).steps
        tuning = b.tuning()
        mem = b.memory_bytes()
    t_batch = time.perf_counter() - t0
    # the tile widths and launch forms the autotuner chooses from, each fixed, on the same batch: the
    # time loop alone (alw_batch_run after the arena is built), twice each in alternating order
    forms = [(64, False), (32, False), (64, True)]
    widths = {f"{w}x32{', one launch per stage' if one else ', one launch per Hamiltonian'}": []
              for w, one in forms}
    for w, one in forms + forms:
        with native.Batch(precision="mixed", weights=args.weights, stream=stream) as bw:
            for inst, ph in zip(insts, phis):
                bw.add(nx=inst.n, ny=inst.n, ham=inst.ham, phi0=ph, t_final=inst.t_final, **kw)
            bw.set_tuning(order=tuning["order"], steps_per_graph=tuning["steps_per_graph"], run=tuning["run"],
                          tile_w=w, one_launch=one)
            bw.build()
            t1 = time.perf_counter()
            bw.run()
            widths[f"{w}x32{', one launch per stage' if one else ', one launch per Hamiltonian'}"].append(
                time.perf_counter() - t1)
    widths = {k: {"run_s": v, "solves_per_s": len(insts) / min(v)} for k, v in widths.items()}
    serial_n = min(len(insts), args.serial_count)
    t0 = time.perf_counter()
    for inst, ph in list(zip(insts, phis))[:serial_n]:
        with native.Solver(dim=2, nx=inst.n, ny=inst.n, ham=inst.ham, precision="mixed", weights=args.weights,
                           stream=stream, **kw) as s:
            s.set_phi0(ph)
            s.step_to(inst.t_final)
            s.get_phi()
    t_serial = time.perf_counter() - t0
    ok = all(bool((o == o).all()) for o in outs)
    return {"instances": len(insts), "solves_per_s": len(insts) / t_batch,
            "serial_solves_per_s": serial_n / t_serial, "speedup_vs_serial": (len(insts) / t_batch) / (serial_n / t_serial),
            "point_updates_per_s": node_steps / t_batch, "wall_s": t_batch, "graph_replays": replays,
            "tuning": tuning, "fixed_tunings_time_loop": widths, "device_bytes": mem, "serial_sample": serial_n,
            "finite": ok}


def bench_serving(args, stream, rate):
    """Poisson arrivals of solves (128^2..2048^2, the batch mix) into the continuous-batching server
    under an HBM budget; latency from arrival to result, against one-at-a-time plain solves."""
    import threading

    from paper_1909_13263_gb300 import inputs, native

    reqs = inputs.request_stream(rate, args.serve_count, 128, 2048)
    phis = [inputs.instance_phi0(i)[0] for _, i in reqs]
    kw = dict(xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0)
    with native.Server(hbm_budget_bytes=int(args.serve_budget_gb * 2**30), max_slots=256, max_side=2048,
                       weights=args.weights, stream=stream) as srv:
        srv.set_round_steps(args.serve_round_steps)
        if args.serve_round_tiles is not None:
            srv.set_round_tiles(args.serve_round_tiles)
        ids = [None] * len(reqs)
        t0 = time.perf_counter()
        for k, ((at, inst), ph) in enumerate(zip(reqs, phis)):
            delay = t0 + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids[k] = srv.submit(nx=inst.n, ny=inst.n, ham=inst.ham, phi0=ph, t_final=inst.t_final, **kw)
        lat = []
        for rid in ids:
            done, info, _ = srv.poll(rid, timeout=600.0, fetch=True)
            lat.append(info["latency_s"])
        makespan = time.perf_counter() - t0
        rounds = srv.stats()["rounds"]
    served = {"rate_per_s": rate, "requests": len(reqs), "solves_per_s": len(reqs) / makespan,
              "rounds": rounds, "round_steps": args.serve_round_steps,
              "round_tiles": "default" if args.serve_round_tiles is None else args.serve_round_tiles,
              **_latency_summary(lat)}
    # one-at-a-time plain solves of the same arrivals (FIFO, a single worker)
    lat_s = []
    done_at = 0.0
    t0 = time.perf_counter()
    for (at, inst), ph in zip(reqs, phis):
        delay = t0 + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        with native.Solver(dim=2, nx=inst.n, ny=inst.n, ham=inst.ham, precision="mixed", weights=args.weights,
                           stream=stream, **kw) as s:
            s.set_phi0(ph)
            s.step_to(inst.t_final)
            s.get_phi()
        done_at = time.perf_counter() - t0
        lat_s.append(done_at - at)
    serial = {"solves_per_s": len(reqs) / done_at, **_latency_summary(lat_s)}
    return {"served": served, "serial": serial,
            "p99_speedup_vs_serial": serial["p99_s"] / served["p99_s"],
            "solves_per_s_vs_serial": served["solves_per_s"] / serial["solves_per_s"],
            "budget_gb": args.serve_budget_gb}


def _host_description() -> dict:
    import platform

    d = {"machine": platform.machine(), "cores": _host_cores(), "cpu_count": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:") or line.startswith("Vendor ID:"):
                k, v = line.split(":", 1)
                d[k.strip().lower().replace(" ", "_")] = v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return d


def run_oracle_report(args):
    """The FP64 CPU oracle timed on the host cores (one JSON line): one core, and every core at once with
    one independent instance per core, for the 1D accuracy workload at N = 40, 80, 160, 320 and for
    Example 3 on 400^2 and 2048^2; 8192^2 extrapolated from the 2048^2 cost per node and step.  Each
    sample is sized for about half a second of one-core work (at least one step)."""
    import oracle

    oracle.build()
    cores = args.cpu_cores or _host_cores()
    pool = OraclePool(cores)
    out = {"report": "oracle", "unit": "point-updates/s", "host": _host_description(), "workers": cores}
    # per-node-step cost guesses (s) that size the samples; the measured cost replaces them
    guess = {"k1": 6e-7, "ex3": 1.6e-6}
    for kind, sizes, name in (("k1", (40, 80, 160, 320), "k1_burgers1d"), ("ex3", (400, 2048), "ex3_burgers2d")):
        rows = {}
        for n in sizes:
            nodes = n if kind == "k1" else n * n
            steps = max(1, int(0.5 / (guess[kind] * nodes)))
            t0, t1, st, _ = _oracle_case(kind, n, steps)
            one = nodes * st / (t1 - t0)
            allc, span, st2 = pool.rate_case(kind, n, steps)
            rows[f"{n}" if kind == "k1" else f"{n}sq"] = {
                "steps": st, "ms_per_step_one_core": 1e3 * (t1 - t0) / st, "one_core": one,
                "all_cores": allc, "all_cores_span_s": span}
        out[name] = rows
    big = out["ex3_burgers2d"]["2048sq"]
    n8 = 8192 * 8192
    out["ex3_burgers2d"]["8192sq_extrapolated"] = {
        "ms_per_step_one_core": 1e3 * n8 / big["one_core"], "one_core": big["one_core"],
        "all_cores": big["all_cores"], "ms_per_step_all_cores": 1e3 * n8 / big["all_cores"],
        "from": "2048^2 cost per node and step"}
    pool.close()
    print(json.dumps(out), flush=True)
    return 0


def run_sizes_report(args):
    """Device throughput of one RK3 step by grid size and precision (one JSON line).

    Example 3 (Burgers, periodic) on 400^2, 2048^2 and 8192^2 and Example 10 (sin(p+q), linear
    extrapolation) on 1024^2 and 4096^2, in MIXED, FP32 and FP64, plus FP64 Example 3 from 80^2 to
    1024^2, arc-length weights: CUDA events on the solver's stream around a timed run of RK3 steps
    after warm-up steps."""
    import torch

    from paper_1909_13263_gb300 import inputs, native

    native.load()
    native.use_torch_allocator(True)
    stream = torch.cuda.Stream()
    out = {"report": "sizes", "unit": "point-updates/s", "weights": args.weights}
    cases = [("ex3_burgers2d", n, "burgers2d", "periodic", -2.0, 2.0) for n in (400, 2048, 8192)]
    cases += [("ex10_sin2d_linextrap", n, "sin2d", "linextrap", -1.0, 1.0) for n in (1024, 4096)]
    for name, n, ham, bc, lo, hi in cases:
        x, _ = inputs.axis(n, lo, hi, bc)
        phi0 = inputs.phi0_negcos_diag_2d(x, x) if ham == "burgers2d" else inputs.phi0_riemann_2d(x, x)
        row = {}
        for prec in ("mixed", "fp32", "fp64"):
            with torch.cuda.stream(stream):
                with native.Solver(dim=2, nx=n, ny=n, bc=bc, xlo=lo, xhi=hi, ylo=lo, yhi=hi, ham=ham,
                                   precision=prec, weights=args.weights, stream=stream) as s:
                    s.set_phi0(phi0)
                    s.advance(3)
                    torch.cuda.synchronize()
                    # about 0.3 s of timed work (at least 3 steps)
                    rate_guess = {"fp64": 2.0e8}.get(prec, 2.0e10)
                    steps = max(3, min(2000, int(0.3 * rate_guess / (n * n))))
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    s.advance(steps)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / steps
            row[prec] = {"ms_per_step": ms, "point_updates_per_s": n * n / (ms * 1e-3), "steps": steps}
        out[f"{name}_{n}sq"] = row
    # FP64 at the paper's grid sizes (Example 3)
    fp64 = {}
    for n in (80, 160, 320, 640, 1024):
        x, _ = inputs.axis(n, -2.0, 2.0, "periodic")
        with torch.cuda.stream(stream):
            with native.Solver(dim=2, nx=n, ny=n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham="burgers2d",
                               precision="fp64", weights=args.weights, stream=stream) as s:
                s.set_phi0(inputs.phi0_negcos_diag_2d(x, x))
                s.advance(3)
                torch.cuda.synchronize()
                steps = max(3, min(400, int(0.3 * 2.0e8 / (n * n))))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.advance(steps)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
        fp64[f"{n}sq"] = {"ms_per_step": ms, "point_updates_per_s": n * n / (ms * 1e-3), "steps": steps}
    out["ex3_burgers2d_fp64_paper_sizes"] = fp64
    print(json.dumps(out), flush=True)
    return 0


def bench_precision(args, stream):
    """Errors of the MIXED path (the timed precision) against FP64 and the exact solution.

    Example 10 (sin(p + q), pi(|y| - |x|), linear extrapolation; no closed-form solution) on 1024^2 to
    t = 1: MIXED against the FP64 path, max |e| and mean |e|.  Example 3 on 2048^2 to t = 0.5/pi^2:
    FP64 and MIXED against the exact solution (characteristics) and MIXED against FP64."""
    import numpy as np

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import exact
    from paper_1909_13263_gb300 import inputs, native

    out = {"norms": "max = max |e|, l1 = mean |e| over the nodes"}
    n = args.precision_ex10_n
    x, _ = inputs.axis(n, -1.0, 1.0, "linextrap")
    phi0 = inputs.phi0_riemann_2d(x, x)
    res = {}
    for prec in ("fp64", "mixed"):
        with native.Solver(dim=2, nx=n, ny=n, bc="linextrap", xlo=-1.0, xhi=1.0, ylo=-1.0, yhi=1.0,
                           ham="sin2d", precision=prec, stream=stream) as s:
            s.set_phi0(phi0)
            steps = s.step_to(1.0)
            res[prec] = s.get_phi()
    d = np.abs(res["mixed"] - res["fp64"])
    # also over the window |x|, |y| <= 1/2, away from the corners, where this problem (linear extrapolation)
    # amplifies rounding-level differences
    inner = np.ix_(np.abs(x) <= 0.5, np.abs(x) <= 0.5)
    out[f"ex10_sin2d_linextrap_{n}sq_t1"] = {"steps": steps, "mixed_vs_fp64_max": float(d.max()),
                                             "mixed_vs_fp64_l1": float(d.mean()),
                                             "mixed_vs_fp64_max_inner": float(d[inner].max()),
                                             "mixed_vs_fp64_l1_inner": float(d[inner].mean())}
    n = args.precision_ex3_n
    x, _ = inputs.axis(n, -2.0, 2.0, "periodic")
    tf = 0.5 / math.pi**2
    ex = exact.negcos_diag_2d("burgers2d", x, x, tf)
    res = {}
    for prec in ("fp64", "mixed"):
        with native.Solver(dim=2, nx=n, ny=n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham="burgers2d",
                           precision=prec, stream=stream) as s:
            s.set_phi0(inputs.phi0_negcos_diag_2d(x, x))
            s.step_to(tf)
            res[prec] = s.get_phi()
    row = {}
    for prec, phi in res.items():
        e = np.abs(phi - ex)
        row[f"{prec}_vs_exact_max"] = float(e.max())
        row[f"{prec}_vs_exact_l1"] = float(e.mean())
    d = np.abs(res["mixed"] - res["fp64"])
    row["mixed_vs_fp64_max"] = float(d.max())
    row["mixed_vs_fp64_l1"] = float(d.mean())
    row["mixed_l1_ratio_to_fp64"] = row["mixed_vs_exact_l1"] / row["fp64_vs_exact_l1"]
    out[f"ex3_burgers2d_{n}sq"] = row
    return out


def bench_fp64(args, stream):
    """The FP64 path (the oracle-parity precision) on the bench grid: RK3 steps timed with CUDA events."""
    import torch

    from paper_1909_13263_gb300 import inputs, native

    n = args.n
    x, _ = inputs.axis(n, -2.0, 2.0, "periodic")
    with native.Solver(dim=2, nx=n, ny=n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham="burgers2d",
                       precision="fp64", weights=args.weights, alpha_mode="global_lagged", stream=stream) as s:
        s.set_phi0(inputs.phi0_negcos_diag_2d(x, x))
        s.advance(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.advance(args.fp64_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.fp64_steps
    return {"workload": f"ex3_burgers2d_{n}sq", "value": n * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "steps": args.fp64_steps, "bound": "fp64 pipe",
            "fp64_pipe_note": "ncu: FP64 pipe 86 % busy on this kernel (profiles/stage_kernel_fp64_ex3_arclength_1024.md)"}


def run_ours(args):
    import numpy as np
    import torch

    from paper_1909_13263_gb300 import inputs, native

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    native.load()
    native.use_torch_allocator(True)
    stream = torch.cuda.Stream()
    n = args.n
    x, dx = inputs.axis(n, -2.0, 2.0, "periodic")
    tf = 0.5 / math.pi**2
    kw = dict(dim=2, nx=n, ny=n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham="burgers2d", weights=args.weights,
              precision=args.precision, alpha_mode="global_lagged")
    with torch.cuda.stream(stream):
        xs = torch.tensor(x, device="cuda", dtype=torch.float64)
        phi0_dev = -torch.cos(math.pi * (xs[None, :] + xs[:, None]) / 2.0)
        s = native.Solver(stream=stream, **kw)
        s.set_phi0(phi0_dev)
        del phi0_dev
        s.advance(args.warmup)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as cs:
            torch.cuda.synchronize()
            ev0.record(stream)
            s.advance(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        s.sync()
        ms = ev0.elapsed_time(ev1)
        clocks = cs.summary()
        # per-stage device time of the stage kernel, each stage launched alone (events on the launching
        # stream): a breakdown only -- the roofline uses the launches inside the timed graph replays
        st = s.get_state()
        dt = 0.6 / (st.alpha[0] / dx + st.alpha[1] / dx)
        reps = 5
        stage_ms = [0.0, 0.0, 0.0]
        for _ in range(reps):
            for k in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s.run_stage(k + 1, dt)
                b.record(stream)
                b.synchronize()
                stage_ms[k] += a.elapsed_time(b) / reps
        s.sync()
        s.close()
    ms = max_over_ranks(ms)
    value = ws * n * n * args.steps / (ms * 1e-3)

    # end to end: host phi0 -> device -> RK3 solve to t = 0.5/pi^2 -> host phi
    e2e = None
    if not args.no_e2e:
        phi0_host = inputs.phi0_negcos_diag_2d(x, x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = native.Solver(stream=stream, **kw)
        s2.set_phi0(phi0_host)
        nsteps = s2.step_to(tf)
        phi = s2.get_phi()
        el = time.perf_counter() - t0
        s2.close()
        el = max_over_ranks(el)
        e2e = {"value": ws * n * n * nsteps / el, "unit": UNIT,
               "h2d_bytes_per_step": 8 * n * n / nsteps, "d2h_bytes_per_step": 8 * n * n / nsteps,
               "solve": f"t = 0.5/pi^2 in {nsteps} RK3 steps, {el:.3f} s wall",
               "finite": bool(np.isfinite(phi).all())}
        del phi0_host, phi

    batched = serving = None
    if not args.no_batch:
        with torch.cuda.stream(stream):
            batched = bench_batched(args, stream)
    if not args.no_serve:
        with torch.cuda.stream(stream):
            rates = [float(r) for r in args.serve_rates.split(",") if r]
            runs = [bench_serving(args, stream, r) for r in rates]
            top = max(runs, key=lambda r: r["served"]["rate_per_s"])
            serving = {"sweep": runs, "rates_per_s": rates,
                       "solves_per_s_vs_serial_at_highest_rate": top["solves_per_s_vs_serial"],
                       "p99_not_above_serial_at_every_rate": all(r["served"]["p99_s"] <= r["serial"]["p99_s"]
                                                                 for r in runs)}
    precision = fp64 = None
    if not args.no_precision:
        with torch.cuda.stream(stream):
            precision = bench_precision(args, stream)
    if not args.no_fp64:
        with torch.cuda.stream(stream):
            fp64 = bench_fp64(args, stream)

    if rank != 0:
        return 0
    peaks, src = _peaks()
    algo = ALGO.get((args.weights, args.precision), ALGO[("arclength", "mixed")])
    pts = n * n
    # the dominant kernel's average launch duration inside the timed region: a periodic grid's RK3 step
    # graph holds exactly the three stage launches (no ghost or reduction kernels), so the per-launch
    # average is the graph-timed step time / 3 (graph gaps included: achieved is, if anything, low)
    launch_ms = ms / (3 * args.steps)
    bytes_launch = sum(algo["bytes"]) * pts / 3.0       # algorithmic bytes of an average stage launch
    hbm_achieved = bytes_launch / (launch_ms * 1e-3) / 1e9
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    mufu_achieved = algo["mufu"] * pts / (launch_ms * 1e-3) / 1e9        # Gop/s
    mufu_peak = SM_COUNT * MUFU_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e9
    traffic = _traffic()
    roof = {
        "kernel": "stage2d_kernel (3 launches per RK3 step; per-launch average over the timed graph replays)",
        "bound": "hbm",
        "unit": "GB/s",
        "achieved": hbm_achieved,
        "peak": hbm_peak,
        "frac": hbm_achieved / hbm_peak,
        "peak_source": f"{src}: MEASURED_PEAKS.json hbm_gbs (copy bandwidth)" if src == "measured" else src,
        "algorithmic_bytes_per_launch": bytes_launch,
        "algorithmic_bytes_per_point_step": sum(algo["bytes"]),
        "launch_ms": launch_ms,
        "traffic": (traffic["dram_bytes_per_point_step"] * pts / 3.0) if traffic else None,
        "traffic_source": traffic.get("measured_on") if traffic else "no capture of the current kernel",
        "stage_ms_isolated": stage_ms,
        "alu": {"unit": "Gop/s", "achieved": mufu_achieved, "peak": mufu_peak, "frac": mufu_achieved / mufu_peak,
                "mufu_per_point_stage": algo["mufu"], "mufu_per_point_stage_full_sweep": algo.get("mufu_full"),
                "peak_source": f"measured 16 MUFU ops/SM/clk (rsqrt, sqrt, lg2, sin) x {SM_COUNT} SMs x "
                               f"{SM_MAX_MHZ:.0f} MHz"},
        "fp32": {"achieved_tflops": algo["flops"] * pts / (launch_ms * 1e-3) / 1e12,
                 "peak_tflops": SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12},
    }
    # instruction issue: thread instructions per node and stage from the same ncu capture as the traffic
    # (arc length, MIXED) against 4 schedulers x 32 lanes per SM and clock
    if traffic and traffic.get("thread_instructions_per_point_stage") and \
            (args.weights, args.precision) == ("arclength", "mixed"):
        inst = traffic["thread_instructions_per_point_stage"]
        achieved = sum(inst) / 3.0 * pts / (launch_ms * 1e-3) / 1e12
        peak = SM_COUNT * 4 * 32 * SM_MAX_MHZ * 1e6 / 1e12
        roof["issue"] = {"achieved_tinst_s": achieved, "peak_tinst_s": peak, "frac": achieved / peak,
                         "peak_source": f"derived: {SM_COUNT} SMs x 4 schedulers x 32 lanes x {SM_MAX_MHZ:.0f} MHz",
                         "thread_instructions_per_point_stage": inst}
        if traffic.get("counters"):
            # issue slots, resident warps and pipe activity of the same launches (one-pass ncu counters)
            roof["ncu_counters"] = {k: v for k, v in traffic["counters"].items() if k != "note"}
    cpu = None
    if not args.no_cpu and ws >= 1:
        import oracle

        oracle.build()
        r1, el1, stp = cpu_oracle_rate(args.cpu_n, args.cpu_steps)
        cores = args.cpu_cores or _host_cores()
        pool = OraclePool(cores)
        r, el, stp = pool.rate(args.cpu_n, args.cpu_steps)
        pool.close()
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{stp} RK3 steps of Example 3 on {cores} independent {args.cpu_n}x{args.cpu_n} grids, "
                         f"one process per core ({el:.1f} s wall)",
               "one_core": {"value": r1, "sample": f"{stp} RK3 steps of Example 3 on one {args.cpu_n}x{args.cpu_n} "
                                                    f"grid ({el1:.1f} s)"}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
        "config": {"workload": f"ex3_burgers2d_{n}sq", "nx": n, "ny": n, "precision": args.precision,
                   "weights": args.weights, "hamiltonian": "(p+q+1)^2/2", "alpha": "global_lagged",
                   "step": "one TVD-RK3 step (3 fused stage kernels)",
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{ws}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
        "batched": batched,
        "serving": serving,
        "precision": precision,
        "fp64": fp64,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_precision_report(args):
    """Errors of the float paths against FP64 and against the exact solution (one JSON line).

    Example 3 (periodic, exact solution by characteristics) to t = 0.5/pi^2 (default 400^2 and
    2048^2): L1 (mean |e|) and max |e| of FP64, MIXED and FP32 against the exact solution, and of
    MIXED and FP32 against FP64.  Example 10 (sin(p+q), pi(|y|-|x|), linear extrapolation) to t = 1
    (default 1024^2): MIXED and FP32 against FP64 (no exact solution).  Plus FP64 throughput at
    2048^2."""
    import numpy as np
    import torch

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import exact
    from paper_1909_13263_gb300 import inputs, native

    native.load()
    native.use_torch_allocator(True)
    out = {"report": "precision"}
    precs = [v for v in args.report_precisions.split(",") if v]
    tf = 0.5 / math.pi**2
    for n in [int(v) for v in args.report_ex3_sizes.split(",") if v]:
        x, dx = inputs.axis(n, -2.0, 2.0, "periodic")
        phi0 = inputs.phi0_negcos_diag_2d(x, x)
        ex = exact.negcos_diag_2d("burgers2d", x, x, tf)
        res = {}
        for prec in precs:
            with native.Solver(dim=2, nx=n, ny=n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham="burgers2d",
                               precision=prec) as s:
                s.set_phi0(phi0)
                s.step_to(tf)
                res[prec] = s.get_phi()
        row = {}
        for prec, phi in res.items():
            e = np.abs(phi - ex)
            row[prec] = {"l1_vs_exact": float(e.mean()), "linf_vs_exact": float(e.max())}
            if prec != "fp64" and "fp64" in res:
                d = np.abs(phi - res["fp64"])
                row[prec].update({"l1_vs_fp64": float(d.mean()), "linf_vs_fp64": float(d.max()),
                                  "l1_ratio_to_fp64": float(e.mean() / np.abs(res["fp64"] - ex).mean())})
        out[f"ex3_burgers2d_{n}sq"] = row
    for n in [int(v) for v in args.report_ex10_sizes.split(",") if v]:
        x, dx = inputs.axis(n, -1.0, 1.0, "linextrap")
        phi0 = inputs.phi0_riemann_2d(x, x)
        res = {}
        for prec in ("fp64", "mixed", "fp32"):
            with native.Solver(dim=2, nx=n, ny=n, bc="linextrap", xlo=-1.0, xhi=1.0, ylo=-1.0, yhi=1.0,
                               ham="sin2d", precision=prec) as s:
                s.set_phi0(phi0)
                steps = s.step_to(1.0)
                res[prec] = s.get_phi()
        row = {"steps": steps}
        inner = np.ix_(np.abs(x) <= 0.5, np.abs(x) <= 0.5)   # the window away from the corners
        for prec in ("mixed", "fp32"):
            d = np.abs(res[prec] - res["fp64"])
            row[prec] = {"l1_vs_fp64": float(d.mean()), "linf_vs_fp64": float(d.max()),
                         "l1_vs_fp64_inner": float(d[inner].mean()), "linf_vs_fp64_inner": float(d[inner].max())}
        if n == min(int(v) for v in args.report_ex10_sizes.split(",") if v):
            # conditioning: the FP64 result's change under a 1e-8 perturbation of phi0 (seeded normal noise);
            # with linear extrapolation two corners amplify rounding-level differences by many orders
            pert = phi0 + 1e-8 * np.random.default_rng(7).standard_normal(phi0.shape)
            with native.Solver(dim=2, nx=n, ny=n, bc="linextrap", xlo=-1.0, xhi=1.0, ylo=-1.0, yhi=1.0,
                               ham="sin2d", precision="fp64") as s:
                s.set_phi0(pert)
                s.step_to(1.0)
                d = np.abs(s.get_phi() - res["fp64"])
            row["fp64_under_1e-8_perturbation"] = {"l1": float(d.mean()), "linf": float(d.max()),
                                                   "l1_inner": float(d[inner].mean()),
                                                   "linf_inner": float(d[inner].max())}
        out[f"ex10_sin2d_linextrap_{n}sq"] = row
        del res
    # FP64 throughput (the parity path): RK3 steps of Example 3 on 2048^2
    n = 2048
    x, dx = inputs.axis(n, -2.0, 2.0, "periodic")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with native.Solver(dim=2, nx=n, ny=n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham="burgers2d",
                           precision="fp64", stream=stream) as s:
            s.set_phi0(inputs.phi0_negcos_diag_2d(x, x))
            s.advance(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.advance(10)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 10
    out["fp64_ex3_2048sq"] = {"ms_per_step": ms, "point_updates_per_s": n * n / (ms * 1e-3)}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--precision", choices=["mixed", "fp32", "fp64"], default="mixed")
    ap.add_argument("--weights", choices=["arclength", "jp"], default="arclength")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-n", type=int, default=512)
    ap.add_argument("--cpu-steps", type=int, default=20)
    ap.add_argument("--ref-n", type=int, default=128)
    ap.add_argument("--cpu-cores", type=int, default=0,
                    help="oracle worker processes for the CPU figures (default: every core this process may use)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--serial-count", type=int, default=128)
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--precision-ex10-n", type=int, default=1024)
    ap.add_argument("--precision-ex3-n", type=int, default=2048)
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--serve-round-steps", type=int, default=4)
    ap.add_argument("--serve-round-tiles", type=int, default=None,
                    help="tile limit of a server round (default: the server's own, four kernel waves; 0: none)")
    ap.add_argument("--serve-rates", type=str, default="50,200,1000,2000",
                    help="comma-separated Poisson arrival rates of the serving sweep (req/s)")
    ap.add_argument("--report", choices=["", "precision", "sizes", "oracle"], default="",
                    help="precision: errors of the float paths against FP64 and the exact solution; sizes: "
                         "device throughput by grid size; oracle: the FP64 CPU oracle timed on the host cores")
    ap.add_argument("--report-ex3-sizes", type=str, default="400,2048",
                    help="precision report: grid sides of Example 3 (comma-separated)")
    ap.add_argument("--report-precisions", type=str, default="fp64,mixed,fp32",
                    help="paths of the precision report's Example 3 rows (Example 10 always runs all three)")
    ap.add_argument("--report-ex10-sizes", type=str, default="1024",
                    help="precision report: grid sides of Example 10 (comma-separated)")
    ap.add_argument("--serve-count", type=int, default=400)
    ap.add_argument("--serve-budget-gb", type=float, default=60.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.report == "precision":
        return run_precision_report(args)
    if args.report == "sizes":
        return run_sizes_report(args)
    if args.report == "oracle":
        return run_oracle_report(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

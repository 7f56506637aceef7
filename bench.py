"""Benchmark: effective field + LLG torque inside adaptive Dormand-Prince
RK45 on the large ferromagnet workload (1024 x 1024 x 8 cells of 2x2x1 nm,
demag + exchange + uniaxial anisotropy + interfacial DMI, tol 1e-5).

One benchmark step is one DP45 attempt (six field evaluations, the error
estimate read back, accept/reject).  The metric counts field evaluations:
Mcell-evals/s = sum over evaluations of cells x sublattices / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs N independent replicas (one per rank, launched by torchrun), as
the path does not shard a single grid; value = all ranks' cell-evals / max
time.  `--impl reference` times the FP64 CPU oracle instead (rank 0 only).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "field+torque Mcell-evals/s"
METRIC_FULL = "field+torque Mcell-evals/s & served solves/s (p50/p99) vs plain path @ stated err"
UNIT = "Mcell-evals/s"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def kernel_bytes(g, nk_avg, nparts=1, nsub=1, mel=False):
    """Algorithmic DRAM bytes per launch of each pass (per eval):
    each array that a pass must read or write, once."""
    nx, ny, nz = g["shape"]
    n = nx * ny * nz
    kxn = g["Px"] // 2 + 1
    kyn = g["Py"] // 2 + 1
    kzn = g["Pz"] // 2 + 1
    krow = (6 * kzn + 3) // 4 * 4
    spec = 3 * kxn * ny * nz * 8            # x-transformed spectrum, complex64
    khat = kxn * kyn * krow * 4             # kernel octant rows, float32
    part = 12 * n                            # one 3-vector field, float32
    return {
        # read y and the n_k earlier stages, write the stage, write the spectrum
        "pass_a": part * nparts * (1 + nk_avg) + part * nparts + spec,
        # spectrum in and out, kernel octant in
        "pass_b": 2 * spec + khat,
        # spectrum in, stage m in, k out (+ strain in)
        "field": spec + part * nsub * 2 + (24 * n if mel else 0),
    }


def eval_flops(g, nsub=1):
    """Algorithmic FP32 flops of one field evaluation (the FFT counted as
    5 N log2 N per complex transform of length N): the forward x transform
    of real row pairs (pass A), the y transforms both ways, the z transforms
    both ways and the 3x3 multiply (36 flops per frequency, pass B), the
    inverse x transform (pass C) and ~150 flops of local field and torque per
    cell and sublattice."""
    import math
    nx, ny, nz = g["shape"]
    Px, Py, Pz = g["Px"], g["Py"], g["Pz"]
    kxn = Px // 2 + 1

    def fft(n):
        return 5.0 * n * math.log2(n) if n > 1 else 0.0
    x = 3 * nz * ((ny + 1) // 2) * fft(Px)
    y = 2 * 3 * nz * kxn * fft(Py)
    z = 2 * 3 * kxn * Py * fft(Pz)
    mult = 36.0 * kxn * Py * Pz
    return 2 * x + y + z + mult + 150.0 * nx * ny * nz * nsub


FLOOR_BYTES = 99   # compulsory DRAM bytes per cell-eval of the large ferromagnet (m, k, kernel, one spectrum round trip)


def geometry(shape):
    def nice(n):
        if n == 1:
            return 1
        c = [p for p in (2 ** k for k in range(1, 14)) if p >= 2 * n - 1][:1]
        c += [p for p in (3 * 2 ** k for k in range(1, 13)) if p >= 2 * n - 1][:1]
        return min(c)
    return {"shape": shape, "Px": nice(shape[0]), "Py": nice(shape[1]), "Pz": nice(shape[2])}


def traffic_from_profile(kernel):
    """ncu DRAM bytes per launch recorded for this kernel's sources, or None
    if any of them changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[kernel]
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, "paper_2411_18194_gb300", "csrc", f), "rb").read())
        return rec["dram_bytes_per_launch"] if h.hexdigest()[:16] == rec["source_sha"] else None
    except Exception:
        return None


def reduce_over_ranks(maxes, sums, device):
    """Whole-job numbers of independent replicas: the max over ranks of each
    value in `maxes` (times) and the sum of each value in `sums` (work,
    throughputs).  Identity when not running distributed."""
    import torch
    mx = torch.tensor([float(v) for v in maxes], dtype=torch.float64, device=device)
    sm = torch.tensor([float(v) for v in sums], dtype=torch.float64, device=device)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx.tolist(), sm.tolist()


def _oracle_evals(seconds):
    """Field+torque evaluations of the FP64 oracle (numpy) on a 128x128x8
    sub-grid of the large-ferromagnet workload (same materials, cell size)
    for about `seconds`: (evaluations, elapsed s, cells)."""
    import numpy as np
    from inputs import config_c2, random_unit_vectors
    from oracle import dp45
    w = config_c2()
    p = w.problem
    p.shape = (128, 128, 8)
    p.regions = np.zeros((8, 128, 128), dtype=np.uint8)
    m = random_unit_vectors(w.seed, p.shape).astype(np.float64)
    o = dp45.Oracle(p)
    st = dp45.State([m])
    n = 0
    t0 = time.perf_counter()
    while True:
        o.rhs(st)
        n += 1
        el = time.perf_counter() - t0
        if el > seconds:
            break
    return n, el, 128 * 128 * 8


def cpu_worker(seconds):
    """One oracle process of the all-cores baseline (spawned, one thread)."""
    return _oracle_evals(seconds)


def cpu_model():
    """The host CPU's model name as lscpu reports it (else the machine type)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip() + " (" + platform.machine() + ")"
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(seconds=15.0):
    """The FP64 oracle as it stands (numpy), on the host cores: one process
    per core (spawned, one thread each: the numpy FFTs and element-wise work
    of the oracle do not thread), and one thread alone, each on the same
    128 x 128 x 8 sub-grid of the workload for about `seconds`."""
    import multiprocessing
    n1, el1, cells = _oracle_evals(seconds)
    single = n1 * cells / el1 / 1e6
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    with multiprocessing.get_context("spawn").Pool(cores) as pool:
        res = pool.map(cpu_worker, [seconds] * cores)
    total = sum(n * c / el for n, el, c in res) / 1e6
    evals = sum(n for n, _, _ in res)
    return {"value": total, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": "%d field+torque evaluations of a 128x128x8 sub-grid of the workload (same materials, "
                      "cell size), FP64 numpy, %d processes of one thread for %.0f s" % (evals, cores, seconds),
            "single_thread": {"value": single, "cores": 1,
                              "sample": "%d evaluations of the same sub-grid in %.1f s" % (n1, el1)}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from inputs import config_c2, random_unit_vectors
    from oracle import dp45
    w = config_c2()
    p = w.problem
    p.shape = (128, 128, 8)
    p.regions = np.zeros((8, 128, 128), dtype=np.uint8)
    m = random_unit_vectors(w.seed, p.shape).astype(np.float64)
    o = dp45.Oracle(p)
    st = dp45.State([m])
    k1 = o.rhs(st)
    dt = 1e-14
    for _ in range(args.warmup):
        st2, _, _ = o.attempt(st, k1, dt)
    e0 = o.evals
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st2, _, _ = o.attempt(st, k1, dt)
    el = time.perf_counter() - t0
    cells = 128 * 128 * 8
    value = (o.evals - e0) * cells / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "metric_full": METRIC_FULL, "value": value,
            "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random m0)",
            "config": {"workload": "ferromagnet 1024x1024x8 (2x2x1 nm), demag+exchange+anisotropy+iDMI, "
                                   "adaptive DP45 tol 1e-5; each step a bounded sample: one DP45 attempt "
                                   "on a 128x128x8 sub-grid", "cells_per_step_eval": cells},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "DP45 attempts (6 evaluations each) on a 128x128x8 sub-grid, "
                                       "FP64 numpy, one thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


WORKLOADS = {
    "c2": "ferromagnet 1024x1024x8 cells of 2x2x1 nm, Ms 1.1e6, A 1.6e-11, Ku 8e5 (z), iDMI 3e-3, "
          "alpha 0.1; demag+exchange+anisotropy+iDMI; adaptive DP45 tol 1e-5 from dt 1e-14",
    "c1": "ferromagnet 64x64x1 cells of 4 nm, Ms 8e5, A 1.3e-11, alpha 0.02, B = 10 mT along z; "
          "demag+exchange+Zeeman; fixed DP45 dt 1e-13",
    "c3": "two-sublattice antiferromagnet 1024x256x1 cells of 2 nm with magnetoelastic coupling and "
          "elastodynamics (biaxial anisotropy, A0 -4e-11, A12 -1e-12); fixed DP45 dt 5e-15",
    "c5": "served stream of relax-to-equilibrium solves: seeded Poisson arrivals (200 req/s), grids 64^2x1 "
          "to 1024^2x4 of 4x4x2 nm, Ms 8e5, A 1.3e-11, alpha 0.5, |B| <= 50 mT, random m0; adaptive DP45 "
          "(tol 1e-5) until max|m x B| <= torque tol or max time; 150 GB admission budget",
    "c4": "256 independent ferromagnets, seeded nx, ny in {32..512} (2^k, 3*2^k), nz in {1,2,4}, 2 nm cells, "
          "Ms 4e5-1.4e6, A 5e-12-2e-11, alpha 0.01-0.5, demag+exchange, random m0, fixed DP45 step per "
          "instance (stability bound); batched: one launch per pass per stage, graph per lock step",
}


def run_serve(args):
    """C5 as its own benchmark line."""
    line = serve_measure(args, init=True)
    if line is not None:
        print(json.dumps(line))


def serve_measure(args, init):
    """C5: continuous-batching relax server against the plain path (each
    request relaxed alone, in arrival order) on the same request stream.
    Returns the benchmark line on rank 0 (None elsewhere)."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1 and init:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from inputs import serve_requests
    from paper_2411_18194_gb300 import serve

    def stream_of_requests():
        return [serve.Request(i, w, t, args.torque_tol, args.max_time)
                for i, (t, w) in enumerate(serve_requests(args.requests, rate_hz=args.rate))]

    # warm-up: every distinct geometry once (spectrum builds, tuned shapes,
    # module loading) so that both paths start warm
    seen = set()
    for r in stream_of_requests():
        key = (tuple(r.workload.problem.shape), tuple(r.workload.problem.cell))
        if key not in seen:
            seen.add(key)
            mag = serve._make_magnet(r.workload, 1e-14)
            mag.step(1)
            mag.close()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    srv = serve.RelaxServer(budget_bytes=args.budget_gb * 1e9, attempts_per_round=args.attempts)
    served = srv.run(stream_of_requests())
    peak = srv.peak_members
    srv.close()
    clk = clocks.stop()
    st = serve.latency_stats(served)
    plain = serve.latency_stats(serve.serve_one_at_a_time(stream_of_requests()))
    (span,), (solves,) = reduce_over_ranks([st["span_s"]], [st["solves"]], "cuda")
    if rank == 0:
        line = {
            "metric": "served solves/s", "metric_full": METRIC_FULL, "value": solves / span,
            "unit": "solves/s", "n_gpus": ws, "steps": args.requests, "warmup": args.warmup,
            "ms_per_step": span / max(1, st["solves"]) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded arrivals, grids, fields, m0)",
            "config": {"workload": WORKLOADS["c5"], "requests": args.requests, "rate_hz": args.rate,
                       "torque_tol_T": args.torque_tol, "max_time_s": args.max_time,
                       "budget_gb": args.budget_gb, "attempts_per_round": args.attempts,
                       "peak_members": peak, "parallelism": "replicas",
                       "step": "one request (relax solve)"},
            "latency_s": {"p50": st["p50_s"], "p99": st["p99_s"], "mean": st["mean_s"]},
            "time_capped_fraction": st["time_capped_fraction"],
            "plain_path": {"solves_per_s": plain["solves_per_s"], "p50": plain["p50_s"], "p99": plain["p99_s"],
                           "mean": plain["mean_s"], "time_capped_fraction": plain["time_capped_fraction"],
                           "what": "each request relaxed alone (mmp_relax) in arrival order"},
            "speedup_vs_plain": (solves / span) / plain["solves_per_s"],
            "clocks": clk,
        }
    if ws > 1 and init:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line if rank == 0 else None


def run_batch(args):
    """C4 as its own benchmark line."""
    line = batch_measure(args, init=True)
    if line is not None:
        print(json.dumps(line))


def batch_measure(args, init):
    """C4: the batch path against the plain one-at-a-time path on the same
    instances (same shapes, same steps; results are bitwise equal).
    Returns the benchmark line on rank 0 (None elsewhere)."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1 and init:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2411_18194_gb300 as pkg
    from inputs import batch_instances
    insts = batch_instances(args.instances)
    mags = []
    t0 = time.perf_counter()
    for w in insts:
        mag = pkg.Magnet.from_problem(w.problem)
        mag.set_m(0, torch.from_numpy(w.m0[0]).cuda())
        mag.set_solver(adaptive=False, dt=w.dt)
        mags.append(mag)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    shapes = {}
    for mag in mags:
        sh, _ = mag.autotune(batch=True)
        shapes[mag.shape] = sh
    t_tune = time.perf_counter() - t0
    cells = [int(np.prod(w.problem.shape)) for w in insts]
    evals_per_step = 6 * sum(cells)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # batched path
    b = pkg.Batch(stream)
    for mag in mags:
        b.add(mag, "steps", args.warmup + args.steps)
    b.advance(args.warmup)          # first stages, graph capture, warm-up steps
    clocks = ClockSampler(local)
    barrier()
    l0 = b.launches()
    clocks.start()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    b.advance(args.steps)
    stop.record(stream)
    barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(stop)
    launches = b.launches() - l0
    b.close()
    # per-pass device times (traced lock steps, direct launches) for the roofline
    b = pkg.Batch(stream)
    for mag in mags:
        b.add(mag, "steps", 3)
    b.advance(1)
    b.profile(True)
    b.advance(2)
    prof = b.profile_read()
    b.profile(False)
    b.close()
    # plain path: the same instances one at a time, same step count
    for mag in mags:
        mag.step(1)
    barrier()
    p0 = time.perf_counter()
    for mag in mags:
        mag.step(args.steps)
    barrier()
    ms_plain = (time.perf_counter() - p0) * 1e3
    # end to end with host buffers: per lock step every state in from pinned
    # host memory, one batched step, every state back
    hosts = [torch.from_numpy(w.m0[0]).pin_memory() for w in insts]
    outs = [torch.empty_like(h).pin_memory() for h in hosts]
    e2e_steps = max(3, args.steps // 10)
    b = pkg.Batch(stream)
    for mag in mags:
        b.add(mag, "steps", e2e_steps + 1)
    b.advance(1)
    barrier()
    q0 = time.perf_counter()
    for _ in range(e2e_steps):
        for mag, h in zip(mags, hosts):
            mag.set_m(0, h)
        b.advance(1)
        for mag, o in zip(mags, outs):
            mag.get_m(0, o)
    barrier()
    e2e_s = time.perf_counter() - q0
    b.close()
    for mag in mags:
        mag.close()
    (t_max, t_plain), (all_evals,) = reduce_over_ranks([ms, ms_plain], [evals_per_step * args.steps], "cuda")
    value = all_evals / (t_max * 1e-3) / 1e6
    plain = all_evals / (t_plain * 1e-3) / 1e6
    e2e_value = evals_per_step * e2e_steps / e2e_s / 1e6
    _, (e2e_all,) = reduce_over_ranks([], [e2e_value], "cuda")
    peak, src = peaks()
    step_bytes = 0
    pass_bytes = {"pass_a": 0, "pass_b": 0, "field": 0}
    nk_avg = (0 + 1 + 2 + 3 + 4 + 5 + 5) / 7.0
    for w in insts:
        kb = kernel_bytes(geometry(w.problem.shape), nk_avg)
        step_bytes += 6 * sum(kb.values())
        for k in pass_bytes:
            pass_bytes[k] += kb[k]
    # dominant pass: all its launches of one stage (pass B: one per z group)
    dom = max(prof, key=lambda k: prof[k][1])
    per_stage = {k: v[1] / 12.0 for k, v in prof.items()}    # 2 traced lock steps x 6 stages
    achieved = pass_bytes[dom] / (per_stage[dom] * 1e-3) / 1e9
    share = {k: round(v[1] / sum(x[1] for x in prof.values()), 4) for k, v in prof.items()}
    nbytes = 12 * sum(cells)
    if rank == 0:
        line = {
            "metric": METRIC, "metric_full": METRIC_FULL, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded sizes, materials, random m0)",
            "config": {"workload": WORKLOADS["c4"], "instances": len(insts), "cells": sum(cells),
                       "parallelism": "replicas",
                       "step": "one lock step: one fixed DP45 step of every instance (6 evaluations each)",
                       "l2": "inputs larger than L2 (%.1f GB of state, stages, spectra)" % (
                           sum(cells) * 150e-9),
                       "setup_s": round(t_setup, 2), "autotune_s": round(t_tune, 2),
                       "distinct_shapes": len(shapes)},
            "plain_path": {"value": plain, "unit": UNIT, "ms_per_step": t_plain / args.steps,
                           "what": "the same instances stepped one at a time through mmp_step"},
            "speedup_vs_plain": value / plain,
            "solves_per_s": {"batched": len(insts) * ws / (t_max * 1e-3),
                             "plain": len(insts) * ws / (t_plain * 1e-3),
                             "solve": "%d fixed DP45 steps of one instance" % args.steps},
            "roofline": {"kernel": "batched " + dom + " (all its launches of one stage)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "peak_source": src, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "bytes_per_stage": pass_bytes[dom],
                         "ms_per_stage": per_stage[dom]},
            "kernel_share": share,
            "whole_step_gbs": step_bytes * args.steps / (ms * 1e-3) / 1e9,
            "cpu_baseline": None,
            "e2e": {"value": e2e_all, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                    "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clk,
        }
    if ws > 1 and init:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line if rank == 0 else None


def pass_b_ms(mag, engine, evals=12):
    """Mean device time of pass B (CUDA events) over `evals` field evaluations
    of the magnet's current state with the given engine bits."""
    mag.set_shape(engine=engine)
    mag.eval_field(0)
    mag.eval_field(0)
    mag.profile(True)
    for _ in range(evals):
        mag.eval_field(0)
    n, ms = mag.profile_read()["pass_b"]
    mag.profile(False)
    return ms / n


def tensor_core_study(mag_c2):
    """Pass B with the final DFT32 of its y transforms on the CUDA cores and
    on the tensor cores (split TF32), on the large ferromagnet and on the
    largest batched instance (512x512x1, solo context)."""
    import torch
    import paper_2411_18194_gb300 as pkg
    from inputs import Problem, random_unit_vectors
    out = {}
    base = mag_c2.get_shape()
    if not base["engine"] & 1:
        return None
    e0 = base["engine"] & ~4
    out["c2_1024x1024x8"] = {"cuda_cores_ms": pass_b_ms(mag_c2, e0), "tensor_cores_ms": pass_b_ms(mag_c2, e0 | 4)}
    mag_c2.set_shape(**base)
    p = Problem((512, 512, 1), (2e-9, 2e-9, 2e-9), 1, frozenset({"DEMAG", "EXCH"}))
    p.set("MS", 1.4e6).set("AEX", 2e-11).set("ALPHA", 0.5)
    m = pkg.Magnet.from_problem(p)
    m.set_m(0, torch.from_numpy(random_unit_vectors(777, p.shape)).cuda())
    e = m.get_shape()["engine"] & ~4
    out["batched_512x512x1"] = {"cuda_cores_ms": pass_b_ms(m, e), "tensor_cores_ms": pass_b_ms(m, e | 4)}
    m.close()
    for v in out.values():
        v["tensor_over_cuda"] = v["tensor_cores_ms"] / v["cuda_cores_ms"]
    out["what"] = ("pass B per launch (CUDA events, mean of 12) with the final length-32 DFT of every y "
                   "transform on the CUDA cores or as a split-TF32 GEMM on the tensor cores (tcgen05, "
                   "engine bit 4); the benchmark value uses the autotuned shape")
    return out


def spectrum_build_study():
    """Cold build of a geometry's demag kernel spectrum (what a server pays
    to admit a new grid): first field evaluation of a fresh context minus a
    second one, for the largest served grid and the large ferromagnet's
    grid (cell sizes not used before, so nothing is cached)."""
    import time
    import torch
    import paper_2411_18194_gb300 as pkg
    from inputs import Problem, random_unit_vectors
    out = {}
    for shape, cell in (((1024, 1024, 4), (4e-9, 4e-9, 2e-9)), ((1024, 1024, 8), (2.000001e-9, 2e-9, 1e-9))):
        p = Problem(shape, cell, 1, frozenset({"DEMAG", "EXCH"}))
        p.set("MS", 8e5).set("AEX", 1.3e-11).set("ALPHA", 0.5)
        m = pkg.Magnet.from_problem(p)
        m.set_m(0, torch.from_numpy(random_unit_vectors(31, shape)).cuda())
        nx, ny, nz = shape
        B = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
        T = torch.empty_like(B)
        t = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m.eval_field(0, B, T)
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
        m.close()
        out["%dx%dx%d" % shape] = {"cold_ms": round(1e3 * (t[0] - t[1]), 2), "first_eval_ms": round(1e3 * t[0], 2),
                                   "warm_eval_ms": round(1e3 * t[1], 3)}
    out["what"] = ("demag kernel spectrum built on the device: Newell (FP64) below the cutoff, the far-field "
                   "expansion in FP32 above it, FP64 FFTs along axes of padded length >= 64; cold_ms = first "
                   "field evaluation of a new geometry minus the second")
    return out


# the batched and served halves of the metric as they ride along the default
# line: their own workloads, compact (bounded run time)
EXTRA_C4 = {"instances": 256, "steps": 10, "warmup": 3}
EXTRA_C5 = {"requests": 12, "rate": 200.0, "torque_tol": 1e-4, "max_time": 1e-8, "budget_gb": 150.0,
            "attempts": 4, "warmup": 3}


def extras(args):
    """Compact batched (C4) and served (C5) sub-objects of the default line."""
    import argparse
    a4 = argparse.Namespace(**vars(args))
    a4.__dict__.update(EXTRA_C4)
    l4 = batch_measure(a4, init=False)
    a5 = argparse.Namespace(**vars(args))
    a5.__dict__.update(EXTRA_C5)
    l5 = serve_measure(a5, init=False)
    if l4 is None or l5 is None:
        return None
    batched = {
        "workload": WORKLOADS["c4"], "instances": l4["config"]["instances"], "steps": l4["steps"],
        "solve": l4["solves_per_s"]["solve"],
        "solves_per_s": l4["solves_per_s"]["batched"], "plain_solves_per_s": l4["solves_per_s"]["plain"],
        "mcell_evals_per_s": l4["value"], "plain_mcell_evals_per_s": l4["plain_path"]["value"],
        "speedup_vs_plain": l4["speedup_vs_plain"], "ms_per_lock_step": l4["ms_per_step"],
        "roofline_frac": l4["roofline"]["frac"], "clocks": l4["clocks"],
        "what": "all instances advanced together (one launch per pass per stage, lock steps from a CUDA "
                "graph) against the same instances stepped one at a time; results bitwise equal"}
    served = {
        "workload": WORKLOADS["c5"], "requests": l5["config"]["requests"],
        "torque_tol_T": l5["config"]["torque_tol_T"], "max_time_s": l5["config"]["max_time_s"],
        "solves_per_s": l5["value"], "p50_s": l5["latency_s"]["p50"], "p99_s": l5["latency_s"]["p99"],
        "time_capped_fraction": l5["time_capped_fraction"],
        "plain_solves_per_s": l5["plain_path"]["solves_per_s"], "plain_p50_s": l5["plain_path"]["p50"],
        "plain_p99_s": l5["plain_path"]["p99"], "speedup_vs_plain": l5["speedup_vs_plain"],
        "peak_members": l5["config"]["peak_members"], "clocks": l5["clocks"],
        "what": "continuous batching (admission by memory budget, joins between lock steps) against each "
                "request relaxed alone in arrival order; a solve relaxes to max|m x B| <= torque tol or "
                "the max simulated time"}
    return {"batched": batched, "served": served}


def run_gpu(args):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_2411_18194_gb300 as pkg
    from inputs import config_c1, config_c2, config_c3
    w = {"c1": config_c1, "c2": config_c2, "c3": config_c3}[args.workload]()
    p = w.problem
    nx, ny, nz = p.shape
    ncell = nx * ny * nz * p.n_sub
    mag = pkg.Magnet.from_problem(p)
    for s_, m_ in enumerate(w.m0):
        mag.set_m(s_, torch.from_numpy(m_).cuda())
    if w.u0 is not None:
        mag.set_elastic(torch.from_numpy(w.u0).cuda(), torch.from_numpy(w.v0).cuda())
    m0 = torch.from_numpy(w.m0[0]).cuda()
    mag.set_solver(adaptive=w.adaptive, dt=w.dt, tol=w.tol, dt_min=1e-18, dt_max=1e-11)
    t0 = time.perf_counter()
    if args.shape:
        shape = mag.set_shape(**parse_shape(args.shape))
    else:
        shape, tuned_ms = mag.autotune()      # launch shape chosen by timing (outside the timed region)
    t_tune = time.perf_counter() - t0

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up (also builds the demag kernel spectrum)
    for _ in range(args.warmup):
        mag.step(1)
    # the timed region runs untraced (fixed steps then replay from a graph);
    # per-kernel device times come from a traced run of a few steps after it
    if not w.adaptive:
        mag.step(2)                      # capture the fixed-step graph before timing
    clocks = ClockSampler(local)
    barrier()
    e0 = mag.time()["evals"]
    clocks.start()
    stream = torch.cuda.current_stream()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    if w.adaptive:
        attempts = 0
        while attempts < args.steps:
            mag.step(1)                  # one attempt (read-back, controller)
            attempts += 1
    else:
        mag.step(args.steps)             # fixed steps: pairs replayed from a graph
    stop.record(stream)
    barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(stop)
    tinfo = mag.time()
    evals = tinfo["evals"] - e0
    traced_steps = min(args.steps, 20)
    mag.profile(True)
    e_tr = mag.time()["evals"]
    for _ in range(traced_steps):
        mag.step(1)
    prof = mag.profile_read()
    mag.profile(False)
    tr_evals = mag.time()["evals"] - e_tr
    launches = int(round(sum(v[0] for v in prof.values()) * evals / max(tr_evals, 1)))
    (t_max,), (all_evals,) = reduce_over_ranks([ms], [evals * ncell], "cuda")
    value = all_evals / (t_max * 1e-3) / 1e6

    # roofline of the dominant kernel
    g = geometry(p.shape)
    nk_avg = (0 + 1 + 2 + 3 + 4 + 5 + 5) / 7.0   # k vectors read by stage assembly per eval (a72 = 0)
    kb = kernel_bytes(g, nk_avg, nparts=p.n_sub + (2 if "ELASTIC" in p.terms else 0), nsub=p.n_sub,
                      mel="MEL" in p.terms)
    dom = max((k for k in prof if k in kb) if any(k in kb for k in prof) else prof,
              key=lambda k: prof[k][1])
    n_l, tot_ms = prof[dom]
    avg_s = tot_ms / n_l * 1e-3
    peak, src = peaks()
    achieved = kb.get(dom, 0) / avg_s / 1e9
    share = {k: round(v[1] / sum(x[1] for x in prof.values()), 4) for k, v in prof.items()}

    # end to end through the public API with host buffers: per step the state
    # (magnetisation of sublattice 0) is copied in from pinned host memory and
    # read back.
    host_in = torch.from_numpy(w.m0[0]).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    mag.get_m(0, host_in)
    e2e_steps = max(5, args.steps // 10)
    barrier()
    e1 = mag.time()["evals"]
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mag.set_m(0, host_in)
        mag.step(1)
        mag.get_m(0, host_out)
        host_in, host_out = host_out, host_in
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_evals = mag.time()["evals"] - e1
    e2e_value = e2e_evals * ncell / e2e_s / 1e6
    _, (e2e_all,) = reduce_over_ranks([], [e2e_value], "cuda")
    nbytes = 12 * nx * ny * nz

    # fixed-step single instance: the same context as the one member of a
    # batch, whose lock steps replay from a CUDA graph (launch-bound grids)
    graph_path = None
    if args.workload == "c1":
        mag.set_shape(R=1, stage_kernel=0, engine=0)
        bt = pkg.Batch(stream)
        bt.add(mag, "steps", args.warmup + args.steps)
        bt.advance(args.warmup)
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        bt.advance(args.steps)
        g1.record(stream)
        barrier()
        gms = g0.elapsed_time(g1)
        glaunch = bt.launches()
        bt.close()
        graph_path = {"value": 6 * args.steps * ncell / (gms * 1e-3) / 1e6, "unit": UNIT,
                      "ms_per_step": gms / args.steps, "launches_total": glaunch,
                      "what": "the same context as the only member of an mmp_batch: fixed lock steps "
                              "replayed from a CUDA graph (shape R=1, kernel rows from L2)"}

    if rank == 0:
        line = {
            "metric": METRIC, "metric_full": METRIC_FULL, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded random m0)",
            "config": {"workload": WORKLOADS[args.workload],
                       "cells": nx * ny * nz, "sublattices": p.n_sub, "parallelism": "replicas",
                       "step": "one DP45 attempt (6 field evaluations + error readback)",
                       "evals": evals, "accepted": tinfo["steps"], "rejected": tinfo["rejected"],
                       "sim_time_s": tinfo["t"], "dt_s": tinfo["dt"],
                       "shape": shape, "autotune_s": round(t_tune, 2),
                       "l2": ("inputs larger than L2 (state + stages + spectra ~1.3 GB)" if args.workload == "c2"
                              else "working set fits in L2; no flush between steps")},
            "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak,
                         "peak_source": src, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic_from_profile(dom) if args.workload == "c2" else None,
                         "bytes_per_launch": kb.get(dom),
                         "avg_launch_ms": avg_s * 1e3, "launches": n_l},
            "kernel_share": share,
            "cpu_baseline": cpu_baseline() if not args.no_cpu_baseline and args.workload == "c2" else None,
            "e2e": {"value": e2e_all, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clk,
        }
        # path-level figures: effective algorithmic bandwidth (the passes'
        # bytes, and the compulsory floor) and achieved FP32 rate
        cell_evals = nx * ny * nz * p.n_sub
        per_eval_bytes = sum(kb.values())
        rate = value * 1e6 / cell_evals                 # evaluations per second
        line["path"] = {
            "algorithmic_bytes_per_cell_eval": round(per_eval_bytes / cell_evals, 1),
            "algorithmic_gbs": round(rate * per_eval_bytes / 1e9, 1),
            "floor_bytes_per_cell_eval": FLOOR_BYTES,
            "floor_gbs": round(value * 1e6 * FLOOR_BYTES / 1e9, 1),
            "fp32_gflop_per_eval": round(eval_flops(g, p.n_sub) / 1e9, 3),
            "fp32_gflops": round(rate * eval_flops(g, p.n_sub) / 1e9, 1),
        }
        # the ALU ceiling: measured FP32 FMA throughput (dependent-free FMA
        # chains at full occupancy, CUDA events), with the clock seen meanwhile
        fsamp = ClockSampler(local)
        fsamp.start()
        pk_gflops, pk_ms = pkg.fp32_peak(reps=200)
        fclk = fsamp.stop()
        line["path"]["fp32_peak_gflops"] = round(pk_gflops, 1)
        line["path"]["fp32_frac"] = round(line["path"]["fp32_gflops"] / pk_gflops, 4)
        line["path"]["fp32_peak_clock"] = fclk
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        line["path"]["fp32_peak_how"] = ("mmp_fp32_peak: best of 200 launches of 8 independent FMA chains per "
                                         "thread, %d blocks x 256 threads, %.3f ms each" % (8 * nsm, pk_ms))
        if graph_path:
            line["graph_path"] = graph_path
    if args.workload == "c2" and not args.no_extras:
        tcs = tensor_core_study(mag)
        if rank == 0 and tcs is not None:
            line["tensor_core_stage"] = tcs
        sbs = spectrum_build_study()
        if rank == 0:
            line["demag_spectrum_build"] = sbs
    mag.close()
    del mag
    if args.workload == "c2" and not args.no_extras:
        ex = extras(args)
        if rank == 0 and ex is not None:
            line.update(ex)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def parse_shape(text):
    """--shape ty,radix_x,radix_y,R,stage_kernel[,tyc[,engine]]"""
    v = [int(x) for x in text.split(",")]
    return dict(zip(("ty", "radix_x", "radix_y", "R", "stage_kernel", "tyc", "engine"), v))


def run_profile_evals(args):
    """Set-up plus N field evaluations and N DP45 attempts of the same
    workload, without timing (a short command for ncu captures)."""
    import torch
    import paper_2411_18194_gb300 as pkg
    from inputs import config_c2
    w = config_c2()
    mag = pkg.Magnet.from_problem(w.problem)
    mag.set_m(0, torch.from_numpy(w.m0[0]).cuda())
    mag.set_solver(adaptive=True, dt=w.dt, tol=w.tol)
    if args.shape:
        mag.set_shape(**parse_shape(args.shape))
    else:
        mag.autotune()                   # the shape the benchmark times
    for _ in range(args.profile_evals):
        mag.eval_field(0)
        mag.step(1)
    mag.sync()
    mag.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="c2: leave out the batched (C4) and served (C5) sub-objects")
    ap.add_argument("--profile-evals", type=int, default=0)
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5"],
                    help="c2 (default, the benchmark line); c1, c3 for the other single workloads; "
                         "c4 the batch of uneven instances; c5 the served request stream")
    ap.add_argument("--instances", type=int, default=256, help="c4: number of instances")
    ap.add_argument("--shape", default="", help="single workloads: ty,radix_x,radix_y,R,stage_kernel[,tyc] "
                                                "instead of the autotuned shape (profiling commands)")
    ap.add_argument("--requests", type=int, default=48, help="c5: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="c5: mean arrival rate (1/s)")
    ap.add_argument("--torque-tol", type=float, default=1e-4, help="c5: relax torque tolerance (T)")
    ap.add_argument("--max-time", type=float, default=10e-9, help="c5: relax max simulated time (s)")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="c5: admission budget (GB)")
    ap.add_argument("--attempts", type=int, default=4, help="c5: lock-step attempts between admissions")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile_evals:
        run_profile_evals(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "c4":
        run_batch(args)
    elif args.workload == "c5":
        run_serve(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

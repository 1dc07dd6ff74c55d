"""Throughput of the spectral-element time step on GB300.

One "step" is one leapfrog time step of the whole hot path over the mesh:
gather, GLL gradient, metric, transposed contraction, deterministic
assembly, inverse mass, source, Kahan-compensated update and receiver traces.
Workload (default): the graded heterogeneous mesh, 512 x 512 quads on the
unit square, widths graded 8x toward (0,0), interior vertices perturbed by up
to 20% of the local width, order 4 (4,198,401 GLL nodes), c ~ U[1,3] per
element, Ricker f0 = 10 at the centre, dt = 0.3 CFL, 2000 steps, Hilbert
ordering, FP32 bulk with the Kahan leapfrog and FP64 precompute/traces.

Metric: GLL node-updates/s = nodes x steps / time (higher is better).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (its own shot; weak
scaling, no collective on the data path); rank 0 prints one JSON line.
`--impl reference` times the FP64 CPU oracle (the C/OpenMP restatement, all
host cores) on the same workload instead.

Besides the headline (FP32 bulk + Kahan, Hilbert order) the line carries the
rest of the metric "FP32 vs FP64 at stated error": the FP64 and plain FP32
rates on the same mesh (`precisions`), the errors of FP32+Kahan against FP64
on the GPU over the workload's 2000 steps and of both precisions against the
CPU oracle over the first steps (`error`), and the multilayered
4096 x 1024 model (67M nodes), the largest single-GPU workload
(`workloads`).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "GLL node-updates/s (order 4)"
UNIT = "node-updates/s"
WORKLOAD = "graded_512x512_p4"
L2_BYTES = 129 * 2 ** 20
# algorithmic DRAM bytes per node-update at p = 4 (1.5625 element slots per
# node; connectivity 4 B/slot, stored metric 12 B/slot FP32 or 24 B FP64;
# node state: FP32 three-level u r/w, u_prev r, s r; Kahan u, delta, c r/w,
# s r; FP64 three-level as FP32 with 8-byte values)
ALGO_BYTES = {"fp32": 41.0, "fp32_kahan": 53.0, "fp64": 76.0}
# the first-order system with Heun steps, per node-update at p = 4: velocity
# per slot (2 values) read/written 7 times, connectivity twice, node values
# (U, U~, dU, s) read/written 9 times
ALGO_BYTES_HEUN = {"fp32": 136.0, "fp64": 272.0}
# FP64: GB300's double-precision rate is far below its FP32 rate, so the FP64
# leapfrog is bound by arithmetic. Flops per node-update at p = 4: per element
# 8 (p+1)^3 + 6 (p+1)^2 = 1150 (two derivative contractions of 2 (p+1)^3 each
# way, 6 per point for the metric), times 262,144 / 4,198,401 elements per node,
# plus 5 for the node update (f - Ku, 2u - u_prev, one FMA). Peak: the nominal 1.25 TFLOP/s, i.e. 152 SMs x
# 2.07 GHz x 4 FP64 flop per SM-clock.
FLOPS_FP64_LEAPFROG = 1150.0 * 262144 / 4198401 + 5.0
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32_kahan", choices=["fp32_kahan", "fp64", "fp32"])
    ap.add_argument("--ordering", default="hilbert",
                    choices=["hilbert", "rowmajor", "random", "none", "connectivity", "distance", "hilbert_wide"])
    ap.add_argument("--n", type=int, default=512, help="quads per side of the graded mesh")
    ap.add_argument("--workload", default="graded", choices=["graded", "layered", "homogeneous", "batched", "adjoint"],
                    help="graded 512x512 (default), the layered 4096x1024 model (67M nodes), or batched shots")
    ap.add_argument("--batch-shots", type=int, default=64)
    ap.add_argument("--batch-nmin", type=int, default=64)
    ap.add_argument("--batch-nmax", type=int, default=1024)
    ap.add_argument("--batch-stream", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="sem_batch_set_stream: -1 automatic, 1 every order streamed, 2 clock-driven one launch per "
                         "step, 0 one launch per order and step with counters")
    ap.add_argument("--no-compare", action="store_true", help="skip the per-ordering comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline only: skip the other precisions, the error block and the layered model")
    ap.add_argument("--metric", default="bilinear", choices=["bilinear", "stored"],
                    help="FP32 geometric factors formed per point from the bilinear map (default) or "
                         "computed in FP64, rounded once and streamed")
    ap.add_argument("--scheme", default="leapfrog", choices=["leapfrog", "heun"],
                    help="leapfrog (default) or the paper's first-order system with Heun steps")
    ap.add_argument("--band", type=int, default=-1,
                    help="steps per band of the streamed wavefront order (-1 = library default, 0 = step order)")
    ap.add_argument("--window", type=int, default=0, help="levels per wavefront tile (0 = automatic)")
    ap.add_argument("--eb", type=int, default=0, help="elements per block (0 = library default)")
    ap.add_argument("--threads", type=int, default=0, help="threads per block (0 = library default)")
    ap.add_argument("--stream", type=int, default=-1,
                    help="steps per streamed launch (0 = one launch per step; -1 = library default)")
    return ap.parse_args()


def max_over_ranks(torch, dist, x, world, device):
    """The largest of every rank's x (the job takes as long as its slowest
    rank); x itself for one rank."""
    if world <= 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, nodes_per_rank, steps, seconds):
    """Whole-job node-updates/s: every rank advances its own replica (weak
    scaling), timed by the slowest rank."""
    return world * nodes_per_rank * steps / seconds


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(args, rank=0):
    if args.workload == "layered":
        m = gen.layered(4096, 1024)
    elif args.workload == "homogeneous":
        m = gen.unit_square(args.n)
    else:
        m = gen.graded(args.n)
    # replicas: each rank shoots from its own source position
    if rank:
        g = gen.SplitMix64(gen.DEFAULT_SEED + 100 + rank)
        m["src_xy"] = (0.25 + 0.5 * g.uniform(), 0.25 + 0.5 * g.uniform())
    return m


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        self.t0 = time.time()

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        rows = []
        try:
            with open(self.f.name) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.f.name)
        return rows

    @staticmethod
    def summarize(rows):
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_handle(P, m, precision, ordering, nsteps_cap, eb=0, threads=0, scheme="leapfrog", stream=-1,
                tiling=(-1, 0), metric="bilinear"):
    h = P.SEM(m["coords"], m["quads"], 4, precision)
    if scheme != "leapfrog":
        h.sem_set_scheme(scheme)
    if metric != "bilinear":
        h.sem_set_metric(metric)
    if stream >= 0:
        h.sem_set_stream(stream)
    h.sem_set_stream_tiling(*tiling)
    h.sem_reorder(ordering)
    h.sem_set_model(m["vel"], m["rho"])
    if eb or threads:
        h.sem_set_tuning(eb, threads)
    h.sem_set_source(m["f0"], m["t0"], m["amp"], *m["src_xy"])
    h.sem_set_receivers(m["receivers"], nsteps_cap)
    h.sem_set_dt(0.3 * h.sem_cfl_dt())
    return h


def time_steps(torch, h, k):
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    h.sem_step(k)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def oracle_c(m):
    """The C/OpenMP FP64 oracle on a workload mesh (all host cores)."""
    from oracle import cpp
    return cpp.SEMC(m["coords"], m["quads"], 4, m["vel"], m["rho"], validate=False)


def cpu_baseline(m, dt, budget_s=12.0, S=None):
    """The FP64 CPU oracle (the C/OpenMP restatement, as it stands) on the
    same mesh: leapfrog steps with source and receivers after 2 warm-up
    steps, as many as fit in about budget_s seconds, on all host cores; then
    2 steps on one thread. Returns (node-updates/s all cores, steps, busy
    threads, node-updates/s one thread)."""
    from oracle import cpp
    S = S or oracle_c(m)
    src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
    t = time.perf_counter()
    u, up, _ = S.run(2, dt, src=src, receivers=m["receivers"])
    per = max((time.perf_counter() - t) / 2, 1e-6)
    k = int(max(2, min(2000, budget_s / per)))
    t, c = time.perf_counter(), time.process_time()
    S.run(k, dt, src=src, receivers=m["receivers"], u0=u, u_prev=up, step0=2)
    el, cpu = time.perf_counter() - t, time.process_time() - c
    S1 = cpp.SEMC(m["coords"], m["quads"], 4, m["vel"], m["rho"], threads=1, validate=False)
    t = time.perf_counter()
    S1.run(2, dt, src=src)
    el1 = time.perf_counter() - t
    S1.close()
    return S.n_nodes * k / el, k, cores_busy(cpu, el), S.n_nodes * 2 / el1


def kernel_source_digest():
    """sha256 of the CUDA kernel sources: a recorded ncu traffic figure is
    only reported while the kernels it was measured on are unchanged."""
    import hashlib
    hsh = hashlib.sha256()
    for f in ("sem_kernels.cu", "sem_kernels.cuh", "sem_plan.h"):
        with open(os.path.join(ROOT, "paper_2104_08416_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()


def recorded_traffic(precision, ordering, kernel, stream_order="step", workload=WORKLOAD, metric="bilinear"):
    """DRAM bytes per step of the step kernel from the committed ncu records
    (same workload, precision, metric source, ordering, kernel sources and
    order of the streamed units); None when no record matches."""
    tfile = os.path.join(ROOT, "profiles", "sem_step_kernel_traffic.json")
    try:
        with open(tfile) as fh:
            tj = json.load(fh)
    except (OSError, ValueError):
        return None
    digest = kernel_source_digest()
    for r in (tj.get("records", []) if isinstance(tj, dict) else []):
        try:
            if (r.get("workload") == workload and r.get("precision") == precision and r.get("ordering") == ordering
                    and r.get("metric", "bilinear") == metric
                    and str(r.get("kernel", "")).startswith(kernel + "<") and r.get("kernel_sha256") == digest
                    and r.get("stream_order", "step") == stream_order):
                return float(r["dram_bytes_per_launch"]) / float(r.get("steps_per_launch", 1))
        except (ValueError, KeyError, TypeError):
            continue
    return None


def cores_busy(cpu_s, wall_s):
    """Threads a timed CPU region kept busy on average: process CPU time over
    wall time (the NumPy oracle's gathers, einsum and bincount run on one)."""
    return max(1, int(round(cpu_s / max(wall_s, 1e-9))))


def threads_used():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, world, rank):
    """--impl reference: the FP64 CPU oracle (the C/OpenMP restatement, as it
    stands, on all host cores) on the same workload as the GPU line: W
    untimed leapfrog steps, then K timed steps with source and receivers."""
    if rank != 0:
        return
    if args.workload == "layered":
        m, wname = gen.layered(4096, 1024), "layered_4096x1024_p4"
    elif args.workload == "homogeneous":
        m, wname = gen.unit_square(args.n), f"homogeneous_{args.n}x{args.n}_p4"
    else:
        m, wname = gen.graded(args.n), (WORKLOAD if args.n == 512 else f"graded_{args.n}x{args.n}_p4")
    from oracle import sem as osem
    S = oracle_c(m)
    dt = 0.3 * osem.cfl_dt(m["coords"], m["quads"], 4, m["vel"])
    src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
    u, up, _ = S.run(args.warmup, dt, src=src, receivers=m["receivers"])
    t, c = time.perf_counter(), time.process_time()
    S.run(args.steps, dt, src=src, receivers=m["receivers"], u0=u, u_prev=up, step0=args.warmup)
    el, cpu = time.perf_counter() - t, time.process_time() - c
    v = S.n_nodes * args.steps / el
    sample = (f"{wname} ({S.n_nodes} nodes), {args.steps} leapfrog steps of the FP64 C/OpenMP oracle "
              f"(dense element matrices) after {args.warmup} untimed")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wname, "sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores_busy(cpu, el), "host_threads": threads_used(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_batched(args, P, torch):
    """Batched shots (C4): 64 independent layered models of n x n quads (n
    uniform in [nmin, nmax]), orders 3..7, one Ricker source each, advanced by
    sem_batch_step (streamed: per order one launch per 64-step block over the
    blocks of all its shots, captured in a CUDA graph; block sizes autotuned
    on 24-step streamed trials). Reported against the same shots in FP64 on
    the GPU (batched likewise: the plain FP64 GPU path), with the error of
    the batched run against that FP64 run after the same steps, and against
    the batched handles stepped one shot at a time with sem_step."""
    shots = gen.batched(args.batch_shots, args.batch_nmin, args.batch_nmax)
    K = args.steps if args.steps != 2000 else 1000
    W = args.warmup
    cap = W + K + 8

    def build_all(prec):
        t0 = time.perf_counter()
        hs = []
        for m in shots:
            h = P.SEM(m["coords"], m["quads"], m["order"], prec)
            h.sem_reorder(args.ordering)
            h.sem_set_model(m["vel"], m["rho"])
            h.sem_set_source(m["f0"], m["t0"], m["amp"], *m["src_xy"])
            h.sem_set_receivers(m["receivers"], cap + K)
            h.sem_set_dt(0.3 * h.sem_cfl_dt())
            hs.append(h)
        b = P.SEMBatch(hs, autotune_steps=24)
        b.sem_batch_set_stream(args.batch_stream)
        b.sem_batch_step(W)
        torch.cuda.synchronize()
        return hs, b, time.perf_counter() - t0

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    hs, b, setup_s = build_all(args.precision)
    nodes = sum(h.n_nodes for h in hs)
    elems = sum(m["quads"].shape[0] for m in shots)
    sampler = ClockSampler(0)
    time.sleep(0.2)
    el = timed(lambda: b.sem_batch_step(K))
    clocks = ClockSampler.summarize(sampler.stop())
    info = b.sem_batch_info()
    mode = b.sem_batch_mode()
    u32 = [h.sem_read_wavefield() for h in hs]
    # the same handles one shot at a time (each streams on its own)
    el_solo = timed(lambda: [h.sem_step(K) for h in hs])
    b.sem_batch_destroy()
    for h in hs:
        h.sem_destroy()
    # the plain FP64 GPU path on the same shots and steps
    h64, b64, setup64 = build_all("fp64")
    el64 = timed(lambda: b64.sem_batch_step(K))
    errs = [rel_l2(u, h.sem_read_wavefield()) for u, h in zip(u32, h64)]
    b64.sem_batch_destroy()
    for h in h64:
        h.sem_destroy()
    line = {
        "metric": "GLL node-updates/s (batched shots, orders 3-7)", "value": nodes * K / el, "unit": UNIT,
        "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": 1e3 * el / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32_kahan": "f32", "fp32": "f32", "fp64": "f64"}[args.precision], "data": "synthetic",
        "config": {"workload": f"batched_{args.batch_shots}_shots_{args.batch_nmin}-{args.batch_nmax}_p3-7",
                   "shots": len(hs), "nodes": nodes, "elements": elems, "precision": args.precision,
                   "ordering": args.ordering, "autotuned": info, "mode": mode, "setup_s": setup_s},
        "one_shot_at_a_time": {"value": nodes * K / el_solo, "unit": UNIT, "ms_per_step": 1e3 * el_solo / K},
        "fp64_gpu": {"value": nodes * K / el64, "unit": UNIT, "ms_per_step": 1e3 * el64 / K, "setup_s": setup64},
        "error_vs_fp64_gpu": {"steps": W + K, "max_rel_l2_over_shots": max(errs),
                              "median_rel_l2_over_shots": float(np.median(errs)), "tolerance": 1e-5},
        "gpu_launches": int((K // mode["steps_per_launch"] + 1) * (mode["streamed_classes"] + 1)
                            + K * (len(info["orders"]) - mode["streamed_classes"]) + len(hs)),
        "clocks": clocks,
    }
    print(json.dumps(line))


def run_adjoint(args, P, torch):
    """Velocity gradient of the L2 trace misfit: 256 x 256 quads, order 4,
    layered true model, smoothed start model, 8 shots, 3000 steps; the
    gradient from sem_misfit_gradient (forward with checkpoints, recompute,
    adjoint), FP64 and FP32, timed per gradient over all shots."""
    from paper_2104_08416_gb300.autograd import Survey
    c = gen.adjoint_case()
    m = c["mesh"]
    n = args.steps if args.steps != 2000 else 3000
    h = P.SEM(m["coords"], m["quads"], 4, "fp64")
    h.sem_reorder(args.ordering)
    h.sem_set_model(c["vel_true"], m["rho"])
    dt = 0.3 * h.sem_cfl_dt()
    N = h.n_nodes
    h.sem_destroy()
    d_obs = []
    for sx, sy in c["sources"]:
        t = P.SEM(m["coords"], m["quads"], 4, "fp64")
        t.sem_reorder(args.ordering)
        t.sem_set_model(c["vel_true"], m["rho"])
        t.sem_set_source(c["f0"], c["t0"], c["amp"], sx, sy)
        t.sem_set_receivers(c["receivers"], n)
        t.sem_set_dt(dt)
        t.sem_step(n)
        d_obs.append(t.sem_read_traces())
        t.sem_destroy()
    v0 = np.asarray(c["vel_start"], dtype=np.float64)
    res = {}
    for prec in ("fp64", "fp32"):
        sv = Survey(m["coords"], m["quads"], 4, c["sources"], c["receivers"], d_obs, n, dt, c["f0"], c["t0"],
                    c["amp"], rho=m["rho"], precision=prec, ordering=args.ordering)
        sv.misfit_and_gradient(v0)                     # warm-up (builds the handles)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 2
        for _ in range(reps):
            J, g = sv.misfit_and_gradient(v0)
        torch.cuda.synchronize()
        el = (time.perf_counter() - t0) / reps
        sv.close()
        res[prec] = (J, g, el)
    J64, g64, t64 = res["fp64"]
    J32, g32, t32 = res["fp32"]
    shots = len(c["sources"])
    # a gradient = forward + recomputed forward + adjoint: three passes of
    # N x n node updates per shot
    line = {
        "metric": "adjoint gradient, node-updates/s (3 passes per shot)", "value": 3 * shots * N * n / t64,
        "unit": UNIT, "n_gpus": 1, "steps": n, "warmup": 1, "ms_per_step": 1e3 * t64 / (shots * n),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "adjoint_256x256_p4_8shots", "nodes": N, "shots": shots, "steps": n,
                   "checkpoints": "ceil(sqrt(steps))", "ordering": args.ordering},
        "seconds_per_gradient": {"fp64": t64, "fp32": t32},
        "misfit": {"fp64": J64, "fp32": J32},
        "fp32_vs_fp64": {"gradient_rel_l2": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64)),
                         "misfit_rel": abs(J32 - J64) / J64},
    }
    print(json.dumps(line))


def step_rate(P, torch, m, precision, k, w, ordering="hilbert", metric="bilinear"):
    """node-updates/s and the step kernel's time per step of one precision on
    a workload mesh: w untimed steps, k timed, k more with per-launch events."""
    h = make_handle(P, m, precision, ordering, w + 2 * k + 8, metric=metric)
    h.sem_step(w)
    torch.cuda.synchronize()
    el = time_steps(torch, h, k)
    h.sem_profile_enable(True)
    time_steps(torch, h, k)
    bms, bl, oms, ol = h.sem_profile_read()
    h.sem_profile_enable(False)
    spl, nopen = h.sem_launch_info()
    block_bytes, _ = h.sem_traffic_model()
    N = h.n_nodes
    h.sem_destroy()
    return {"node_updates_per_s": N * k / el, "ms_per_step": 1e3 * el / k, "steps": k,
            "step_kernel_us": 1e3 * bms / k, "launches": int(bl), "steps_per_launch": k / max(bl, 1),
            "kernel": "sem_stream_kernel" if spl > 1 else "sem_step_kernel",
            "compulsory_bytes_per_step": block_bytes, "nodes": N}


def hbm_roofline(r, precision, peak, peak_kind, workload, ordering="hilbert", metric="bilinear"):
    """Roofline of the step kernel from a step_rate() result: algorithmic
    bytes per node-update times the node updates of one launch over the
    launch's mean event time, and, where an ncu record of the same kernel
    sources exists, the DRAM traffic per step and its fraction of the peak."""
    N, spl = r["nodes"], r["steps_per_launch"]
    launch_us = r["step_kernel_us"] * spl
    algo = ALGO_BYTES[precision]
    achieved = algo * N * spl / (launch_us * 1e-6) / 1e9
    tps = recorded_traffic(precision, ordering, r["kernel"], "step", workload, metric)
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "peak_kind": peak_kind, "kernel": r["kernel"], "launch_us": launch_us, "steps_per_launch": spl,
           "algorithmic_bytes_per_node_update": algo, "traffic": None if tps is None else tps * spl,
           "traffic_per_step": tps, "dram_frac": None,
           "compulsory_bytes_per_step": r["compulsory_bytes_per_step"],
           "compulsory_frac": r["compulsory_bytes_per_step"] / (r["step_kernel_us"] * 1e-6) / 1e9 / peak}
    if tps is not None:
        out["dram_gbs"] = tps / (r["step_kernel_us"] * 1e-6) / 1e9
        out["dram_frac"] = out["dram_gbs"] / peak
    return out


def fp64_roofline(r):
    """The FP64 leapfrog is bound by GB300's FP64 arithmetic rate."""
    fl = FLOPS_FP64_LEAPFROG * r["nodes"] / (r["step_kernel_us"] * 1e-6) / 1e12
    return {"bound": "alu", "achieved": fl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": fl / FP64_PEAK_TFLOPS, "peak_kind": "derived (nominal FP64 rate)",
            "flops_per_node_update": FLOPS_FP64_LEAPFROG, "kernel": r["kernel"]}


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def error_block(P, torch, m, nsteps=2000, S=None):
    """The stated error of the FP32 path: (1) FP32+Kahan against FP64, both
    on the GPU, after the workload's nsteps steps from rest (wavefield and
    receiver traces); (2) both precisions against the FP64 C oracle over the
    first 10 steps from a smooth field cos(3 pi x) cos(2 pi y) that puts signal
    on every node (u^-1 from the oracle's K and M), with the source on."""
    out = {}
    res = {}
    variants = (("fp64", "fp64", "bilinear"), ("fp32_kahan", "fp32_kahan", "bilinear"),
                ("fp32_kahan_stored_metric", "fp32_kahan", "stored"))
    for name, prec, metric in variants:
        h = make_handle(P, m, prec, "hilbert", nsteps, metric=metric)
        h.sem_step(nsteps)
        res[name] = (h.sem_read_wavefield(), h.sem_read_traces())
        h.sem_destroy()
    tr64 = res["fp64"][1]
    reached = bool(np.abs(tr64).max() > 0)
    for name in ("fp32_kahan", "fp32_kahan_stored_metric"):
        out[f"{name}_vs_fp64_gpu"] = {"steps": nsteps, "wavefield_rel_l2": rel_l2(res[name][0], res["fp64"][0]),
                                      # None while the wavefront has not reached the receivers
                                      "traces_rel_l2": rel_l2(res[name][1], tr64) if reached else None,
                                      "tolerance": 1e-5}
    if S is not None:
        n = 10
        h = make_handle(P, m, "fp64", "hilbert", n)
        dt = 0.3 * h.sem_cfl_dt()
        xy = h.sem_node_coordinates()
        h.sem_destroy()
        u0 = np.cos(3.0 * np.pi * xy[:, 0]) * np.cos(2.0 * np.pi * xy[:, 1])
        um1 = u0 - 0.5 * dt * dt * S.apply_K(u0) / S.M
        src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
        u_ref, _, tr_ref = S.run(n, dt, src=src, receivers=m["receivers"], u0=u0, u_prev=um1)
        vs = {"steps": n, "start": "cos(3 pi x) cos(2 pi y)"}
        for name, prec, metric, tol in (("fp64", "fp64", "bilinear", 1e-12),
                                        ("fp32_kahan", "fp32_kahan", "bilinear", 1e-5),
                                        ("fp32_kahan_stored_metric", "fp32_kahan", "stored", 1e-5)):
            h = make_handle(P, m, prec, "hilbert", n, metric=metric)
            h.sem_set_dt(dt)
            h.sem_set_state(u0, um1, 0)
            h.sem_step(n)
            vs[name] = {"wavefield_rel_l2": rel_l2(h.sem_read_wavefield(), u_ref),
                        "traces_rel_l2": rel_l2(h.sem_read_traces(), tr_ref), "tolerance": tol}
            h.sem_destroy()
        out["vs_cpu_oracle"] = vs
    return out


def layered_line(P, torch, K, peak, peak_kind):
    """The multilayered 4096 x 1024 model (67,129,345 nodes; the largest
    single-GPU workload) in FP32+Kahan, Hilbert order: rate, roofline, and the
    error against FP64 after 300 steps on every 16th node and on the traces."""
    m = gen.layered(4096, 1024)
    k = max(K, 100)
    r = step_rate(P, torch, m, "fp32_kahan", k, 3)
    line = {"workload": "layered_4096x1024_p4", "nodes": r["nodes"], "elements": int(m["quads"].shape[0]),
            "value": r["node_updates_per_s"], "unit": UNIT, "ms_per_step": r["ms_per_step"], "steps": k,
            "roofline": hbm_roofline(r, "fp32_kahan", peak, peak_kind, "layered_4096x1024_p4")}
    n = 300
    res = {}
    for prec in ("fp64", "fp32_kahan"):
        h = make_handle(P, m, prec, "hilbert", n)
        h.sem_step(n)
        res[prec] = (h.sem_read_wavefield()[::16], h.sem_read_traces())
        h.sem_destroy()
    reached = bool(np.abs(res["fp64"][1]).max() > 0)
    line["error"] = {"fp32_kahan_vs_fp64_gpu": {
        "steps": n, "wavefield_rel_l2_every_16th_node": rel_l2(res["fp32_kahan"][0], res["fp64"][0]),
        # None while the wavefront has not reached the surface receivers
        "traces_rel_l2": rel_l2(res["fp32_kahan"][1], res["fp64"][1]) if reached else None,
        "tolerance": 1e-5}}
    return line


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2104_08416_gb300 import build as _build
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    import paper_2104_08416_gb300 as P
    P.load()
    P.sem_set_allocator_torch()
    if args.workload in ("batched", "adjoint"):
        if rank == 0:
            (run_batched if args.workload == "batched" else run_adjoint)(args, P, torch)
        if world > 1:
            dist.destroy_process_group()
        return

    K, W = args.steps, args.warmup
    m = workload(args, rank)
    if args.workload == "layered":
        wname = "layered_4096x1024_p4"
    elif args.workload == "homogeneous":
        wname = f"homogeneous_{args.n}x{args.n}_p4"
    else:
        wname = WORKLOAD if args.n == 512 else f"graded_{args.n}x{args.n}_p4"
    cap = W + 2 * K + 8
    h = make_handle(P, m, args.precision, args.ordering, cap, args.eb, args.threads, args.scheme, args.stream,
                    (args.band, args.window), args.metric)
    N = h.n_nodes
    # warm-up (the first call builds the device data)
    h.sem_step(W)
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if rank == 0 else None
    time.sleep(0.2)
    # timed region: K steps, barrier + sync on both sides
    if world > 1:
        dist.barrier()
    el = time_steps(torch, h, K)
    el = max_over_ranks(torch, dist, el, world, "cuda")
    # second pass with per-kernel events for the roofline
    h.sem_profile_enable(True)
    prof_el = time_steps(torch, h, K)
    bms, bl, oms, ol = h.sem_profile_read()
    h.sem_profile_enable(False)
    block_bytes, open_bytes = h.sem_traffic_model()
    spl, nopen = h.sem_launch_info()
    band, window = h.sem_stream_order()
    time.sleep(0.2)
    clocks = ClockSampler.summarize(sampler.stop()) if sampler else None
    u = h.sem_read_wavefield()
    finite = bool(np.isfinite(u).all())
    h.sem_destroy()

    # end to end through the public API with host buffers, set-up excluded
    # like the reference arm's: the K steps' inputs (the source table, host
    # to device) and results (the receiver traces of every step, device to
    # host) cross the boundary inside the timed region; the handle was set up
    # and its device data built before it (timed apart: setup_s), and the
    # final wavefield read-back is timed apart too (wavefield_s)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2 = make_handle(P, m, args.precision, args.ordering, K, args.eb, args.threads, args.scheme, args.stream,
                     (args.band, args.window), args.metric)
    h2.sem_read_mass()                 # builds the device data
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    h2d0, d2h0 = h2.sem_transfer_bytes()
    t0 = time.perf_counter()
    h2.sem_step(K)
    tr = h2.sem_read_traces()
    torch.cuda.synchronize()
    e2e_el = time.perf_counter() - t0
    h2d, d2h = h2.sem_transfer_bytes()
    h2d, d2h = h2d - h2d0, d2h - d2h0
    t0 = time.perf_counter()
    u2 = h2.sem_read_wavefield()
    wavefield_s = time.perf_counter() - t0
    h2.sem_destroy()
    e2e_el = max_over_ranks(torch, dist, e2e_el, world, "cuda")

    # ordering comparison (the paper's locality claim, restated on the GPU)
    orderings = None
    if rank == 0 and not args.no_compare:
        orderings = {}
        kk = min(K, 500)
        for kind in ("hilbert", "rowmajor", "random", "none", "connectivity", "distance", "hilbert_wide"):
            hh = make_handle(P, m, args.precision, kind, W + 2 * kk + 8, args.eb, args.threads, args.scheme, args.stream,
                    (args.band, args.window))
            hh.sem_step(W)
            t_ord = time_steps(torch, hh, kk)
            hh.sem_profile_enable(True)
            time_steps(torch, hh, kk)
            b_ms, b_l, o_ms, o_l = hh.sem_profile_read()   # kk steps
            bb, ob = hh.sem_traffic_model()
            spl_o, no = hh.sem_launch_info()
            hh.sem_destroy()
            # which kernel ran: DENSE plans (orderings whose node numbering
            # follows the element order) may stream; GATHER plans launch once
            # per step (--stream 0 makes every ordering do so)
            orderings[kind] = {"node_updates_per_s": N * kk / t_ord, "ms_per_step": 1e3 * t_ord / kk,
                               "step_kernel_us": 1e3 * b_ms / kk, "open_nodes": no,
                               "kernel": "sem_stream_kernel" if spl_o > 1 else "sem_step_kernel",
                               "step_bytes_model": bb}
    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peak, peak_kind = read_peaks()
    full = args.workload == "graded" and args.n == 512 and args.scheme == "leapfrog" and world == 1
    cpu = None
    S_c = None
    if not args.no_cpu_baseline and world == 1 and args.workload == "graded":
        from oracle import sem as osem
        S_c = oracle_c(m)
        dt_w = 0.3 * osem.cfl_dt(m["coords"], m["quads"], 4, m["vel"])
        v, k, busy, v1 = cpu_baseline(m, dt_w, S=S_c)
        cpu = {"value": v, "unit": UNIT, "cores": busy, "host_threads": threads_used(), "kind": "oracle",
               "one_core": v1,
               "sample": f"{k} leapfrog steps (after 2 untimed) of the FP64 C/OpenMP oracle on the full {wname} "
                         f"mesh ({N} nodes) on all host threads, set-up excluded; one_core: 2 steps on one thread"}
    extra = {}
    if full and args.precision == "fp32_kahan" and args.ordering == "hilbert" and not args.no_extra:
        kk = max(K, 200)
        precs = {}
        for prec in ("fp64", "fp32", "fp32_kahan_stored_metric"):
            if prec == "fp32_kahan_stored_metric":
                r = step_rate(P, torch, m, "fp32_kahan", kk, 3, metric="stored")
                precs[prec] = {"value": r["node_updates_per_s"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                               "steps": kk, "note": "FP32+Kahan streaming G_q computed in FP64 and rounded once "
                                                    "(12 B per GLL point) instead of forming it from the bilinear map",
                               "roofline": hbm_roofline(r, "fp32_kahan", peak, peak_kind, WORKLOAD,
                                                        metric="stored")}
                continue
            r = step_rate(P, torch, m, prec, kk, 3)
            precs[prec] = {"value": r["node_updates_per_s"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                           "steps": kk,
                           "roofline": fp64_roofline(r) if prec == "fp64" else
                           hbm_roofline(r, prec, peak, peak_kind, WORKLOAD)}
            if prec == "fp64":
                precs[prec]["roofline"]["hbm_frac"] = hbm_roofline(r, prec, peak, peak_kind, WORKLOAD)["frac"]
        extra["precisions"] = precs
        extra["error"] = error_block(P, torch, m, 2000, S_c)
        extra["workloads"] = {"layered_4096x1024_p4": layered_line(P, torch, K, peak, peak_kind)}
    if S_c is not None:
        S_c.close()

    # the profiled pass covers K steps in bl step-kernel launches (one step
    # each, or several when the time loop is streamed)
    blk_us = 1e3 * bms / K
    launch_us = 1e3 * bms / max(bl, 1)
    steps_per_launch = K / max(bl, 1)
    # algorithmic bytes of one step-kernel launch: the per-node-update figure
    # of the hot path times the node updates one launch makes
    algo = (ALGO_BYTES_HEUN if args.scheme == "heun" else ALGO_BYTES)[args.precision]
    achieved = algo * N * steps_per_launch / (launch_us * 1e-6) / 1e9
    kname = "sem_stream_kernel" if spl > 1 else "sem_step_kernel"
    sorder = {"band_steps": band, "window_levels": window} if band > 0 else "step"
    traffic_step = recorded_traffic(args.precision, args.ordering, kname, sorder, wname, args.metric)
    traffic = None if traffic_step is None else traffic_step * steps_per_launch
    dram_gbs = None if traffic_step is None else traffic_step / (blk_us * 1e-6) / 1e9
    value = job_rate(world, N, K, el)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * el / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32_kahan": "f32", "fp32": "f32", "fp64": "f64"}[args.precision], "data": "synthetic",
        "config": {"workload": wname, "nodes": N, "elements": m["quads"].shape[0], "order": 4,
                   "precision": args.precision, "ordering": args.ordering, "scheme": args.scheme,
                   "metric": args.metric,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "stream_order": sorder,
                   "l2": (f"per-step working set {block_bytes / 1e6:.0f} MB > L2 {L2_BYTES / 1e6:.0f} MB, no flush"
                          if block_bytes > L2_BYTES else
                          f"per-step working set {block_bytes / 1e6:.1f} MB fits in L2, no flush (small workload)"),
                   "finite": finite},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_per_step": traffic_step,
                     "dram_gbs": dram_gbs, "dram_frac": None if dram_gbs is None else dram_gbs / peak,
                     "kernel": kname, "peak_kind": peak_kind,
                     "steps_per_launch": steps_per_launch, "launch_us": launch_us,
                     "step_kernel_us": blk_us, "open_kernel_us_per_run": 1e3 * oms / max(ol, 1),
                     "algorithmic_bytes_per_launch": algo * N * steps_per_launch,
                     "compulsory_bytes_per_step": block_bytes, "compulsory_gbs": block_bytes / (blk_us * 1e-6) / 1e9,
                     "open_bytes_per_launch": open_bytes,
                     "open_nodes": nopen, "profiled_ms_per_step": 1e3 * prof_el / K,
                     "algorithmic_bytes_per_node_update": algo,
                     "algorithmic_gbs_per_step": algo * N * K / el / 1e9},
        "cpu_baseline": cpu,
        "e2e": {"value": world * N * K / e2e_el, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
                "d2h_bytes_per_step": d2h / K,
                "includes": "K steps through sem_step with the source table uploaded and every step's receiver "
                            "traces read back by sem_read_traces; set-up excluded (as in the reference arm)",
                "setup_s": setup_s, "wavefield_readback_s": wavefield_s,
                "with_setup": world * N * K / (e2e_el + setup_s)},
        "gpu_launches": int(bl + ol),
        "clocks": clocks,
        "orderings": orderings,
    }
    line.update(extra)
    if args.precision == "fp64" and args.scheme == "leapfrog" and args.n == 512 and args.workload == "graded":
        # FP64 arithmetic bound: the roofline is the FP64 ALU rate
        fl = FLOPS_FP64_LEAPFROG * N * steps_per_launch / (launch_us * 1e-6) / 1e12
        line["roofline"].update({"bound": "alu", "achieved": fl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                 "frac": fl / FP64_PEAK_TFLOPS, "peak_kind": "derived (nominal FP64 rate)",
                                 "flops_per_node_update": FLOPS_FP64_LEAPFROG,
                                 "hbm_frac": achieved / peak})
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

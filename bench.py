#!/usr/bin/env python
"""Benchmark of the polynomial-diagram objective+gradient hot path.

Workload: a 1024 x 1024 pixel grid on [-1,1]^2 labelled by a seeded
degree-4 polynomial diagram with N = 500 grains (degree <= 1 Legendre
coefficients from uniform sites, degree >= 2 coefficients normal with spread
1/(2N); 485 grains are non-empty), 2% boundary label noise, fitted at
degree 4 (K = 15) with eps = 1e-3.  One
step is one objective + gradient evaluation (features, logits, log-sum-exp,
objective and gradient reductions) at the generating parameters.

Metric: pixel x grain objective+gradient evaluations per second
(P * N_eff per step).  ``value`` is timed on the device with CUDA events
with inputs resident in HBM and L2 flushed between steps (a 256 MiB write,
not timed); ``e2e`` is the same metric through the public API with the
step's inputs copied from pinned host memory and its outputs copied back
inside the timed region.

``--impl reference`` times the FP64 CPU oracle (the only reference this
method has) on a bounded band of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_20816_gb300 import synth  # noqa: E402

SHAPE = (1024, 1024)
N_GRAINS = 500
DEG = 4
EPS = 1e-3
NOISE = 0.02
SEED = synth.SEED_BASE + 1
WORKLOAD = ("2D 1024x1024, N=500 degree-4 polynomial diagram, 2% boundary noise, "
            "fit degree 4 (K=15), eps=1e-3")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["fp64", "fp32", "bf16", "bf16x3"],
                    help="bf16x3 (default): tcgen05 logits with three-term bf16 operands, fp32 accumulation and "
                         "log-sum-exp, fp16 gradient operands, double final reductions; fp32: CUDA-core path")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-fit", action="store_true",
                    help="skip the time-to-fit leg of the default run (about 100 s, mostly the FP64 reference fit)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP32, dense and early-parameter lines and the time-to-fit leg")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target duration of the CPU oracle sample")
    ap.add_argument("--newton-iters", type=int, default=30,
                    help="--workload config3: Newton-CG iterations of the 256^3 fits")
    ap.add_argument("--train-maps", type=int, default=3000,
                    help="--workload fit: 256^2 maps the warm-start network is trained on")
    ap.add_argument("--fit-maps", type=int, default=4,
                    help="--workload fit: 512^2, N = 300 maps of the warm-start evaluation")
    ap.add_argument("--workload", default="config2", choices=["config2", "batched", "fit", "config3"],
                    help="config2: the headline line; batched: 256 maps in one persistent launch vs per-map "
                         "launches; fit: time to the FP64 objective for the precision schedules; config3: "
                         "the 256^3 workload per degree and precision")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "source": "fallback"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for t, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((t, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sel = [r for r in rows if self.t0 and self.t1 and self.t0 - 0.05 <= r[0] <= self.t1 + 0.05] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in sel for q in range(4) if r[3][q].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": max(r[2] for r in sel),
                "reasons": reasons, "samples": len(sel)}


# ---------------------------------------------------------------------------
# the workload
# ---------------------------------------------------------------------------
def make_workload_gpu(pd, torch):
    """Rasterise the generating diagram with the library's own assignment."""
    y, z = synth.poly_params(SEED, N_GRAINS, 2, pd.pd_K(2, DEG))
    th = pd.pd_theta_from_apd(2, DEG, y, np.zeros(N_GRAINS)).numpy()
    th[:, 3:] = z[:, 3:]
    grid = pd.Grid(SHAPE)
    lab, _, _ = pd.pd_assign(grid, N_GRAINS, DEG, torch.from_numpy(th).cuda())
    lab = synth.boundary_noise(lab.cpu().numpy(), SHAPE, NOISE, SEED + 7)
    lab, n_eff, used = synth.compact(lab)
    return grid, lab.astype(np.int32), n_eff, np.ascontiguousarray(th[used])


def oracle_band(rows: int, r0=None):
    """A band of `rows` grid rows of the same workload (starting at row r0,
    centred by default), as an explicit point list labelled by the oracle
    (only the CPU legs call this).  Every generated grain stays in the
    objective (the band alone would empty most of them), so the cost per
    pixel is that of the whole workload."""
    import oracle as O
    n1, n2 = SHAPE
    if r0 is None:
        r0 = (n2 - rows) // 2
    xs = -1.0 + (2.0 * np.arange(n1) + 1.0) / n1
    ys = -1.0 + (2.0 * np.arange(r0, r0 + rows) + 1.0) / n2
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    g = O.Grid(coords=np.stack([X.reshape(-1), Y.reshape(-1)], 1))
    y, z = synth.poly_params(SEED, N_GRAINS, 2, O.K(2, DEG))
    th = O.theta_from_apd(2, DEG, y, np.zeros(N_GRAINS))
    th[:, 3:] = z[:, 3:]
    lab, _ = O.assign(g, N_GRAINS, DEG, th)
    lab = synth.boundary_noise(lab, (n1, rows), NOISE, SEED + 7)
    return O, g, lab.astype(np.int32), N_GRAINS, np.ascontiguousarray(th)


def _oracle_worker(args):
    """One host core: the oracle's objective+gradient on its own band, with
    wall-clock start and end (the process pool is spawned, never forked)."""
    rows, r0, barrier = args
    O, g, lab, n, th = oracle_band(rows, r0)
    barrier.wait()                          # every worker has built its band
    t0 = time.time()
    O.objective_grad(g, lab, n, DEG, EPS, th)
    return t0, time.time(), g.P * n


def cpu_oracle_all_cores(rows: int):
    """The oracle on every host core at once: one spawned process per core,
    each on its own band of `rows` rows; pairs of all bands over the wall time
    from the first start to the last end."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    r0s = [(SHAPE[1] - rows) * q // max(1, cores - 1) for q in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man, ctx.Pool(cores) as pool:
        barrier = man.Barrier(cores)
        res = pool.map(_oracle_worker, [(rows, r0, barrier) for r0 in r0s], chunksize=1)
    t0 = min(r[0] for r in res)
    t1 = max(r[1] for r in res)
    pairs = sum(r[2] for r in res)
    return {"value": pairs / (t1 - t0), "unit": "pixel*grain/s", "cores": cores, "kind": "oracle",
            "sample": "objective+gradient of the FP64 C oracle, one process per host core (%d), each on its "
                      "own %d-row band (%d pixels x %d grains), %.1f s wall" % (cores, rows, rows * SHAPE[0],
                                                                               N_GRAINS, t1 - t0)}


def cpu_oracle_rate(target_s: float):
    """Time the oracle's objective+gradient on a band sized for ~target_s."""
    O, g, lab, n, th = oracle_band(8)
    t = time.perf_counter()
    O.objective_grad(g, lab, n, DEG, EPS, th)
    per_px = (time.perf_counter() - t) / g.P
    rows = int(max(8, min(SHAPE[1], target_s / (per_px * SHAPE[0]))))
    O, g, lab, n, th = oracle_band(rows)
    t = time.perf_counter()
    O.objective_grad(g, lab, n, DEG, EPS, th)
    dt = time.perf_counter() - t
    one = {"value": g.P * n / dt, "unit": "pixel*grain/s", "cores": 1, "kind": "oracle",
           "sample": "objective+gradient of the FP64 C oracle (single thread) on a %d-row band "
                     "(%d pixels x %d grains) of the same workload, %.1f s" % (rows, g.P, n, dt)}
    # every core: bands sized so that each process runs about as long
    try:
        one["all_cores"] = cpu_oracle_all_cores(max(2, rows))
    except Exception as e:  # the single-thread figure stands on its own
        one["all_cores"] = {"unavailable": repr(e)[:200]}
    one["host_cores"] = os.cpu_count()
    return one


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps, warm = max(1, args.steps), max(0, args.warmup)
    per_step = max(0.5, min(3.0, 120.0 / (steps + warm)))
    O, g, lab, n, th = oracle_band(8)
    t = time.perf_counter()
    O.objective_grad(g, lab, n, DEG, EPS, th)
    per_px = (time.perf_counter() - t) / g.P
    rows = int(max(2, min(SHAPE[1], per_step / (per_px * SHAPE[0]))))
    O, g, lab, n, th = oracle_band(rows)
    for _ in range(warm):
        O.objective_grad(g, lab, n, DEG, EPS, th)
    t = time.perf_counter()
    for _ in range(steps):
        O.objective_grad(g, lab, n, DEG, EPS, th)
    dt = time.perf_counter() - t
    value = g.P * n * steps / dt
    line = {
        "impl": "reference", "metric": "pixel*grain objective+gradient evaluations per second",
        "value": value, "unit": "pixel*grain/s", "n_gpus": args.gpus, "steps": steps, "warmup": warm,
        "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_rows": rows, "sample_pixels": g.P, "grains": n},
        "cpu_baseline": {"value": value, "unit": "pixel*grain/s", "cores": 1, "kind": "oracle",
                         "sample": "FP64 C oracle, single thread, %d-row band (%d pixels) of the workload "
                                   "per step" % (rows, g.P)},
        "e2e": {"value": value, "unit": "pixel*grain/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def ncu_traffic():
    """DRAM bytes (read + write) per launch of kernels captured with ncu:
    the profile summaries under profiles/ carry lines
        bench-traffic: kernel=<name> bytes_per_launch=<B> scale=<s> source_sha256=<h>
    (B measured on the captured launch, s the factor to one launch of this
    workload, 1 when the capture ran it).  A figure is used only while the
    library's sources hash to h, i.e. for the very code that was measured;
    otherwise the traffic is reported as null."""
    from paper_2605_20816_gb300 import build
    cur = build.source_hash()
    out = {}
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return out
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith((".md", ".txt")):
            continue
        with open(os.path.join(pdir, fn)) as f:
            for line in f:
                if "bench-traffic:" not in line:
                    continue
                kv = dict(t.split("=", 1) for t in line.split("bench-traffic:", 1)[1].split() if "=" in t)
                if kv.get("source_sha256") == cur and "kernel" in kv:
                    out[kv["kernel"]] = (float(kv["bytes_per_launch"]) * float(kv.get("scale", "1")),
                                         "profiles/" + fn)
    return out


# ---------------------------------------------------------------------------
# replicas (one process per GPU, no data-path collective): the timing rule
# ---------------------------------------------------------------------------
def job_ms(ms_local: float, world: int, device) -> float:
    """Whole-job time of the timed region: the maximum over the ranks."""
    if world <= 1:
        return ms_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, pixels: int, grains: int, ms_step: float) -> float:
    """Pixel-grain pairs per second of all replicas (each evaluates the whole
    workload once per step: weak scaling)."""
    return world * pixels * grains / (ms_step * 1e-3)


def time_steps(torch, fn, steps, flush):
    """Device milliseconds per call of fn (CUDA events on the current stream,
    L2 flushed before every call, untimed)."""
    stream = torch.cuda.current_stream()
    for _ in range(2):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for q in range(steps):
        flush.fill_(q & 0xFF)
        ev[q][0].record(stream)
        fn()
        ev[q][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def time_to_fit(pd, grid, lab, N):
    """Time to reach the FP64 plain fit's objective: Phi_ref is Phi after
    1000 FP64 L-BFGS iterations from theta = 0 (the paper's budget, Sec.
    5.2); a form has reached it when Phi >= Phi_ref - 1e-8 |Phi_ref|.  The
    plain FP32 form and the BF16X3 (tensor-core) forms, plain and
    eps-annealed (ANNEAL), each run a first phase of up to 3000 iterations
    that leaves when its relative gain per iteration drops below 1e-7, then
    FP64 refinement; a target met in the first phase must hold in FP64."""
    warm_up_fits(pd, grid, lab, N)
    t = time.perf_counter()
    _, ref = pd.pd_fit(grid, lab, N, DEG, EPS, max_iter=1000, prec=pd.PD_FP64)
    rows = {"fp64_plain": {"seconds": time.perf_counter() - t, "iters": ref["iters"], "evals": ref["evals"],
                           "phi": ref["phi"]}}
    target = ref["phi"] - 1e-8 * abs(ref["phi"])
    for name, prec, kw in (("fp32_then_fp64", pd.PD_FP32, {}), ("bf16x3_then_fp64", pd.PD_BF16X3, {}),
                           ("anneal_bf16x3_then_fp64", pd.PD_BF16X3, ANNEAL)):
        t = time.perf_counter()
        _, rep = pd.pd_fit(grid, lab, N, DEG, EPS, max_iter=3000, prec=prec, refine_iter=1000, target_phi=target,
                           switch_rtol=1e-7, **kw)
        rows[name] = {"seconds": time.perf_counter() - t, "iters": rep["iters"], "iters_phase1": rep["iters_phase1"],
                      "evals": rep["evals"], "phi": rep["phi"], "reached": rep["phi"] >= target,
                      "stages": rep["stages"]}
    best = min(("bf16x3_then_fp64", "anneal_bf16x3_then_fp64"),
               key=lambda k: rows[k]["seconds"] if rows[k]["reached"] else float("inf"))
    ok = rows["fp32_then_fp64"]["reached"] and rows[best]["reached"]
    return {"phi_ref": ref["phi"], "target": target, "runs": rows, "schedule": best,
            "anneal": "eps0 = 10 eps, factor 0.25, 100 iterations per stage, then the normal schedule at eps",
            "multiple_vs_fp32": rows["fp32_then_fp64"]["seconds"] / rows[best]["seconds"] if ok else None}


# eps-annealing of the fit schedules (stages 1e-2, 2.5e-3, then eps = 1e-3)
ANNEAL = dict(anneal_eps0=1e-2, anneal_factor=0.25, anneal_iter=100)


def warm_up_fits(pd, grid, lab, N):
    """One short fit per precision before any fit is timed, so that the
    kernels' first-use cost (module loading) is not counted in a fit."""
    for prec in (pd.PD_FP64, pd.PD_FP32, pd.PD_BF16X3):
        pd.pd_fit(grid, lab, N, DEG, EPS, max_iter=2, prec=prec)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2605_20816_gb300 import pd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    prec = pd.PREC[args.prec]

    grid, lab_np, N, th_np = make_workload_gpu(pd, torch)
    P = grid.P
    K = pd.pd_K(2, DEG)
    lab = torch.from_numpy(lab_np).cuda()
    th = torch.from_numpy(th_np).cuda()
    obj = torch.empty((), dtype=torch.float64, device="cuda")
    grad = torch.empty((N, K), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        pd.pd_objective_grad(grid, lab, N, th, DEG, EPS, prec=prec, obj_out=obj, grad_out=grad)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
        time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.mark(True)
    for s in range(args.steps):
        flush.fill_(s & 0xFF)           # evict the previous step's data from L2 (not timed)
        ev[s][0].record(stream)
        step()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    sampler.mark(False)
    if world > 1:
        dist.barrier()
    ms = job_ms(sum(a.elapsed_time(b) for a, b in ev), world, "cuda")
    clocks = sampler.stop() if not args.no_clocks else None
    ms_step = ms / args.steps
    value = job_value(world, P, N, ms_step)

    # traced pass: per-kernel device time of the same steps
    pd.pd_prof_enable(True)
    for s in range(args.steps):
        flush.fill_(s & 0xFF)
        step()
    torch.cuda.synchronize()
    prof = pd.pd_prof_read()
    pd.pd_prof_enable(False)
    launches = sum(c for c, _ in prof.values()) // args.steps

    # end to end through the public API from pinned host buffers
    h_lab = torch.from_numpy(lab_np).pin_memory()
    h_th = torch.from_numpy(th_np).pin_memory()
    h_obj = torch.empty((), dtype=torch.float64).pin_memory()
    h_grad = torch.empty((N, K), dtype=torch.float64).pin_memory()
    d_lab = torch.empty_like(lab)
    d_th = torch.empty_like(th)
    e2e_steps = max(5, args.steps // 4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        d_lab.copy_(h_lab, non_blocking=True)
        d_th.copy_(h_th, non_blocking=True)
        o, g = pd.pd_objective_grad(grid, d_lab, N, d_th, DEG, EPS, prec=prec, obj_out=obj, grad_out=grad)
        h_obj.copy_(o, non_blocking=True)
        h_grad.copy_(g, non_blocking=True)
        stream.synchronize()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    assert math.isfinite(float(h_obj.item()))

    extras = {}
    if world == 1 and not args.no_extras:
        # the plain FP32 form (CUDA cores) on the same evaluation
        n_x = max(5, min(args.steps, 50))
        ms32 = time_steps(torch, lambda: pd.pd_objective_grad(grid, lab, N, th, DEG, EPS, prec=pd.PD_FP32,
                                                             obj_out=obj, grad_out=grad), n_x, flush)
        extras["fp32"] = {"ms_per_step": ms32, "value": P * N / (ms32 * 1e-3), "dtype": "f32",
                          "what": "CUDA-core FP32 evaluation (tile-relative logits, float-float centre offsets)"}
        # every pair visited: the pair skipping of the tensor-core passes off
        os.environ["PD_TC_NO_SKIP"] = "1"
        try:
            msd = time_steps(torch, step, n_x, flush)
        finally:
            del os.environ["PD_TC_NO_SKIP"]
        extras["dense"] = {"ms_per_step": msd, "value": P * N / (msd * 1e-3),
                           "what": "the headline evaluation visiting every (tile, grain block) pair"}
        # a parameter taken early in a fit (20 L-BFGS iterations from 0): a
        # diffuse diagram, on which skipping leaves out fewer pairs
        th_e, _ = pd.pd_fit(grid, lab, N, DEG, EPS, max_iter=20, prec=prec)
        mse = time_steps(torch, lambda: pd.pd_objective_grad(grid, lab, N, th_e, DEG, EPS, prec=prec,
                                                            obj_out=obj, grad_out=grad), n_x, flush)
        extras["early_theta"] = {"ms_per_step": mse, "value": P * N / (mse * 1e-3),
                                 "what": "the headline evaluation at theta after 20 L-BFGS iterations from 0"}
        # accuracy of the headline precision and of FP32 against FP64 on the
        # same inputs (objective relative; gradient in 2-norm relative)
        o64, g64 = pd.pd_objective_grad(grid, lab, N, th, DEG, EPS, prec=pd.PD_FP64)
        acc = {}
        for nm in sorted({args.prec, "fp32"} - {"fp64"}):
            o_, g_ = pd.pd_objective_grad(grid, lab, N, th, DEG, EPS, prec=pd.PREC[nm])
            acc[nm] = {"phi_rel": abs(o_.item() - o64.item()) / abs(o64.item()),
                       "grad_rel": float(torch.linalg.norm(g_ - g64) / torch.linalg.norm(g64))}
        extras["accuracy_vs_fp64"] = acc
        # the arg-min assignment with the mismatch count (Err^G), fast path
        # (fp32 with a certified margin) and the double-precision kernel
        mis = torch.empty((), dtype=torch.int64, device="cuda")
        lab_out = torch.empty_like(lab)

        def assign():
            pd.pd_assign(grid, N, DEG, th, ref_labels=lab, out=lab_out, mismatch_out=mis)
        msa = time_steps(torch, assign, n_x, flush)
        os.environ["PD_ASSIGN_FP64"] = "1"
        try:
            msa64 = time_steps(torch, assign, max(3, n_x // 10), flush)
        finally:
            del os.environ["PD_ASSIGN_FP64"]
        extras["assign"] = {"ms": msa, "ms_fp64_kernel": msa64, "err": int(mis.item()) / P,
                            "what": "arg-min assignment and Err^G at the generating parameters"}
        if not args.no_fit:
            extras["time_to_fit"] = time_to_fit(pd, grid, lab, N)
    if rank != 0:
        return 0
    pk = peaks()
    # measured unit throughputs (the library's own microbenchmarks)
    units = {"ffma_per_s": pd.pd_microbench(0), "ex2_per_s": pd.pd_microbench(1),
             "dfma_per_s": pd.pd_microbench(2)}
    # dominant kernel and its roofline
    top = max(prof.items(), key=lambda kv: kv[1][1])
    name, (cnt, tot_ms) = top
    avg_s = tot_ms / cnt * 1e-3
    traffic = ncu_traffic()
    if args.prec in ("fp32", "fp64"):
        # CUDA-core passes: bound by FMA issue; algorithmic work of either
        # pass is one K-long contraction, 2K flop per pixel-grain pair
        algo = P * N * 2 * K
        peak = 2 * (units["ffma_per_s"] if args.prec == "fp32" else units["dfma_per_s"]) / 1e12
        achieved = algo / avg_s / 1e12
        roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic.get(name, (None, None))[0],
                "traffic_source": traffic.get(name, (None, None))[1],
                "peak_source": "measured %s FMA throughput x 2 flop (pd_microbench)" % args.prec.upper()}
    else:
        # tensor-core passes: the contractions run on tcgen05; each pass
        # must evaluate one soft-assignment exponential per pixel-grain pair
        # on the MUFU, which binds
        algo = P * N
        peak = units["ex2_per_s"] / 1e12
        achieved = algo / avg_s / 1e12
        roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tex2/s",
                "frac": achieved / peak, "traffic": traffic.get(name, (None, None))[0],
                "traffic_source": traffic.get(name, (None, None))[1],
                "peak_source": "measured MUFU ex2 throughput (pd_microbench)"}
    # the whole evaluation against its binding unit: one exponential per
    # pixel-grain pair is the method's algorithmic minimum (the logits and
    # gradient contractions need 4K flop per pair, far below the tensor or
    # FMA peaks), so the step is measured in exponentials per second
    step_ex2 = P * N / (ms_step * 1e-3) / 1e12
    roof["step"] = {"achieved": step_ex2, "peak": units["ex2_per_s"] / 1e12, "unit": "Tex2/s",
                    "frac": step_ex2 / (units["ex2_per_s"] / 1e12),
                    "basis": "one ex2 per pixel-grain pair per evaluation over ms_per_step"}
    cpu = cpu_oracle_rate(args.cpu_seconds) if world == 1 or rank == 0 else None
    line = {
        "metric": "pixel*grain objective+gradient evaluations per second",
        "value": value, "unit": "pixel*grain/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3"}[args.prec],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "pixels": P, "grains": N, "K": K, "eps": EPS,
                   "l2": "flushed between steps (256 MiB write, untimed)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "clocks": clocks,
        "e2e": {"value": world * P * N / (e2e_ms * 1e-3), "unit": "pixel*grain/s",
                "h2d_bytes_per_step": 4 * P + 8 * N * K, "d2h_bytes_per_step": 8 + 8 * N * K},
        "gpu_launches": launches * args.steps,
        "kernels_per_step": {k: {"launches": c // args.steps, "ms": t / args.steps} for k, (c, t) in prof.items()},
        "roofline": roof,
        "unit_peaks": units,
        "cpu_baseline": cpu,
    }
    line.update(extras)
    for k in ("fp32", "dense", "early_theta"):
        if k in line:
            line[k]["frac_of_ex2_peak"] = P * N / (line[k]["ms_per_step"] * 1e-3) / units["ex2_per_s"]
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """256 2-D maps, sides and grain counts uniform in [128, 1024] and
    [20, 2000], seeded degree-3 polynomial diagrams fitted at degree 3 (K=10),
    eps = 1e-3: one sweep = the objective and gradient of every map, as one
    batch (a captured CUDA graph) against one call per map, in BF16X3 on the
    tensor cores (the headline) and FP32 on the CUDA cores."""
    import torch

    from paper_2605_20816_gb300 import pd
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    d, eps, n_maps = 3, 1e-3, 256
    shapes = synth.batched_shapes(synth.SEED_BASE + 3, n_maps)
    maps = []
    work = 0
    for q, (n1, n2, N0) in enumerate(shapes):
        K = pd.pd_K(2, d)
        y, z = synth.poly_params(synth.SEED_BASE + 1000 + q, N0, 2, K)
        th = pd.pd_theta_from_apd(2, d, y, np.zeros(N0)).numpy()
        th[:, 3:] = z[:, 3:]
        grid = pd.Grid((n1, n2))
        lab, _, _ = pd.pd_assign(grid, N0, d, torch.from_numpy(th).cuda())
        lab, n, used = synth.compact(lab.cpu().numpy())
        tt = torch.from_numpy(np.ascontiguousarray(th[used])).cuda()
        maps.append((grid, torch.from_numpy(lab.astype(np.int32)).cuda(), n, tt,
                     torch.empty((), dtype=torch.float64, device="cuda"), torch.empty_like(tt)))
        work += grid.P * n
    stream = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 30))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    rows = {}
    for name in ("bf16x3", "fp32"):
        prec = pd.PREC[name]
        t0 = time.perf_counter()
        batch = pd.Batch(maps, d, eps, prec=prec, autotune=True)
        t_plan = time.perf_counter() - t0
        ms_batch = timed(batch.eval, max(3, args.warmup))
        phis = [m[4].item() for m in maps]

        def loop():
            for grid, lab, n, tt, obj, grad in maps:
                pd.pd_objective_grad(grid, lab, n, tt, d, eps, prec=prec, obj_out=obj, grad_out=grad)
        ms_loop = timed(loop, 2)
        same = all(m[4].item() == ph for m, ph in zip(maps, phis))
        rows[name] = {"ms_per_sweep": ms_batch, "value": work / (ms_batch * 1e-3),
                      "per_map_launches": {"ms_per_sweep": ms_loop, "value": work / (ms_loop * 1e-3)},
                      "speedup_vs_per_map": ms_loop / ms_batch, "autotune": batch.info(), "plan_seconds": t_plan,
                      "objectives_equal_per_map_calls": same}
        batch.close()
    head = rows["bf16x3"]
    line = {"metric": "pixel*grain objective+gradient evaluations per second (batched maps)",
            "value": head["value"], "unit": "pixel*grain/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_sweep"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
            "config": {"workload": "256 2-D maps, sides U[128,1024], N U[20,2000], degree-3 diagrams, fit degree 3 "
                                   "(K=10), eps=1e-3", "pixel_grain_per_sweep": work,
                       "maps": n_maps},
            "runs": rows}
    print(json.dumps(line))
    return 0


def run_fit(args):
    """Time to reach the FP64 plain fit's objective (<= 1e-8 relative).

    Config 2 (1024^2, N = 485, degree 4): the plain FP32 form against the
    tensor-core forms (BF16X3 first phase, plain, eps-annealed, and from the
    learned warm start), each followed by FP64 refinement.  Config 5 (512^2, N = 300,
    degree 4, a few seeded maps): the same per map, and the batched,
    warm-started BF16X3 + FP64 form fitting all maps at once against the
    plain FP32 form fitting them one by one.  A first phase may run up to
    3000 iterations and leaves early when its relative gain per iteration
    drops below 1e-7; a target met in it must hold in FP64.  The network is
    trained here on --train-maps seeded 256^2 degree-4 maps (N uniform in
    [50, 400]); data generation and training are timed but not counted."""
    import torch

    from paper_2605_20816_gb300 import pd, warmstart
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))

    def fit(grid, lab, N, prec, target, theta0=None, anneal=False):
        init = pd.PD_INIT_ZERO if theta0 is None else pd.PD_INIT_GIVEN
        t = time.perf_counter()
        _, rep = pd.pd_fit(grid, lab, N, DEG, EPS, theta=theta0, init=init, max_iter=3000, prec=prec,
                           refine_iter=1000, target_phi=target, switch_rtol=1e-7, **(ANNEAL if anneal else {}))
        return {"seconds": time.perf_counter() - t, "iters": rep["iters"], "iters_phase1": rep["iters_phase1"],
                "evals": rep["evals"], "phi": rep["phi"], "reached": rep["phi"] >= target}

    def reference(grid, lab, N):
        t = time.perf_counter()
        _, ref = pd.pd_fit(grid, lab, N, DEG, EPS, max_iter=1000, prec=pd.PD_FP64)
        return ref, time.perf_counter() - t

    # the learned warm start
    t = time.perf_counter()
    X, T = warmstart.dataset(args.train_maps, seed0=5_000_000, side=256, grains=(50, 400))
    t_data = time.perf_counter() - t
    t = time.perf_counter()
    net = pd.MLP(135, 256, 256, 15, seed=1)
    losses = warmstart.train(net, X, T, epochs=40, batch=4096, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t

    def warm(grid, lab, N):
        t = time.perf_counter()
        th0, _ = pd.pd_warm_start(net, grid, lab, N, DEG, EPS, prec=pd.PD_BF16X3)
        torch.cuda.synchronize()
        return th0, time.perf_counter() - t

    # config 2
    grid, lab_np, N, _ = make_workload_gpu(pd, torch)
    lab = torch.from_numpy(lab_np).cuda()
    warm_up_fits(pd, grid, lab, N)
    ref, t_ref = reference(grid, lab, N)
    target = ref["phi"] - 1e-8 * abs(ref["phi"])
    rows = {"fp64_plain": {"seconds": t_ref, "iters": ref["iters"], "evals": ref["evals"], "phi": ref["phi"]},
            "fp32_then_fp64": fit(grid, lab, N, pd.PD_FP32, target),
            "bf16x3_then_fp64": fit(grid, lab, N, pd.PD_BF16X3, target),
            "anneal_bf16x3_then_fp64": fit(grid, lab, N, pd.PD_BF16X3, target, anneal=True)}
    th0, t_pred = warm(grid, lab, N)
    rows["warm_bf16x3_then_fp64"] = fit(grid, lab, N, pd.PD_BF16X3, target, th0)
    rows["warm_bf16x3_then_fp64"]["seconds"] += t_pred
    best = min(("bf16x3_then_fp64", "anneal_bf16x3_then_fp64", "warm_bf16x3_then_fp64"),
               key=lambda k: rows[k]["seconds"] if rows[k]["reached"] else float("inf"))

    # config 5: per map, then batched
    maps5, targets5, per_map = [], [], []
    for q in range(args.fit_maps):
        g5, l5, n5, _ = warmstart.diagram(6_000_000 + q, (512, 512), 300, DEG)
        r5, t_r5 = reference(g5, l5, n5)
        tg = r5["phi"] - 1e-8 * abs(r5["phi"])
        row = {"grains": n5, "fp64_plain_seconds": t_r5, "phi_ref": r5["phi"],
               "fp32_then_fp64": fit(g5, l5, n5, pd.PD_FP32, tg),
               "bf16x3_then_fp64": fit(g5, l5, n5, pd.PD_BF16X3, tg),
               "anneal_bf16x3_then_fp64": fit(g5, l5, n5, pd.PD_BF16X3, tg, anneal=True)}
        w0, t_w = warm(g5, l5, n5)
        row["warm_bf16x3_then_fp64"] = fit(g5, l5, n5, pd.PD_BF16X3, tg, w0)
        row["warm_bf16x3_then_fp64"]["seconds"] += t_w
        per_map.append(row)
        maps5.append((g5, l5, n5))
        targets5.append(tg)
    plain_total = sum(r["fp32_then_fp64"]["seconds"] for r in per_map)
    batched = {"plain_fp32_then_fp64_seconds": plain_total}
    for name, use_warm, anneal in (("cold", False, False), ("warm", True, False), ("anneal", False, True)):
        t = time.perf_counter()
        if use_warm:
            thetas = [warm(g5, l5, n5)[0] for g5, l5, n5 in maps5]
        else:
            thetas = [torch.zeros((n5, pd.pd_K(2, DEG)), dtype=torch.float64, device="cuda") for _, _, n5 in maps5]
        reps = pd.pd_fit_batched(maps5, thetas, DEG, EPS, init=pd.PD_INIT_GIVEN, max_iter=3000, prec=pd.PD_BF16X3,
                                 refine_iter=1000, switch_rtol=1e-7, targets=targets5,
                                 **(ANNEAL if anneal else {}))
        t_b = time.perf_counter() - t
        batched[name] = {"seconds": t_b, "reached": all(r["phi"] >= tg for r, tg in zip(reps, targets5)),
                         "iters": [r["iters"] for r in reps], "multiple_vs_plain_fp32": plain_total / t_b}
    net.close()
    line = {"metric": "time to the FP64 plain-fit objective (<=1e-8 relative)", "value": rows[best]["seconds"],
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "schedule": best,
            "speedup_vs_fp32_then_fp64": rows["fp32_then_fp64"]["seconds"] / rows[best]["seconds"],
            "config": {"workload": WORKLOAD, "reference": "FP64 plain fit, 1000 L-BFGS iterations from theta=0",
                       "phi_ref": ref["phi"]},
            "warm_start": {"train_maps": args.train_maps, "train_grains": int(X.shape[0]),
                           "data_seconds": t_data, "train_seconds": t_train, "epochs": 40,
                           "loss_first": losses[0], "loss_last": losses[-1]},
            "runs": rows,
            "config5": {"workload": "512^2, N = 300 requested, degree-4 diagrams, eps = 1e-3, %d maps" % args.fit_maps,
                        "per_map": per_map,
                        "batched_bf16x3_then_fp64": batched}}
    print(json.dumps(line))
    return 0


def run_config3(args):
    """The 3-D workload: 256^3 voxels, N = 2000 grains requested from a seeded
    anisotropic power diagram (compacted to the non-empty grains), fit degree
    2 (K = 10) and 3 (K = 20), eps = 1e-3: device time of one objective+
    gradient evaluation per precision (L2 flushed between steps), and the
    relative difference of the reduced-precision objectives from FP64."""
    import torch

    from paper_2605_20816_gb300 import pd
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    shape, n0, eps = (256, 256, 256), 2000, 1e-3
    y, w, A = synth.apd_params(synth.SEED_BASE + 2, n0, dim=3)
    th2 = pd.pd_theta_from_apd(3, 2, y, w, A).cuda()
    grid = pd.Grid(shape)
    lab, _, _ = pd.pd_assign(grid, n0, 2, th2)
    lab_np, N, used = synth.compact(lab.cpu().numpy())
    lab = torch.from_numpy(lab_np.astype(np.int32)).cuda()
    th2 = th2[torch.from_numpy(used).cuda()].contiguous()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    P = grid.P
    rows = {}
    for d in (2, 3):
        K = pd.pd_K(3, d)
        th = torch.zeros((N, K), dtype=torch.float64, device="cuda")
        th[:, :10] = th2
        phi64 = pd.pd_objective_grad(grid, lab, N, th, d, eps, prec=pd.PD_FP64, want_grad=False)[0].item()
        for name in ("fp32", "bf16x3"):
            prec = pd.PREC[name]
            try:
                pd.pd_objective_grad(grid, lab, N, th, d, eps, prec=prec)
            except pd.PdError as e:
                rows["d%d_%s" % (d, name)] = {"unsupported": str(e)}
                continue
            steps = max(3, min(args.steps, 10))
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            stream = torch.cuda.current_stream()
            obj = None
            for q in range(steps):
                flush.fill_(q & 0xFF)
                ev[q][0].record(stream)
                obj, _ = pd.pd_objective_grad(grid, lab, N, th, d, eps, prec=prec)
                ev[q][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev) / steps
            row = {"ms_per_eval": ms, "pixel_grain_per_s": P * N / (ms * 1e-3),
                   "phi_rel_vs_fp64": abs(obj.item() - phi64) / abs(phi64)}
            if d == 2:
                # one Hessian-vector product (the inner step of Newton-CG)
                v = torch.from_numpy(synth.random_theta(synth.SEED_BASE + 50, N, K, 1.0)).cuda()
                pd.pd_hvp(grid, lab, N, th, v, d, eps, prec=prec)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(3):
                    pd.pd_hvp(grid, lab, N, th, v, d, eps, prec=prec)
                e1.record(stream)
                torch.cuda.synchronize()
                row["hvp_ms"] = e0.elapsed_time(e1) / 3
            rows["d%d_%s" % (d, name)] = row
    # Newton-CG fits at d = 2, every inner step a Hessian-vector product of
    # eq. (hess), from theta = 0 (at eps = 1e-3 the moment heuristic of Sec.
    # 5.5.2 starts in a saturated soft assignment, Phi about -64, from which
    # Newton-CG barely moves: the oracle shows the same on a 32^3 map), for a
    # fixed budget of Newton iterations; the map is separable, so Phi has no
    # finite maximiser and the budget, not a tolerance, ends the fit.  The
    # report's Phi and Err^G are taken in double precision.
    fits = {}
    for name in ("bf16x3", "fp32"):
        t = time.perf_counter()
        _, rep = pd.pd_fit(grid, lab, N, 2, eps, init=pd.PD_INIT_ZERO, method=pd.PD_METHOD_NEWTON_CG,
                           max_iter=args.newton_iters, max_cg=25, prec=pd.PREC[name])
        fits[name] = {"seconds": time.perf_counter() - t, "iters": rep["iters"], "evals": rep["evals"],
                      "hvps": rep["hvps"], "phi": rep["phi"], "err": rep["err"], "status": rep["status"]}
    fits["speedup_bf16x3_vs_fp32"] = fits["fp32"]["seconds"] / fits["bf16x3"]["seconds"]
    line = {"metric": "pixel*grain objective+gradient evaluations per second (3-D)", "unit": "pixel*grain/s",
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "3D 256^3 voxels, N=2000 requested (anisotropic power diagram), eps=1e-3",
                       "voxels": P, "grains": N, "l2": "flushed between steps"},
            "runs": rows,
            "newton_cg_fit_d2": {"budget": "%d Newton iterations, at most 25 CG steps each" % args.newton_iters,
                                 "init": "theta = 0", "runs": fits}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "fit":
        return run_fit(args)
    if args.workload == "config3":
        return run_config3(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Throughput of isolated-system Poisson solves on GB300.

One step = one whole solve (x forward, y forward, z forward x Green's
spectrum x z inverse, y inverse, x inverse) of the 256^3 multi-sphere
workload (doubled mesh 512^3, h = 1/256, 8 seeded homogeneous spheres plus a
Gaussian blob) in FP32, inputs resident in HBM.  Four source/potential pairs
(512 MB, more than the 129 MB L2) rotate between steps.  Also measured:
the same solve in FP64, the end-to-end rate through ipf_solve_host (host
buffers, copies inside the timed region), mean per-pass device times and
the roofline of the dominant pass.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --impl reference the FP64 CPU oracle is timed instead (host cores,
Green's spectrum built once outside the timed steps, as the paper's
Create/Solve split does).  Multi-GPU runs are independent replicas: each
rank solves its own stream of workloads; no collective is on the data path.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_BENCH = 256
METRIC = "isolated solves/s & HBM GB/s at 256^3 (FP32 vs FP64); serving p50/p99 ms"
WORKLOAD = "multisphere-256: 256^3 cells (doubled mesh 512^3), h=1/256, 8 spheres + Gaussian, seed 0"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="isofft", choices=["isofft", "reference"])
    ap.add_argument("--cells", type=int, default=N_BENCH, help="cells per axis of the workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--no-paper-scale", action="store_true",
                    help="skip the 1152^3 solve (the paper's largest ladder point)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# algorithmic bytes (what each pass must move at least once)
# ---------------------------------------------------------------------------
def pass_bytes(N, M, es):
    """Per-pass algorithmic HBM bytes of one solve; es = bytes per real."""
    Nx, Ny, Nz = N
    Mx, My, Mz = M
    K = Mx // 2
    c = 2 * es
    src = es * Nx * Ny * Nz
    wy = c * K * Ny * Nz            # x spectra of the active rows
    wall = c * K * My * Nz          # after the y pass
    g = es * (My // 2 + 1) * (Mz // 2 + 1) * (K + 1)
    return {
        "x_forward": src + wy,
        "y_forward": wy + wall,
        "z_convolve": 2 * wall + g,
        "y_inverse": wall + wy,
        "x_inverse": wy + src,
    }


PASSES = ["x_forward", "y_forward", "z_convolve", "y_inverse", "x_inverse"]
KERNELS = {"x_forward": "k_x_forward", "y_forward": "k_y_forward", "z_convolve": "k_z_convolve",
           "y_inverse": "k_y_inverse", "x_inverse": "k_x_inverse"}


def kernel_times(passes, nbytes):
    """Mean device ms, algorithmic bytes and GB/s per kernel."""
    out = {}
    for name, ms, b in [(KERNELS[p], passes[i], nbytes[p]) for i, p in enumerate(PASSES)]:
        out[name] = {"ms": ms, "bytes": b, "gbs": b / (ms / 1e3) / 1e9 if ms > 0 else 0.0}
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic(kernel, tag):
    """DRAM bytes per launch from the committed ncu summary of `kernel` on
    this workload, if the kernel sources are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, tag))
    if not os.path.exists(path):
        return None
    want = sources_digest()
    traffic, digest = None, None
    for line in open(path):
        if line.startswith("traffic_bytes_per_launch:"):
            traffic = float(line.split(":", 1)[1])
        if line.startswith("sources_sha256:"):
            digest = line.split(":", 1)[1].strip()
    return traffic if digest == want else None


# the sources that define the pass kernels (a change to any of them makes a
# committed ncu summary stale)
KERNEL_SOURCES = ("df64.cuh", "fft_engine.cuh", "launch.h", "passes.cuh", "passes_inst.cu", "tma.cuh")


def sources_digest():
    """Digest of the kernel sources' code (comments and blank lines left
    out, so that a comment edit does not make a capture stale)."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1106_0557_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        t = open(os.path.join(csrc, fn)).read()
        t = re.sub(r"/\*.*?\*/", "", t, flags=re.S)
        t = re.sub(r"//[^\n]*", "", t)
        h.update("\n".join(line.rstrip() for line in t.splitlines() if line.strip()).encode())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id is not None:
            cmd.insert(1, "--id=%s" % self.gpu_id)
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed helpers (replicas only: a barrier and a max of times)
# ---------------------------------------------------------------------------
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "isofft" else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(value, ws, device=None):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, ws, device=None):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline field)
# ---------------------------------------------------------------------------
def time_oracle(n, steps, budget_s, warmup=0, keep=False):
    """Times full oracle solves of the workload.  With `keep`, also returns
    the oracle's potentials of the workload's FP64 source and of that source
    rounded to FP32 (the exact input of the FP32 GPU solve), the references
    of the GPU results' error statement."""
    import oracle
    from paper_1106_0557_gb300 import sources
    w = sources.multi_sphere(n, seed=0)
    src = w.source()
    M = oracle.doubled_mesh(w.N)
    Gt = oracle.green_spectrum(M, w.h)
    for _ in range(warmup):
        oracle.solve_with_spectrum(src, M, Gt)
    times = []
    phi = None
    t_start = time.perf_counter()
    for _ in range(steps):
        t0 = time.perf_counter()
        phi = oracle.solve_with_spectrum(src, M, Gt)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s:
            break
    if not keep:
        return len(times), sum(times), oracle.num_threads()
    refs = {"f64": phi, "f32": oracle.solve_with_spectrum(src.astype(np.float32).astype(np.float64), M, Gt)}
    return len(times), sum(times), oracle.num_threads(), refs


def potential_errors(potentials, refs):
    """Normwise max|phi - ref| / max|ref|, pointwise max |phi - ref| / |ref|
    (well defined: the potential of a non-negative source is negative
    everywhere) and the L1 norm of Eq. 11, sum |phi - ref| / sum |ref|, of
    each dtype's GPU potential against the FP64 oracle on the same input;
    FP64 and df64 solve the FP64 source, FP32 its FP32 rounding."""
    tol = {"f32": 1e-5, "f64": 1e-12, "df64": 1e-12}
    out = {}
    for dt, phi in potentials.items():
        ref = refs["f32" if dt == "f32" else "f64"]
        d = np.abs(phi - ref)
        out[dt] = {"normwise": float(d.max() / np.abs(ref).max()), "pointwise": float((d / np.abs(ref)).max()),
                   "l1": float(d.sum() / np.abs(ref).sum()), "tol": tol[dt], "cells": int(ref.size),
                   "ref": "full-grid FP64 oracle solve"}
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    n = args.cells
    # one untimed solve stands for the warm-up (a full oracle solve takes
    # seconds); the timed solves stop after 150 s of CPU work
    warm = 1 if args.warmup > 0 else 0
    done, secs, cores = time_oracle(n, max(1, args.steps), budget_s=150.0, warmup=warm)
    value = done / secs
    sample = ("%d full %d^3 FP64 oracle solve(s) (doubled mesh %d^3, recursive FFT) after %d untimed, Green's "
              "spectrum built before timing; capped at 150 s of CPU work" % (done, n, 2 * n, warm))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": done, "warmup": warm, "ms_per_step": 1e3 * secs / done, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": [n, n, n], "M": [2 * n] * 3},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the paper's largest mesh
# ---------------------------------------------------------------------------
def run_paper_scale(steps=20, warmup=3):
    """The Sec. 4.2 spheroid at 1152^3 cells (doubled mesh 2304^3), FP32,
    in place: the mesh of the paper's largest weak-scaling run (~1 s per
    solve on 13 824 Opteron cores).  Set-up (the Green's spectrum) is
    excluded, as the paper computes it once at initialisation."""
    import torch

    from paper_1106_0557_gb300 import Plan, native, sources
    w = sources.paper_spheroid(1152)
    t0 = time.perf_counter()
    plan = Plan(w.N, w.h, "f32", flags=native.IPF_FLAG_PASS_EVENTS)
    setup_s = time.perf_counter() - t0
    src = sources.rasterize_torch(w.bodies, w.N, w.h, w.lo, dtype=torch.float32)
    for _ in range(warmup):
        plan.solve(src, src)
    torch.cuda.synchronize()
    plan.pass_times()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.solve(src, src)
    e1.record()
    torch.cuda.synchronize()
    plan.check()
    ms = e0.elapsed_time(e1) / steps
    passes = plan.pass_times()
    pb = pass_bytes(w.N, plan.padded_shape, 4)
    nbytes = sum(pb[k] for k in PASSES)
    plan.close()
    del src
    torch.cuda.empty_cache()
    native.ipf_greens_cache_trim(0)
    return {"workload": "Sec. 4.2 spheroid (e=0.9, a=0.5) in [-1,1]^3, 1152^3 cells, doubled mesh 2304^3, FP32, "
                        "in place", "ms_per_solve": round(ms, 3), "steps": steps,
            "hbm_gbs_algorithmic": round(nbytes / (ms / 1e3) / 1e9, 1),
            "kernels": {KERNELS[k]: {"ms": round(t, 3), "gbs": round(pb[k] / (t / 1e3) / 1e9, 1)}
                        for k, t in zip(PASSES, passes)},
            "setup_s": round(setup_s, 2),
            "paper": "about 1 s per solve on ~13 000 Opteron cores (Cray XT-4), same mesh"}


# ---------------------------------------------------------------------------
# batched and served solves
# ---------------------------------------------------------------------------
def run_batch(steps=50, count=64):
    """64 independent grids (each axis from {32,48,64,96,128}), FP32, as one
    batch captured in a CUDA graph and replayed; also the same batch
    submitted without a graph."""
    import torch

    from paper_1106_0557_gb300 import native, sources
    from paper_1106_0557_gb300.solver import BatchGraph, Plan, submit_batch
    wl = sources.ragged_batch(count)
    plans = [Plan(w.N, w.h, "f32") for w in wl]
    srcs = [torch.from_numpy(w.source(np.float32)).cuda() for w in wl]
    outs = [torch.empty_like(x) for x in srcs]
    nbytes = 0
    for p, w in zip(plans, wl):
        b = pass_bytes(w.N, p.padded_shape, 4)
        nbytes += sum(b[k] for k in PASSES)
    res = {"grids": count, "workload": "ragged batch, each axis from {32,48,64,96,128}, seed = grid index",
           "how": {"graph": "per-grid passes on 8 library streams, captured in a CUDA graph",
                   "submit": "the same without the graph",
                   "fused": "one launch per pass over a table of every grid's work items (ISOFFT_BATCH_FUSED=1)",
                   "one": "one persistent launch for all five passes, per-(grid, pass) completion counters "
                          "(ISOFFT_BATCH_FUSED=2)"}}
    for mode in ("graph", "submit", "fused", "one"):
        os.environ["ISOFFT_BATCH_FUSED"] = {"fused": "1", "one": "2"}.get(mode, "0")
        if mode == "graph":
            bg = BatchGraph(plans, srcs, outs)
            run = bg.replay
        else:
            def run():
                submit_batch(plans, srcs, outs)
        for _ in range(3):
            run()
        torch.cuda.synchronize()
        l0 = native.ipf_launch_count()
        run()
        torch.cuda.synchronize()
        launches = native.ipf_launch_count() - l0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[mode] = {"ms_per_batch": round(ms, 4), "solves_per_s": round(count / (ms / 1e3), 1),
                     "hbm_gbs_algorithmic": round(nbytes / (ms / 1e3) / 1e9, 1),
                     "launches_per_batch": None if mode == "graph" else launches}
    os.environ.pop("ISOFFT_BATCH_FUSED", None)
    for p in plans:
        p.close()
    return res


def run_serving(n_requests, slots, fp64_class="df64", express_slots=2, plan_workers=4):
    """Config 5: cubic N log-uniform in [32, 384], 70 % FP32 (tolerance
    1e-5) / 30 % FP64 class (tolerance 1e-12, served with the `fp64_class`
    dtype), HBM budget 120 GB, continuous batching over `slots` streams with
    plans created on the server's background thread.
    * Saturated throughput: all requests at t = 0, warm (after one pass).
    * Poisson arrivals at 0.5, 0.8 and 0.95 x that rate (0.8 headlined), each
      load point from a cold start: a fresh server and an empty spectrum
      cache, so every shape's first request waits for its plan and Green's
      spectrum to be built (their latency counts).  Two admission policies:
      first come first served on every slot ("fcfs"), and `express_slots`
      slots, on high-priority streams, kept for requests no costlier than
      an FP32 128^3 solve ("express", the headline).  Plans are built by
      `plan_workers` background threads.
    * The FP32 class served vs the same shapes solved one at a time in plain
      FP64 (plan set-up excluded)."""
    import torch

    from paper_1106_0557_gb300 import native, serving, sources
    spec = sources.serving_requests(count=n_requests, seed=0)
    cls = lambda d: fp64_class if d == "f64" else d
    mk = lambda arr: [serving.Request(r["id"], r["n"], cls(r["dtype"]), r["seed"], a) for r, a in zip(spec, arr)]
    be = serving.TorchBackend(slots=slots)
    reqs = mk(np.zeros(len(spec)))
    be.prepare(reqs)
    srv = serving.Server(be, budget_bytes=120e9, slots=slots, async_plans=True, plan_workers=plan_workers)
    serving.saturated_throughput(srv, be, reqs)  # warm-up pass: plans and spectra
    sat = serving.saturated_throughput(srv, be, reqs)
    peak = srv.peak_bytes
    srv.close()
    policies = {"fcfs": 0, "express": express_slots}
    sweeps = {}
    for pol, nexp in policies.items():
        sweep = []
        be.set_express(nexp)
        for load in (0.5, 0.8, 0.95):
            r = load * sat["solves_per_s"]
            native.ipf_greens_cache_trim(0)
            srv = serving.Server(be, budget_bytes=120e9, slots=slots, async_plans=True, express_slots=nexp,
                                 plan_workers=plan_workers)
            rq = mk(serving.poisson_arrivals(len(spec), r, seed=1))
            srv.run(rq)
            peak = max(peak, srv.peak_bytes)
            st = serving.latency_stats(rq)
            cheap = serving.Server(be, slots=slots, express_slots=1).small
            st_s = serving.latency_stats([q for q in rq if cheap(q)])
            st_l = serving.latency_stats([q for q in rq if not cheap(q)])
            srv.close()
            # requests that found no plan of their shape: the first of each shape
            seen, first = set(), []
            for q in sorted(rq, key=lambda q: q.arrival):
                if (q.n, q.dtype) not in seen:
                    seen.add((q.n, q.dtype))
                    first.append(q.latency)
            sweep.append({"load": load, "rate": round(r, 1), "p50_ms": round(st["p50_ms"], 3),
                          "p99_ms": round(st["p99_ms"], 3), "solves_per_s": round(st["solves_per_s"], 1),
                          "small_p50_p99_ms": [round(st_s["p50_ms"], 3), round(st_s["p99_ms"], 3)],
                          "large_p50_p99_ms": [round(st_l["p50_ms"], 3), round(st_l["p99_ms"], 3)],
                          "cold_shapes": len(first), "cold_p50_ms": round(float(np.percentile(first, 50)) * 1e3, 3)})
            if load == 0.8 and pol == "express":
                rate, lat = r, st
        sweeps[pol] = sweep
    be.set_express(0)
    # FP32 class served (saturated, warm) vs plain unbatched FP64 on the same shapes
    sub = [q for q in reqs if q.dtype == "f32"][:300]
    srv = serving.Server(be, budget_bytes=120e9, slots=slots, async_plans=True, plan_workers=plan_workers)
    serving.saturated_throughput(srv, be, sub)
    served32 = serving.saturated_throughput(srv, be, sub)
    srv.close()
    # plain path: one FP64 solve at a time on one stream, plan set-up excluded
    shapes = [q.n for q in sub]
    plain_s = 0.0
    stream = torch.cuda.current_stream().cuda_stream
    for n in shapes:
        p = native.ipf_plan_create((n,) * 3, (1.0 / n,) * 3, "f64")
        src = be.source(n, "f64")
        out = torch.empty_like(src)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        native.ipf_solve(p, src.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        plain_s += time.perf_counter() - ts
        native.ipf_plan_destroy(p)
    plain64 = len(shapes) / plain_s
    return {"requests": len(spec), "slots": slots, "budget_gb": 120,
            "mix": "cubic N log-uniform [32,384], 70%% f32 / 30%% FP64-class served as %s" % fp64_class,
            "plans": "created on background threads; admission looks ahead past requests whose plan is "
                     "being built",
            "saturated_solves_per_s": round(sat["solves_per_s"], 1),
            "policy": "express: %d of %d slots, on high-priority streams, kept for requests no costlier than "
                      "an FP32 128^3 solve (small = %s); large requests first come first served on the others; "
                      "plans built by %d background threads" % (
                          express_slots, slots, "FP32 N <= 128, df64 N <= 72", plan_workers),
            "poisson_rate": round(rate, 1), "p50_ms": round(lat["p50_ms"], 3), "p99_ms": round(lat["p99_ms"], 3),
            "solves_per_s": round(lat["solves_per_s"], 1),
            "load_sweep": sweeps["express"], "load_sweep_fcfs": sweeps["fcfs"],
            "load_sweep_start": "cold: fresh server, empty spectrum cache",
            "f32_served_solves_per_s": round(served32["solves_per_s"], 1),
            "f64_plain_unbatched_solves_per_s": round(plain64, 1),
            "f32_served_over_f64_plain": round(served32["solves_per_s"] / plain64, 2),
            "peak_bytes": int(peak)}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def host_copy_rates(hsrc, hphi, stream, reps=20):
    """Plain pinned-host <-> device copy rates of one solve's buffers, the
    floor under the end-to-end rate: each direction alone, and both at once
    on two streams."""
    import torch
    d = torch.empty(hsrc.shape, dtype=hsrc.dtype, device="cuda")
    d2 = torch.empty_like(d)
    other = torch.cuda.Stream()
    out = {}
    for name in ("h2d", "d2h", "both"):
        for rep in range(reps + 3):
            if rep == 3:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            if name in ("h2d", "both"):
                with torch.cuda.stream(stream):
                    d.copy_(hsrc, non_blocking=True)
            if name in ("d2h", "both"):
                with torch.cuda.stream(other):
                    hphi.copy_(d2, non_blocking=True)
        torch.cuda.synchronize()
        secs = (time.perf_counter() - t0) / reps
        out["ms_" + name] = round(secs * 1e3, 4)
        out["gbs_" + name] = round(hsrc.numel() * hsrc.element_size() * (2 if name == "both" else 1)
                                   / secs / 1e9, 1)
    return out


def run_isofft(args, ws, rank, local):
    import torch

    from paper_1106_0557_gb300 import native, sources
    from paper_1106_0557_gb300.solver import Plan

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    native.lib()
    n = args.cells
    w = sources.multi_sphere(n, seed=0)
    src64 = w.source()
    N = w.N
    stream = torch.cuda.current_stream()

    forms = {}  # y-pass forms the plans picked
    potentials = {}  # the last timed solve's potential per dtype (host, FP64)

    def timed_solves(dtype, steps, warmup, pool=4):
        tdt = torch.float32 if dtype == "f32" else torch.float64  # df64 reads and writes FP64 arrays
        plan = Plan(N, w.h, dtype, flags=native.IPF_FLAG_PASS_EVENTS)
        forms[dtype] = [("tiles", "streamed", "narrow tiles")[v] for v in plan.variants]
        base = torch.from_numpy(src64).to(dev, tdt)
        srcs = [base.clone() for _ in range(pool)]
        outs = [torch.empty_like(base) for _ in range(pool)]
        for i in range(warmup):
            plan.solve(srcs[i % pool], outs[i % pool])
        torch.cuda.synchronize()
        plan.pass_times()  # reset the accumulated pass means
        barrier(ws)
        torch.cuda.synchronize()
        l0 = native.ipf_launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(steps):
            plan.solve(srcs[i % pool], outs[i % pool])
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        plan.check(stream)  # raises if a bounded device wait gave up
        ms = ev0.elapsed_time(ev1)
        launches = native.ipf_launch_count() - l0
        passes = plan.pass_times()
        M = plan.padded_shape
        phi = outs[(steps - 1) % pool]
        finite = bool(torch.isfinite(phi).all().item())
        potentials[dtype] = phi.double().cpu().numpy()
        plan.close()
        del srcs, outs
        torch.cuda.empty_cache()
        return ms, launches, passes, M, finite

    peak, peak_kind = measured_peaks()
    gpu_uuid = None
    try:
        gpu_uuid = torch.cuda.get_device_properties(local).uuid
        gpu_uuid = "GPU-" + str(gpu_uuid)
    except Exception:
        gpu_uuid = str(local)

    # FP32: the headline
    with ClockSampler(gpu_uuid) as clk:
        ms32, launches, passes32, M, finite32 = timed_solves("f32", args.steps, args.warmup)
    clocks = clk.summary()
    ms32 = reduce_max(ms32, ws, dev)
    total = reduce_sum(args.steps, ws, dev)
    value = total / (ms32 / 1e3)
    bytes32 = pass_bytes(N, M, 4)
    gbs32 = sum(v["bytes"] for v in kernel_times(passes32, bytes32).values()) / (ms32 / args.steps / 1e3) / 1e9

    # FP64 (fewer steps: the FP64 units of this part are a small fraction of FP32)
    steps64 = max(3, args.steps // 10)
    ms64, _, passes64, _, finite64 = timed_solves("f64", steps64, max(3, args.warmup // 4))
    ms64 = reduce_max(ms64, ws, dev)
    value64 = reduce_sum(steps64, ws, dev) / (ms64 / 1e3)
    bytes64 = pass_bytes(N, M, 8)
    gbs64 = sum(v["bytes"] for v in kernel_times(passes64, bytes64).values()) / (ms64 / steps64 / 1e3) / 1e9

    # FP64-class float pairs on the FP32 units (same FP64 buffers)
    stepsdf = max(3, args.steps // 4)
    msdf, _, passesdf, _, finitedf = timed_solves("df64", stepsdf, max(3, args.warmup // 4))
    msdf = reduce_max(msdf, ws, dev)
    valuedf = reduce_sum(stepsdf, ws, dev) / (msdf / 1e3)
    bytesdf = pass_bytes(N, M, 8)
    kdf = kernel_times(passesdf, bytesdf)
    gbsdf = sum(kdf[k]["bytes"] for k in kdf) / (msdf / stepsdf / 1e3) / 1e9

    # end to end through the public host-buffer entry point
    plan = Plan(N, w.h, "f32")
    hsrc = torch.from_numpy(src64.astype(np.float32)).pin_memory()
    hphi = torch.empty_like(hsrc).pin_memory()
    sh = stream.cuda_stream
    for _ in range(3):
        native.ipf_solve_host(plan.handle, hsrc.data_ptr(), hphi.data_ptr(), sh)
    e2e_steps = max(3, min(args.steps, 200))
    # untimed: the asynchronous path warmed the same way as it is timed
    for _ in range(max(3, e2e_steps // 10)):
        native.ipf_solve_host_async(plan.handle, hsrc.data_ptr(), hphi.data_ptr(), sh)
    native.ipf_plan_host_wait(plan.handle)
    # the headline e2e: solves enqueued back to back through the public
    # asynchronous host-buffer call, every one copying its source in and its
    # potential out, one wait at the end
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        native.ipf_solve_host_async(plan.handle, hsrc.data_ptr(), hphi.data_ptr(), sh)
    native.ipf_plan_host_wait(plan.handle)
    t_e2e = time.perf_counter() - t0
    barrier(ws)
    # and one blocking host solve at a time
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        native.ipf_solve_host(plan.handle, hsrc.data_ptr(), hphi.data_ptr(), sh)
    t_block = time.perf_counter() - t0
    barrier(ws)
    plan.close()
    t_e2e = reduce_max(t_e2e, ws, dev)
    e2e_value = reduce_sum(e2e_steps, ws, dev) / t_e2e
    block_value = reduce_sum(e2e_steps, ws, dev) / reduce_max(t_block, ws, dev)
    io_bytes = hsrc.numel() * hsrc.element_size()
    copy_rates = host_copy_rates(hsrc, hphi, stream)

    # roofline of the dominant kernel (the longest mean device time)
    k32 = kernel_times(passes32, bytes32)
    k64 = kernel_times(passes64, bytes64)
    dname = max(k32, key=lambda k: k32[k]["ms"])
    achieved = k32[dname]["bytes"] / (k32[dname]["ms"] / 1e3) / 1e9
    traffic = profile_traffic(dname, "f32_%d" % n)

    batch = None if args.no_batch else run_batch()
    paper_scale = None if args.no_paper_scale else run_paper_scale()
    serve = None if args.no_serve else run_serving(args.serve_requests, args.serve_slots)

    cpu = None
    errors = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        done, secs, cores, refs = time_oracle(n, 1, budget_s=60.0, keep=True)
        cpu = {"value": done / secs, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": "%d full %d^3 FP64 oracle solve (doubled mesh %d^3), Green's spectrum built "
                         "before timing" % (done, n, 2 * n)}
        errors = potential_errors(potentials, refs)

    if rank != 0:
        return
    per_kernel = {}
    for k in k32:
        per_kernel[k] = {"ms_f32": round(k32[k]["ms"], 5), "gbs_f32": round(k32[k]["gbs"], 1),
                         "ms_f64": round(k64[k]["ms"], 5), "gbs_f64": round(k64[k]["gbs"], 1),
                         "algorithmic_bytes_f32": k32[k]["bytes"]}
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": list(N), "M": list(M), "h": w.h[0],
                   "y_pass_forms": forms,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "4 rotating src/phi pairs (%d MB) > 129 MB L2" % (8 * 4 * n ** 3 // 2 ** 20)},
        "hbm_gbs": round(gbs32, 1),
        "fp64": {"value": value64, "unit": "solves/s", "ms_per_step": ms64 / steps64, "steps": steps64,
                 "hbm_gbs": round(gbs64, 1)},
        "df64": {"value": valuedf, "unit": "solves/s", "ms_per_step": msdf / stepsdf, "steps": stepsdf,
                 "hbm_gbs": round(gbsdf, 1), "what": "FP64-class float-pair arithmetic on the FP32 units, "
                 "FP64 buffers, tolerance 1e-12",
                 "kernels": {k: {"ms": round(v["ms"], 5), "gbs": round(v["gbs"], 1)} for k, v in kdf.items()}},
        "kernels": per_kernel,
        "roofline": {"bound": "hbm", "kernel": dname, "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "algorithmic_bytes": k32[dname]["bytes"]},
        "e2e": {"value": e2e_value, "unit": "solves/s", "steps": e2e_steps, "h2d_bytes_per_step": io_bytes,
                "d2h_bytes_per_step": io_bytes, "how": "ipf_solve_host_async back to back, one ipf_plan_host_wait",
                "blocking_solves_per_s": round(block_value, 1), "plain_copies": copy_rates},
        "batch": batch,
        "serving": serve,
        "paper_scale": paper_scale,
        "cpu_baseline": cpu,
        "max_rel_err": errors,
        "gpu_launches": launches,
        "clocks": clocks,
        "finite": finite32 and finite64 and finitedf,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_isofft(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Command line: timed solves of one mesh shape on cuda:0.

    python -m paper_1106_0557_gb300 solve --n NX NY NZ [--h HX HY HZ]
        [--dtype f32|f64|df64] [--repeat K] [--warmup W] [--seed S]

Builds the library if needed, creates a plan (reporting its set-up time:
the Green's spectrum and the y-pass timing), solves a seeded multi-sphere
source (the benchmark's distribution on the given mesh) W + K times, and
prints one JSON line with the mean device time per solve and per pass and
the algorithmic HBM GB/s of each pass.  The solves are in place, so the
device holds the plan's workspace, its spectrum and one source array.
"""
import argparse
import json
import sys
import time


def _pass_bytes(N, M, es):
    Nx, Ny, Nz = N
    K = M[0] // 2
    c = 2 * es
    src = es * Nx * Ny * Nz
    wy = c * K * Ny * Nz
    wall = c * K * M[1] * Nz
    g = es * (M[1] // 2 + 1) * (M[2] // 2 + 1) * (K + 1)
    return [src + wy, wy + wall, 2 * wall + g, wall + wy, wy + src]


def _solve(args):
    import torch

    from . import native, sources
    from .solver import Plan

    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    N = tuple(args.n)
    h = tuple(args.h) if args.h else tuple(1.0 / n for n in N)
    native.lib()
    t0 = time.perf_counter()
    plan = Plan(N, h, args.dtype, flags=native.IPF_FLAG_PASS_EVENTS)
    setup = time.perf_counter() - t0
    bodies = sources.multi_sphere_bodies(sources.rng(args.seed))
    tdt = torch.float32 if args.dtype == "f32" else torch.float64
    src = sources.rasterize_torch(bodies, N, h, dtype=tdt)
    for _ in range(args.warmup):
        plan.solve(src, src)
    torch.cuda.synchronize()
    plan.pass_times()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.repeat):
        plan.solve(src, src)
    e1.record()
    torch.cuda.synchronize()
    plan.check()
    ms = e0.elapsed_time(e1) / max(1, args.repeat)
    passes = plan.pass_times() if args.repeat else [0.0] * 5
    M = plan.padded_shape
    es = 4 if args.dtype == "f32" else 8
    nbytes = _pass_bytes(N, M, es)
    names = ["x_forward", "y_forward", "z_convolve", "y_inverse", "x_inverse"]
    out = {"n": list(N), "m": list(M), "h": list(h), "dtype": args.dtype, "setup_s": round(setup, 4),
           "ms_per_solve": round(ms, 4), "solves": args.repeat,
           "passes": {k: {"ms": round(t, 4), "gbs": round(b / (t / 1e3) / 1e9, 1) if t > 0 else None}
                      for k, t, b in zip(names, passes, nbytes)}}
    plan.close()
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1106_0557_gb300")
    sub = ap.add_subparsers(dest="cmd", required=True)
    sp = sub.add_parser("solve", help="timed solves of one mesh shape")
    sp.add_argument("--n", type=int, nargs=3, required=True, metavar=("NX", "NY", "NZ"))
    sp.add_argument("--h", type=float, nargs=3, metavar=("HX", "HY", "HZ"), help="cell widths (default 1/N)")
    sp.add_argument("--dtype", default="f32", choices=["f32", "f64", "df64"])
    sp.add_argument("--repeat", type=int, default=10)
    sp.add_argument("--warmup", type=int, default=3)
    sp.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    if args.cmd == "solve":
        _solve(args)
    return 0


if __name__ == "__main__":
    sys.exit(main())

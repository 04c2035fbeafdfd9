"""Run single operator applications of a named workload, for profiling.

    python -m paper_2505_22797_gb300.profile_ops --op forward --workload c2 --reps 3

Builds the inputs of the workload (seeded synthetic), runs `--warmup`
untimed applications and then `--reps` applications of the chosen operator
(forward A, adjoint A^T, dbeta, conv, the Core Stage interpolation,
its transpose, a Core Stage solve of --grid-iters CG steps, or one whole
PnP reconstruction) in the chosen precision, timing each
with CUDA events on the current stream, and prints one line per operator.
It is the small, self-contained command to put under a profiler.
"""
from __future__ import annotations

import argparse
import os
import sys

import torch

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2505_22797_gb300 import api, build  # noqa: E402
from paper_2505_22797_gb300 import synthetic as syn  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--op", choices=["forward", "adjoint", "dbeta", "conv", "interp", "interp_T", "grid",
                                     "pnp", "all"], default="all")
    ap.add_argument("--workload", default="c2", help="c1, c2, c2_partial, c4, c5 or 3d")
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--grid-iters", type=int, default=2,
                    help="CG steps of the grid op (a fixed count: rel_tol 0)")
    ap.add_argument("--kernel", action="store_true",
                    help="report the operator kernel alone (library event timing, mean of reps)")
    args = ap.parse_args(argv)

    build.build()
    api.load()
    three = args.workload == "3d"
    cfg = syn.config3("3d") if three else syn.config(args.workload)
    m, g = cfg["model"], cfg["grid"]
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    r = torch.as_tensor(cfg["r"], dtype=dt, device="cuda")
    v = torch.as_tensor(cfg["v"], dtype=dt, device="cuda")
    c = torch.as_tensor(cfg["c"], dtype=dt, device="cuda")
    out = torch.empty_like(c)
    if three:
        s = api.mpi_forward3(m, g, r, v, c)
        field = torch.stack([c * (1.0 - 0.1 * q) for q in range(9)]).contiguous()
        s3 = torch.empty_like(s)
        ops = {
            "forward": lambda: api.mpi_forward3(m, g, r, v, c, s=s),
            "adjoint": lambda: api.mpi_adjoint3(m, g, r, v, s, c_out=out),
            "conv": lambda: api.mpi_conv3(m, g, c, out=out),
            "interp": lambda: api.mpi_interp3(g, r, v, field, s=s3),
            "interp_T": lambda: api.mpi_interp3_adjoint(g, r, v, s, Ahat=field),
            "grid": lambda: api.mpi_grid3(g, r, v, s, gamma=1e-7, max_iter=args.grid_iters, rel_tol=0.0),
        }
    else:
        s = api.mpi_forward(m, g, r, v, c)
        field = torch.stack([c, 0.5 * c, 0.25 * c, c]).contiguous()
        s2 = torch.empty_like(s)
        ops = {
            "forward": lambda: api.mpi_forward(m, g, r, v, c, s=s),
            "adjoint": lambda: api.mpi_adjoint(m, g, r, v, s, c_out=out),
            "dbeta": lambda: api.mpi_dbeta(m, g, r, v, c, s),
            "conv": lambda: api.mpi_conv(m, g, c, out=out),
            "interp": lambda: api.mpi_interp(g, r, v, field, s=s2),
            "interp_T": lambda: api.mpi_interp_adjoint(g, r, v, s, Ahat=field),
            "grid": lambda: api.mpi_grid(g, r, v, s, gamma=1e-7, max_iter=args.grid_iters, rel_tol=0.0),
            # one whole reconstruction of the workload (its PnP iterations and CG
            # steps); nu0 = 1e-3 of the mean diagonal of A^T A from 4 probes
            "pnp": lambda: api.mpi_pnp_solve(m, g, r, v, s, cfg["n_it"], cfg["n_cg"], nu0,
                                             clip_pct=cfg["clip_pct"], rho_out=out),
        }
        gen = torch.Generator(device="cpu").manual_seed(7)
        fro = 0.0
        for _ in range(4):
            z = (torch.randint(0, 2, tuple(c.shape), generator=gen) * 2 - 1).to("cuda", dt)
            fro += float(torch.sum(api.mpi_forward(m, g, r, v, z).double() ** 2)) / 4
        nu0 = 1e-3 * fro / c.numel()
    names = [n for n in ops if n != "pnp"] if args.op == "all" else [args.op]
    pairs = c.numel() * r.shape[0]
    stream = torch.cuda.current_stream()
    for name in names:
        fn = ops[name]
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        # the timed repetitions run inside an NVTX range named after the op,
        # for a profiler's range filter (ncu --nvtx --nvtx-include "<op>/")
        torch.cuda.nvtx.range_push(name)
        for _ in range(args.reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        torch.cuda.nvtx.range_pop()
        best = min(ms)
        apps = 2 * cfg["n_it"] * (cfg["n_cg"] + 1) + 1 if name == "pnp" else 1
        rate = "" if name in ("conv", "interp", "interp_T", "grid") else f"  {apps * pairs / best / 1e6:.1f} Gpair/s"
        line = f"{args.workload} {args.dtype} {name}: best {best:.3f} ms of {args.reps}{rate}"
        if args.kernel and name in ("forward", "adjoint", "dbeta", "conv"):
            cls = {"forward": api.PROF_FORWARD, "adjoint": api.PROF_ADJOINT,
                   "dbeta": api.PROF_DBETA, "conv": api.PROF_CONV}[name]
            api.mpi_profile_enable(True)
            for _ in range(args.reps):
                fn()
            n, tot = api.mpi_profile_read(cls)
            api.mpi_profile_enable(False)
            kms = tot / max(n, 1)
            line += f" | kernel {kms:.4f} ms"
            if name != "conv":
                line += f" = {pairs / kms / 1e6:.1f} Gpair/s"
        print(line, flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

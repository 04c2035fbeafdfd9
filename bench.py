"""Benchmark of the GB300 MPI reconstruction path.

One step = one full ZeroShot-PnP reconstruction (Algorithm 1) of the
128 x 128 spiral workload (T = 65536 samples, 2 channels, 100 PnP iterations
of 20 CG steps, 5x5 Gaussian denoiser, 5th-percentile trimming) with the
forward operator A in FP32 and FP64 CG vectors/inner products.  Every step
applies A and A^T 4201 times; the metric counts (voxel, sample) pairs per
second over the whole reconstruction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank reconstructs its own copy of the workload on its
own GPU (independent problems: weak scaling, no data-path collective); rank 0
prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic per-pair operation counts (FP32 operations, XU transcendental
# operations) of the two closed-form regimes of a pair:
#   "far"  (u < 144, z < 12): the full closed form.  Forward: 2 for the squared
#          distance, 10 for a and d from rsqrt/exp2/rcp, 6 to accumulate c a
#          and c d (y.W) y.  Adjoint: 2 + 10 + 5 (quadratic form, scaling,
#          accumulation).
#   "vfar" (u >= 144): exp(-2z) is below FP32 resolution and a, d take their
#          asymptotic form (rsqrt and 4 FP32 operations instead of 10 + 3 XU).
#          The adjoint evaluates a uW + d P there as a polynomial in 1/z in
#          nested form: 2 (distance) + 2 (quadratic form) + 5, one rsqrt.
# Pairs near the FFP (u < 1, the Taylor series) are a ~1e-4 fraction and are
# counted as "far".  The algorithmic count of a launch is the pair-weighted
# mix, with the vfar fraction measured on the workload's geometry.
ALG_OPS = {"k_forward": {"far": (18, 3), "vfar": (12, 1)},
           "k_adjoint": {"far": (17, 3), "vfar": (9, 1)}}
VFAR_U32 = 144.0


def vfar_fraction(model, grid, r, stride=64):
    """Fraction of (voxel, sample) pairs with |beta G (x - r)|^2 >= 144, on
    every `stride`-th sample (exact over all voxels of those samples)."""
    B = model["beta"] * np.asarray(model["G"], dtype=np.float64)
    xs = grid["x0"] + (np.arange(grid["nx"]) + 0.5) * grid["dx"]
    ys = grid["y0"] + (np.arange(grid["ny"]) + 0.5) * grid["dy"]
    X, Y = np.meshgrid(xs, ys)
    P = np.stack([X.ravel(), Y.ravel()], 1) @ B.T
    Rb = np.asarray(r, dtype=np.float64)[::stride] @ B.T
    n_far = 0
    for k in range(0, Rb.shape[0], 256):
        d = P[None, :, :] - Rb[k:k + 256, None, :]
        n_far += int(np.count_nonzero(np.einsum("tvi,tvi->tv", d, d) >= VFAR_U32))
    return n_far / (P.shape[0] * Rb.shape[0])


def issue_bound_gpair(sm_count, sm_mhz, n_fp32, n_xu):
    """Pairs per second (1e9 units) the SMs can issue when a pair costs n_fp32
    FP32 and n_xu XU operations: per SM and clock at most 128 thread
    instructions in all, 128 on the FP32 pipe and 32 on the XU pipe."""
    per_clk = min(128.0 / (n_fp32 + n_xu), 128.0 / n_fp32, 32.0 / n_xu)
    return sm_count * sm_mhz * 1e6 * per_clk / 1e9


def mixed_ops(kernel, f_vfar):
    (a32, axu), (b32, bxu) = ALG_OPS[kernel]["far"], ALG_OPS[kernel]["vfar"]
    return (1 - f_vfar) * a32 + f_vfar * b32, (1 - f_vfar) * axu + f_vfar * bxu

METRIC = "A/Aᵀ Gvoxel·samples/s and PnP recon/s, FP32 batched vs FP64 plain, ≤1e-5 err"
UNIT = "Gvoxel·samples/s"
WORKLOAD = "c2"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _config_desc(cfg, extra=None):
    g = cfg["grid"]
    d = {"workload": f"{g['nx']}x{g['ny']} voxels, 24x24 mm, Archimedean spiral (32 turns), "
                     f"T={cfg['r'].shape[0]} samples, 2 channels, {cfg['n_it']} PnP iterations x "
                     f"{cfg['n_cg']} CG steps, 5x5 Gaussian denoiser, 5th-percentile trimming",
         "grid": [g["nx"], g["ny"]], "samples": int(cfg["r"].shape[0]), "pnp_iterations": cfg["n_it"],
         "cg_steps": cfg["n_cg"], "operator_applications_per_step": 2 * cfg["n_it"] * (cfg["n_cg"] + 1) + 1,
         "l2": "256 MiB buffer written between timed steps (inputs ~1.5 MB fit in L2)"}
    if extra:
        d.update(extra)
    return d


# ---------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle.

def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    if world > 1:
        # torchrun gives every rank OMP_NUM_THREADS=1; the other ranks exit
        # without work, so rank 0's oracle takes the host's cores as at N = 1
        # (set before the oracle library, and with it OpenMP, is loaded).
        os.environ["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)
    from oracle import oracle
    from paper_2505_22797_gb300 import synthetic as syn
    cfg = syn.config(WORKLOAD)
    m, g = cfg["model"], cfg["grid"]
    T_sub = 32768
    r, v = cfg["r"][:T_sub], cfg["v"][:T_sub]
    c = cfg["c"]
    s = np.random.default_rng(1).normal(size=(2, T_sub))
    pairs = 2 * g["nx"] * g["ny"] * T_sub
    oracle.build()
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.forward(m, g, r, v, c)
        oracle.adjoint(m, g, r, v, s)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = pairs * len(times) / tot / 1e9
    sample = (f"one A and one A^T application of the 128x128 workload on its first {T_sub} "
              f"samples ({pairs:.3e} pairs) per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config_desc(cfg, {"sample": sample}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Our arm.

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = os.path.join("/tmp", f"mpi_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.fh.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[4:8]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# Sources that define the operator kernels and their launch configuration.
KERNEL_SOURCES = ["common.cuh", "langevin.cuh", "pair_kernels.cuh", "pair_ops.cuh", "pair_ops.cu"]


def code_only(text: str) -> str:
    """C/CUDA source without comments and blank space: what a digest of the
    kernel code should see (editing a comment changes no counter)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def kernel_digest(read=None):
    """sha256 prefix of the code of the operator kernels' sources; `read(f)`
    returns a source's text (default: the working tree)."""
    if read is None:
        def read(f):
            return open(os.path.join(ROOT, "paper_2505_22797_gb300", "csrc", f)).read()
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(code_only(read(f)).encode())
    return h.hexdigest()[:16]


def _traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was captured on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    ent = d.get(kernel)
    if not ent or ent.get("source_digest") != kernel_digest():
        return None
    return ent.get("dram_bytes_per_launch")


def measure_batched(api, syn, dev, stream, n_it_timed=1):
    """The 64-frame workload (grids 64^2..256^2, T in [8192, 131072], FP32,
    20 CG steps per PnP iteration) through one batch plan: one untimed run
    that autotunes and captures the graph, then one timed run of
    `n_it_timed` PnP iterations (after A^T of the data).  The full 50-iteration
    reconstruction rate is extrapolated from the per-iteration time."""
    import torch
    frames = syn.batch_frames(64)
    f32 = torch.float32
    r, v, s_list, specs, nu0 = [], [], [], [], []
    pairs_app = 0
    gen = torch.Generator(device="cpu").manual_seed(11)
    for fr in frames:
        m, g = fr["model"], fr["grid"]
        rr = torch.as_tensor(fr["r"], dtype=f32, device=dev)
        vv = torch.as_tensor(fr["v"], dtype=f32, device=dev)
        cc = torch.as_tensor(fr["c"], dtype=f32, device=dev)
        sc = api.mpi_forward(m, g, rr, vv, cc)
        sn = syn.add_noise(sc.cpu().numpy().astype(np.float64), fr["noise_frac"], fr["noise_seed"])
        z = (torch.randint(0, 2, (g["ny"], g["nx"]), generator=gen) * 2 - 1).to(dev, f32)
        fro = float(torch.sum(api.mpi_forward(m, g, rr, vv, z).double() ** 2))
        N = g["nx"] * g["ny"]
        nu0.append(1e-3 * fro / N)
        r.append(rr)
        v.append(vv)
        s_list.append(torch.as_tensor(sn, dtype=f32, device=dev))
        specs.append((m, g, rr.shape[0]))
        pairs_app += N * rr.shape[0]
    n_cg = frames[0]["n_cg"]
    plan = api.BatchPlan(specs, nu0, n_it_timed, n_cg, flags=api.MPI_BATCH_AUTOTUNE)
    rho = plan.run(r, v, s_list)  # tunes, captures
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.run(r, v, s_list, rho_out=rho)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    info = plan.info()
    plan.close()
    apps = 2 * n_it_timed * (n_cg + 1) + 1
    rate = pairs_app * apps / (ms * 1e-3)
    n_it_full = frames[0]["n_it"]
    recon_s = pairs_app * (2 * n_it_full * (n_cg + 1) + 1) / rate
    return {"frames": len(frames), "pairs_per_application": pairs_app,
            "timed": f"{n_it_timed} PnP iteration(s) x {n_cg} CG steps + A^T of the data, all frames",
            "ms": ms, "gpair_per_s": rate / 1e9,
            "recon_per_s_extrapolated": len(frames) / recon_s,
            "batch_s_extrapolated": recon_s, "plan": info}


def measure_paper_pipeline(api, syn, dev, stream):
    """The paper's two-stage reconstruction (Core Stage with gamma = 1e-7 and
    CG to 1e-3 relative residual, then ZeroShot-PnP with the trace-kernel
    convolution, 10 iterations of 20 CG steps) on the scanner-shaped
    synthetic scan (Lissajous 17/16, 1632 samples, 24 mm FoV, 1 % noise) at
    the paper's 21x21 and 100x100 grids, FP32, timed end to end on the
    device.  Beside it, on the same data: the direct-operator PnP (A instead
    of Core Stage + C, same 10 x 20 iterations) and the single-channel form
    (channel x only: one-channel Core Stage, then PnP with the (0, 0) entry of
    the kernel matrix).  Quality is the relative L2 distance to the phantom.
    The paper's times (Table runtimes: CPU 0.46 s / 5.84 s, RTX A6000 1.56 s /
    3.36 s, with a DRUNet denoiser) are context only."""
    import torch
    f32 = torch.float32
    out = {}
    paper = {21: (0.46, 1.56), 100: (5.84, 3.36)}

    def frob2(apply, n, probes=4):
        gen = torch.Generator(device="cpu").manual_seed(5)
        acc = 0.0
        for _ in range(probes):
            z = (torch.randint(0, 2, (n, n), generator=gen) * 2 - 1).to(dev, f32)
            acc += float(torch.sum(apply(z).double() ** 2)) / probes
        return acc

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3, res

    for n in (21, 100):
        g = syn.square_grid(n)
        m = syn.default_model()
        r_np, v_np = syn.lissajous(1632, 17, 16)
        c_np = syn.ellipses(g, np.random.default_rng(101))
        c_t = torch.as_tensor(c_np, dtype=torch.float64)
        r = torch.as_tensor(r_np, dtype=f32, device=dev)
        v = torch.as_tensor(v_np, dtype=f32, device=dev)
        s_clean = api.mpi_forward(m, g, r, v, torch.as_tensor(c_np, dtype=f32, device=dev))
        s = torch.as_tensor(syn.add_noise(s_clean.cpu().numpy().astype(np.float64), 0.01, 201),
                            dtype=f32, device=dev)
        N = n * n
        nu_c = 1e-3 * frob2(lambda z: api.mpi_conv(m, g, z), n) / N
        nu_c00 = 1e-3 * frob2(lambda z: api.mpi_conv_component(m, g, 0, z), n) / N
        nu_a = 1e-3 * frob2(lambda z: api.mpi_forward(m, g, r, v, z), n) / N

        def err(rho):
            return float(torch.linalg.norm(rho.double().cpu() - c_t) / torch.linalg.norm(c_t))

        def two_stage():
            _, u, it = api.mpi_grid(g, r, v, s, gamma=1e-7, max_iter=10000, rel_tol=1e-3,
                                    return_iters=True)
            return it, api.mpi_pnp_solve(m, g, None, None, u.contiguous(), 10, 20, nu_c,
                                         op=api.MPI_OP_CONV)

        def direct():
            return api.mpi_pnp_solve(m, g, r, v, s, 10, 20, nu_a)

        s_x = s[0].contiguous()

        def single_x():
            _, a00, it = api.mpi_grid(g, r, v, s_x, gamma=1e-7, max_iter=10000, rel_tol=1e-3,
                                      return_iters=True, channel=0)
            return it, api.mpi_pnp_solve(m, g, None, None, a00.contiguous(), 10, 20, nu_c00,
                                         op=api.MPI_OP_CONV, kernel_component=0)

        # the same pipelines with the continuous Laplacian as the regulariser
        # (the stencil with 1/dx^2, 1/dy^2; lengths in mm) at the paper's gamma
        def two_stage_scaled():
            _, u, it = api.mpi_grid(g, r, v, s, gamma=1e-7, max_iter=10000, rel_tol=1e-3,
                                    return_iters=True, lap_scaled=True)
            return it, api.mpi_pnp_solve(m, g, None, None, u.contiguous(), 10, 20, nu_c,
                                         op=api.MPI_OP_CONV)

        def single_x_scaled():
            _, a00, it = api.mpi_grid(g, r, v, s_x, gamma=1e-7, max_iter=10000, rel_tol=1e-3,
                                      return_iters=True, channel=0, lap_scaled=True)
            return it, api.mpi_pnp_solve(m, g, None, None, a00.contiguous(), 10, 20, nu_c00,
                                         op=api.MPI_OP_CONV, kernel_component=0)

        t2, (it2, rho2) = timed(two_stage)
        td, rhod = timed(direct)
        t1, (it1, rho1) = timed(single_x)
        t3, (it3, rho3) = timed(two_stage_scaled)
        t4, (it4, rho4) = timed(single_x_scaled)
        out[f"{n}x{n}"] = {
            "s": t2, "core_stage_cg_steps": it2, "rel_err_vs_phantom": err(rho2),
            "direct_A_pnp": {"s": td, "rel_err_vs_phantom": err(rhod)},
            "single_channel_x": {"s": t1, "core_stage_cg_steps": it1, "rel_err_vs_phantom": err(rho1)},
            "two_stage_scaled_laplacian": {"s": t3, "core_stage_cg_steps": it3, "rel_err_vs_phantom": err(rho3)},
            "single_channel_x_scaled_laplacian": {"s": t4, "core_stage_cg_steps": it4,
                                                  "rel_err_vs_phantom": err(rho4)},
            "paper_cpu_s": paper[n][0], "paper_rtx_a6000_s": paper[n][1]}
    return out


def measure_transfer(api, syn, dev, stream, s_model):
    """Transfer-function correction of the workload's signal (two channels,
    T = 65 536, synthetic receive chain, SNR thresholds 0.04 / 0.01): device
    time of one call, mean of 5, and its parity-relevant shape."""
    import torch
    s_np = s_model.double().cpu().numpy()
    T = s_np.shape[1]
    a_hat = syn.transfer_function(T)
    raw, snr = syn.measured_signal(s_np, a_hat, 0.01, 5)
    d_raw = torch.as_tensor(raw, dtype=torch.float32, device=dev)
    d_a = torch.as_tensor(a_hat, dtype=torch.complex128, device=dev)
    d_snr = torch.as_tensor(snr, dtype=torch.float64, device=dev)
    out = torch.empty_like(d_raw)
    api.mpi_transfer_correct(d_raw, d_a, d_snr, [0.04, 0.01], out=out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        api.mpi_transfer_correct(d_raw, d_a, d_snr, [0.04, 0.01], out=out)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / 5
    return {"ms": ms, "samples": int(T), "channels": int(s_np.shape[0]),
            "note": "FP64 device DFTs (Stockham radix-4), per call incl. scratch and twiddle setup"}


# 3-D pairs: "far" 25 FP32 + 3 XU (3 differences, 3 for |y|^2, 10 for a, d,
# 9 for the dot products and accumulation); "vfar" replaces the 10 + 3 XU of
# a, d by 4 + 1 XU; the adjoint's vfar pair term is nested in 1/z (one
# operation fewer).
ALG_OPS_3D = {"k_forward3": {"far": (25, 3), "vfar": (19, 1)},
              "k_adjoint3": {"far": (25, 3), "vfar": (18, 1)}}


def vfar_fraction3(model3, grid3, r, stride=64):
    """vfar_fraction for a 3-D grid and trajectory."""
    B = model3["beta"] * np.asarray(model3["G"], dtype=np.float64)
    xs = grid3["x0"] + (np.arange(grid3["nx"]) + 0.5) * grid3["dx"]
    ys = grid3["y0"] + (np.arange(grid3["ny"]) + 0.5) * grid3["dy"]
    zs = grid3["z0"] + (np.arange(grid3["nz"]) + 0.5) * grid3["dz"]
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) @ B.T
    Rb = np.asarray(r, dtype=np.float64)[::stride] @ B.T
    n_far = 0
    for k in range(0, Rb.shape[0], 64):
        d = P[None, :, :] - Rb[k:k + 64, None, :]
        n_far += int(np.count_nonzero(np.einsum("tvi,tvi->tv", d, d) >= VFAR_U32))
    return n_far / (P.shape[0] * Rb.shape[0])


def measure_ffp3d(api, syn, dev, stream, sm_count, sm_max):
    """The 3-D FFP workload (48 x 48 x 24 voxels, 3-D Lissajous, T = 65 536,
    three channels): kernel-only rates of A and A^T (library event timing,
    mean of 5 applications each) against their issue bound, one ZeroShot-PnP
    reconstruction (20 iterations x 20 CG steps, FP32) timed on the device,
    and the two-stage form (3-D Core Stage, then PnP with the 3-D
    convolution) on the same data."""
    import torch
    f32 = torch.float32
    cfg = syn.config3("3d")
    m, g = cfg["model"], cfg["grid"]
    r = torch.as_tensor(cfg["r"], dtype=f32, device=dev)
    v = torch.as_tensor(cfg["v"], dtype=f32, device=dev)
    c = torch.as_tensor(cfg["c"], dtype=f32, device=dev)
    N, T = cfg["c"].size, cfg["r"].shape[0]
    s_clean = api.mpi_forward3(m, g, r, v, c)
    s = torch.as_tensor(syn.add_noise(s_clean.cpu().numpy().astype(np.float64), cfg["noise_frac"],
                                      cfg["noise_seed"]), dtype=f32, device=dev)
    out = {}
    f_vfar = vfar_fraction3(m, g, cfg["r"])
    cout = torch.empty_like(c)
    for name, cls, fn in (("k_forward3", api.PROF_FORWARD, lambda: api.mpi_forward3(m, g, r, v, c, s=s_clean)),
                          ("k_adjoint3", api.PROF_ADJOINT, lambda: api.mpi_adjoint3(m, g, r, v, s, c_out=cout))):
        fn()
        torch.cuda.synchronize()
        api.mpi_profile_enable(True)
        for _ in range(5):
            fn()
        n, tot = api.mpi_profile_read(cls)
        api.mpi_profile_enable(False)
        ms = tot / max(n, 1)
        (a32, axu), (b32, bxu) = ALG_OPS_3D[name]["far"], ALG_OPS_3D[name]["vfar"]
        n_fp32, n_xu = (1 - f_vfar) * a32 + f_vfar * b32, (1 - f_vfar) * axu + f_vfar * bxu
        peak = issue_bound_gpair(sm_count, sm_max, n_fp32, n_xu)
        rate = N * T / (ms * 1e-3) / 1e9
        out[name] = {"avg_launch_ms": ms, "gpair_per_s": rate, "peak": peak, "frac": rate / peak,
                     "peak_basis": (f"issue bound, {n_fp32:.2f} FP32 + {n_xu:.3f} XU algorithmic ops per "
                                    f"pair ({f_vfar:.4f} of the pairs in the asymptotic regime)")}
    gen = torch.Generator(device="cpu").manual_seed(5)
    fro = 0.0
    for _ in range(4):
        z = (torch.randint(0, 2, tuple(c.shape), generator=gen) * 2 - 1).to(dev, f32)
        fro += float(torch.sum(api.mpi_forward3(m, g, r, v, z).double() ** 2)) / 4
    nu0 = 1e-3 * fro / N
    n_it, n_cg = cfg["n_it"], cfg["n_cg"]
    rho = torch.empty_like(c)
    api.mpi_pnp_solve3(m, g, r, v, s, 1, 1, nu0, rho_out=rho)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    api.mpi_pnp_solve3(m, g, r, v, s, n_it, n_cg, nu0, rho_out=rho)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    apps = 1 + n_it * (2 * (n_cg + 1))
    c64 = torch.as_tensor(cfg["c"], dtype=torch.float64)
    out["pnp"] = {"iterations": n_it, "cg_steps": n_cg, "s": ms * 1e-3,
                  "gpair_per_s": apps * N * T / (ms * 1e-3) / 1e9,
                  "rel_err_vs_phantom": float(torch.linalg.norm(rho.double().cpu() - c64) / torch.linalg.norm(c64))}
    # The paper's two-stage form in three dimensions: the 9-component Core
    # Stage (gamma = 1e-7, CG to 1e-3 relative residual), then PnP with the
    # 3-D trace-kernel convolution on its trace, same iteration counts.
    fro_c = 0.0
    for _ in range(4):
        z = (torch.randint(0, 2, tuple(c.shape), generator=gen) * 2 - 1).to(dev, f32)
        fro_c += float(torch.sum(api.mpi_conv3(m, g, z).double() ** 2)) / 4
    nu_c = 1e-3 * fro_c / N
    rho2 = torch.empty_like(c)

    def core_stage():
        return api.mpi_grid3(g, r, v, s, gamma=1e-7, max_iter=10000, rel_tol=1e-3, return_iters=True)

    core_stage()
    torch.cuda.synchronize()
    e0.record(stream)
    _, u, it = core_stage()
    e1.record(stream)
    e1.synchronize()
    ms_core = e0.elapsed_time(e1)
    e0.record(stream)
    api.mpi_pnp_solve3(m, g, None, None, u.contiguous(), n_it, n_cg, nu_c, op=api.MPI_OP_CONV, rho_out=rho2)
    e1.record(stream)
    e1.synchronize()
    ms_pnp_c = e0.elapsed_time(e1)
    out["two_stage"] = {"s": (ms_core + ms_pnp_c) * 1e-3, "core_stage_s": ms_core * 1e-3,
                        "core_stage_cg_steps": int(it), "core_stage_ms_per_cg_step": ms_core / max(it, 1),
                        "pnp_conv_s": ms_pnp_c * 1e-3,
                        "rel_err_vs_phantom": float(torch.linalg.norm(rho2.double().cpu() - c64)
                                                    / torch.linalg.norm(c64))}
    out["workload"] = "48x48x24 voxels, 24x24x12 mm, G = 2.5 T/m diag(-1/2, -1/2, 1), 3-D Lissajous 17/16/15, T=65536, 3 channels"
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2505_22797_gb300 import api, build
    from paper_2505_22797_gb300 import synthetic as syn
    if world > 1:
        # one rank compiles (if the sources changed); the others then find the
        # library built instead of compiling the same objects concurrently
        if rank == 0:
            build.build()
        dist.barrier()
    build.build()
    api.load()

    dev = torch.device("cuda", local)
    cfg = syn.config(WORKLOAD)
    m, g = cfg["model"], cfg["grid"]
    N, T = g["nx"] * g["ny"], cfg["r"].shape[0]
    n_it, n_cg = cfg["n_it"], cfg["n_cg"]
    f32 = torch.float32
    r = torch.as_tensor(cfg["r"], dtype=f32, device=dev)
    v = torch.as_tensor(cfg["v"], dtype=f32, device=dev)
    c = torch.as_tensor(cfg["c"], dtype=f32, device=dev)
    s_clean = api.mpi_forward(m, g, r, v, c)
    s_np = syn.add_noise(s_clean.cpu().numpy().astype(np.float64), cfg["noise_frac"], cfg["noise_seed"])
    s = torch.as_tensor(s_np, dtype=f32, device=dev)
    # nu0 = 1e-3 ||A||_F^2 / N with ||A||_F^2 from 4 Rademacher probes (E ||A z||^2).
    gen = torch.Generator(device="cpu").manual_seed(7)
    fro = 0.0
    for _ in range(4):
        z = (torch.randint(0, 2, (g["ny"], g["nx"]), generator=gen) * 2 - 1).to(dev, f32)
        fro += float(torch.sum(api.mpi_forward(m, g, r, v, z).double() ** 2)) / 4
    nu0 = 1e-3 * fro / N
    rho = torch.empty((g["ny"], g["nx"]), dtype=f32, device=dev)
    apps = 2 * n_it * (n_cg + 1) + 1
    pairs_step = apps * N * T
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        api.mpi_pnp_solve(m, g, r, v, s, n_it, n_cg, nu0, clip_pct=cfg["clip_pct"], rho_out=rho)

    from paper_2505_22797_gb300 import multirank

    def barrier():
        multirank.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # --- timed region (device time per step, L2 flushed between steps) ------
    stream = torch.cuda.current_stream()
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    gpu_id = f"GPU-{uuid}" if uuid is not None else str(local)
    launches0 = api.mpi_kernel_launches()
    api.mpi_profile_enable(True)
    step_ms = []
    with ClockSampler(gpu_id) as clocks:
        barrier()
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        barrier()
    launches = api.mpi_kernel_launches() - launches0
    prof = {k: api.mpi_profile_read(k) for k in (api.PROF_FORWARD, api.PROF_ADJOINT)}
    api.mpi_profile_enable(False)
    # every rank reconstructs its own problem: all ranks' units over the
    # slowest rank's time
    local_s = sum(step_ms) * 1e-3
    total_ms = multirank.max_over_ranks(local_s) * 1e3
    value = multirank.job_rate(pairs_step * args.steps, local_s) / 1e9
    recon_per_s = multirank.job_rate(args.steps, local_s)

    # --- end to end through the public API, host buffers ------------------------
    h_r = torch.as_tensor(cfg["r"], dtype=f32).pin_memory()
    h_v = torch.as_tensor(cfg["v"], dtype=f32).pin_memory()
    h_s = s.cpu().pin_memory()
    h_rho = torch.empty((g["ny"], g["nx"]), dtype=f32).pin_memory()
    d_r, d_v, d_s = torch.empty_like(r), torch.empty_like(v), torch.empty_like(s)
    e2e_ms = []
    barrier()
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d_r.copy_(h_r, non_blocking=True)
        d_v.copy_(h_v, non_blocking=True)
        d_s.copy_(h_s, non_blocking=True)
        api.mpi_pnp_solve(m, g, d_r, d_v, d_s, n_it, n_cg, nu0, clip_pct=cfg["clip_pct"], rho_out=rho)
        h_rho.copy_(rho, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    barrier()
    e2e_local_s = sum(e2e_ms) * 1e-3
    e2e_tot = multirank.max_over_ranks(e2e_local_s) * 1e3
    e2e_value = multirank.job_rate(pairs_step * len(e2e_ms), e2e_local_s) / 1e9
    h2d = (h_r.numel() + h_v.numel() + h_s.numel()) * 4
    d2h = h_rho.numel() * 4

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # --- roofline of the dominant kernel ----------------------------------------
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    clk = clocks.summary()
    sm_max = peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
    (nf, fms), (na, ams) = prof[api.PROF_FORWARD], prof[api.PROF_ADJOINT]
    dom, n_l, ms_l = ("k_forward", nf, fms) if fms >= ams else ("k_adjoint", na, ams)
    # Algorithmic instructions per pair of the closed-form branch (FP32 ops,
    # XU ops): every one occupies an issue slot (128 thread-instructions per
    # SM per cycle), FP32 ops the FP32 pipe (128 lanes), XU ops the XU pipe
    # (32 results per SM per cycle on GB300, inferred from ncu's pct-of-peak).
    f_vfar = vfar_fraction(m, g, cfg["r"])
    n_fp32, n_xu = mixed_ops(dom, f_vfar)
    peak_gpair = issue_bound_gpair(sm_count, sm_max, n_fp32, n_xu)
    achieved = (N * T) / (ms_l / n_l * 1e-3) / 1e9 if n_l else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_gpair, "unit": "Gpair/s",
                "frac": achieved / peak_gpair if achieved else None, "traffic": _traffic(dom),
                "kernel": dom, "launches": n_l, "avg_launch_ms": ms_l / n_l if n_l else None,
                "peak_basis": (f"issue bound: {sm_count} SMs x {sm_max:.0f} MHz x 128 thread-instructions"
                               f"/clk / ({n_fp32:.2f} FP32 + {n_xu:.3f} XU algorithmic ops per pair: "
                               f"{f_vfar:.4f} of the pairs in the asymptotic regime u >= 144)"),
                "other": {"k_forward_avg_ms": fms / nf if nf else None,
                          "k_adjoint_avg_ms": ams / na if na else None,
                          "share_of_step": (fms + ams) / total_ms if total_ms else None}}

    # --- FP64 plain form (one A and one A^T application) -----------------------
    f64 = torch.float64
    r64, v64, c64 = r.double(), v.double(), c.double()
    s64 = api.mpi_forward(m, g, r64, v64, c64)
    api.mpi_adjoint(m, g, r64, v64, s64)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    api.mpi_forward(m, g, r64, v64, c64, s=s64)
    api.mpi_adjoint(m, g, r64, v64, s64)
    e1.record(stream)
    e1.synchronize()
    f64_ms = e0.elapsed_time(e1)
    f64_rate = 2 * N * T / (f64_ms * 1e-3) / 1e9
    fp64_plain = {"gpair_per_s": f64_rate, "recon_s_extrapolated": pairs_step / (f64_rate * 1e9),
                  "note": "one FP64 A and one FP64 A^T application, extrapolated to the "
                          f"{apps} applications of a reconstruction"}

    # --- batched form: 64 frames of uneven size in one plan ----------------------
    batched = None
    if world == 1 and not args.no_batch:
        batched = measure_batched(api, syn, dev, stream)

    # --- the paper's own two-stage pipeline, for context ------------------------
    paper_pipeline = None
    if world == 1 and not args.no_batch:
        paper_pipeline = measure_paper_pipeline(api, syn, dev, stream)

    # --- preprocessing: transfer-function correction --------------------------
    transfer = None
    if world == 1 and not args.no_batch:
        transfer = measure_transfer(api, syn, dev, stream, s)

    # --- the three-dimensional FFP --------------------------------------------
    ffp3d = None
    if world == 1 and not args.no_batch:
        ffp3d = measure_ffp3d(api, syn, dev, stream, sm_count, sm_max)

    # --- CPU baseline: the oracle on a bounded sample -----------------------
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        from oracle import oracle
        oracle.build()
        T_sub = T
        rr_, vv_ = cfg["r"][:T_sub], cfg["v"][:T_sub]
        ss_ = np.random.default_rng(1).normal(size=(2, T_sub))
        t0 = time.perf_counter()
        oracle.forward(m, g, rr_, vv_, cfg["c"])
        oracle.adjoint(m, g, rr_, vv_, ss_)
        dt = time.perf_counter() - t0
        cpu = {"value": 2 * N * T_sub / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
               "kind": "oracle",
               "sample": f"one A and one A^T application of the workload ({T_sub} samples, "
                         f"{2 * N * T_sub:.3e} pairs, {dt:.1f} s)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config_desc(cfg, {"precision": "FP32 operator, FP64 CG vectors and inner products",
                                         "nu0": nu0}),
            "recon_per_s": recon_per_s,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": len(e2e_ms),
                    "recon_per_s": len(e2e_ms) * world / (e2e_tot * 1e-3)},
            "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "fp64_plain": fp64_plain, "batched": batched, "paper_pipeline": paper_pipeline,
            "ffp3d": ffp3d, "transfer_correction": transfer,
            "clocks": clk, "impl": "ours"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the secondary measurements (64-frame batch, paper pipeline, 3-D FFP)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

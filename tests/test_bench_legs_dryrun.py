"""The benchmark's paper-pipeline leg run on the CPU with a stand-in binding
built on the FP64 oracle (CUDA events stubbed): checks the leg's own logic
(the calls it makes, their arguments, the record it returns) without a GPU.
The numbers it produces are the oracle's, not a measurement."""
import os
import sys
import types

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2505_22797_gb300 import synthetic as syn  # noqa: E402

pytestmark = pytest.mark.slow


class _Event:
    def __init__(self, **kw):
        self.t = 0.0

    def record(self, stream=None):
        import time
        self.t = time.perf_counter()

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3


def _fake_api(orc):
    T = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64)  # noqa: E731
    N = lambda t: t.detach().double().cpu().numpy()  # noqa: E731

    def conv_fft(kern, x):
        ny, nx = x.shape
        shape = (2 * ny, 2 * nx)
        y = np.fft.irfft2(np.fft.rfft2(x, shape) * np.fft.rfft2(kern, shape), shape)
        return y[ny - 1:2 * ny - 1, nx - 1:2 * nx - 1]

    def kernel(m, g, comp=None):
        return orc.conv_kernel(m, g, component=None if comp is None else (comp // 2, comp % 2))

    api = types.SimpleNamespace(MPI_OP_FORWARD=0, MPI_OP_CONV=1, calls=[])

    def mpi_forward(m, g, r, v, c, s=None, stream=None):
        return T(orc.forward(m, g, N(r), N(v), N(c)))

    def mpi_conv(m, g, z, out=None, stream=None):
        return T(conv_fft(kernel(m, g), N(z)))

    def mpi_conv_component(m, g, comp, z, out=None, stream=None):
        return T(conv_fft(kernel(m, g, comp), N(z)))

    def mpi_grid(g, r, v, s, gamma=1e-7, max_iter=10000, rel_tol=1e-3, return_iters=False, channel=None,
                 lap_scaled=False, **kw):
        api.calls.append(("grid", g["nx"], gamma, channel, lap_scaled))
        lap = "scaled" if lap_scaled else "bare"
        if channel is None:
            A, u, h = orc.core_stage(g, N(r), N(v), N(s), gamma, max_iter, rel_tol=rel_tol, lap=lap)
        else:
            A, u, h = orc.core_stage_channel(g, N(r), N(v), N(s).reshape(-1), channel, gamma, max_iter,
                                             rel_tol=rel_tol, lap=lap)
        return (T(A), T(u), len(h) - 1) if return_iters else (T(A), T(u))

    def mpi_pnp_solve(m, g, r, v, data, n_iter, n_cg, nu0, clip_pct=5.0, op=0, kernel_component=None, **kw):
        api.calls.append(("pnp", g["nx"], op, kernel_component))
        shape = (g["ny"], g["nx"])
        if op == 1:
            k = kernel(m, g, kernel_component)
            C = lambda x: conv_fft(k, x.reshape(shape))  # noqa: E731
            return T(orc.pnp(C, C, N(data), shape, n_iter, n_cg, nu0, clip_pct))
        # with A (the direct form): one iteration of one CG step keeps the
        # stand-in cheap; only the leg's bookkeeping is checked here
        rr, vv = N(r), N(v)
        return T(orc.pnp(lambda x: orc.forward(m, g, rr, vv, x.reshape(shape)),
                         lambda y: orc.adjoint(m, g, rr, vv, y), N(data), shape, 1, 1, nu0, clip_pct))

    for f in (mpi_forward, mpi_conv, mpi_conv_component, mpi_grid, mpi_pnp_solve):
        setattr(api, f.__name__, f)
    return api


def test_paper_pipeline_leg_logic(orc, monkeypatch):
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    api = _fake_api(orc)
    out = bench.measure_paper_pipeline(api, syn, "cpu", None)
    assert set(out) == {"21x21", "100x100"}
    for n, rec in ((21, out["21x21"]), (100, out["100x100"])):
        for key in ("s", "core_stage_cg_steps", "rel_err_vs_phantom", "direct_A_pnp", "single_channel_x",
                    "two_stage_scaled_laplacian", "single_channel_x_scaled_laplacian", "paper_cpu_s",
                    "paper_rtx_a6000_s"):
            assert key in rec, key
        for k in ("two_stage_scaled_laplacian", "single_channel_x_scaled_laplacian"):
            assert rec[k]["core_stage_cg_steps"] > 0 and np.isfinite(rec[k]["rel_err_vs_phantom"])
    # the scaled regulariser keeps the fine grid near the coarse one (reading of the regulariser)
    assert out["100x100"]["two_stage_scaled_laplacian"]["rel_err_vs_phantom"] < 0.45
    assert out["100x100"]["single_channel_x_scaled_laplacian"]["rel_err_vs_phantom"] < 0.6
    grids = [c for c in api.calls if c[0] == "grid"]
    assert {(c[1], c[3], c[4]) for c in grids} == {(n, ch, sc) for n in (21, 100) for ch in (None, 0)
                                                   for sc in (False, True)}
    assert all(c[2] == 1e-7 for c in grids)
    pnps = [c for c in api.calls if c[0] == "pnp"]
    assert ("pnp", 100, 1, 0) in pnps and ("pnp", 100, 0, None) in pnps

"""GPU parity of the ZeroShot-PnP solve (Algorithm 1), the trace-kernel
convolution, the built-in denoiser and its callback path, against the FP64
oracle on seeded synthetic inputs."""
import os

import numpy as np
import pytest
import torch

from paper_2505_22797_gb300 import api
from paper_2505_22797_gb300 import synthetic as syn
from tests.gpu_util import dev, host, rel_l2, roundoff_spread, rounded, tol

pytestmark = pytest.mark.gpu
DTYPES = [torch.float32, torch.float64]


def _data(orc, cfg, dt):
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    s = rounded(syn.add_noise(orc.forward(m, g, r, v, c), cfg["noise_frac"], cfg["noise_seed"]), dt)
    nu0 = orc.nu0_from_frob2(orc.frob2(m, g, r, v), g["nx"] * g["ny"])
    return m, g, r, v, s, nu0


def _oracle_pnp(orc, m, g, r, v, s, n_it, n_cg, nu0, clip=5.0, record=None):
    shape = (g["ny"], g["nx"])
    return orc.pnp(lambda x: orc.forward(m, g, r, v, x), lambda y: orc.adjoint(m, g, r, v, y), s,
                   shape, n_it, n_cg, nu0, clip_pct=clip, record=record)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(24, 20, 900), (37, 29, 1500)])
def test_pnp_forward_small(orc, dt, shape):
    cfg = syn.small(*shape, traj="spiral", seed=21)
    m, g, r, v, s, nu0 = _data(orc, cfg, dt)
    rec = []
    want = _oracle_pnp(orc, m, g, r, v, s, 4, 4, nu0, record=rec)
    got, info = api.mpi_pnp_solve(m, g, dev(r, dt), dev(v, dt), dev(s, dt), 4, 4, nu0,
                                  with_info=True)
    assert rel_l2(host(got), want) <= tol(dt)
    for k in range(4):
        assert abs(info[k][0] - rec[k]["sigma"]) <= 10 * tol(dt) * rec[k]["sigma"]
        assert abs(info[k][1] - rec[k]["nu"]) <= 10 * tol(dt) * rec[k]["nu"]
        assert abs(info[k][3] - rec[k]["clip"]) <= 10 * tol(dt) * (abs(rec[k]["clip"]) + rec[k]["sigma"])


@pytest.mark.parametrize("dt", DTYPES)
def test_pnp_c1_well_posed(orc, dt):
    """The 32x32 Lissajous workload, 50 PnP iterations of 5 CG steps: the
    setting where the iteration is stable under round-off (the oracle's own
    1-ulp spread is ~1e-14), held to the strict 1e-5 / 1e-12 bar."""
    cfg = syn.config("c1")
    m, g, r, v, s, nu0 = _data(orc, cfg, dt)
    want = _oracle_pnp(orc, m, g, r, v, s, cfg["n_it"], 5, nu0)
    got = api.mpi_pnp_solve(m, g, dev(r, dt), dev(v, dt), dev(s, dt), cfg["n_it"], 5, nu0)
    err = rel_l2(host(got), want)
    print(f"c1 PnP 50x5 {dt}: rel-L2 vs oracle {err:.3e}")
    assert err <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
def test_pnp_c1_full(orc, dt):
    """The 32x32 Lissajous workload as configured: 50 PnP iterations of 20 CG
    steps.  The error against the oracle is held to ten times the oracle's
    own round-off spread at the same precision (never below the 1e-5 / 1e-12
    bar)."""
    cfg = syn.config("c1")
    m, g, r, v, s, nu0 = _data(orc, cfg, dt)
    want = _oracle_pnp(orc, m, g, r, v, s, cfg["n_it"], cfg["n_cg"], nu0)
    got = api.mpi_pnp_solve(m, g, dev(r, dt), dev(v, dt), dev(s, dt), cfg["n_it"], cfg["n_cg"], nu0)
    err = rel_l2(host(got), want)
    spread = roundoff_spread(orc, m, g, r, v, s, cfg["n_it"], cfg["n_cg"], nu0, dt)
    print(f"c1 PnP 50x20 {dt}: rel-L2 vs oracle {err:.3e}, oracle round-off spread {spread:.3e}")
    assert err <= max(tol(dt), 10 * spread)


@pytest.fixture(scope="module")
def c2_well_posed(orc):
    """The 128 x 128 spiral workload (every 8th sample of the 32-turn spiral,
    8192 samples, velocities per sample of the subsampled trajectory) with the
    oracle's Algorithm 1 at 3 PnP iterations of 5 CG steps.  Inputs are
    rounded to FP32 once, so the one oracle run (and its per-iteration record)
    serves both precisions of the GPU path."""
    cfg = syn.config("c2")
    m, g = cfg["model"], cfg["grid"]
    f32 = torch.float32
    r = rounded(cfg["r"][::8], f32)
    v = rounded(cfg["v"][::8] * 8.0, f32)
    c = rounded(cfg["c"], f32)
    s = rounded(syn.add_noise(orc.forward(m, g, r, v, c), cfg["noise_frac"], cfg["noise_seed"]), f32)
    nu0 = orc.nu0_from_frob2(orc.frob2(m, g, r, v), g["nx"] * g["ny"])
    rec = []
    want = _oracle_pnp(orc, m, g, r, v, s, 3, 5, nu0, clip=cfg["clip_pct"], record=rec)
    return m, g, r, v, s, nu0, want, rec, cfg["clip_pct"]


@pytest.mark.parametrize("dt", DTYPES)
def test_pnp_c2_grid_well_posed(c2_well_posed, dt):
    """Algorithm 1 on the 128 x 128 grid (the percentile select and the
    variance run over 16 384 values in one block) at the strict bar: the
    reconstruction within 1e-5 (FP32) / 1e-12 (FP64) of the oracle, and per
    iteration sigma, nu and the 5th-percentile clip value."""
    m, g, r, v, s, nu0, want, rec, clip = c2_well_posed
    got, info = api.mpi_pnp_solve(m, g, dev(r, dt), dev(v, dt), dev(s, dt), 3, 5, nu0, clip_pct=clip,
                                  with_info=True)
    err = rel_l2(host(got), want)
    print(f"128x128 PnP 3x5 {dt}: rel-L2 vs oracle {err:.3e}")
    assert err <= tol(dt)
    for k in range(3):
        sig, nu, _, pclip = info[k]
        assert abs(sig - rec[k]["sigma"]) <= 10 * tol(dt) * rec[k]["sigma"]
        assert abs(nu - rec[k]["nu"]) <= 10 * tol(dt) * rec[k]["nu"]
        assert abs(pclip - rec[k]["clip"]) <= 10 * tol(dt) * (abs(rec[k]["clip"]) + rec[k]["sigma"])


def test_pnp_no_clip_zero_iters_and_deterministic(orc):
    dt = torch.float32
    cfg = syn.small(16, 16, 600, seed=4)
    m, g, r, v, s, nu0 = _data(orc, cfg, dt)
    want = _oracle_pnp(orc, m, g, r, v, s, 2, 3, nu0, clip=-1.0)
    args = (m, g, dev(r, dt), dev(v, dt), dev(s, dt))
    a = host(api.mpi_pnp_solve(*args, 2, 3, nu0, clip_pct=-1.0))
    b = host(api.mpi_pnp_solve(*args, 2, 3, nu0, clip_pct=-1.0))
    assert rel_l2(a, want) <= tol(dt)
    assert np.array_equal(a, b)
    z = host(api.mpi_pnp_solve(*args, 0, 3, nu0))
    assert not z.any()


@pytest.mark.parametrize("dt", DTYPES)
def test_pnp_conv_operator(orc, dt):
    """Algorithm 1 with C_h (the paper's deconvolution stage) on a trace image."""
    cfg = syn.small(19, 14, 10, seed=9)
    m, g = cfg["model"], cfg["grid"]
    K = orc.conv_kernel(m, g)
    c = rounded(cfg["c"], dt)
    u = rounded(orc.conv(g, K, c) + 0.01 * np.random.default_rng(3).normal(size=c.shape), dt)
    nu0 = 1e-3 * np.sum(K * K)
    want = orc.pnp(lambda x: orc.conv(g, K, x), lambda y: orc.conv(g, K, y), u, c.shape, 3, 5, nu0)
    got = api.mpi_pnp_solve(m, g, None, None, dev(u, dt), 3, 5, nu0, op=api.MPI_OP_CONV)
    assert rel_l2(host(got), want) <= tol(dt)


def test_pnp_callback_and_errors(orc):
    dt = torch.float32
    cfg = syn.small(12, 10, 300, seed=2)
    m, g, r, v, s, nu0 = _data(orc, cfg, dt)
    seen = []

    def halve(x, out, sigma):
        seen.append(float(sigma.item()))
        out.copy_(x * 0.5)
    got = api.mpi_pnp_solve(m, g, dev(r, dt), dev(v, dt), dev(s, dt), 2, 3, nu0, denoise=halve)
    want = orc.pnp(lambda x: orc.forward(m, g, r, v, x), lambda y: orc.adjoint(m, g, r, v, y), s,
                   (10, 12), 2, 3, nu0, denoise=lambda img, sig: img * 0.5)
    assert len(seen) == 2
    assert rel_l2(host(got), want) <= tol(dt)

    def broken(x, out, sigma):
        raise RuntimeError("denoiser failure")
    with pytest.raises(api.MPIError) as e:
        api.mpi_pnp_solve(m, g, dev(r, dt), dev(v, dt), dev(s, dt), 2, 3, nu0, denoise=broken)
    assert e.value.status == api.MPI_ERR_CALLBACK
    os.environ["MPI_FAULT"] = "alloc"
    try:
        with pytest.raises(api.MPIError) as e:
            api.mpi_pnp_solve(m, g, dev(r, dt), dev(v, dt), dev(s, dt), 2, 3, nu0)
        assert e.value.status == api.MPI_ERR_NOMEM
    finally:
        del os.environ["MPI_FAULT"]
    # the library still works after the injected failures
    again = api.mpi_pnp_solve(m, g, dev(r, dt), dev(v, dt), dev(s, dt), 2, 3, nu0)
    assert np.isfinite(host(again)).all()


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(1, 1), (5, 3), (33, 17), (64, 64)])
def test_conv_and_denoiser(orc, dt, shape):
    nx, ny = shape
    g = syn.square_grid(nx, 24.0, ny)
    m = syn.default_model()
    x = rounded(np.random.default_rng(nx).normal(size=(ny, nx)), dt)
    want = orc.conv(g, orc.conv_kernel(m, g), x)
    assert rel_l2(host(api.mpi_conv(m, g, dev(x, dt))), want) <= tol(dt)
    assert rel_l2(host(api.mpi_denoise_gaussian5(dev(x, dt))), orc.gaussian5(x)) <= tol(dt)


def test_conv_non_diagonal_gradient(orc):
    dt = torch.float64
    g = syn.square_grid(21, 24.0, 13)
    m = dict(syn.default_model(), G=[[2.1e-3, 4e-4], [4e-4, -2.6e-3]])
    x = np.random.default_rng(1).normal(size=(13, 21))
    want = orc.conv(g, orc.conv_kernel(m, g), x)
    assert rel_l2(host(api.mpi_conv(m, g, dev(x, dt))), want) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("comp", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_conv_kernel_component(orc, dt, comp):
    """Entry (a, b) of beta K(beta G y) G as convolution kernel (Sec. 3.6),
    non-diagonal G so that all four entries differ."""
    g = syn.square_grid(23, 24.0, 14)
    m = dict(syn.default_model(), G=[[2.1e-3, 4e-4], [-3e-4, -2.6e-3]])
    x = rounded(np.random.default_rng(5).normal(size=(14, 23)), dt)
    want = orc.conv(g, orc.conv_kernel(m, g, component=comp), x)
    got = api.mpi_conv_component(m, g, 2 * comp[0] + comp[1], dev(x, dt))
    assert rel_l2(host(got), want) <= tol(dt)
    tr = api.mpi_conv_component(m, g, -1, dev(x, dt))
    assert rel_l2(host(tr), orc.conv(g, orc.conv_kernel(m, g), x)) <= tol(dt)


def test_pnp_single_channel_deconvolution(orc):
    """Algorithm 1 on the (0, 0) kernel entry (channel-x data, Sec. 3.6),
    FP64, few steps so that CG round-off stays at the FP64 bar."""
    dt = torch.float64
    g = syn.square_grid(21, 24.0)
    m = syn.default_model()
    u = np.random.default_rng(8).normal(size=(21, 21))
    kern = orc.conv_kernel(m, g, component=(0, 0))
    op = lambda x: orc.conv(g, kern, x)  # noqa: E731
    want = orc.pnp(op, op, u, (21, 21), 3, 4, 0.05)
    got = api.mpi_pnp_solve(m, g, None, None, dev(u, dt), 3, 4, 0.05, op=api.MPI_OP_CONV,
                            kernel_component=0)
    assert rel_l2(host(got), want) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
def test_pnp_forward_single_channel(orc, dt):
    """Algorithm 1 with the direct operator on channel x only (p = [(1, 0)],
    the partial-data setting of Sec. 3.6): s has one row."""
    cfg = syn.small(26, 22, 1100, traj="spiral", seed=31)
    cfg["model"] = dict(cfg["model"], p=[[1.0, 0.0]])
    m, g, r, v, s, nu0 = _data(orc, cfg, dt)
    assert s.shape == (1, 1100)
    want = _oracle_pnp(orc, m, g, r, v, s, 4, 4, nu0)
    got = api.mpi_pnp_solve(m, g, dev(r, dt), dev(v, dt), dev(s, dt), 4, 4, nu0)
    assert rel_l2(host(got), want) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(80, 80), (128, 128), (97, 113), (181, 64), (300, 20)])
def test_conv_fft_route(orc, dt, shape):
    """Grids of 4096 voxels and more (FP32; 1024 in FP64) take the FFT route (circular convolution
    on a padded grid): same linear convolution as the oracle's direct sum."""
    nx, ny = shape
    g = syn.square_grid(nx, 24.0, ny)
    for m in (syn.default_model(), dict(syn.default_model(), G=[[2.1e-3, 4e-4], [4e-4, -2.6e-3]])):
        x = rounded(np.random.default_rng(nx + ny).normal(size=(ny, nx)), dt)
        want = orc.conv(g, orc.conv_kernel(m, g), x)
        assert rel_l2(host(api.mpi_conv(m, g, dev(x, dt))), want) <= tol(dt)
    comp = orc.conv_kernel(m, g, component=(1, 0))
    got = api.mpi_conv_component(m, g, 2, dev(x, dt))
    assert rel_l2(host(got), orc.conv(g, comp, x)) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(512, 512), (2048, 4), (8, 1024), (4, 1100)])
def test_conv_fft_route_large(orc, dt, shape):
    """The three-launch FFT route at 512 x 512 and at its limits (4096-point
    rows, 2048-point columns), and a grid past them (4096-point columns: the
    nine-launch route), every output against the oracle's FFT realisation of
    the same linear convolution."""
    nx, ny = shape
    g = syn.square_grid(nx, 24.0, ny)
    m = syn.default_model()
    x = rounded(np.random.default_rng(nx * 3 + ny).normal(size=(ny, nx)), dt)
    want = orc.conv_fft(orc.conv_kernel(m, g), x)
    assert rel_l2(host(api.mpi_conv(m, g, dev(x, dt))), want) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
def test_pnp_conv_fft_route(orc, dt):
    """Algorithm 1 with C on a 100 x 100 grid (FFT route), few steps."""
    g = syn.square_grid(100, 24.0)
    m = syn.default_model()
    u = rounded(np.random.default_rng(12).normal(size=(100, 100)) + 1.0, dt)
    kern = orc.conv_kernel(m, g)
    op = lambda x: orc.conv(g, kern, x)  # noqa: E731
    want = orc.pnp(op, op, u, (100, 100), 2, 3, 0.05)
    got = api.mpi_pnp_solve(m, g, None, None, dev(u, dt), 2, 3, 0.05, op=api.MPI_OP_CONV)
    assert rel_l2(host(got), want) <= tol(dt)

"""GPU parity of the three-dimensional field-free point (Sec. 2 with n = 3):
forward and adjoint operators, the 3-D trace-kernel convolution, the volume
denoiser and Algorithm 1 with either operator, against the FP64 oracle on
seeded synthetic inputs."""
import numpy as np
import pytest
import torch

from paper_2505_22797_gb300 import api
from paper_2505_22797_gb300 import synthetic as syn
from tests.gpu_util import dev, host, rel_l2, rounded, tol

pytestmark = pytest.mark.gpu
DTYPES = [torch.float32, torch.float64]
G_GEN = [[-1.1e-3, 3e-4, -2e-4], [3e-4, -1.4e-3, 1e-4], [-2e-4, 1e-4, 2.3e-3]]

CASES = [
    dict(nx=1, ny=1, nz=1, T=7),                         # degenerate grid, one partial tile
    dict(nx=13, ny=11, nz=5, T=1500),                    # several tiles, ragged tails
    dict(nx=20, ny=17, nz=9, T=3001, G=G_GEN),           # general G
    dict(nx=9, ny=8, nz=7, T=700, n_ch=1),               # one channel
    dict(nx=16, ny=16, nz=8, T=1024, n_ch=2),            # exact tile multiples
]


def _case(cs, dt):
    cfg = syn.small3(cs["nx"], cs["ny"], cs["nz"], cs["T"], seed=cs["nx"], n_ch=cs.get("n_ch", 3))
    m = cfg["model"]
    if "G" in cs:
        m = dict(m, G=cs["G"])
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    return m, cfg["grid"], r, v, c


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("cs", CASES, ids=lambda c: f"{c['nx']}x{c['ny']}x{c['nz']}_{c['T']}")
def test_forward3_adjoint3(orc, dt, cs):
    m, g, r, v, c = _case(cs, dt)
    s = api.mpi_forward3(m, g, dev(r, dt), dev(v, dt), dev(c, dt))
    assert rel_l2(host(s), orc.forward3(m, g, r, v, c)) <= tol(dt)
    y = rounded(np.random.default_rng(3).normal(size=s.shape), dt)
    got = api.mpi_adjoint3(m, g, dev(r, dt), dev(v, dt), dev(y, dt))
    assert rel_l2(host(got), orc.adjoint3(m, g, r, v, y)) <= tol(dt)


def test_forward3_far_trajectory(orc):
    """A trajectory 40 mm above the volume: every staged pass takes the
    closed-form-only loop."""
    dt = torch.float32
    m, g, r, v, c = _case(dict(nx=12, ny=10, nz=6, T=900), dt)
    r = r + np.array([0.0, 0.0, 40.0])
    s = api.mpi_forward3(m, g, dev(r, dt), dev(v, dt), dev(c, dt))
    assert rel_l2(host(s), orc.forward3(m, g, r, v, c)) <= tol(dt)
    y = rounded(np.random.default_rng(4).normal(size=s.shape), dt)
    got = api.mpi_adjoint3(m, g, dev(r, dt), dev(v, dt), dev(y, dt))
    assert rel_l2(host(got), orc.adjoint3(m, g, r, v, y)) <= tol(dt)


@pytest.mark.parametrize("T", [257, 901])
def test_adjoint3_asymptotic_odd_batches(orc, T):
    """A trajectory far above the volume: every staged pass takes the packed
    asymptotic form, and an odd sample count leaves the last staged pair with
    one real sample (its partner carries zero weight)."""
    dt = torch.float32
    m, g, r, v, c = _case(dict(nx=12, ny=10, nz=6, T=T), dt)
    r = r + np.array([0.0, 0.0, 400.0])
    s = api.mpi_forward3(m, g, dev(r, dt), dev(v, dt), dev(c, dt))
    assert rel_l2(host(s), orc.forward3(m, g, r, v, c)) <= tol(dt)
    y = rounded(np.random.default_rng(5).normal(size=s.shape), dt)
    got = api.mpi_adjoint3(m, g, dev(r, dt), dev(v, dt), dev(y, dt))
    assert rel_l2(host(got), orc.adjoint3(m, g, r, v, y)) <= tol(dt)


def test_empty_trajectory3():
    g = syn.box_grid3(4, 3, 2)
    m = syn.default_model3()
    z = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    out = api.mpi_adjoint3(m, g, z, z, torch.zeros((3, 0), dtype=torch.float32, device="cuda"))
    assert torch.count_nonzero(out).item() == 0
    s = api.mpi_forward3(m, g, z, z, torch.ones((2, 3, 4), dtype=torch.float32, device="cuda"))
    assert s.shape == (3, 0)


@pytest.mark.parametrize("dt", DTYPES)
def test_full_size_sampled(orc, dt):
    """The 48 x 48 x 24 / 65 536-sample workload at full size, in the launch
    configuration of the benchmark: 24 seeded samples of A c (all channels)
    and 24 seeded voxels of A^T y, computed one by one by the oracle."""
    cfg = syn.config3("3d")
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    rng = np.random.default_rng(17)
    s = host(api.mpi_forward3(m, g, dev(r, dt), dev(v, dt), dev(c, dt)))
    ts = np.sort(rng.choice(r.shape[0], 24, replace=False))
    want = orc.forward3(m, g, r[ts], v[ts], c)
    assert rel_l2(s[:, ts], want) <= tol(dt)
    y = rounded(rng.normal(size=(3, r.shape[0])), dt)
    a = host(api.mpi_adjoint3(m, g, dev(r, dt), dev(v, dt), dev(y, dt))).reshape(-1)
    vs = np.sort(rng.choice(a.size, 24, replace=False))
    assert rel_l2(a[vs], orc.adjoint3(m, g, r, v, y, sel=vs)) <= tol(dt)


def test_adjoint_identity_full_size():
    """<A c, y> = <c, A^T y> on the full 3-D workload, FP64."""
    dt = torch.float64
    cfg = syn.config3("3d")
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (dev(cfg[k], dt) for k in ("r", "v", "c"))
    y = dev(np.random.default_rng(2).normal(size=(3, cfg["r"].shape[0])), dt)
    lhs = float(torch.sum(api.mpi_forward3(m, g, r, v, c) * y))
    rhs = float(torch.sum(c * api.mpi_adjoint3(m, g, r, v, y)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_forward3_deterministic():
    dt = torch.float32
    cfg = syn.small3(14, 12, 6, 2048)
    args = [dev(cfg[k], dt) for k in ("r", "v", "c")]
    a = api.mpi_forward3(cfg["model"], cfg["grid"], *args)
    b = api.mpi_forward3(cfg["model"], cfg["grid"], *args)
    assert torch.equal(a, b)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(1, 1, 1), (9, 7, 5), (17, 13, 6)])
def test_conv3_and_denoiser(orc, dt, shape):
    nx, ny, nz = shape
    g = syn.box_grid3(nx, ny, nz)
    for m in (syn.default_model3(), dict(syn.default_model3(), G=G_GEN)):
        x = rounded(np.random.default_rng(nx).normal(size=(nz, ny, nx)), dt)
        want = orc.conv3(g, orc.conv_kernel3(m, g), x)
        assert rel_l2(host(api.mpi_conv3(m, g, dev(x, dt))), want) <= tol(dt)
    assert rel_l2(host(api.mpi_denoise_gaussian5_3d(dev(x, dt))), orc.gaussian5_3d(x)) <= tol(dt)


def _pnp3_oracle(orc, m, g, r, v, s, n_it, n_cg, nu0):
    shape = (g["nz"], g["ny"], g["nx"])
    return orc.pnp(lambda x: orc.forward3(m, g, r, v, x), lambda y: orc.adjoint3(m, g, r, v, y), s,
                   shape, n_it, n_cg, nu0, denoise=lambda x, sig: orc.gaussian5_3d(x))


@pytest.mark.parametrize("dt", DTYPES)
def test_pnp3_forward(orc, dt):
    cfg = syn.small3(12, 10, 6, 1200, seed=5)
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    s = rounded(syn.add_noise(orc.forward3(m, g, r, v, c), 0.01, 31), dt)
    nu0 = 1e-3 * orc.frob2_3(m, g, r, v) / c.size
    want = _pnp3_oracle(orc, m, g, r, v, s, 3, 4, nu0)
    got = api.mpi_pnp_solve3(m, g, dev(r, dt), dev(v, dt), dev(s, dt), 3, 4, nu0)
    assert rel_l2(host(got), want) <= tol(dt)


def test_pnp3_conv_and_callback(orc):
    dt = torch.float64
    g = syn.box_grid3(9, 8, 5)
    m = syn.default_model3()
    u = np.random.default_rng(6).normal(size=(5, 8, 9)) + 1.0
    kern = orc.conv_kernel3(m, g)
    op = lambda x: orc.conv3(g, kern, x)  # noqa: E731
    want = orc.pnp(op, op, u, (5, 8, 9), 3, 4, 0.05, denoise=lambda x, sig: orc.gaussian5_3d(x))
    got = api.mpi_pnp_solve3(m, g, None, None, dev(u, dt), 3, 4, 0.05, op=api.MPI_OP_CONV)
    assert rel_l2(host(got), want) <= tol(dt)
    seen = []

    def den(tin, tout, tsig):
        seen.append(tin.shape)
        tout.copy_(0.5 * tin)
    want_cb = orc.pnp(op, op, u, (5, 8, 9), 2, 3, 0.05, denoise=lambda x, sig: 0.5 * x)
    got_cb = api.mpi_pnp_solve3(m, g, None, None, dev(u, dt), 2, 3, 0.05, op=api.MPI_OP_CONV,
                                denoise=den)
    assert seen == [(5, 8, 9)] * 2
    assert rel_l2(host(got_cb), want_cb) <= tol(dt)


def test_bad_arguments3():
    g = syn.box_grid3(4, 3, 2)
    r = torch.zeros((5, 3), dtype=torch.float32, device="cuda")
    c = torch.zeros((2, 3, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(api.MPIError):
        api.mpi_forward3(dict(syn.default_model3(), G=[[0.0] * 3] * 3), g, r, r, c)
    with pytest.raises(api.MPIError):
        api.mpi_forward3(syn.default_model3(), dict(g, nz=0), r, r, c)
    with pytest.raises(ValueError):
        api.mpi_forward3(syn.default_model3(), g, r[:, :2].contiguous(), r[:, :2].contiguous(), c)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(24, 20, 18), (65, 9, 16)])
def test_conv3_fft_route(orc, dt, shape):
    """Volumes of 8192 voxels and more (FP32; 512 in FP64) take the FFT
    route: the same linear 3-D convolution as the oracle's direct sum."""
    nx, ny, nz = shape
    g = syn.box_grid3(nx, ny, nz)
    for m in (syn.default_model3(), dict(syn.default_model3(), G=G_GEN)):
        x = rounded(np.random.default_rng(nx * ny).normal(size=(nz, ny, nx)), dt)
        want = orc.conv3(g, orc.conv_kernel3(m, g), x)
        assert rel_l2(host(api.mpi_conv3(m, g, dev(x, dt))), want) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(48, 48, 24), (100, 90, 1), (3, 3, 1100)])
def test_conv3_fft_route_sizes(orc, dt, shape):
    """The five-launch route on the 3-D workload's 48 x 48 x 24 volume, and
    volumes past its size rule (one plane; 1100 planes, 4096-point z
    transforms) on the multi-pass route: every output against the oracle."""
    nx, ny, nz = shape
    g = syn.box_grid3(nx, ny, nz)
    m = dict(syn.default_model3(), G=G_GEN)
    x = rounded(np.random.default_rng(nx + 7 * nz).normal(size=(nz, ny, nx)), dt)
    want = orc.conv3(g, orc.conv_kernel3(m, g), x)
    assert rel_l2(host(api.mpi_conv3(m, g, dev(x, dt))), want) <= tol(dt)


def test_pnp3_conv_fft_route(orc):
    dt = torch.float32
    g = syn.box_grid3(24, 20, 18)
    m = syn.default_model3()
    u = rounded(np.random.default_rng(13).normal(size=(18, 20, 24)) + 1.0, dt)
    kern = orc.conv_kernel3(m, g)
    op = lambda x: orc.conv3(g, kern, x)  # noqa: E731
    want = orc.pnp(op, op, u, (18, 20, 24), 2, 3, 0.05, denoise=lambda x, sig: orc.gaussian5_3d(x))
    got = api.mpi_pnp_solve3(m, g, None, None, dev(u, dt), 2, 3, 0.05, op=api.MPI_OP_CONV)
    assert rel_l2(host(got), want) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(9, 7, 5), (24, 20, 18)])
def test_conv3_weighted_trace_kernel(orc, dt, shape):
    """mpi_conv3_kernel(kernel = 1): the convolution with beta tr K(beta G y)
    on the direct and the FFT route, for the traceless default gradient and a
    general one."""
    nx, ny, nz = shape
    g = syn.box_grid3(nx, ny, nz)
    for m in (syn.default_model3(), dict(syn.default_model3(), G=G_GEN)):
        x = rounded(np.random.default_rng(nx + 1).normal(size=(nz, ny, nx)), dt)
        want = orc.conv3(g, orc.conv_kernel3_trK(m, g), x)
        assert rel_l2(host(api.mpi_conv3_kernel(m, g, 1, dev(x, dt))), want) <= tol(dt)
        want0 = orc.conv3(g, orc.conv_kernel3(m, g), x)
        assert rel_l2(host(api.mpi_conv3_kernel(m, g, 0, dev(x, dt))), want0) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
def test_weighted_trace3(orc, dt):
    g = syn.box_grid3(7, 6, 5)
    for m in (syn.default_model3(), dict(syn.default_model3(), G=G_GEN)):
        A = rounded(np.random.default_rng(3).normal(size=(9, 5, 6, 7)), dt)
        want = orc.weighted_trace3(m, A)
        assert rel_l2(host(api.mpi_weighted_trace3(m, g, dev(A, dt))), want) <= tol(dt)


def test_pnp3_conv_weighted_trace_kernel(orc):
    """PnP with kernel = 1 convolves with beta tr K(beta G y).  That kernel is
    ~1e3 times the traceless trace kernel, so nu0 = 0.05 leaves C^T C + nu I
    badly conditioned: at 3 x 4 steps the oracle's own one-ulp spread is
    6.5e-13 and a GB300 run differed by 4.8e-12.  At 2 x 2 steps the spread is
    1e-15, and the strict FP64 bar applies."""
    dt = torch.float64
    g = syn.box_grid3(9, 8, 5)
    m = syn.default_model3()
    u = np.random.default_rng(7).normal(size=(5, 8, 9)) + 1.0
    kern = orc.conv_kernel3_trK(m, g)
    op = lambda x: orc.conv3(g, kern, x)  # noqa: E731
    want = orc.pnp(op, op, u, (5, 8, 9), 2, 2, 0.05, denoise=lambda x, sig: orc.gaussian5_3d(x))
    got = api.mpi_pnp_solve3(m, g, None, None, dev(u, dt), 2, 2, 0.05, op=api.MPI_OP_CONV, kernel=1)
    assert rel_l2(host(got), want) <= tol(dt)

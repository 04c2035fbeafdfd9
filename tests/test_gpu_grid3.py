"""GPU parity of the three-dimensional Core Stage (Eq. first:step with
n = 3): tensor-product cosine interpolation, its transpose and the CG solve
for the 9 (or, one channel measured, 3) components, against the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_2505_22797_gb300 import api
from paper_2505_22797_gb300 import synthetic as syn
from tests.gpu_util import dev, host, rel_l2, rounded, tol

pytestmark = pytest.mark.gpu
DTYPES = [torch.float32, torch.float64]


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(1, 1, 1, 7), (2, 3, 1, 40), (5, 4, 3, 300), (17, 13, 6, 3001),
                                   (48, 48, 24, 65536)])
def test_interp3_and_transpose(orc, dt, shape):
    """Several blocks of samples with a ragged tail; the Lissajous reaches
    past the outer voxel centres, so positions clamp to the node hull; the
    last shape is the 3-D FFP workload (48 x 48 x 24, 65 536 samples)."""
    nx, ny, nz, T = shape
    g = syn.box_grid3(nx, ny, nz)
    rng = np.random.default_rng(nx * 7 + nz + T)
    r, v = syn.lissajous3(T, 17, 16, 15)
    r, v = rounded(r, dt), rounded(v, dt)
    A = rounded(rng.normal(size=(9, nz, ny, nx)), dt)
    s = rounded(rng.normal(size=(3, T)), dt)
    assert rel_l2(host(api.mpi_interp3(g, dev(r, dt), dev(v, dt), dev(A, dt))),
                  orc.interp3(g, r, v, A)) <= tol(dt)
    assert rel_l2(host(api.mpi_interp3_adjoint(g, dev(r, dt), dev(v, dt), dev(s, dt))),
                  orc.interp3_T(g, r, v, s)) <= tol(dt)


def test_interp3_T_dense_cell(orc):
    """Thousands of samples in one cell: long per-cell lists, many work units
    per node, ordered combine; matches the FP64 sums."""
    dt = torch.float64
    g = syn.box_grid3(6, 5, 4)
    T = 6000
    rng = np.random.default_rng(1)
    r = np.stack([0.5 + 0.2 * rng.uniform(size=T), -0.4 + 0.2 * rng.uniform(size=T),
                  0.3 + 0.2 * rng.uniform(size=T)], 1)
    v = rng.normal(size=(T, 3))
    s = rng.normal(size=(3, T))
    assert rel_l2(host(api.mpi_interp3_adjoint(g, dev(r, dt), dev(v, dt), dev(s, dt))),
                  orc.interp3_T(g, r, v, s)) <= tol(dt)


def test_interp3_transpose_is_deterministic():
    g = syn.box_grid3(20, 18, 9)
    r, v = syn.lissajous3(20000, 17, 16, 15)
    s = np.random.default_rng(2).normal(size=(3, 20000))
    dt = torch.float32
    a = host(api.mpi_interp3_adjoint(g, dev(r, dt), dev(v, dt), dev(s, dt)))
    b = host(api.mpi_interp3_adjoint(g, dev(r, dt), dev(v, dt), dev(s, dt)))
    assert np.array_equal(a, b)


def test_interp3_empty_trajectory():
    g = syn.box_grid3(4, 3, 2)
    z = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    A = api.mpi_interp3_adjoint(g, z, z, torch.zeros((3, 0), dtype=torch.float64, device="cuda"))
    assert host(A).shape == (9, 2, 3, 4) and not host(A).any()
    Ahat, u = api.mpi_grid3(g, z, z, torch.zeros((3, 0), dtype=torch.float64, device="cuda"),
                            gamma=1e-3, max_iter=5, rel_tol=0.0)
    assert not host(Ahat).any() and not host(u).any()


def _signal3(orc, cfg, dt):
    g, m = cfg["grid"], cfg["model"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    return g, r, v, rounded(orc.forward3(m, g, r, v, c), dt)


@pytest.mark.parametrize("dt", DTYPES)
def test_core_stage3_fixed_iterations(orc, dt):
    cfg = syn.small3(14, 12, 6, 3000, seed=5)
    g, r, v, s = _signal3(orc, cfg, dt)
    gamma = 1e-4
    want, want_u, hist = orc.core_stage3(g, r, v, s, gamma, max_iter=25)
    A, u, n = api.mpi_grid3(g, dev(r, dt), dev(v, dt), dev(s, dt), gamma=gamma, max_iter=25,
                            rel_tol=0.0, return_iters=True)
    assert A.shape == (9, 6, 12, 14)
    assert n == len(hist) - 1
    assert rel_l2(host(A), want) <= tol(dt)
    assert rel_l2(host(u), want_u) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", [0, 1, 2])
def test_core_stage3_single_channel(orc, dt, k):
    """Only channel k measured: the row (A_k0, A_k1, A_k2) and A_kk after a
    fixed number of CG steps match the oracle's single-channel solve."""
    cfg = syn.small3(11, 10, 5, 1800, seed=11 + k)
    g, r, v, s = _signal3(orc, cfg, dt)
    gamma = 1e-4
    want, want_kk, hist = orc.core_stage3(g, r, v, s[k], gamma, max_iter=20, channel=k)
    A, akk, n = api.mpi_grid3(g, dev(r, dt), dev(v, dt), dev(s[k], dt), gamma=gamma, max_iter=20,
                              rel_tol=0.0, return_iters=True, channel=k)
    assert A.shape == (3, 5, 10, 11)
    assert n == len(hist) - 1
    assert rel_l2(host(A), want) <= tol(dt)
    assert rel_l2(host(akk), want_kk) <= tol(dt)


def test_core_stage3_tolerance_fp64(orc):
    """The paper's parameters (gamma = 1e-7, rel. tol 1e-3) in FP64: the same
    stopping step as the oracle, and the trace within the oracle's own
    sensitivity to one-ulp data perturbations (times 20, never below the
    1e-12 bar)."""
    dt = torch.float64
    cfg = syn.small3(16, 16, 8, 4000, seed=3)
    g, r, v, s = _signal3(orc, cfg, dt)
    want, want_u, hist = orc.core_stage3(g, r, v, s, 1e-7, max_iter=10000, rel_tol=1e-3)
    ulp = np.random.default_rng(0).choice([-1.0, 1.0], size=s.shape) * np.spacing(np.abs(s))
    _, pert_u, hist_p = orc.core_stage3(g, r, v, s + ulp, 1e-7, max_iter=10000, rel_tol=1e-3)
    assert len(hist_p) == len(hist)
    bound = max(1e-12, 20 * rel_l2(pert_u, want_u))
    _, u, n = api.mpi_grid3(g, dev(r, dt), dev(v, dt), dev(s, dt), gamma=1e-7, max_iter=10000,
                            rel_tol=1e-3, return_iters=True)
    assert n == len(hist) - 1
    err = rel_l2(host(u), want_u)
    print(f"3-D core stage gamma=1e-7: {n} CG steps, rel-L2 {err:.2e}, bound {bound:.2e}")
    assert err <= bound


def test_core_stage3_full_size_fp32(orc):
    """The 3-D FFP workload's geometry (48 x 48 x 24 voxels, 65 536 samples,
    three channels): 20 CG steps of the FP32 operator against the oracle.
    The data are the oracle's measurement of a smooth 9-component field
    (Gaussian bumps) with 1 % noise: a realistic signal at a fraction of the
    cost of the 3-D forward model on the CPU."""
    dt = torch.float32
    cfg = syn.config3("3d")
    g = cfg["grid"]
    r, v = rounded(cfg["r"], dt), rounded(cfg["v"], dt)
    zs, ys, xs = np.meshgrid(*[np.linspace(-1, 1, n) for n in (g["nz"], g["ny"], g["nx"])], indexing="ij")
    rng = np.random.default_rng(12)
    A_true = np.stack([np.exp(-((xs - a) ** 2 + (ys - b) ** 2 + (zs - c) ** 2) / 0.3)
                       for a, b, c in rng.uniform(-0.5, 0.5, size=(9, 3))])
    s = orc.interp3(g, r, v, A_true)
    s = rounded(s + 0.01 * np.abs(s).max() * rng.normal(size=s.shape), dt)
    want, want_u, hist = orc.core_stage3(g, r, v, s, 1e-7, max_iter=20)
    A, u, n = api.mpi_grid3(g, dev(r, dt), dev(v, dt), dev(s, dt), gamma=1e-7, max_iter=20,
                            rel_tol=0.0, return_iters=True)
    assert n == 20
    assert rel_l2(host(A), want) <= tol(dt)
    assert rel_l2(host(u), want_u) <= tol(dt)


def test_core_stage3_rejects_bad_arguments():
    g = syn.box_grid3(4, 4, 2)
    r = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    s = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(api.MPIError):
        api.mpi_grid3(g, r, r, s, max_iter=1, channel=3)
    with pytest.raises(api.MPIError):
        api.mpi_grid3(g, r, r, torch.zeros((3, 3), dtype=torch.float64, device="cuda"), gamma=-1.0)
    with pytest.raises(api.MPIError):
        api.mpi_interp3({**g, "dz": 0.0}, r, r, torch.zeros((9, 2, 4, 4), dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("dt", DTYPES)
def test_core_stage3_scaled_laplacian(orc, dt):
    """lap_scaled in three dimensions (1/dx^2, 1/dy^2, 1/dz^2 on a grid with
    dy != dx): fixed CG steps against the oracle's scaled 3-D Core Stage."""
    cfg = syn.small3(12, 10, 6, 2500, seed=7)
    g = cfg["grid"]
    assert g["dy"] != g["dx"]
    g, r, v, s = _signal3(orc, cfg, dt)
    want, want_u, hist = orc.core_stage3(g, r, v, s, 1e-3, max_iter=20, lap="scaled")
    A, u, n = api.mpi_grid3(g, dev(r, dt), dev(v, dt), dev(s, dt), gamma=1e-3, max_iter=20, rel_tol=0.0,
                            return_iters=True, lap_scaled=True)
    assert n == len(hist) - 1
    assert rel_l2(host(A), want) <= tol(dt)
    assert rel_l2(host(u), want_u) <= tol(dt)

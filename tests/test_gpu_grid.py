"""GPU parity of the Core Stage: cosine interpolation, its transpose and the
CG solve of Eq. first:step, against the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_2505_22797_gb300 import api
from paper_2505_22797_gb300 import synthetic as syn
from tests.gpu_util import dev, host, rel_l2, rounded, tol

pytestmark = pytest.mark.gpu
DTYPES = [torch.float32, torch.float64]


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(1, 1, 7), (1, 9, 300), (11, 1, 300), (2, 3, 40), (17, 13, 700),
                                   (64, 64, 8192)])
def test_interp_and_transpose(orc, dt, shape):
    nx, ny, T = shape
    g = syn.square_grid(nx, 24.0, ny)
    rng = np.random.default_rng(nx * 7 + T)
    r, v = syn.lissajous(T, 5, 4, amp=13.0)  # overshoots the node hull: clamping
    r, v = rounded(r, dt), rounded(v, dt)
    A = rounded(rng.normal(size=(4, ny, nx)), dt)
    s = rounded(rng.normal(size=(2, T)), dt)
    assert rel_l2(host(api.mpi_interp(g, dev(r, dt), dev(v, dt), dev(A, dt))),
                  orc.interp(g, r, v, A)) <= tol(dt)
    assert rel_l2(host(api.mpi_interp_adjoint(g, dev(r, dt), dev(v, dt), dev(s, dt))),
                  orc.interp_T(g, r, v, s)) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
def test_interp_T_dense_cell(dt):
    """Thousands of samples in one cell (a trajectory that dwells): the
    cell's run spans many work units; result matches FP64 sums."""
    g = syn.square_grid(8, 8.0)
    T = 5000
    rng = np.random.default_rng(0)
    r = rounded(0.3 + 0.1 * rng.uniform(size=(T, 2)), dt)
    v = rounded(rng.normal(size=(T, 2)), dt)
    s = rounded(rng.normal(size=(2, T)), dt)
    from oracle import oracle as orc
    assert rel_l2(host(api.mpi_interp_adjoint(g, dev(r, dt), dev(v, dt), dev(s, dt))),
                  orc.interp_T(g, r, v, s)) <= tol(dt)


@pytest.mark.parametrize("T, n_cells, run", [(0, 1, 1), (1, 1, 1), (3000, 1, 1), (2047, 5, 9),
                                             (2049, 255, 3), (5000, 256, 40), (9001, 70000, 12),
                                             (1 << 20, 511 * 511, 30), (1 << 20, 47 * 47 * 23, 2000)])
def test_cell_order_stable(T, n_cells, run):
    """The binning step on its own: bit-equal to a stable sort by cell (zero
    to three radix passes, a ragged last tile, runs of one cell as a
    trajectory leaves them, up to thousands long) and run offsets equal to
    the cumulative cell counts."""
    rng = np.random.default_rng(T + n_cells + run)
    lengths = rng.integers(1, run + 1, size=T + 1)
    keys = np.repeat(rng.integers(0, n_cells, size=T + 1), lengths)[:T].astype(np.int32)
    lst, off = api.mpi_cell_order(torch.from_numpy(keys).cuda(), n_cells)
    torch.cuda.synchronize()
    assert np.array_equal(lst.cpu().numpy(), np.argsort(keys, kind="stable"))
    want = np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=n_cells))])
    assert np.array_equal(off.cpu().numpy(), want)
    lst2, none = api.mpi_cell_order(torch.from_numpy(keys).cuda(), n_cells, with_offset=False)
    assert none is None and torch.equal(lst2, lst)


def test_core_stage_full_size_fp32(orc):
    """The 512 x 512 / 2^20-sample geometry (cells of up to ~1900 samples,
    each spread over many work units of the one-pass normal product): 20 CG
    steps of the FP32 solve against the oracle.  The data are the oracle's
    measurement of a smooth 4-component field with 1 % noise."""
    dt = torch.float32
    cfg = syn.config("c5")
    g = cfg["grid"]
    r, v = rounded(cfg["r"], dt), rounded(cfg["v"], dt)
    ys, xs = np.meshgrid(*[np.linspace(-1, 1, n) for n in (g["ny"], g["nx"])], indexing="ij")
    rng = np.random.default_rng(21)
    A_true = np.stack([np.exp(-((xs - a) ** 2 + (ys - b) ** 2) / 0.2) for a, b in rng.uniform(-0.5, 0.5, (4, 2))])
    s = orc.interp(g, r, v, A_true)
    s = rounded(s + 0.01 * np.abs(s).max() * rng.normal(size=s.shape), dt)
    want, want_u, _ = orc.core_stage(g, r, v, s, 1e-7, max_iter=20)
    A, u, n = api.mpi_grid(g, dev(r, dt), dev(v, dt), dev(s, dt), gamma=1e-7, max_iter=20, rel_tol=0.0,
                           return_iters=True)
    assert n == 20
    assert rel_l2(host(A), want) <= tol(dt)
    assert rel_l2(host(u), want_u) <= tol(dt)


def test_cell_order_rejects_bad_arguments():
    keys = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(api.MPIError):
        api.mpi_cell_order(keys, 0)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("steps", [30, 37])
def test_core_stage_fixed_iterations(orc, dt, steps):
    """Fixed CG step counts: 30 steps run step by step; 37 run as two
    replays of the 16-step graph and 5 more steps."""
    cfg = syn.small(20, 18, 2000, seed=5)
    g, m = cfg["grid"], cfg["model"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    s = rounded(orc.forward(m, g, r, v, c), dt)
    gamma = 1e-4
    want, want_u, hist = orc.core_stage(g, r, v, s, gamma, max_iter=steps)
    A, u, n = api.mpi_grid(g, dev(r, dt), dev(v, dt), dev(s, dt), gamma=gamma, max_iter=steps,
                           rel_tol=0.0, return_iters=True)
    assert n == len(hist) - 1
    assert rel_l2(host(A), want) <= tol(dt)
    assert rel_l2(host(u), want_u) <= tol(dt)


def test_core_stage_tolerance_fp64(orc):
    """Paper parameters (gamma = 1e-7, rel. tol 1e-3): same stopping step as
    the oracle's textbook loop, and the same result to within the problem's
    own round-off sensitivity.  With gamma = 1e-7 the normal matrix is badly
    conditioned, so CG amplifies rounding-order differences; the bound is
    taken from the oracle itself: the spread of its result when the data are
    perturbed by one unit in the last place, times 20 (and never below the
    1e-12 FP64 bar)."""
    dt = torch.float64
    cfg = syn.config("c1")
    g, m = cfg["grid"], cfg["model"]
    r, v, c = cfg["r"], cfg["v"], cfg["c"]
    s = orc.forward(m, g, r, v, c)
    want, want_u, hist = orc.core_stage(g, r, v, s, 1e-7, max_iter=10000, rel_tol=1e-3)
    ulp = np.random.default_rng(0).choice([-1.0, 1.0], size=s.shape) * np.spacing(np.abs(s))
    _, pert_u, hist_p = orc.core_stage(g, r, v, s + ulp, 1e-7, max_iter=10000, rel_tol=1e-3)
    assert len(hist_p) == len(hist)
    bound = max(1e-12, 20 * rel_l2(pert_u, want_u))
    A, u, n = api.mpi_grid(g, dev(r, dt), dev(v, dt), dev(s, dt), gamma=1e-7, max_iter=10000,
                           rel_tol=1e-3, return_iters=True)
    assert n == len(hist) - 1
    err = rel_l2(host(u), want_u)
    print(f"core stage gamma=1e-7: {n} CG steps, rel-L2 {err:.2e}, sensitivity bound {bound:.2e}")
    assert err <= bound


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", [0, 1])
def test_core_stage_single_channel(orc, dt, k):
    """Sec. 3.6: only channel k measured.  The two components (A_k0, A_k1)
    and the diagonal A_kk after a fixed number of CG steps match the oracle's
    single-channel Core Stage."""
    cfg = syn.small(19, 17, 1500, seed=11 + k)
    g, m = cfg["grid"], cfg["model"]
    r, v, c = (rounded(cfg[key], dt) for key in ("r", "v", "c"))
    s_k = rounded(orc.forward(m, g, r, v, c)[k], dt)
    gamma = 1e-4
    want, want_kk, hist = orc.core_stage_channel(g, r, v, s_k, k, gamma, max_iter=25)
    A, akk, n = api.mpi_grid(g, dev(r, dt), dev(v, dt), dev(s_k, dt), gamma=gamma, max_iter=25,
                             rel_tol=0.0, return_iters=True, channel=k)
    assert A.shape == (2, 17, 19)
    assert n == len(hist) - 1
    assert rel_l2(host(A), want) <= tol(dt)
    assert rel_l2(host(akk), want_kk) <= tol(dt)


def test_core_stage_single_channel_tolerance(orc):
    """Single channel at the paper's parameters (gamma = 1e-7, rel. tol 1e-3),
    FP64: same stopping step as the oracle; result within the oracle's own
    one-ulp sensitivity (times 20, never below the 1e-12 bar)."""
    dt = torch.float64
    cfg = syn.small(24, 24, 3000, seed=21)
    g, m = cfg["grid"], cfg["model"]
    r, v, c = cfg["r"], cfg["v"], cfg["c"]
    s_k = orc.forward(m, g, r, v, c)[0]
    want, want_kk, hist = orc.core_stage_channel(g, r, v, s_k, 0, 1e-7, 10000, rel_tol=1e-3)
    ulp = np.random.default_rng(1).choice([-1.0, 1.0], size=s_k.shape) * np.spacing(np.abs(s_k))
    _, pert_kk, hist_p = orc.core_stage_channel(g, r, v, s_k + ulp, 0, 1e-7, 10000, rel_tol=1e-3)
    assert len(hist_p) == len(hist)
    bound = max(1e-12, 20 * rel_l2(pert_kk, want_kk))
    _, akk, n = api.mpi_grid(g, dev(r, dt), dev(v, dt), dev(s_k, dt), gamma=1e-7, max_iter=10000,
                             rel_tol=1e-3, return_iters=True, channel=0)
    assert n == len(hist) - 1
    assert rel_l2(host(akk), want_kk) <= bound


def test_core_stage_channel_rejects_bad_selector():
    g = syn.square_grid(4, 8.0)
    r = torch.zeros((3, 2), dtype=torch.float64, device="cuda")
    s = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(api.MPIError):
        api.mpi_grid(g, r, r, s, max_iter=1, channel=2)


@pytest.mark.parametrize("dt", DTYPES)
def test_core_stage_scaled_laplacian(orc, dt):
    """lap_scaled: the regulariser is the Laplacian with 1/dx^2, 1/dy^2 (an
    anisotropic grid here); fixed CG steps against the oracle's scaled Core
    Stage."""
    cfg = syn.small(20, 14, 2000, seed=6)
    g, m = cfg["grid"], cfg["model"]
    assert g["dx"] != g["dy"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    s = rounded(orc.forward(m, g, r, v, c), dt)
    want, want_u, hist = orc.core_stage(g, r, v, s, 1e-3, max_iter=30, lap="scaled")
    A, u, n = api.mpi_grid(g, dev(r, dt), dev(v, dt), dev(s, dt), gamma=1e-3, max_iter=30, rel_tol=0.0,
                           return_iters=True, lap_scaled=True)
    assert n == len(hist) - 1
    assert rel_l2(host(A), want) <= tol(dt)
    assert rel_l2(host(u), want_u) <= tol(dt)

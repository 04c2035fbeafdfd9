"""GPU parity of the pair operators (forward A, adjoint A^T, d/dbeta) against
the FP64 oracle, through the C ABI, on seeded synthetic inputs: small cases
spanning several work items with ragged tails, edge cases, and the full-size
workloads (all outputs where the oracle is fast enough, seeded samples of
outputs elsewhere)."""
import numpy as np
import pytest
import torch

from paper_2505_22797_gb300 import api
from paper_2505_22797_gb300 import synthetic as syn
from tests.gpu_util import dev, host, rel_l2, rounded, tol

pytestmark = pytest.mark.gpu
DTYPES = [torch.float32, torch.float64]


def _case(nx, ny, T, traj="lissajous", seed=7, G=None, p=None):
    cfg = syn.small(nx, ny, T, traj, seed)
    if G is not None:
        cfg["model"] = dict(cfg["model"], G=G)
    if p is not None:
        cfg["model"] = dict(cfg["model"], p=p)
    return cfg


CASES = [
    dict(nx=37, ny=29, T=777),                          # ragged in every direction
    dict(nx=32, ny=32, T=1632),                         # exact tiles
    dict(nx=64, ny=48, T=3000, traj="spiral"),
    dict(nx=33, ny=65, T=2049, G=[[2.1e-3, 4e-4], [3e-4, -2.6e-3]]),   # non-diagonal G
    dict(nx=20, ny=17, T=515, p=[[0.6, 0.8]]),          # one channel
    dict(nx=1, ny=1, T=5),
    dict(nx=7, ny=1, T=1),
]


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(str(c[k]) for k in ("nx", "ny", "T")))
def test_forward_adjoint_small(orc, dt, case):
    cfg = _case(**case)
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    want = orc.forward(m, g, r, v, c)
    got = host(api.mpi_forward(m, g, dev(r, dt), dev(v, dt), dev(c, dt)))
    assert rel_l2(got, want) <= tol(dt)
    s = rounded(np.random.default_rng(3).normal(size=want.shape), dt)
    want_g = orc.adjoint(m, g, r, v, s)
    got_g = host(api.mpi_adjoint(m, g, dev(r, dt), dev(v, dt), dev(s, dt)))
    assert rel_l2(got_g, want_g) <= tol(dt)


@pytest.mark.parametrize("shift", [60.0, 0.6])
def test_packed_asymptotic_tiers(orc, shift):
    """FP32 on a ragged grid with the trajectory moved sideways: far (every
    pair in the packed asymptotic tiers of the forward row loop and the
    adjoint's sample groups, the last group partial) and near the grid's edge
    (asymptotic, closed-form and mixed segments and groups side by side)."""
    dt = torch.float32
    cfg = _case(37, 29, 1001, "spiral", seed=11)
    m, g = cfg["model"], cfg["grid"]
    r = rounded(cfg["r"] + np.array([shift * 12.0, 0.0]), dt)
    v, c = (rounded(cfg[k], dt) for k in ("v", "c"))
    want = orc.forward(m, g, r, v, c)
    got = host(api.mpi_forward(m, g, dev(r, dt), dev(v, dt), dev(c, dt)))
    assert rel_l2(got, want) <= tol(dt)
    s = rounded(np.random.default_rng(8).normal(size=want.shape), dt)
    want_g = orc.adjoint(m, g, r, v, s)
    got_g = host(api.mpi_adjoint(m, g, dev(r, dt), dev(v, dt), dev(s, dt)))
    assert rel_l2(got_g, want_g) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
def test_dbeta_small(orc, dt):
    cfg = _case(41, 23, 1500, "spiral")
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    gs = rounded(np.random.default_rng(5).normal(size=(2, 1500)), dt)
    want = orc.dbeta(m, g, r, v, c, gs)
    got = float(host(api.mpi_dbeta(m, g, dev(r, dt), dev(v, dt), dev(c, dt), dev(gs, dt))))
    assert abs(got - want) <= tol(dt) * abs(want)


@pytest.mark.parametrize("dt", DTYPES)
def test_empty_trajectory(dt):
    cfg = _case(9, 8, 10)
    m, g = cfg["model"], cfg["grid"]
    z = torch.zeros((0, 2), dtype=dt, device="cuda")
    s = api.mpi_forward(m, g, z, z, dev(cfg["c"], dt))
    assert s.shape == (2, 0)
    out = torch.full((8, 9), 7.0, dtype=dt, device="cuda")
    api.mpi_adjoint(m, g, z, z, torch.zeros((2, 0), dtype=dt, device="cuda"), c_out=out)
    assert float(host(out).max()) == 0.0 and float(host(out).min()) == 0.0
    d = api.mpi_dbeta(m, g, z, z, dev(cfg["c"], dt), torch.zeros((2, 0), dtype=dt, device="cuda"))
    assert float(host(d)) == 0.0


def test_invalid_arguments_rejected_before_launch():
    cfg = _case(9, 8, 10)
    r, v, c = (dev(cfg[k], torch.float32) for k in ("r", "v", "c"))
    bad = dict(cfg["model"], beta=-1.0)
    with pytest.raises(api.MPIError) as e:
        api.mpi_forward(bad, cfg["grid"], r, v, c)
    assert e.value.status == api.MPI_ERR_INVALID
    bad_g = dict(cfg["grid"], nx=0)
    with pytest.raises(api.MPIError):
        api.mpi_adjoint(cfg["model"], bad_g, r, v, torch.zeros((2, 10), device="cuda"))
    sing = dict(cfg["model"], G=[[1.0, 2.0], [2.0, 4.0]])
    with pytest.raises(api.MPIError):
        api.mpi_forward(sing, cfg["grid"], r, v, c)


def test_deterministic_fp32():
    cfg = syn.config("c1")
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (dev(cfg[k], torch.float32) for k in ("r", "v", "c"))
    a = host(api.mpi_forward(m, g, r, v, c))
    b = host(api.mpi_forward(m, g, r, v, c))
    assert np.array_equal(a, b)
    s = dev(a, torch.float32)
    assert np.array_equal(host(api.mpi_adjoint(m, g, r, v, s)), host(api.mpi_adjoint(m, g, r, v, s)))


@pytest.mark.parametrize("dt", DTYPES)
def test_c1_full(orc, dt):
    """32x32 Lissajous workload, every output."""
    cfg = syn.config("c1")
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    want = orc.forward(m, g, r, v, c)
    got = host(api.mpi_forward(m, g, dev(r, dt), dev(v, dt), dev(c, dt)))
    assert rel_l2(got, want) <= tol(dt)
    s = rounded(want, dt)
    assert rel_l2(host(api.mpi_adjoint(m, g, dev(r, dt), dev(v, dt), dev(s, dt))),
                  orc.adjoint(m, g, r, v, s)) <= tol(dt)


def test_c2_full_forward_and_sampled_adjoint(orc):
    """128x128 spiral workload, T = 65536, FP32: every output of A; A^T on a
    seeded sample of 256 voxels (each needs a full pass over the samples)."""
    dt = torch.float32
    cfg = syn.config("c2")
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    want = orc.forward(m, g, r, v, c)
    got = host(api.mpi_forward(m, g, dev(r, dt), dev(v, dt), dev(c, dt)))
    assert rel_l2(got, want) <= tol(dt)
    s = rounded(syn.add_noise(want, 0.01, 202), dt)
    sel = np.random.default_rng(11).choice(128 * 128, 256, replace=False)
    want_g = orc.adjoint(m, g, r, v, s, sel=sel)
    got_g = host(api.mpi_adjoint(m, g, dev(r, dt), dev(v, dt), dev(s, dt))).reshape(-1)[sel]
    assert rel_l2(got_g, want_g) <= tol(dt)


def test_c2_adjoint_identity_fp64():
    """<A c, s> = <c, A^T s> on the full 128x128 / 65536 workload (a property
    that holds at any size), FP64 on the GPU."""
    dt = torch.float64
    cfg = syn.config("c2")
    m, g = cfg["model"], cfg["grid"]
    r, v = dev(cfg["r"], dt), dev(cfg["v"], dt)
    rng = np.random.default_rng(12)
    c = dev(rng.normal(size=(128, 128)), dt)
    s = dev(rng.normal(size=(2, 65536)), dt)
    lhs = float(torch.sum(api.mpi_forward(m, g, r, v, c) * s))
    rhs = float(torch.sum(c * api.mpi_adjoint(m, g, r, v, s)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


def test_c5_sampled_rows(orc):
    """512x512 / 2^20-sample workload (FP32): 512 seeded samples of A
    (rows of s) and 64 seeded voxels of A^T against the oracle."""
    dt = torch.float32
    cfg = syn.config("c5")
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    got = host(api.mpi_forward(m, g, dev(r, dt), dev(v, dt), dev(c, dt)))
    rows = np.sort(np.random.default_rng(13).choice(r.shape[0], 512, replace=False))
    want = orc.forward(m, g, r[rows], v[rows], c)
    assert rel_l2(got[:, rows], want) <= tol(dt)
    s = rounded(np.random.default_rng(14).normal(size=got.shape) * np.abs(got).max(), dt)
    vox = np.random.default_rng(15).choice(512 * 512, 64, replace=False)
    got_g = host(api.mpi_adjoint(m, g, dev(r, dt), dev(v, dt), dev(s, dt))).reshape(-1)[vox]
    assert rel_l2(got_g, orc.adjoint(m, g, r, v, s, sel=vox)) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
def test_samples_on_voxel_centres(orc, dt):
    """Samples exactly on voxel centres (u = 0 for one pair each) and within a
    fraction of a voxel of them: the near-FFP series path of both kernels."""
    g = syn.square_grid(48, 24.0, 40)
    m = syn.default_model()
    xs, ys = syn.voxel_centres(g)
    rng = np.random.default_rng(31)
    ii, jj = rng.integers(0, 48, 600), rng.integers(0, 40, 600)
    jitter = rng.choice([0.0, 0.0, 0.01, 0.05, 0.2], size=(600, 2)) * rng.normal(size=(600, 2))
    r = rounded(np.stack([xs[ii], ys[jj]], 1) + jitter, dt)
    v = rounded(rng.normal(size=(600, 2)) * 0.05, dt)
    c = rounded(rng.uniform(size=(40, 48)), dt)
    want = orc.forward(m, g, r, v, c)
    assert rel_l2(host(api.mpi_forward(m, g, dev(r, dt), dev(v, dt), dev(c, dt))), want) <= tol(dt)
    s = rounded(rng.normal(size=(2, 600)), dt)
    assert rel_l2(host(api.mpi_adjoint(m, g, dev(r, dt), dev(v, dt), dev(s, dt))),
                  orc.adjoint(m, g, r, v, s)) <= tol(dt)

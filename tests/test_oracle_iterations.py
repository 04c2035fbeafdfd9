"""Pins for the oracle's iterations: CG, the percentile trimming, the noise
estimate, the built-in denoiser, the ZeroShot-PnP loop (Algorithm 1) and the
Core Stage solve (Eq. first:step)."""
import numpy as np
import pytest

from paper_2505_22797_gb300 import synthetic as syn


def test_cg_matches_dense_solve(orc):
    rng = np.random.default_rng(0)
    B = rng.normal(size=(8, 8))
    M = B @ B.T + 0.5 * np.eye(8)
    b = rng.normal(size=8)
    x, hist, n_app = orc.cg(lambda z: M @ z, b, np.zeros(8), 8)
    assert np.allclose(x, np.linalg.solve(M, b), rtol=1e-10, atol=1e-12)
    assert n_app == 9
    # A-norm of the error decreases monotonically
    xs = np.linalg.solve(M, b)
    errs = []
    for n in range(0, 8):
        xn, _, _ = orc.cg(lambda z: M @ z, b, np.zeros(8), n)
        errs.append((xn - xs) @ M @ (xn - xs))
    assert all(e2 <= e1 * (1 + 1e-12) for e1, e2 in zip(errs, errs[1:]))


def test_cg_rel_tol_and_zero_rhs(orc):
    M = np.diag([1.0, 2.0, 3.0])
    x, hist, n_app = orc.cg(lambda z: M @ z, np.zeros(3), np.zeros(3), 10)
    assert n_app == 1 and np.all(x == 0)
    b = np.array([1.0, 1.0, 1.0])
    x, hist, _ = orc.cg(lambda z: M @ z, b, np.zeros(3), 100, rel_tol=1e-3)
    assert hist[-1] <= 1e-3 * np.sqrt(3)
    assert len(hist) <= 4


@pytest.mark.parametrize("pct", [0.0, 5.0, 37.3, 100.0])
@pytest.mark.parametrize("n", [1, 2, 17, 1000])
def test_percentile_vs_numpy(orc, pct, n):
    x = np.random.default_rng(n).normal(size=n)
    assert abs(orc.percentile_value(x, pct) - np.percentile(x, pct)) <= 1e-15 * (1 + abs(np.percentile(x, pct)))
    got = orc.percentile_clamp(x, pct)
    assert np.array_equal(got, np.maximum(x, orc.percentile_value(x, pct)))


def test_variance_vs_numpy(orc):
    x = np.random.default_rng(1).normal(3.0, 2.0, size=5000)
    assert abs(orc.variance(x) - np.var(x)) < 1e-13 * np.var(x)
    assert orc.variance(np.full(7, 2.5)) == 0.0


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (5, 4), (32, 32), (17, 40)])
def test_gaussian5_vs_scipy(orc, shape):
    ndi = pytest.importorskip("scipy.ndimage")
    x = np.random.default_rng(2).normal(size=shape)
    want = ndi.gaussian_filter(x, sigma=1.0, truncate=2.0, mode="reflect")
    assert np.allclose(orc.gaussian5(x), want, rtol=1e-13, atol=1e-14)


def test_pnp_identity_operator_closed_form(orc):
    """With O = I, CG solves (1 + nu) x = d + nu rho2 in one step, so each
    iteration of Algorithm 1 has a closed form; run it with numpy/scipy
    routines and compare."""
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(4)
    d = rng.normal(size=(9, 7)) + 1.0
    nu0 = 0.3
    rec = []
    got = orc.pnp(lambda x: x, lambda x: x, d, (9, 7), n_it=4, n_cg=3, nu0=nu0,
                  clip_pct=5.0, record=rec)
    rho2 = np.zeros_like(d)
    nu, lam = nu0, None
    for k in range(4):
        rho1 = (d + nu * rho2) / (1 + nu)
        rho1 = np.maximum(rho1, np.percentile(rho1, 5.0))
        sig = np.sqrt(np.var(rho1))
        if k == 0:
            lam = nu0 * sig**2
        rho2 = ndi.gaussian_filter(rho1, 1.0, truncate=2.0, mode="reflect")
        nu = lam / sig**2
        assert abs(rec[k]["sigma"] - sig) < 1e-13
        assert abs(rec[k]["nu"] - nu) < 1e-13 * nu
    assert np.allclose(got, rho2, rtol=1e-12, atol=1e-13)
    # nu_1 = nu0 (Algorithm 1: lambda is fixed from the first sigma)
    assert abs(rec[0]["nu"] - nu0) < 1e-15


def test_pnp_no_clip_and_callback(orc):
    rng = np.random.default_rng(5)
    d = rng.normal(size=(4, 4))
    seen = []

    def den(img, sigma):
        seen.append(sigma)
        return img * 0.5
    out = orc.pnp(lambda x: 2 * x, lambda x: 2 * x, d, (4, 4), 2, 4, 0.1, clip_pct=-1,
                  denoise=den)
    # first iteration: (4 + nu0) rho1 = 2 d  (O^T O = 4 I), no clipping
    rho1 = 2 * d / 4.1
    assert abs(seen[0] - np.std(rho1)) < 1e-13
    assert out.shape == (4, 4) and len(seen) == 2


def test_core_stage_vs_dense_solve(orc):
    grid = syn.square_grid(5, 10.0, 4)
    rng = np.random.default_rng(3)
    T = 60
    r, v = syn.lissajous(T, 3, 2, amp=5.0)
    s = rng.normal(size=(2, T))
    gamma = 1e-2
    N = 20
    # dense normal matrix from unit vectors
    cols = []
    for k in range(4 * N):
        e = np.zeros(4 * N)
        e[k] = 1
        E = e.reshape(4, 4, 5)
        lap = np.stack([orc.laplacian(grid, orc.laplacian(grid, E[m])) for m in range(4)])
        cols.append((orc.interp_T(grid, r, v, orc.interp(grid, r, v, E)) / T + gamma * lap).reshape(-1))
    Mn = np.stack(cols, 1)
    assert np.allclose(Mn, Mn.T, atol=1e-12)
    b = (orc.interp_T(grid, r, v, s) / T).reshape(-1)
    want = np.linalg.solve(Mn, b)
    Ahat, u, hist = orc.core_stage(grid, r, v, s, gamma, max_iter=400)
    assert np.allclose(Ahat.reshape(-1), want, rtol=1e-7, atol=1e-9 * np.abs(want).max())
    assert np.allclose(u, Ahat[0] + Ahat[3])
    Ahat2, _, hist2 = orc.core_stage(grid, r, v, s, gamma, max_iter=10000, rel_tol=1e-3)
    assert hist2[-1] <= 1e-3 * np.linalg.norm(b) and len(hist2) < 400


@pytest.mark.parametrize("k", [0, 1])
def test_core_stage_single_channel_vs_dense_solve(orc, k):
    """Sec. 3.6: only channel k measured; the two components (A_k0, A_k1) from
    CG equal the dense normal-equation solution."""
    grid = syn.square_grid(5, 10.0, 4)
    rng = np.random.default_rng(7 + k)
    T = 70
    r, v = syn.lissajous(T, 3, 2, amp=5.0)
    s_k = rng.normal(size=T)
    gamma = 1e-2
    N = 20
    cols = []
    for q in range(2 * N):
        e = np.zeros(2 * N)
        e[q] = 1
        E = e.reshape(2, 4, 5)
        E4 = np.zeros((4, 4, 5))
        E4[2 * k:2 * k + 2] = E
        Ms = orc.interp(grid, r, v, E4)[k]
        s2 = np.zeros((2, T))
        s2[k] = Ms
        MtM = orc.interp_T(grid, r, v, s2)[2 * k:2 * k + 2] / T
        lap = np.stack([orc.laplacian(grid, orc.laplacian(grid, E[m])) for m in range(2)])
        cols.append((MtM + gamma * lap).reshape(-1))
    Mn = np.stack(cols, 1)
    s2 = np.zeros((2, T))
    s2[k] = s_k
    b = (orc.interp_T(grid, r, v, s2)[2 * k:2 * k + 2] / T).reshape(-1)
    want = np.linalg.solve(Mn, b)
    A, Akk, _ = orc.core_stage_channel(grid, r, v, s_k, k, gamma, max_iter=300)
    assert np.allclose(A.reshape(-1), want, rtol=1e-7, atol=1e-9 * np.abs(want).max())
    assert np.array_equal(Akk, A[k])

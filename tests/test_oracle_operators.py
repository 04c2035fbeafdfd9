"""Pins for the oracle's operators: the forward model A (sign, G, beta, v and
channel projection), its adjoint, d/dbeta, the cosine interpolation of the
Core Stage, the Laplacian and the sampled-kernel convolution.  Each check is
against something other than the oracle itself: mpmath derivatives of the
magnetisation, an FFT route, dense brute force, scipy routines, identities."""
import math

import numpy as np
import pytest

from paper_2505_22797_gb300 import synthetic as syn

mp = pytest.importorskip("mpmath")


@pytest.fixture(autouse=True)
def _mp_precision():
    """40 significant digits for every mpmath reference here, restored after."""
    with mp.workdps(40):
        yield


def _tiny(nx=4, ny=3, T=6, seed=0, G=None, p=None, beta=900.0, fov=6.0):
    rng = np.random.default_rng(seed)
    grid = {"nx": nx, "ny": ny, "x0": -fov / 2, "y0": -fov / 2 + 0.3,
            "dx": fov / nx, "dy": fov / ny * 0.9}
    model = {"beta": beta, "G": G if G is not None else [[2.5e-3, 0.0], [0.0, 2.5e-3]],
             "p": p if p is not None else [[1.0, 0.0], [0.0, 1.0]]}
    r = rng.uniform(-fov / 2, fov / 2, size=(T, 2))
    v = rng.normal(size=(T, 2)) * 0.1
    c = rng.uniform(0, 1, size=(ny, nx))
    return grid, model, r, v, c


def _mp_signal_integrand(model, grid, c, rt):
    """sum_x c_x p_k^T L(beta |H|) H/|H|, H = G(x - r(t)), in mpmath."""
    G = [[mp.mpf(g) for g in row] for row in model["G"]]
    beta = mp.mpf(model["beta"])
    P = model["p"]
    out = [mp.mpf(0)] * len(P)
    for j in range(grid["ny"]):
        for i in range(grid["nx"]):
            x = [mp.mpf(grid["x0"]) + (i + mp.mpf(0.5)) * mp.mpf(grid["dx"]),
                 mp.mpf(grid["y0"]) + (j + mp.mpf(0.5)) * mp.mpf(grid["dy"])]
            d = [x[0] - rt[0], x[1] - rt[1]]
            H = [G[0][0] * d[0] + G[0][1] * d[1], G[1][0] * d[0] + G[1][1] * d[1]]
            h = mp.sqrt(H[0] ** 2 + H[1] ** 2)
            z = beta * h
            L = mp.coth(z) - 1 / z
            for k in range(len(P)):
                out[k] += mp.mpf(c[j, i]) * L * (P[k][0] * H[0] + P[k][1] * H[1]) / h
    return out


@pytest.mark.parametrize("G", [[[2.5e-3, 0.0], [0.0, 2.5e-3]], [[-1e-3, 3e-4], [3e-4, 2e-3]]])
def test_forward_is_time_derivative_of_magnetisation(orc, G):
    """s_k(t) = -d/dt sum_x c_x p_k^T L(beta|H|) H/|H|, H = G(x - r(t))
    (Eq. signal and the time-derivative identity of Sec. 2 with dH/dt = -G r';
    the constant -mu0 m R is dropped as in Eq. core:formula, which leaves the
    minus sign of dH/dt).  Analytic Lissajous trajectory, mpmath derivative."""
    grid, model, _, _, c = _tiny(G=G)
    model["p"] = [[1.0, 0.0], [0.0, 1.0]]
    Ax, Ay, fx, fy = 2.5, 2.0, 0.013, 0.011

    def rr(t):
        return [Ax * mp.sin(2 * mp.pi * fx * t), Ay * mp.sin(2 * mp.pi * fy * t + mp.mpf(0.3))]

    ts = [3.0, 17.0, 40.0]
    r = np.array([[float(u) for u in rr(mp.mpf(t))] for t in ts])
    v = np.array([[float(Ax * 2 * mp.pi * fx * mp.cos(2 * mp.pi * fx * t)),
                   float(Ay * 2 * mp.pi * fy * mp.cos(2 * mp.pi * fy * t + mp.mpf(0.3)))]
                  for t in ts])
    s = orc.forward(model, grid, r, v, c)
    for q, t in enumerate(ts):
        for k in range(2):
            ref = -mp.diff(lambda tt: _mp_signal_integrand(model, grid, c, rr(tt))[k], mp.mpf(t))
            assert abs(s[k, q] - float(ref)) <= 1e-11 * max(1.0, abs(float(ref))), (t, k)


def test_forward_fft_route(orc):
    """With samples on voxel centres, A c = p_k^T [(Kmat * c)(r_t)] G v_t where
    Kmat(o) = beta K(beta G o) is sampled on all voxel offsets and the
    convolution runs through a zero-padded FFT (the double-convolution form of
    Eq. signal:noA)."""
    nx, ny = 7, 5
    grid, model, _, _, c = _tiny(nx=nx, ny=ny)
    grid["dx"] = grid["dy"] = 0.8
    rng = np.random.default_rng(3)
    ii, jj = rng.integers(0, nx, 9), rng.integers(0, ny, 9)
    r = np.stack([grid["x0"] + (ii + 0.5) * grid["dx"], grid["y0"] + (jj + 0.5) * grid["dy"]], 1)
    v = rng.normal(size=(9, 2))
    G = np.array(model["G"])
    offs = np.stack(np.meshgrid((np.arange(2 * nx - 1) - (nx - 1)) * grid["dx"],
                                (np.arange(2 * ny - 1) - (ny - 1)) * grid["dy"]), -1)
    Km = model["beta"] * orc.kernel_matrix(model["beta"] * offs @ G.T)  # [KY, KX, 2, 2]
    sy, sx = 3 * ny - 2, 3 * nx - 2
    field = np.zeros((2, 2, ny, nx))
    for a in range(2):
        for b in range(2):
            full = np.fft.irfft2(np.fft.rfft2(Km[..., a, b], (sy, sx)) * np.fft.rfft2(c, (sy, sx)),
                                 (sy, sx))
            field[a, b] = full[ny - 1:2 * ny - 1, nx - 1:2 * nx - 1]
    want = np.stack([field[:, :, jj[q], ii[q]] @ (G @ v[q]) for q in range(9)], 1)
    got = orc.forward(model, grid, r, v, c)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def _dense(orc, model, grid, r, v):
    """Dense matrix of A ([n_ch*T, N]) built entry by entry from the pair term."""
    nx, ny = grid["nx"], grid["ny"]
    P = np.asarray(model["p"], dtype=float).reshape(-1, 2)
    T = r.shape[0]
    M = np.zeros((P.shape[0] * T, nx * ny))
    for t in range(T):
        for j in range(ny):
            for i in range(nx):
                x = np.array([grid["x0"] + (i + 0.5) * grid["dx"], grid["y0"] + (j + 0.5) * grid["dy"]])
                Jw = orc.pair(model, x, r[t], v[t])
                for k in range(P.shape[0]):
                    M[k * T + t, j * nx + i] = P[k] @ Jw
    return M


@pytest.mark.parametrize("n_ch", [1, 2])
def test_brute_force_8x8(orc, n_ch):
    grid, model, r, v, c = _tiny(nx=8, ny=8, T=12, seed=5)
    model["p"] = [[0.8, 0.6], [-0.6, 0.8]][:n_ch]
    M = _dense(orc, model, grid, r, v)
    s = orc.forward(model, grid, r, v, c)
    assert np.allclose(s.reshape(-1), M @ c.reshape(-1), rtol=1e-13, atol=1e-15)
    y = np.random.default_rng(9).normal(size=s.shape)
    g = orc.adjoint(model, grid, r, v, y)
    assert np.allclose(g.reshape(-1), M.T @ y.reshape(-1), rtol=1e-13, atol=1e-15)
    assert abs(orc.frob2(model, grid, r, v) - np.sum(M * M)) < 1e-12 * np.sum(M * M)
    sel = np.array([0, 9, 63, 17])
    assert np.allclose(orc.adjoint(model, grid, r, v, y, sel=sel), (M.T @ y.reshape(-1))[sel],
                       rtol=1e-13)


def test_adjoint_identity(orc):
    cfg = syn.small(13, 9, 300, "spiral")
    rng = np.random.default_rng(2)
    c = rng.normal(size=(9, 13))
    s = rng.normal(size=(2, 300))
    lhs = np.sum(orc.forward(cfg["model"], cfg["grid"], cfg["r"], cfg["v"], c) * s)
    rhs = np.sum(c * orc.adjoint(cfg["model"], cfg["grid"], cfg["r"], cfg["v"], s))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + abs(rhs))


def _mp_forward(model, grid, r, v, c, beta):
    """A(c; beta) in mpmath from the Jacobian form J w = beta K(beta G(x-r)) G v."""
    G = [[mp.mpf(g) for g in row] for row in model["G"]]
    P = model["p"]
    T = r.shape[0]
    s = [[mp.mpf(0)] * T for _ in P]
    for t in range(T):
        w = [G[0][0] * v[t, 0] + G[0][1] * v[t, 1], G[1][0] * v[t, 0] + G[1][1] * v[t, 1]]
        for j in range(grid["ny"]):
            for i in range(grid["nx"]):
                x = [grid["x0"] + (i + 0.5) * grid["dx"], grid["y0"] + (j + 0.5) * grid["dy"]]
                d = [mp.mpf(x[0]) - r[t, 0], mp.mpf(x[1]) - r[t, 1]]
                y = [beta * (G[0][0] * d[0] + G[0][1] * d[1]), beta * (G[1][0] * d[0] + G[1][1] * d[1])]
                z = mp.sqrt(y[0] ** 2 + y[1] ** 2)
                L = mp.coth(z) - 1 / z
                Lp = 1 / z**2 - 1 / mp.sinh(z) ** 2
                a = L / z
                dd = (Lp - a) / z**2
                yw = y[0] * w[0] + y[1] * w[1]
                Jw = [beta * (a * w[0] + dd * yw * y[0]), beta * (a * w[1] + dd * yw * y[1])]
                for k in range(len(P)):
                    s[k][t] += mp.mpf(c[j, i]) * (P[k][0] * Jw[0] + P[k][1] * Jw[1])
    return s


def test_dbeta_vs_mpmath_derivative(orc):
    """d/dbeta <g, A(c; beta)> against mpmath's numerical derivative of an
    independent high-precision forward."""
    grid, model, r, v, c = _tiny(nx=3, ny=3, T=4, seed=11, beta=700.0)
    gs = np.random.default_rng(4).normal(size=(2, 4))

    def obj(b):
        s = _mp_forward(model, grid, r, v, c, b)
        return sum(gs[k, t] * s[k][t] for k in range(2) for t in range(4))
    ref = float(mp.diff(obj, mp.mpf(model["beta"])))
    got = orc.dbeta(model, grid, r, v, c, gs)
    assert abs(got - ref) <= 1e-12 * abs(ref)


def test_dbeta_central_difference(orc):
    cfg = syn.small(16, 16, 400)
    m = dict(cfg["model"])
    gs = np.random.default_rng(8).normal(size=(2, 400))
    h = 1e-6 * m["beta"]
    mp_, mm_ = dict(m, beta=m["beta"] + h), dict(m, beta=m["beta"] - h)
    fd = (np.sum(gs * orc.forward(mp_, cfg["grid"], cfg["r"], cfg["v"], cfg["c"]))
          - np.sum(gs * orc.forward(mm_, cfg["grid"], cfg["r"], cfg["v"], cfg["c"]))) / (2 * h)
    got = orc.dbeta(m, cfg["grid"], cfg["r"], cfg["v"], cfg["c"], gs)
    assert abs(got - fd) <= 1e-7 * abs(fd)


# ---------------------------------------------------------------------------
# Cosine interpolation and the Laplacian (Core Stage, Eq. first:step)

def test_interp_exact_at_nodes_and_partition_of_unity(orc):
    grid = syn.square_grid(6, 12.0, 5)
    xs, ys = syn.voxel_centres(grid)
    rng = np.random.default_rng(0)
    A = rng.normal(size=(4, 5, 6))
    ii, jj = rng.integers(0, 6, 20), rng.integers(0, 5, 20)
    r = np.stack([xs[ii], ys[jj]], 1)
    v = rng.normal(size=(20, 2))
    s = orc.interp(grid, r, v, A)
    want = np.stack([A[0, jj, ii] * v[:, 0] + A[1, jj, ii] * v[:, 1],
                     A[2, jj, ii] * v[:, 0] + A[3, jj, ii] * v[:, 1]])
    assert np.allclose(s, want, rtol=1e-14, atol=1e-15)
    # constants are reproduced anywhere (including outside the node hull)
    rr = rng.uniform(-8, 8, size=(50, 2))
    vv = rng.normal(size=(50, 2))
    Ac = np.broadcast_to(np.array([1.5, -2.0, 0.25, 3.0])[:, None, None], (4, 5, 6)).copy()
    s = orc.interp(grid, rr, vv, Ac)
    assert np.allclose(s[0], 1.5 * vv[:, 0] - 2.0 * vv[:, 1], rtol=1e-13)
    assert np.allclose(s[1], 0.25 * vv[:, 0] + 3.0 * vv[:, 1], rtol=1e-13)


def test_interp_hand_example(orc):
    """Quarter of the way between nodes 1 and 2 along x, on node row 2:
    weight (1 - cos(pi/4))/2 on node 2."""
    grid = {"nx": 4, "ny": 4, "x0": 0.0, "y0": 0.0, "dx": 1.0, "dy": 1.0}
    A = np.zeros((4, 4, 4))
    A[0, 2, 1], A[0, 2, 2] = 10.0, 20.0
    r = np.array([[1.75, 2.5]])
    v = np.array([[1.0, 0.0]])
    w1 = (1 - math.cos(math.pi / 4)) / 2
    assert abs(orc.interp(grid, r, v, A)[0, 0] - (10.0 * (1 - w1) + 20.0 * w1)) < 1e-14


def test_interp_adjoint(orc):
    grid = syn.square_grid(7, 10.0, 5)
    rng = np.random.default_rng(1)
    r = rng.uniform(-6, 6, size=(200, 2))
    v = rng.normal(size=(200, 2))
    A = rng.normal(size=(4, 5, 7))
    s = rng.normal(size=(2, 200))
    lhs = np.sum(orc.interp(grid, r, v, A) * s)
    rhs = np.sum(A * orc.interp_T(grid, r, v, s))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_laplacian_vs_scipy(orc):
    ndi = pytest.importorskip("scipy.ndimage")
    grid = syn.square_grid(9, 9.0, 6)
    f = np.random.default_rng(3).normal(size=(6, 9))
    assert np.allclose(orc.laplacian(grid, f), ndi.laplace(f, mode="nearest"), rtol=1e-14, atol=1e-14)
    # symmetric (so Lap^T Lap = Lap Lap in the Core Stage)
    n = 54
    D = np.stack([orc.laplacian(grid, np.eye(n)[k].reshape(6, 9)).reshape(-1) for k in range(n)], 1)
    assert np.array_equal(D, D.T)


# ---------------------------------------------------------------------------
# Convolution with the sampled trace kernel (Eq. kernel:trace, Eq. dec:sub:tik)

def test_conv_kernel_isotropic_closed_form(orc):
    """For G = g I: kappa_G(y) = beta g kappa(beta g |y|), kappa = L' + L/z."""
    grid = syn.square_grid(5, 5.0, 4)
    model = syn.default_model()
    g, beta = model["G"][0][0], model["beta"]
    K = orc.conv_kernel(model, grid)
    for jj in range(K.shape[0]):
        for ii in range(K.shape[1]):
            o = ((ii - 4) * grid["dx"], (jj - 3) * grid["dy"])
            z = mp.mpf(beta * g) * mp.sqrt(mp.mpf(o[0]) ** 2 + mp.mpf(o[1]) ** 2)
            kap = (mp.mpf(2) / 3 if z == 0 else
                   1 / z**2 - 1 / mp.sinh(z) ** 2 + (mp.coth(z) - 1 / z) / z)
            assert abs(K[jj, ii] - float(beta * g * kap)) <= 1e-13 * float(beta * g * kap)


def test_conv_is_trace_of_forward_operator(orc):
    """u_i = sum_x c_x kappa_G(x - x_i) equals tr of the 2x2 matrix that the
    forward model applies to v at a sample sitting on voxel centre x_i
    (Eq. convolution:trace), also for a non-diagonal G."""
    grid, model, _, _, c = _tiny(nx=5, ny=4, G=[[-1e-3, 4e-4], [4e-4, 2e-3]])
    model["p"] = [[1.0, 0.0], [0.0, 1.0]]
    xs = grid["x0"] + (np.arange(5) + 0.5) * grid["dx"]
    ys = grid["y0"] + (np.arange(4) + 0.5) * grid["dy"]
    u = orc.conv(grid, orc.conv_kernel(model, grid), c)
    for j in range(4):
        for i in range(5):
            r = np.array([[xs[i], ys[j]], [xs[i], ys[j]]])
            v = np.eye(2)  # two samples at x_ij with v = e_x, e_y
            s = orc.forward(model, grid, r, v, c)
            assert abs(u[j, i] - (s[0, 0] + s[1, 1])) <= 1e-12 * abs(u[j, i])


def test_conv_direct_vs_fft(orc):
    sig = pytest.importorskip("scipy.signal")
    grid = syn.square_grid(11, 12.0, 8)
    model = syn.default_model()
    K = orc.conv_kernel(model, grid)
    x = np.random.default_rng(6).normal(size=(8, 11))
    d = orc.conv(grid, K, x)
    f = orc.conv_fft(K, x)
    full = sig.fftconvolve(K, x, mode="full")
    assert np.allclose(d, f, rtol=1e-12, atol=1e-12 * np.abs(d).max())
    assert np.allclose(d, full[7:15, 10:21], rtol=1e-12, atol=1e-12 * np.abs(d).max())
    y = np.random.default_rng(7).normal(size=(8, 11))
    assert abs(np.sum(orc.conv(grid, K, x) * y) - np.sum(x * orc.conv(grid, K, y))) < 1e-11


def test_conv_kernel_components(orc):
    """Entry (a, b) of beta K(beta G y) G: the (0,0) + (1,1) entries give the
    trace kernel, and each entry is the forward model's matrix entry at voxel
    centres (channel a with v = e_b), also for a non-diagonal G."""
    grid, model, _, _, c = _tiny(nx=5, ny=4, G=[[-1e-3, 4e-4], [4e-4, 2e-3]])
    model["p"] = [[1.0, 0.0], [0.0, 1.0]]
    K = {(a, b): orc.conv_kernel(model, grid, component=(a, b)) for a in range(2) for b in range(2)}
    assert np.allclose(K[0, 0] + K[1, 1], orc.conv_kernel(model, grid), rtol=1e-13, atol=1e-16)
    xs = grid["x0"] + (np.arange(5) + 0.5) * grid["dx"]
    ys = grid["y0"] + (np.arange(4) + 0.5) * grid["dy"]
    for (a, b), Kab in K.items():
        u = orc.conv(grid, Kab, c)
        for j in range(4):
            for i in range(5):
                r = np.array([[xs[i], ys[j]]])
                v = np.eye(2)[b][None]
                s = orc.forward(model, grid, r, v, c)
                assert abs(u[j, i] - s[a, 0]) <= 1e-12 * max(1.0, abs(u[j, i]))

"""Pins for the oracle's three-dimensional field-free-point operators (the
model of Sec. 2 with n = 3): the 3x3 kernel matrix against mpmath's Jacobian
of the magnetisation, the forward model against mpmath's time derivative of
the magnetisation on an analytic 3-D trajectory, the reduction to the pinned
2-D operator on a single slice, a dense brute force of A and A^T, the trace
kernel against the closed form L' + 2 L/z (Eq. kernel:trace with n - 1 = 2),
the 3-D convolution against an FFT route and the volume denoiser against
scipy."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")


@pytest.fixture(autouse=True)
def _mp_precision():
    """40 significant digits for every mpmath reference here, restored after."""
    with mp.workdps(40):
        yield

G3_STD = [[-1.25e-3, 0.0, 0.0], [0.0, -1.25e-3, 0.0], [0.0, 0.0, 2.5e-3]]
G3_GEN = [[-1.1e-3, 3e-4, -2e-4], [3e-4, -1.4e-3, 1e-4], [-2e-4, 1e-4, 2.3e-3]]


def _tiny3(nx=3, ny=4, nz=2, T=5, seed=0, G=None, p=None, beta=900.0, fov=6.0):
    rng = np.random.default_rng(seed)
    grid = {"nx": nx, "ny": ny, "nz": nz, "x0": -fov / 2, "y0": -fov / 2 + 0.3,
            "z0": -fov / 4 - 0.2, "dx": fov / nx, "dy": fov / ny * 0.9, "dz": fov / (2 * nz)}
    model = {"beta": beta, "G": G if G is not None else G3_STD,
             "p": p if p is not None else np.eye(3).tolist()}
    r = rng.uniform(-fov / 3, fov / 3, size=(T, 3))
    v = rng.normal(size=(T, 3)) * 0.1
    c = rng.uniform(0, 1, size=(nz, ny, nx))
    return grid, model, r, v, c


def _centres(grid):
    xs = grid["x0"] + (np.arange(grid["nx"]) + 0.5) * grid["dx"]
    ys = grid["y0"] + (np.arange(grid["ny"]) + 0.5) * grid["dy"]
    zs = grid["z0"] + (np.arange(grid["nz"]) + 0.5) * grid["dz"]
    return xs, ys, zs


def _mp_M3(H, beta):
    h = mp.sqrt(H[0] ** 2 + H[1] ** 2 + H[2] ** 2)
    z = beta * h
    L = mp.coth(z) - 1 / z
    return [L * H[q] / h for q in range(3)]


@pytest.mark.parametrize("H", [(3e-4, -1e-4, 2e-4), (2e-3, 5e-3, -1e-3), (1e-6, -2e-6, 5e-7)])
def test_kernel3_is_jacobian_of_magnetisation(orc, H):
    """beta K(beta H) = d/dH [L(beta|H|) H/|H|] for H in R^3."""
    beta = 2331.350896656040
    J = np.zeros((3, 3))
    for b in range(3):
        for a in range(3):
            def f(hb, a=a, b=b):
                HH = [mp.mpf(h) for h in H]
                HH[b] = hb
                return _mp_M3(HH, beta)[a]
            J[a, b] = float(mp.diff(f, mp.mpf(H[b])))
    K = orc.kernel_matrix3(np.array([[beta * h for h in H]]))[0]
    assert np.allclose(beta * K, J, rtol=1e-12, atol=0)
    assert np.allclose(orc.kernel_matrix3(np.zeros(3)), np.eye(3) / 3, rtol=0, atol=1e-16)


def _mp_integrand3(model, grid, c, rt):
    G = [[mp.mpf(g) for g in row] for row in model["G"]]
    beta = mp.mpf(model["beta"])
    P = model["p"]
    out = [mp.mpf(0)] * len(P)
    for l in range(grid["nz"]):
        for j in range(grid["ny"]):
            for i in range(grid["nx"]):
                x = [mp.mpf(grid["x0"]) + (i + mp.mpf(0.5)) * mp.mpf(grid["dx"]),
                     mp.mpf(grid["y0"]) + (j + mp.mpf(0.5)) * mp.mpf(grid["dy"]),
                     mp.mpf(grid["z0"]) + (l + mp.mpf(0.5)) * mp.mpf(grid["dz"])]
                d = [x[q] - rt[q] for q in range(3)]
                H = [sum(G[a][b] * d[b] for b in range(3)) for a in range(3)]
                M = _mp_M3(H, beta)
                for k in range(len(P)):
                    out[k] += mp.mpf(c[l, j, i]) * sum(P[k][q] * M[q] for q in range(3))
    return out


@pytest.mark.parametrize("G", [G3_STD, G3_GEN])
def test_forward3_is_time_derivative_of_magnetisation(orc, G):
    """s_k(t) = -d/dt sum_x c_x p_k^T L(beta|H|) H/|H|, H = G(x - r(t)), for a
    3-D Lissajous trajectory (mpmath derivative), three channels, the paper's
    G = diag(-1, -1, 2) shape and a general symmetric G."""
    grid, model, _, _, c = _tiny3(G=G)
    amp, fr, ph = (2.0, 1.6, 0.9), (0.013, 0.011, 0.007), (0.0, 0.3, 1.1)

    def rr(t):
        return [amp[q] * mp.sin(2 * mp.pi * fr[q] * t + mp.mpf(ph[q])) for q in range(3)]

    ts = [3.0, 29.0]
    r = np.array([[float(u) for u in rr(mp.mpf(t))] for t in ts])
    v = np.array([[float(amp[q] * 2 * mp.pi * fr[q] * mp.cos(2 * mp.pi * fr[q] * t + mp.mpf(ph[q])))
                   for q in range(3)] for t in ts])
    s = orc.forward3(model, grid, r, v, c)
    for n, t in enumerate(ts):
        for k in range(3):
            ref = -mp.diff(lambda tt: _mp_integrand3(model, grid, c, rr(tt))[k], mp.mpf(t))
            assert abs(s[k, n] - float(ref)) <= 1e-11 * max(1.0, abs(float(ref))), (t, k)


def test_forward3_single_slice_reduces_to_2d(orc):
    """One slice, samples in its plane (r_z = slice centre, v_z = 0) and a
    gradient without x/y-z coupling: y_z = 0 and (G v)_z = 0, so the x and y
    channels equal the pinned 2-D operator and the z channel vanishes."""
    rng = np.random.default_rng(3)
    G2 = [[2.1e-3, 4e-4], [4e-4, -2.6e-3]]
    G3 = [[G2[0][0], G2[0][1], 0.0], [G2[1][0], G2[1][1], 0.0], [0.0, 0.0, 5e-3]]
    g2 = {"nx": 6, "ny": 5, "x0": -3.0, "y0": -2.5, "dx": 1.0, "dy": 1.0}
    g3 = dict(g2, nz=1, z0=0.7, dz=0.4)
    T = 9
    r2 = rng.uniform(-3, 3, size=(T, 2))
    v2 = rng.normal(size=(T, 2)) * 0.1
    r3 = np.concatenate([r2, np.full((T, 1), 0.9)], 1)
    v3 = np.concatenate([v2, np.zeros((T, 1))], 1)
    c = rng.uniform(size=(5, 6))
    m2 = {"beta": 800.0, "G": G2, "p": [[1, 0], [0, 1]]}
    m3 = {"beta": 800.0, "G": G3, "p": np.eye(3).tolist()}
    s2 = orc.forward(m2, g2, r2, v2, c)
    s3 = orc.forward3(m3, g3, r3, v3, c[None])
    assert np.allclose(s3[:2], s2, rtol=1e-13, atol=1e-13 * np.abs(s2).max())
    assert np.abs(s3[2]).max() <= 1e-13 * np.abs(s2).max()
    y = rng.normal(size=(2, T))
    a2 = orc.adjoint(m2, g2, r2, v2, y)
    a3 = orc.adjoint3(m3, g3, r3, v3, np.concatenate([y, rng.normal(size=(1, T))]))
    assert np.allclose(a3[0], a2, rtol=1e-12, atol=1e-13 * np.abs(a2).max())


@pytest.mark.parametrize("n_ch", [1, 2, 3])
def test_forward3_adjoint3_brute_force(orc, n_ch):
    """Dense matrix of A from the pair term (one column per voxel): A c, A^T s,
    sampled A^T and ||A||_F^2 agree with it."""
    p = [[0.6, 0.8, 0.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]][:n_ch]
    grid, model, r, v, c = _tiny3(T=7, seed=n_ch, G=G3_GEN, p=p)
    xs, ys, zs = _centres(grid)
    nz, ny, nx = c.shape
    T = r.shape[0]
    P = np.asarray(p)
    A = np.zeros((n_ch * T, nz * ny * nx))
    for l in range(nz):
        for j in range(ny):
            for i in range(nx):
                col = (l * ny + j) * nx + i
                for t in range(T):
                    Jw = orc.pair3(model, np.array([xs[i], ys[j], zs[l]]), r[t], v[t])
                    for k in range(n_ch):
                        A[k * T + t, col] = P[k] @ Jw
    s = orc.forward3(model, grid, r, v, c)
    assert np.allclose(s.reshape(-1), A @ c.reshape(-1), rtol=1e-12, atol=1e-14)
    y = np.random.default_rng(9).normal(size=(n_ch, T))
    assert np.allclose(orc.adjoint3(model, grid, r, v, y).reshape(-1), A.T @ y.reshape(-1),
                       rtol=1e-12, atol=1e-14)
    sel = np.array([5, 0, nz * ny * nx - 1])
    assert np.allclose(orc.adjoint3(model, grid, r, v, y, sel=sel), (A.T @ y.reshape(-1))[sel],
                       rtol=1e-12, atol=1e-14)
    assert abs(orc.frob2_3(model, grid, r, v) - np.sum(A * A)) <= 1e-12 * np.sum(A * A)


def test_pair3_vs_mpmath(orc):
    """J w for a general G against mpmath's Jacobian applied to G v."""
    model = {"beta": 600.0, "G": G3_GEN, "p": np.eye(3).tolist()}
    x, r, v = np.array([1.2, -0.4, 0.3]), np.array([-0.3, 0.9, -0.2]), np.array([0.05, -0.02, 0.03])
    G = np.array(G3_GEN)
    H0 = G @ (x - r)
    J = np.zeros((3, 3))
    for b in range(3):
        for a in range(3):
            def f(hb, a=a, b=b):
                HH = [mp.mpf(h) for h in H0]
                HH[b] = hb
                return _mp_M3(HH, model["beta"])[a]
            J[a, b] = float(mp.diff(f, mp.mpf(H0[b])))
    assert np.allclose(orc.pair3(model, x, r, v), J @ (G @ v), rtol=1e-12, atol=0)


def test_conv_kernel3_isotropic_closed_form(orc):
    """G = g I: kappa_G(y) = beta g (L'(z) + 2 L(z)/z), z = beta g |y|, the
    trace kernel of Eq. kernel:trace with n - 1 = 2 (2/3 + 1/3 = 1 at y = 0)."""
    g, beta = 2.5e-3, 2331.350896656040
    grid = {"nx": 4, "ny": 3, "nz": 3, "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": 0.4, "dy": 0.5, "dz": 0.3}
    model = {"beta": beta, "G": (g * np.eye(3)).tolist(), "p": np.eye(3).tolist()}
    K = orc.conv_kernel3(model, grid)
    for ll in range(5):
        for jj in range(5):
            for ii in range(7):
                o = [(ii - 3) * 0.4, (jj - 2) * 0.5, (ll - 2) * 0.3]
                z = mp.mpf(beta * g) * mp.sqrt(sum(mp.mpf(q) ** 2 for q in o))
                kap = (mp.mpf(1) if z == 0 else
                       1 / z**2 - 1 / mp.sinh(z) ** 2 + 2 * (mp.coth(z) - 1 / z) / z)
                want = float(beta * g * kap)
                assert abs(K[ll, jj, ii] - want) <= 1e-13 * want


def test_conv3_is_trace_of_forward3(orc):
    """The 3-D convolution equals the trace of the 3x3 matrix the forward
    model applies to v at a sample on a voxel centre (Eq. convolution:trace),
    for the paper's G shape and a general G."""
    for G in (G3_STD, G3_GEN):
        grid, model, _, _, c = _tiny3(nx=3, ny=3, nz=2, G=G)
        xs, ys, zs = _centres(grid)
        u = orc.conv3(grid, orc.conv_kernel3(model, grid), c)
        for l in range(2):
            for j in range(3):
                for i in range(3):
                    r = np.tile([xs[i], ys[j], zs[l]], (3, 1))
                    s = orc.forward3(model, grid, r, np.eye(3), c)
                    assert abs(u[l, j, i] - np.trace(s)) <= 1e-12 * abs(u[l, j, i])


def test_conv3_direct_vs_fft(orc):
    grid, model, _, _, _ = _tiny3(nx=5, ny=4, nz=3)
    K = orc.conv_kernel3(model, grid)
    x = np.random.default_rng(4).normal(size=(3, 4, 5))
    d = orc.conv3(grid, K, x)
    shp = [K.shape[q] + x.shape[q] - 1 for q in range(3)]
    ax = (0, 1, 2)
    full = np.real(np.fft.ifftn(np.fft.fftn(K, shp, ax) * np.fft.fftn(x, shp, ax), axes=ax))
    assert np.allclose(d, full[2:5, 3:7, 4:9], rtol=1e-12, atol=1e-12 * np.abs(d).max())
    y = np.random.default_rng(5).normal(size=(3, 4, 5))
    assert abs(np.sum(orc.conv3(grid, K, x) * y) - np.sum(x * orc.conv3(grid, K, y))) < 1e-10


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (5, 6, 3), (9, 7, 8)])
def test_gaussian5_3d_vs_scipy(orc, shape):
    ndi = pytest.importorskip("scipy.ndimage")
    x = np.random.default_rng(2).normal(size=shape)
    want = ndi.gaussian_filter(x, sigma=1.0, truncate=2.0, mode="reflect")
    assert np.allclose(orc.gaussian5_3d(x), want, rtol=1e-13, atol=1e-14)


def test_trace_kernel_of_a_traceless_gradient_has_almost_no_mean(orc):
    """tr(K(y) G) = a tr G + d y^T G y: for a scalar gradient the sampled trace
    kernel is positive; for the physical, traceless FFP gradient
    g diag(-1/2, -1/2, 1) only d y^T G y remains, which changes sign and sums
    to almost nothing.  beta tr K(beta G y) (the kernel of the
    gradient-weighted trace sum_k A_kk / G_kk) stays positive."""
    grid = {"nx": 12, "ny": 12, "nz": 6, "x0": -6.0, "y0": -6.0, "z0": -3.0, "dx": 1.0, "dy": 1.0, "dz": 1.0}
    g = 2.5e-3
    iso = {"beta": 2331.35, "G": (g * np.eye(3)).tolist(), "p": np.eye(3).tolist()}
    tl = {"beta": 2331.35, "G": np.diag([-g / 2, -g / 2, g]).tolist(), "p": np.eye(3).tolist()}
    k_iso = orc.conv_kernel3(iso, grid)
    k_tl = orc.conv_kernel3(tl, grid)
    assert k_iso.min() > 0.0
    assert k_tl.min() < 0.0 < k_tl.max()
    assert abs(k_tl.sum()) < 0.05 * np.abs(k_tl).sum()
    # beta tr K(beta G y) on the same offsets: positive
    nz, ny, nx = 6, 12, 12
    off = np.stack(np.meshgrid(np.arange(2 * nx - 1) - (nx - 1.0), np.arange(2 * ny - 1) - (ny - 1.0),
                               np.arange(2 * nz - 1) - (nz - 1.0), indexing="xy"), -1).reshape(-1, 3)
    y = tl["beta"] * off @ np.asarray(tl["G"]).T
    K = orc.kernel_matrix3(y).reshape(-1, 3, 3)
    assert np.trace(K, axis1=1, axis2=2).min() > 0.0

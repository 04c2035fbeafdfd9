"""Pins for the oracle's grid-scaled forms: the Laplacian with 1/dx^2, 1/dy^2
(1/dz^2) (exact on quadratics, scipy's stencil over h^2 on isotropic grids,
symmetric, the bare stencil's Core Stage with gamma / h^4), and the kernel of
the gradient-weighted trace tr(Ahat G^-1), beta tr K(beta G y) (the trace
kernel over g for a scalar gradient, tr K(0) = n/3, the closed form
L' + (n - 1) L / z against mpmath, positivity for a traceless gradient, and
tr(Ahat G^-1) of the component-kernel convolutions equal to its convolution)."""
import numpy as np
import pytest

from paper_2505_22797_gb300 import synthetic as syn

mp = pytest.importorskip("mpmath")


@pytest.fixture(autouse=True)
def _mp_precision():
    with mp.workdps(40):
        yield


def test_laplacian_h_exact_on_quadratics_and_scipy(orc):
    g = {"nx": 9, "ny": 7, "x0": -2.0, "y0": 1.0, "dx": 0.5, "dy": 0.3}
    xs = g["x0"] + (np.arange(9) + 0.5) * g["dx"]
    ys = g["y0"] + (np.arange(7) + 0.5) * g["dy"]
    X, Y = np.meshgrid(xs, ys)
    f = 1.5 * X ** 2 - 0.7 * Y ** 2 + 0.3 * X * Y + 2.0 * X - Y + 4.0
    L = orc.laplacian_h(g, f)
    assert np.allclose(L[1:-1, 1:-1], 2 * 1.5 - 2 * 0.7, rtol=0, atol=1e-11)
    ndi = pytest.importorskip("scipy.ndimage")
    gi = {"nx": 9, "ny": 7, "x0": 0.0, "y0": 0.0, "dx": 0.4, "dy": 0.4}
    f = np.random.default_rng(0).normal(size=(7, 9))
    assert np.allclose(orc.laplacian_h(gi, f), ndi.laplace(f, mode="nearest") / 0.16, rtol=1e-13, atol=1e-12)
    n = 63
    D = np.stack([orc.laplacian_h(g, np.eye(n)[k].reshape(7, 9)).reshape(-1) for k in range(n)], 1)
    assert np.allclose(D, D.T, rtol=0, atol=1e-12)


def test_laplacian3_h_exact_on_quadratics(orc):
    g = {"nx": 6, "ny": 5, "nz": 4, "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": 0.5, "dy": 0.25, "dz": 0.8}
    xs = (np.arange(6) + 0.5) * 0.5
    ys = (np.arange(5) + 0.5) * 0.25
    zs = (np.arange(4) + 0.5) * 0.8
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    f = X ** 2 + 2 * Y ** 2 - 0.5 * Z ** 2 + X * Z
    L = orc.laplacian3_h(g, f)
    assert np.allclose(L[1:-1, 1:-1, 1:-1], 2 + 4 - 1, rtol=0, atol=1e-11)
    # one slice: the 2-D scaled Laplacian
    g1 = dict(g, nz=1)
    g2 = {k: g[k] for k in ("nx", "ny", "x0", "y0", "dx", "dy")}
    f1 = np.random.default_rng(1).normal(size=(1, 5, 6))
    assert np.allclose(orc.laplacian3_h(g1, f1)[0], orc.laplacian_h(g2, f1[0]), rtol=1e-14, atol=1e-12)


def test_scaled_core_stage_is_bare_stencil_with_gamma_over_h4(orc):
    g = syn.square_grid(12, 6.0)
    h = g["dx"]
    rng = np.random.default_rng(2)
    r = rng.uniform(-3, 3, size=(200, 2))
    v = rng.normal(size=(200, 2))
    s = rng.normal(size=(2, 200))
    a, ua, _ = orc.core_stage(g, r, v, s, 1e-4, max_iter=30, lap="scaled")
    b, ub, _ = orc.core_stage(g, r, v, s, 1e-4 / h ** 4, max_iter=30)
    assert np.allclose(a, b, rtol=1e-9, atol=1e-12 * np.abs(b).max())


def test_trK_kernel_scalar_gradient_and_origin(orc):
    m = syn.default_model()
    g = syn.square_grid(6, 6.0, 5)
    kt = orc.conv_kernel_trK(m, g)
    kk = orc.conv_kernel(m, g)
    gg = m["G"][0][0]
    assert np.allclose(kt * gg, kk, rtol=1e-14, atol=0)
    assert kt[4, 5] == pytest.approx(m["beta"] * 2.0 / 3.0, rel=1e-14)   # tr K(0) = n/3, n = 2
    m3 = syn.default_model3()
    g3 = {"nx": 5, "ny": 4, "nz": 3, "x0": -2.5, "y0": -2.0, "z0": -1.5, "dx": 1.0, "dy": 1.0, "dz": 1.0}
    k3 = orc.conv_kernel3_trK(m3, g3)
    assert k3[2, 3, 4] == pytest.approx(m3["beta"] * 1.0, rel=1e-14)      # tr K(0) = 1, n = 3
    assert k3.min() > 0.0


@pytest.mark.parametrize("n", [2, 3])
def test_trK_closed_form(orc, n):
    """tr K(y) = L'(z) + (n - 1) L(z)/z (the eigenvalues of K: L' along y,
    L/z across), against mpmath."""
    def L(z):
        return mp.coth(z) - 1 / z

    def Lp(z):
        return 1 / z ** 2 - 1 / mp.sinh(z) ** 2

    if n == 2:
        m = syn.default_model()
        g = {"nx": 4, "ny": 3, "x0": 0.0, "y0": 0.0, "dx": 0.7, "dy": 0.45}
        k = orc.conv_kernel_trK(m, g)
        for jj in range(k.shape[0]):
            for ii in range(k.shape[1]):
                if (jj, ii) == (2, 3):
                    continue
                off = np.array([(ii - 3) * 0.7, (jj - 2) * 0.45])
                y = m["beta"] * np.asarray(m["G"]) @ off
                z = mp.sqrt(mp.mpf(y[0]) ** 2 + mp.mpf(y[1]) ** 2)
                want = m["beta"] * (Lp(z) + (n - 1) * L(z) / z)
                assert abs(k[jj, ii] - float(want)) <= 2e-13 * abs(float(want))
    else:
        m = syn.default_model3()
        g = {"nx": 3, "ny": 3, "nz": 2, "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": 0.6, "dy": 0.5, "dz": 0.9}
        k = orc.conv_kernel3_trK(m, g)
        for ll in range(k.shape[0]):
            for jj in range(k.shape[1]):
                for ii in range(k.shape[2]):
                    if (ll, jj, ii) == (1, 2, 2):
                        continue
                    off = np.array([(ii - 2) * 0.6, (jj - 2) * 0.5, (ll - 1) * 0.9])
                    y = m["beta"] * np.asarray(m["G"]) @ off
                    z = mp.sqrt(sum(mp.mpf(q) ** 2 for q in y))
                    want = m["beta"] * (Lp(z) + (n - 1) * L(z) / z)
                    assert abs(k[ll, jj, ii] - float(want)) <= 2e-13 * abs(float(want))


def test_weighted_trace_of_component_convolutions(orc):
    """Ahat_km at the voxel centres is the convolution of c with the (k, m)
    entry of beta K(beta G y) G; tr(Ahat G^-1) of those equals the convolution
    with beta tr K(beta G y), for a non-diagonal G too."""
    m = {"beta": 900.0, "G": [[2.0e-3, 0.4e-3], [0.4e-3, -1.5e-3]], "p": [[1.0, 0.0], [0.0, 1.0]]}
    g = syn.square_grid(7, 6.0, 6)
    c = np.random.default_rng(3).uniform(size=(6, 7))
    A = np.stack([orc.conv(g, orc.conv_kernel(m, g, component=(k, q)), c) for k in range(2) for q in range(2)])
    want = orc.conv(g, orc.conv_kernel_trK(m, g), c)
    assert np.allclose(orc.weighted_trace(m, A), want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_weighted_trace3_brute_force(orc):
    """Ahat_km(x) = sum_x' c(x') beta [K(beta G (x' - x)) G]_km by brute force
    (the 3x3 kernel matrix, a non-symmetric G); tr(Ahat G^-1) equals the
    convolution of c with beta tr K(beta G y)."""
    G = np.array([[-1.1e-3, 3e-4, -2e-4], [1e-4, -1.4e-3, 2e-4], [-3e-4, 1e-4, 2.3e-3]])
    m = {"beta": 900.0, "G": G.tolist(), "p": np.eye(3).tolist()}
    g = {"nx": 4, "ny": 3, "nz": 2, "x0": -2.0, "y0": -1.5, "z0": -1.0, "dx": 1.0, "dy": 1.0, "dz": 1.0}
    c = np.random.default_rng(4).uniform(size=(2, 3, 4))
    pts = np.array([[(i + 0.5) - 2.0, (j + 0.5) - 1.5, (l + 0.5) - 1.0]
                    for l in range(2) for j in range(3) for i in range(4)])
    cf = c.reshape(-1)
    A = np.zeros((9, 24))
    for a, x in enumerate(pts):
        y = m["beta"] * (pts - x) @ G.T
        K = orc.kernel_matrix3(y).reshape(-1, 3, 3)
        KG = m["beta"] * K @ G
        for k in range(3):
            for q in range(3):
                A[3 * k + q, a] = np.sum(cf * KG[:, k, q])
    A = A.reshape(9, 2, 3, 4)
    kt = orc.conv_kernel3_trK(m, g)
    want = np.zeros(24)
    for a, x in enumerate(pts):
        for b, xp in enumerate(pts):
            o = np.rint(xp - x).astype(int)
            want[a] += kt[o[2] + 1, o[1] + 2, o[0] + 3] * cf[b]
    got = orc.weighted_trace3(m, A).reshape(-1)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())

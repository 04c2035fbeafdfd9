"""Pins for the oracle's three-dimensional Core Stage (Eq. first:step with
n = 3): the tensor-product cosine interpolation (exact at the nodes, partition
of unity, a hand-computed example, the product of three one-dimensional
interpolations for a separable field, the reduction to the pinned 2-D scheme
on one slice), its transpose (adjoint identity), the 7-point Laplacian against
scipy, and the CG solve against a dense solve of the normal equations and
against the pinned 2-D Core Stage on a single slice."""
import math

import numpy as np
import pytest


def _grid3(nx, ny, nz, fov=(10.0, 8.0, 6.0), off=(0.3, -0.2, 0.1)):
    return {"nx": nx, "ny": ny, "nz": nz,
            "x0": -fov[0] / 2 + off[0], "y0": -fov[1] / 2 + off[1], "z0": -fov[2] / 2 + off[2],
            "dx": fov[0] / nx, "dy": fov[1] / ny, "dz": fov[2] / nz}


def _centres(g):
    return (g["x0"] + (np.arange(g["nx"]) + 0.5) * g["dx"],
            g["y0"] + (np.arange(g["ny"]) + 0.5) * g["dy"],
            g["z0"] + (np.arange(g["nz"]) + 0.5) * g["dz"])


def test_interp3_exact_at_nodes_and_partition_of_unity(orc):
    g = _grid3(5, 4, 3)
    xs, ys, zs = _centres(g)
    rng = np.random.default_rng(0)
    A = rng.normal(size=(9, 3, 4, 5))
    n = 30
    ii, jj, ll = rng.integers(0, 5, n), rng.integers(0, 4, n), rng.integers(0, 3, n)
    r = np.stack([xs[ii], ys[jj], zs[ll]], 1)
    v = rng.normal(size=(n, 3))
    s = orc.interp3(g, r, v, A)
    want = np.stack([sum(A[3 * k + m, ll, jj, ii] * v[:, m] for m in range(3)) for k in range(3)])
    assert np.allclose(s, want, rtol=1e-14, atol=1e-14)
    # constants are reproduced anywhere, including outside the node hull
    rr = rng.uniform(-9, 9, size=(60, 3))
    vv = rng.normal(size=(60, 3))
    cst = rng.normal(size=9)
    Ac = np.broadcast_to(cst[:, None, None, None], (9, 3, 4, 5)).copy()
    s = orc.interp3(g, rr, vv, Ac)
    for k in range(3):
        assert np.allclose(s[k], vv @ cst[3 * k:3 * k + 3], rtol=1e-13, atol=1e-13)


def test_interp3_hand_example(orc):
    """A quarter of a cell along x (upper weight (1 - cos(pi/4))/2), half along
    y (1/2) and a third along z ((1 - cos(pi/3))/2 = 1/4): a field that is 1 on
    the upper corner only reads the product of the three upper weights."""
    g = {"nx": 4, "ny": 4, "nz": 4, "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": 1.0, "dy": 1.0, "dz": 1.0}
    A = np.zeros((9, 4, 4, 4))
    A[4, 2, 3, 2] = 1.0           # component (1, 1) at node (i, j, l) = (2, 3, 2)
    r = np.array([[1.5 + 0.25, 2.5 + 0.5, 1.5 + 1.0 / 3.0]])
    v = np.array([[0.0, 2.0, 0.0]])
    want = 2.0 * (1 - math.cos(math.pi / 4)) / 2 * 0.5 * 0.25
    s = orc.interp3(g, r, v, A)
    assert abs(s[1, 0] - want) < 1e-15 and s[0, 0] == 0.0 and s[2, 0] == 0.0


def test_interp3_separable_is_product_of_1d(orc):
    """For a node field f(i) g(j) h(l) the interpolant is the product of the
    three one-dimensional cosine interpolants, each taken from the pinned 2-D
    scheme on a grid one node high."""
    g = _grid3(6, 5, 4)
    rng = np.random.default_rng(2)
    f, gg, h = rng.normal(size=6), rng.normal(size=5), rng.normal(size=4)
    A = np.zeros((9, 4, 5, 6))
    A[0] = h[:, None, None] * gg[None, :, None] * f[None, None, :]
    T = 80
    r = np.stack([rng.uniform(-6, 6, T), rng.uniform(-5, 5, T), rng.uniform(-4, 4, T)], 1)
    v = np.zeros((T, 3))
    v[:, 0] = 1.0
    s = orc.interp3(g, r, v, A)[0]

    def interp1(vals, p, p0, dp):
        n = len(vals)
        g1 = {"nx": n, "ny": 1, "x0": p0, "y0": 0.0, "dx": dp, "dy": 1.0}
        A1 = np.zeros((4, 1, n))
        A1[0, 0] = vals
        rr = np.stack([p, np.full_like(p, 0.5)], 1)
        vv = np.stack([np.ones_like(p), np.zeros_like(p)], 1)
        return orc.interp(g1, rr, vv, A1)[0]

    want = (interp1(f, r[:, 0], g["x0"], g["dx"]) * interp1(gg, r[:, 1], g["y0"], g["dy"]) *
            interp1(h, r[:, 2], g["z0"], g["dz"]))
    assert np.allclose(s, want, rtol=1e-13, atol=1e-14)


def test_interp3_single_slice_reduces_to_2d(orc):
    g3 = _grid3(6, 5, 1)
    g2 = {k: g3[k] for k in ("nx", "ny", "x0", "y0", "dx", "dy")}
    rng = np.random.default_rng(3)
    T = 50
    r = rng.uniform(-6, 6, size=(T, 3))
    v = rng.normal(size=(T, 3))
    A2 = rng.normal(size=(4, 5, 6))
    A3 = np.zeros((9, 1, 5, 6))
    for k in range(2):
        for m in range(2):
            A3[3 * k + m, 0] = A2[2 * k + m]
    s3 = orc.interp3(g3, r, v, A3)
    s2 = orc.interp(g2, r[:, :2], v[:, :2], A2)
    assert np.allclose(s3[:2], s2, rtol=1e-14, atol=1e-14)
    assert np.all(s3[2] == 0.0)


@pytest.mark.parametrize("n_ch", [3, 1])
def test_interp3_adjoint(orc, n_ch):
    g = _grid3(5, 4, 3)
    rng = np.random.default_rng(4 + n_ch)
    T = 300
    r = rng.uniform(-7, 7, size=(T, 3))
    v = rng.normal(size=(T, 3))
    A = rng.normal(size=(3 * n_ch, 3, 4, 5))
    s = rng.normal(size=(n_ch, T))
    lhs = np.sum(orc.interp3(g, r, v, A) * s)
    rhs = np.sum(A * orc.interp3_T(g, r, v, s))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_laplacian3_vs_scipy(orc):
    ndi = pytest.importorskip("scipy.ndimage")
    g = _grid3(5, 4, 3)
    f = np.random.default_rng(5).normal(size=(3, 4, 5))
    assert np.allclose(orc.laplacian3(g, f), ndi.laplace(f, mode="nearest"), rtol=1e-14, atol=1e-14)
    n = 60
    D = np.stack([orc.laplacian3(g, np.eye(n)[k].reshape(3, 4, 5)).reshape(-1) for k in range(n)], 1)
    assert np.array_equal(D, D.T)
    # one slice: the 5-point Laplacian of the pinned 2-D oracle
    g1 = _grid3(5, 4, 1)
    f1 = f[:1]
    g2 = {k: g1[k] for k in ("nx", "ny", "x0", "y0", "dx", "dy")}
    assert np.allclose(orc.laplacian3(g1, f1)[0], orc.laplacian(g2, f1[0]), rtol=0, atol=1e-14)


def _dense_normal(orc, g, r, v, gamma, rows):
    """Dense normal matrix of the Core Stage restricted to channel rows
    `rows`, built from unit vectors."""
    T = r.shape[0]
    nz, ny, nx = g["nz"], g["ny"], g["nx"]
    N = nx * ny * nz
    nc = 3 * len(rows)
    cols = []
    for q in range(nc * N):
        e = np.zeros(nc * N)
        e[q] = 1.0
        E = e.reshape(nc, nz, ny, nx)
        E9 = np.zeros((9, nz, ny, nx))
        for a, k in enumerate(rows):
            E9[3 * k:3 * k + 3] = E[3 * a:3 * a + 3]
        s = orc.interp3(g, r, v, E9)
        s_keep = np.zeros_like(s)
        s_keep[rows] = s[rows]
        MtM = orc.interp3_T(g, r, v, s_keep)
        MtM = np.concatenate([MtM[3 * k:3 * k + 3] for k in rows]) / T
        lap = np.stack([orc.laplacian3(g, orc.laplacian3(g, E[m])) for m in range(nc)])
        cols.append((MtM + gamma * lap).reshape(-1))
    return np.stack(cols, 1)


def test_core_stage3_vs_dense_solve(orc):
    g = _grid3(3, 3, 2)
    rng = np.random.default_rng(6)
    T = 90
    r = rng.uniform(-4, 4, size=(T, 3))
    v = rng.normal(size=(T, 3))
    s = rng.normal(size=(3, T))
    gamma = 1e-2
    Mn = _dense_normal(orc, g, r, v, gamma, [0, 1, 2])
    assert np.allclose(Mn, Mn.T, atol=1e-12)
    b = (orc.interp3_T(g, r, v, s) / T).reshape(-1)
    want = np.linalg.solve(Mn, b)
    Ahat, u, hist = orc.core_stage3(g, r, v, s, gamma, max_iter=600)
    assert np.allclose(Ahat.reshape(-1), want, rtol=1e-7, atol=1e-9 * np.abs(want).max())
    assert np.array_equal(u, Ahat[0] + Ahat[4] + Ahat[8])
    A2, _, hist2 = orc.core_stage3(g, r, v, s, gamma, max_iter=10000, rel_tol=1e-3)
    assert hist2[-1] <= 1e-3 * np.linalg.norm(b) and len(hist2) < 600


@pytest.mark.parametrize("k", [0, 2])
def test_core_stage3_single_channel_vs_dense_solve(orc, k):
    g = _grid3(3, 3, 2)
    rng = np.random.default_rng(8 + k)
    T = 70
    r = rng.uniform(-4, 4, size=(T, 3))
    v = rng.normal(size=(T, 3))
    s_k = rng.normal(size=T)
    gamma = 1e-2
    Mn = _dense_normal(orc, g, r, v, gamma, [k])
    s3 = np.zeros((3, T))
    s3[k] = s_k
    b = orc.interp3_T(g, r, v, s3)[3 * k:3 * k + 3].reshape(-1) / T
    want = np.linalg.solve(Mn, b)
    A, Akk, _ = orc.core_stage3(g, r, v, s_k, gamma, max_iter=400, channel=k)
    assert A.shape == (3, 2, 3, 3)
    assert np.allclose(A.reshape(-1), want, rtol=1e-7, atol=1e-9 * np.abs(want).max())
    assert np.array_equal(Akk, A[k])


def test_core_stage3_single_slice_equals_2d(orc):
    """One slice, no z velocity and a silent third channel: the 9-component
    solve holds the 2-D Core Stage in its (0..1, 0..1) block (the other
    components stay zero and add nothing to any inner product of CG)."""
    g3 = _grid3(6, 5, 1)
    g2 = {k: g3[k] for k in ("nx", "ny", "x0", "y0", "dx", "dy")}
    rng = np.random.default_rng(11)
    T = 120
    r = np.concatenate([rng.uniform(-5, 5, size=(T, 2)), np.zeros((T, 1))], 1)
    v = np.concatenate([rng.normal(size=(T, 2)), np.zeros((T, 1))], 1)
    s = np.concatenate([rng.normal(size=(2, T)), np.zeros((1, T))])
    gamma = 3e-3
    # 20 steps: residual down by 3e4, still far above round-off, so the two
    # sequences of iterates agree to round-off
    A3, u3, h3 = orc.core_stage3(g3, r, v, s, gamma, max_iter=20)
    A2, u2, h2 = orc.core_stage(g2, r[:, :2], v[:, :2], s[:2], gamma, max_iter=20)
    scale = np.abs(A2).max()
    for k in range(2):
        for m in range(2):
            assert np.allclose(A3[3 * k + m, 0], A2[2 * k + m], rtol=0, atol=1e-13 * scale)
    assert np.all(A3[2::3] == 0.0) and np.all(A3[6:] == 0.0)
    assert np.allclose(h3, h2, rtol=1e-12)
    assert np.allclose(u3[0], u2, rtol=0, atol=1e-13 * scale)

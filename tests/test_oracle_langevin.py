"""Pins for the oracle's Langevin family and MPI kernel (Eq. momentum,
Eq. kernel:matrix, Eq. kernel:trace), checked against mpmath at high
precision, closed-form limits and the Jacobian definition."""
import math

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")


@pytest.fixture(autouse=True)
def _mp_precision():
    """90 significant digits for every mpmath reference here, restored after."""
    with mp.workdps(90):
        yield


def _mp_family(z):
    z = mp.mpf(z)
    L = mp.coth(z) - 1 / z
    Lp = 1 / z**2 - 1 / mp.sinh(z) ** 2
    Lpp = -2 / z**3 + 2 * mp.cosh(z) / mp.sinh(z) ** 3
    a = L / z
    d = (Lp - a) / z**2
    e = Lpp / z
    return dict(L=L, Lp=Lp, Lpp=Lpp, a=a, d=d, e=e)


def test_langevin_vs_mpmath(orc):
    zs = np.concatenate([np.logspace(-8, 3, 181), [0.1, 0.5, 1.0, 1.5, 1.99, 2.0, 2.01, 3.0, 10.0]])
    got = orc.langevin(zs)
    worst = 0.0
    for k, z in enumerate(zs):
        ref = _mp_family(z)
        for name, val in ref.items():
            rel = abs(got[name][k] - float(val)) / abs(float(val))
            worst = max(worst, rel)
            assert rel < 2e-14, (name, z, got[name][k], float(val))
    assert worst < 2e-14


def test_langevin_limits(orc):
    g = orc.langevin(np.array([0.0, 1e-7, 1e4]))
    # z -> 0: L ~ z/3, a = L' = 1/3, d = -2/45, e = -2/15 (Taylor of coth)
    assert g["L"][0] == 0.0
    assert abs(g["L"][1] / 1e-7 - 1 / 3) < 1e-15
    for name, lim in (("a", 1 / 3), ("Lp", 1 / 3), ("d", -2 / 45), ("e", -2 / 15)):
        assert abs(g[name][0] - lim) < 1e-16, name
    # z -> inf: L -> 1 - 1/z, L' ~ 1/z^2, a ~ 1/z
    z = 1e4
    assert abs(g["L"][2] - (1 - 1 / z)) < 1e-15
    assert abs(g["Lp"][2] * z * z - 1) < 1e-12
    assert abs(g["a"][2] * z - (1 - 1 / z)) < 1e-12


def test_branch_continuity(orc):
    """Series (z < 2) and closed-form (z >= 2) branches both within a few ulp
    of the exact values on either side of the switch."""
    for z in (2.0 - 1e-13, 2.0, 2.0 + 1e-13):
        got = orc.langevin(np.array([z]))
        ref = _mp_family(z)
        for name, val in ref.items():
            assert abs(got[name][0] - float(val)) <= 2e-15 * abs(float(val)), (name, z)


def _rot(th):
    return np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])


def test_kernel_matrix_structure(orc):
    # K(0) = I/3
    K0 = orc.kernel_matrix(np.zeros((1, 2)))[0]
    assert np.allclose(K0, np.eye(2) / 3, atol=1e-16, rtol=0)
    rng = np.random.default_rng(1)
    ys = rng.normal(size=(50, 2)) * rng.choice([0.01, 0.3, 1.0, 3.0, 30.0], size=(50, 1))
    K = orc.kernel_matrix(ys)
    fam = orc.langevin(np.linalg.norm(ys, axis=1))
    for k, y in enumerate(ys):
        z = np.linalg.norm(y)
        yh = y / z
        yp = np.array([-yh[1], yh[0]])
        # eigenpairs: L' along y, L/z across (Eq. kernel:matrix)
        assert np.allclose(K[k] @ yh, fam["Lp"][k] * yh, rtol=1e-13, atol=1e-16)
        assert np.allclose(K[k] @ yp, fam["L"][k] / z * yp, rtol=1e-13, atol=1e-16)
        # trace = kappa with n = 2 (Eq. kernel:trace)
        assert abs(np.trace(K[k]) - (fam["Lp"][k] + fam["L"][k] / z)) < 1e-14
        # rotation covariance K(Ry) = R K(y) R^T
        R = _rot(0.7 * k)
        KR = orc.kernel_matrix((R @ y)[None])[0]
        assert np.allclose(KR, R @ K[k] @ R.T, rtol=1e-12, atol=1e-15)


def _mp_M(H, beta):
    """Langevin magnetisation direction field L(beta |H|) H/|H| (Eq. momentum)."""
    h = mp.sqrt(H[0] ** 2 + H[1] ** 2)
    z = beta * h
    L = mp.coth(z) - 1 / z
    return [L * H[0] / h, L * H[1] / h]


@pytest.mark.parametrize("H", [(3e-4, -1e-4), (2e-3, 5e-3), (-1e-2, 4e-2), (1e-6, 2e-6)])
def test_kernel_is_jacobian_of_magnetisation(orc, H):
    """beta K(beta H) = d/dH [L(beta|H|) H/|H|]: fixes the beta scaling and the
    form of Eq. kernel:matrix (the time derivative identity of Sec. 2)."""
    beta = 2331.350896656040
    J = np.zeros((2, 2))
    for b in range(2):
        def comp(hb, a):
            HH = [mp.mpf(H[0]), mp.mpf(H[1])]
            HH[b] = hb
            return _mp_M(HH, beta)[a]
        for a in range(2):
            J[a, b] = float(mp.diff(lambda hb: comp(hb, a), mp.mpf(H[b])))
    K = orc.kernel_matrix(np.array([[beta * H[0], beta * H[1]]]))[0]
    assert np.allclose(beta * K, J, rtol=1e-12, atol=0)


def test_pair_vs_mpmath(orc):
    """J w = beta K(beta G(x - r)) G v for a non-diagonal G, against mpmath's
    Jacobian of the magnetisation applied to G v."""
    model = {"beta": 600.0, "G": [[2e-3, 4e-4], [4e-4, -1e-3]], "p": [[1, 0], [0, 1]]}
    x, r, v = np.array([1.2, -0.4]), np.array([-0.3, 0.9]), np.array([0.05, -0.02])
    G = np.array(model["G"])
    H0 = G @ (x - r)
    w = G @ v
    J = np.zeros((2, 2))
    for b in range(2):
        for a in range(2):
            def f(hb, a=a, b=b):
                HH = [mp.mpf(H0[0]), mp.mpf(H0[1])]
                HH[b] = hb
                return _mp_M(HH, model["beta"])[a]
            J[a, b] = float(mp.diff(f, mp.mpf(H0[b])))
    got = orc.pair(model, x, r, v)
    assert np.allclose(got, J @ w, rtol=1e-12, atol=0)


def test_beta_reading_fwhm(orc):
    """The configs' beta gives the trace kernel kappa a 1 mm FWHM at
    mu0 G = 2.5 T/m (reading of the configs' "1 mm PSF")."""
    from paper_2505_22797_gb300.synthetic import BETA_1MM, G_MM
    z_half = BETA_1MM * G_MM * 0.5
    f = orc.langevin(np.array([0.0, z_half]))
    kap0 = f["Lp"][0] + f["a"][0]
    kap = f["Lp"][1] + f["a"][1]
    assert abs(kap / kap0 - 0.5) < 1e-12


def test_hsat_from_table(orc):
    """Eq. hsat with the particle values of Table tab:params_si gives
    mu0 H_sat = 1.760 mT, i.e. beta = 1/(mu0 H_sat) = 568.2 1/T."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_params.json")) as fh:
        P = json.load(fh)
    kb, T, Ms, d = P["k_b"], P["T_B"], P["M_sat"], P["d"]
    mu0_hsat = kb * T / (Ms * math.pi / 6 * d**3)
    assert abs(mu0_hsat - P["mu0_Hsat_T"]) < 5e-7
    assert abs(1 / mu0_hsat - P["beta_per_T"]) < 0.1

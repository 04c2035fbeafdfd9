"""The seeded synthetic inputs (the stand-ins for the paper's scans): every
workload is reproducible from its seeds, has the stated sizes and shapes,
velocities are the time derivative of the positions (per sample), phantoms and
trajectories stay in their stated ranges, and the noise has the stated level."""
import math

import numpy as np
import pytest

from paper_2505_22797_gb300 import synthetic as syn

SIZES = {"c1": (32, 32, 1632), "c2": (128, 128, 65536), "c4": (256, 256, 262144),
         "c5": (512, 512, 1 << 20)}


def _same(a, b):
    for k in ("r", "v", "c"):
        assert np.array_equal(a[k], b[k]), k
    assert a["grid"] == b["grid"] and a["model"] == b["model"]


@pytest.mark.parametrize("name", ["c1", "c2", "c2_partial", "c4", "c5"])
def test_workloads_are_reproducible_and_sized(name):
    a, b = syn.config(name), syn.config(name)
    _same(a, b)
    g = a["grid"]
    if name == "c2_partial":
        assert (g["nx"], g["ny"]) == (128, 128)
        assert a["r"].shape == (round(0.6 * 65536), 2)
    else:
        nx, ny, T = SIZES[name]
        assert (g["nx"], g["ny"]) == (nx, ny) and a["r"].shape == (T, 2) and a["v"].shape == (T, 2)
    assert a["c"].shape == (g["ny"], g["nx"])
    assert a["c"].min() >= 0.0 and a["c"].max() <= 2.0 and a["c"].any()


def _check_velocity(r, v, rel):
    """Central differences of r (one sample apart) against v at interior
    samples: the error of the difference quotient is O(|r'''|)."""
    d = (r[2:] - r[:-2]) / 2.0
    err = np.abs(d - v[1:-1]).max()
    assert err <= rel * np.abs(v).max(), (err, np.abs(v).max())


def test_velocities_are_time_derivatives():
    _check_velocity(*syn.lissajous(1632, 17, 16), 1e-3)
    _check_velocity(*syn.spiral(65536, 32), 1e-3)
    _check_velocity(*syn.lissajous_excited(1 << 16, 17, 16, 24.0, 1.5, 25.0), 1e-3)
    r, v = syn.lissajous3(65536, 17, 16, 15)
    _check_velocity(r, v, 1e-4)


def test_trajectory_ranges():
    r, _ = syn.lissajous(1632, 17, 16)
    assert np.abs(r).max() <= 12.0 + 1e-12
    r, _ = syn.spiral(65536, 32)
    rho = np.hypot(r[:, 0], r[:, 1])
    assert rho.max() <= 12.0 and np.all(np.diff(rho) >= 0)          # outward Archimedean
    th = np.unwrap(np.arctan2(r[1:, 1], r[1:, 0]))
    assert abs((th[-1] - th[0]) / (2 * math.pi) - 32) < 0.01         # 32 turns
    r, _ = syn.lissajous3(65536, 17, 16, 15)
    assert np.all(np.abs(r).max(axis=0) <= np.array([12.0, 12.0, 6.0]) + 1e-12)


def test_phantom_values():
    g = syn.square_grid(64)
    c = syn.ellipses(g, np.random.default_rng(0))
    assert c.min() >= 0.0 and c.max() <= 1.0 and c.any()
    p = syn.point_sources(c, np.random.default_rng(1), n=4, value=2.0)
    assert np.count_nonzero(p == 2.0) == 4 and np.array_equal(p[p != 2.0], c[p != 2.0])
    vs = syn.vessels(g, np.random.default_rng(2))
    assert vs.min() >= 0.0 and vs.max() == pytest.approx(1.0)


def test_noise_level():
    s = np.sin(np.linspace(0, 20, 200000)).reshape(2, -1) * 3.0
    n = syn.add_noise(s, 0.01, 5) - s
    assert abs(n.std() / (0.01 * 3.0) - 1.0) < 0.01 and abs(n.mean()) < 1e-3 * 0.03 * 10
    assert np.array_equal(syn.add_noise(s, 0.01, 5), syn.add_noise(s, 0.01, 5))


def test_batch_frames():
    a, b = syn.batch_frames(), syn.batch_frames()
    assert len(a) == 64
    for fa, fb in zip(a, b):
        _same(fa, fb)
        assert fa["grid"]["nx"] in (64, 96, 128, 192, 256)
        assert 8192 <= fa["r"].shape[0] <= 131072


def test_three_dimensional_workload():
    a, b = syn.config3("3d"), syn.config3("3d")
    _same(a, b)
    g = a["grid"]
    assert (g["nx"], g["ny"], g["nz"]) == (48, 48, 24) and a["r"].shape == (65536, 3)
    assert a["c"].shape == (24, 48, 48) and a["c"].min() >= 0.0 and a["c"].max() <= 1.0
    assert np.asarray(a["model"]["G"]).shape == (3, 3) and len(a["model"]["p"]) == 3

"""Seeded synthetic inputs shaped like the paper's 2-D FFP scans.

This module only draws inputs: voxel grids, field-free-point trajectories with
their analytic velocities, ellipse/point-source/vessel phantoms and additive
Gaussian noise.  It holds none of the reconstruction arithmetic, so both the
CUDA library's tests and the FP64 oracle can be fed from it.

Units: lengths in mm, the selection gradient G in T/mm, beta = 1/(mu0 H_sat) in
1/T, time in samples (velocities are d r / d(sample index)).

The paper's data (the EMWA Bruker scans, Sec. 3.1, and the non-Lissajous
scans of Sec. 3.6) are not available; these generators stand in for them with
the same scanner shape: a 24 mm x 24 mm drive-field FoV, 12 mm drive
amplitudes, mu0 G = diag(2.5, 2.5) T/m, 1632 samples per Lissajous period and
two receive channels p_x = (1, 0), p_y = (0, 1).
"""
from __future__ import annotations

import math

import numpy as np

# beta such that the trace kernel kappa (Eq. kernel:trace, n = 2) has a 1 mm
# FWHM at mu0 G = 2.5 T/m: kappa(z) falls to half its peak at z = 2.914188620820,
# so beta * 2.5e-3 T/mm * 1 mm = 2 * 2.914188620820.
BETA_1MM = 2331.350896656040
G_MM = 2.5e-3  # 2.5 T/m in T/mm


def default_model(beta: float = BETA_1MM, g: float = G_MM, n_ch: int = 2) -> dict:
    p = [[1.0, 0.0], [0.0, 1.0]][:n_ch]
    return {"beta": float(beta), "G": [[g, 0.0], [0.0, g]], "p": p}


def square_grid(n: int, fov_mm: float = 24.0, ny: int | None = None) -> dict:
    """n x ny voxels covering a centred fov_mm x fov_mm square."""
    ny = n if ny is None else ny
    return {"nx": int(n), "ny": int(ny), "x0": -fov_mm / 2, "y0": -fov_mm / 2,
            "dx": fov_mm / n, "dy": fov_mm / ny}


def voxel_centres(grid: dict) -> tuple[np.ndarray, np.ndarray]:
    xs = grid["x0"] + (np.arange(grid["nx"]) + 0.5) * grid["dx"]
    ys = grid["y0"] + (np.arange(grid["ny"]) + 0.5) * grid["dy"]
    return xs, ys


# ---------------------------------------------------------------------------
# Trajectories: r[T, 2] (mm) and v[T, 2] = dr/dt (mm per sample).

def lissajous(T: int, fx: float, fy: float, amp: float = 12.0, phase: float = 0.0):
    """r(t) = amp (sin(2 pi fx t/T + phase), sin(2 pi fy t/T)): fx, fy periods
    per T samples (the scanner's Lissajous of Eq. lissajous, sine phase)."""
    t = np.arange(T, dtype=np.float64)
    wx, wy = 2 * math.pi * fx / T, 2 * math.pi * fy / T
    r = np.stack([amp * np.sin(wx * t + phase), amp * np.sin(wy * t)], axis=1)
    v = np.stack([amp * wx * np.cos(wx * t + phase), amp * wy * np.cos(wy * t)], axis=1)
    return r, v


def lissajous_excited(T: int, fx: float, fy: float, amp: float, amp_e: float, mult_e: float):
    """Lissajous drive plus a fast 1-D excitation along x (the trajectory shape
    of Sec. 3.6): r_x = amp sin(2 pi fx t/T) + amp_e sin(2 pi mult_e fx t/T),
    r_y = amp sin(2 pi fy t/T)."""
    t = np.arange(T, dtype=np.float64)
    wx, wy, we = (2 * math.pi * fx / T, 2 * math.pi * fy / T,
                  2 * math.pi * mult_e * fx / T)
    r = np.stack([amp * np.sin(wx * t) + amp_e * np.sin(we * t), amp * np.sin(wy * t)], axis=1)
    v = np.stack([amp * wx * np.cos(wx * t) + amp_e * we * np.cos(we * t),
                  amp * wy * np.cos(wy * t)], axis=1)
    return r, v


def spiral(T: int, turns: float = 32.0, radius: float = 12.0):
    """Archimedean spiral r(theta) = radius (theta/theta_max)(cos, sin),
    theta = 2 pi turns t/T."""
    t = np.arange(T, dtype=np.float64)
    th_max = 2 * math.pi * turns
    th = th_max * t / T
    dth = th_max / T
    rho = radius * th / th_max
    drho = radius * dth / th_max
    r = np.stack([rho * np.cos(th), rho * np.sin(th)], axis=1)
    v = np.stack([drho * np.cos(th) - rho * np.sin(th) * dth,
                  drho * np.sin(th) + rho * np.cos(th) * dth], axis=1)
    return r, v


def subsample(r, v, keep: float, seed: int):
    """A seeded random subset of the samples (kept in time order)."""
    rng = np.random.default_rng(seed)
    T = r.shape[0]
    idx = np.sort(rng.choice(T, size=max(1, int(round(keep * T))), replace=False))
    return r[idx], v[idx], idx


# ---------------------------------------------------------------------------
# Phantoms: c[ny, nx].

def ellipses(grid: dict, rng, n: int | None = None, semi=(1.5, 6.0),
             centre_frac: float = 0.7) -> np.ndarray:
    xs, ys = voxel_centres(grid)
    X, Y = np.meshgrid(xs, ys)
    fov_x, fov_y = grid["nx"] * grid["dx"], grid["ny"] * grid["dy"]
    cx0, cy0 = grid["x0"] + fov_x / 2, grid["y0"] + fov_y / 2
    if n is None:
        n = int(rng.integers(3, 7))
    c = np.zeros((grid["ny"], grid["nx"]))
    for _ in range(n):
        ex = cx0 + rng.uniform(-0.5, 0.5) * centre_frac * fov_x
        ey = cy0 + rng.uniform(-0.5, 0.5) * centre_frac * fov_y
        a, b = rng.uniform(*semi), rng.uniform(*semi)
        th = rng.uniform(0, math.pi)
        val = rng.uniform(0, 1)
        dx, dy = X - ex, Y - ey
        u = (dx * math.cos(th) + dy * math.sin(th)) / a
        w = (-dx * math.sin(th) + dy * math.cos(th)) / b
        c[u * u + w * w <= 1.0] = val
    return c


def point_sources(c: np.ndarray, rng, n: int = 4, value: float = 2.0) -> np.ndarray:
    c = c.copy()
    flat = rng.choice(c.size, size=n, replace=False)
    c.reshape(-1)[flat] = value
    return c


def _blur(img: np.ndarray, sigma_px: float) -> np.ndarray:
    rad = int(math.ceil(3 * sigma_px))
    k = np.exp(-0.5 * (np.arange(-rad, rad + 1) / sigma_px) ** 2)
    k /= k.sum()
    pad = np.pad(img, rad, mode="reflect")
    tmp = np.apply_along_axis(lambda row: np.convolve(row, k, mode="valid"), 1, pad)
    return np.apply_along_axis(lambda col: np.convolve(col, k, mode="valid"), 0, tmp)


def vessels(grid: dict, rng, n_curves: int = 6, width_px: float = 2.0,
            blur_px: float = 1.5) -> np.ndarray:
    """Smooth random curves (random-phase Fourier paths) rasterised at the given
    width, Gaussian blurred, scaled to [0, 1]."""
    ny, nx = grid["ny"], grid["nx"]
    img = np.zeros((ny, nx))
    jj, ii = np.mgrid[0:ny, 0:nx]
    for _ in range(n_curves):
        s = np.linspace(0, 1, 4 * max(nx, ny))
        px = 0.5 + sum(rng.uniform(-0.25, 0.25) / (h + 1) * np.sin(2 * math.pi * (h + 1) * s
                       + rng.uniform(0, 2 * math.pi)) for h in range(3))
        py = 0.5 + sum(rng.uniform(-0.25, 0.25) / (h + 1) * np.cos(2 * math.pi * (h + 1) * s
                       + rng.uniform(0, 2 * math.pi)) for h in range(3))
        for x, y in zip(px * nx, py * ny):
            j0, i0 = int(y), int(x)
            lo_j, hi_j = max(0, j0 - 2), min(ny, j0 + 3)
            lo_i, hi_i = max(0, i0 - 2), min(nx, i0 + 3)
            d2 = (ii[lo_j:hi_j, lo_i:hi_i] + 0.5 - x) ** 2 + (jj[lo_j:hi_j, lo_i:hi_i] + 0.5 - y) ** 2
            img[lo_j:hi_j, lo_i:hi_i][d2 <= (width_px / 2) ** 2] = 1.0
    img = _blur(img, blur_px)
    mx = img.max()
    return img / mx if mx > 0 else img


def add_noise(s_clean: np.ndarray, frac: float, seed: int) -> np.ndarray:
    """s + N(0, (frac * max|s|)^2), the measurement noise of the configs."""
    rng = np.random.default_rng(seed)
    sig = frac * float(np.max(np.abs(s_clean)))
    return s_clean + rng.normal(0.0, sig, size=s_clean.shape)


# ---------------------------------------------------------------------------
# Named workloads.

def config(name: str) -> dict:
    """The five workloads: inputs without the data s (which needs a forward
    operator; callers add it).  Keys: grid, model, r, v, c, n_it, n_cg,
    noise_frac, noise_seed, clip_pct."""
    m = default_model()
    if name == "c1":  # plain method, 32x32 Lissajous 17/16, T = 1632
        g = square_grid(32)
        r, v = lissajous(1632, 17, 16)
        c = ellipses(g, np.random.default_rng(101))
        return dict(name=name, grid=g, model=m, r=r, v=v, c=c, n_it=50, n_cg=20,
                    noise_frac=0.01, noise_seed=201, clip_pct=5.0)
    if name in ("c2", "c2_partial"):  # 128x128 spiral, T = 65536
        g = square_grid(128)
        r, v = spiral(65536, 32)
        rng = np.random.default_rng(102)
        c = point_sources(ellipses(g, rng), rng)
        if name == "c2_partial":
            r, v, _ = subsample(r, v, 0.6, 302)
        return dict(name=name, grid=g, model=m, r=r, v=v, c=c, n_it=100, n_cg=20,
                    noise_frac=0.01, noise_seed=202, clip_pct=5.0)
    if name == "c4":  # gradients: 256x256 Lissajous, T = 262144
        g = square_grid(256)
        r, v = lissajous(262144, 17, 16)
        c = ellipses(g, np.random.default_rng(104))
        return dict(name=name, grid=g, model=m, r=r, v=v, c=c, n_it=0, n_cg=0,
                    noise_frac=0.01, noise_seed=204, clip_pct=5.0)
    if name == "c5":  # large: 512x512 over 48 mm, excited Lissajous, T = 2^20
        g = square_grid(512, 48.0)
        r, v = lissajous_excited(1 << 20, 17, 16, 24.0, 1.5, 25.0)
        rng = np.random.default_rng(105)
        c = np.maximum(ellipses(g, rng, n=20, semi=(3.0, 12.0)), vessels(g, rng))
        return dict(name=name, grid=g, model=m, r=r, v=v, c=c, n_it=200, n_cg=20,
                    noise_frac=0.02, noise_seed=205, clip_pct=5.0)
    raise ValueError(f"unknown config {name!r}")


def batch_frames(n_frames: int = 64, seed: int = 403, sizes=(64, 96, 128, 192, 256),
                 t_range=(8192, 131072)) -> list[dict]:
    """The batched workload: frames of uneven grid size (uniform over sizes)
    and trajectory length (uniform integer in t_range), each with a Lissajous
    n/(n-1), n in [12, 40], or a 32-turn spiral (50/50)."""
    rng = np.random.default_rng(seed)
    frames = []
    m = default_model()
    for f in range(n_frames):
        n = int(rng.choice(sizes))
        T = int(rng.integers(t_range[0], t_range[1] + 1))
        g = square_grid(n)
        if rng.uniform() < 0.5:
            k = int(rng.integers(12, 41))
            r, v = lissajous(T, k, k - 1)
        else:
            r, v = spiral(T, 32)
        c = ellipses(g, np.random.default_rng(103 + 1000 * f))
        frames.append(dict(name=f"c3_{f}", grid=g, model=m, r=r, v=v, c=c, n_it=50,
                           n_cg=20, noise_frac=0.01, noise_seed=203 + 1000 * f,
                           clip_pct=5.0))
    return frames


def small(nx: int, ny: int, T: int, traj: str = "lissajous", seed: int = 7,
          fov_mm: float = 24.0) -> dict:
    """A small case for parity tests: any grid and length, seeded phantom."""
    g = square_grid(nx, fov_mm, ny)
    m = default_model()
    if traj == "lissajous":
        r, v = lissajous(T, 17 if T > 40 else 3, 16 if T > 40 else 2, amp=fov_mm / 2)
    elif traj == "spiral":
        r, v = spiral(T, max(1.0, min(32.0, T / 64)), radius=fov_mm / 2)
    else:
        raise ValueError(traj)
    c = ellipses(g, np.random.default_rng(seed))
    if not c.any():
        c[ny // 2, nx // 2] = 1.0
    return dict(name=f"small_{nx}x{ny}_{T}_{traj}", grid=g, model=m, r=r, v=v, c=c,
                n_it=3, n_cg=5, noise_frac=0.01, noise_seed=seed + 100, clip_pct=5.0)


# ---------------------------------------------------------------------------
# Three-dimensional field-free point.  The gradient has the paper's shape
# G = g diag(-1/2, -1/2, 1) (diag(-1, -1, 2) up to scale), g = 2.5 T/m along z,
# so the field of view along z is half that along x and y for the same drive
# amplitude in tesla.

def default_model3(beta: float = BETA_1MM, g: float = G_MM, n_ch: int = 3) -> dict:
    G = [[-0.5 * g, 0.0, 0.0], [0.0, -0.5 * g, 0.0], [0.0, 0.0, g]]
    p = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]][:n_ch]
    return {"beta": beta, "G": G, "p": p}


def box_grid3(nx: int, ny: int, nz: int, fov_xy: float = 24.0, fov_z: float = 12.0) -> dict:
    """Voxel grid centred on the origin: fov_xy x fov_xy x fov_z mm."""
    return {"nx": nx, "ny": ny, "nz": nz, "x0": -fov_xy / 2, "y0": -fov_xy / 2, "z0": -fov_z / 2,
            "dx": fov_xy / nx, "dy": fov_xy / ny, "dz": fov_z / nz}


def lissajous3(T: int, fx: float, fy: float, fz: float, amp=(12.0, 12.0, 6.0)):
    """r(t) = (ax sin(2 pi fx t/T), ay sin(2 pi fy t/T), az sin(2 pi fz t/T)),
    the 3-D Lissajous drive; v = dr/dt per sample."""
    t = np.arange(T, dtype=np.float64)
    w = [2 * math.pi * f / T for f in (fx, fy, fz)]
    r = np.stack([amp[q] * np.sin(w[q] * t) for q in range(3)], axis=1)
    v = np.stack([amp[q] * w[q] * np.cos(w[q] * t) for q in range(3)], axis=1)
    return r, v


def ellipsoids(grid3: dict, rng, n: int | None = None, semi=(1.5, 5.0)) -> np.ndarray:
    """Seeded phantom of axis-aligned ellipsoids (centres uniform in the
    central 70 %, semi-axes uniform in `semi` mm, scaled by half along z,
    values U[0, 1], later ones overwrite)."""
    xs = grid3["x0"] + (np.arange(grid3["nx"]) + 0.5) * grid3["dx"]
    ys = grid3["y0"] + (np.arange(grid3["ny"]) + 0.5) * grid3["dy"]
    zs = grid3["z0"] + (np.arange(grid3["nz"]) + 0.5) * grid3["dz"]
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    fov = [grid3["nx"] * grid3["dx"], grid3["ny"] * grid3["dy"], grid3["nz"] * grid3["dz"]]
    cen = [grid3["x0"] + fov[0] / 2, grid3["y0"] + fov[1] / 2, grid3["z0"] + fov[2] / 2]
    if n is None:
        n = int(rng.integers(3, 7))
    c = np.zeros((grid3["nz"], grid3["ny"], grid3["nx"]))
    for _ in range(n):
        e = [cen[q] + rng.uniform(-0.5, 0.5) * 0.7 * fov[q] for q in range(3)]
        a, b, h = rng.uniform(*semi), rng.uniform(*semi), 0.5 * rng.uniform(*semi)
        val = rng.uniform(0, 1)
        c[((X - e[0]) / a) ** 2 + ((Y - e[1]) / b) ** 2 + ((Z - e[2]) / h) ** 2 <= 1.0] = val
    return c


def config3(name: str = "3d") -> dict:
    """The 3-D FFP workload: 48 x 48 x 24 voxels over 24 x 24 x 12 mm, a 3-D
    Lissajous with 17 / 16 / 15 periods per T = 65 536 samples, three
    channels, 1 % noise."""
    if name != "3d":
        raise ValueError(f"unknown 3-D config {name!r}")
    g = box_grid3(48, 48, 24)
    r, v = lissajous3(65536, 17, 16, 15)
    c = ellipsoids(g, np.random.default_rng(106))
    return dict(name=name, grid=g, model=default_model3(), r=r, v=v, c=c, n_it=20, n_cg=20,
                noise_frac=0.01, noise_seed=206, clip_pct=5.0)


def small3(nx: int, ny: int, nz: int, T: int, seed: int = 9, n_ch: int = 3) -> dict:
    """A small 3-D case for parity tests."""
    g = box_grid3(nx, ny, nz)
    big = T > 60
    r, v = lissajous3(T, 17 if big else 3, 16 if big else 2, 15 if big else 1)
    c = ellipsoids(g, np.random.default_rng(seed))
    if not c.any():
        c[nz // 2, ny // 2, nx // 2] = 1.0
    return dict(name=f"small3_{nx}x{ny}x{nz}_{T}", grid=g, model=default_model3(n_ch=n_ch), r=r,
                v=v, c=c, noise_frac=0.01, noise_seed=seed + 100, clip_pct=5.0)


# ---------------------------------------------------------------------------
# Receive chain (the time convolution with a of Eq. core:formula:conva).  The
# measured system matrix from which the paper estimates a_hat and the SNR is
# not available; a synthetic chain stands in: a first-order high-pass (corner
# f_hp bins, so the DC bin is zero), a first-order low-pass (corner f_lp bins)
# and a delay of `delay` samples, per channel with different corners.

def transfer_function(T: int, n_ch: int = 2, f_hp=(3.0, 4.0), f_lp=(900.0, 700.0),
                      delay=(2.5, 3.0)) -> np.ndarray:
    """a_hat [n_ch, T//2 + 1] complex on the DFT bins of one period."""
    f = np.arange(T // 2 + 1, dtype=np.float64)
    out = np.empty((n_ch, f.size), dtype=np.complex128)
    for k in range(n_ch):
        hp = (1j * f / f_hp[k]) / (1 + 1j * f / f_hp[k])
        lp = 1 / (1 + 1j * f / f_lp[k])
        out[k] = hp * lp * np.exp(-2j * np.pi * f * delay[k] / T)
    if T % 2 == 0:  # the Nyquist bin of a real impulse response is real
        out[:, -1] = out[:, -1].real
    return out


def measured_signal(s_model: np.ndarray, a_hat: np.ndarray, noise_frac: float, seed: int):
    """The raw signal of a chain with transfer function a_hat: the model
    signal circularly convolved with a (one period), plus white noise of
    standard deviation noise_frac * max|raw|.  Returns (raw, snr) with the
    per-bin SNR |a_hat s_hat|^2 / (T sigma^2) (signal power over the noise
    power in that bin), the quantity thresholded in Sec. 3.2."""
    s_model = np.atleast_2d(s_model)
    T = s_model.shape[1]
    S = np.fft.rfft(s_model, axis=1) * a_hat
    clean = np.fft.irfft(S, n=T, axis=1)
    sig = noise_frac * np.abs(clean).max()
    raw = clean + np.random.default_rng(seed).normal(0.0, sig, size=clean.shape)
    snr = np.abs(S) ** 2 / (T * sig * sig) if sig > 0 else np.full(S.shape, np.inf)
    return raw, snr

"""FP64 CPU oracle for the MPI reconstruction path (test infrastructure only).

This module and ``mpi_oracle.c`` are the plain, slow, obviously correct
reference the CUDA library is checked against.  Only the test suite, the smoke
check and the CPU-baseline leg of the benchmark may import it; the library
never does, and the two share no code.  Inputs are numpy arrays; a ``model`` is
a mapping with ``beta`` (1/T), ``G`` (2x2, T per length unit) and ``p``
(n_ch x 2 receive directions); a ``grid`` is a mapping with ``nx, ny, x0, y0,
dx, dy`` (voxel centre (x0 + (i+1/2)dx, y0 + (j+1/2)dy)).

The pair sums (A, A^T, d/dbeta, the convolution) live in C for speed; the
iterations (CG, the ZeroShot-PnP loop of Algorithm 1, the Core Stage solve)
are written here step by step in numpy FP64.

Parity status per function (what pins each one lives in tests/test_oracle_*):
  langevin, kernel_matrix, pair, forward, adjoint, dbeta, frob2,
  interp, interp_T, laplacian, conv_kernel, conv, conv_fft, cg,
  percentile_clamp, variance, gaussian5, core_stage: pinned.
  kernel_matrix3, pair3, forward3, adjoint3, frob2_3, conv_kernel3, conv3,
  gaussian5_3d (three-dimensional FFP): pinned.
  interp3, interp3_T, laplacian3, core_stage3 (Core Stage with n = 3): pinned.
  laplacian_h, laplacian3_h, conv_kernel_trK, conv_kernel3_trK,
  weighted_trace, weighted_trace3 (grid-scaled regulariser, gradient-weighted
  trace and its kernel): pinned.
  transfer_correct (DFT division by the transfer function, SNR
  thresholding): pinned.
  pnp: pinned step by step (identity-operator closed form, Algorithm 1
  bookkeeping); the full reconstruction has no printed example in the paper,
  so its end-to-end values are "parity unpinned" at paper level.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmpi_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile mpi_oracle.c with gcc (-O2, OpenMP, IEEE semantics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC",
           "-fno-fast-math", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double)]


class _Model(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("G", ctypes.c_double * 4),
                ("n_ch", ctypes.c_int), ("p", ctypes.c_double * 4)]


class _Grid3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class _Model3(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("G", ctypes.c_double * 9),
                ("n_ch", ctypes.c_int), ("p", ctypes.c_double * 9)]


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.og_langevin.argtypes = [_I64, _D, _D, _D, _D, _D, _D, _D]
            lib.og_kernel_matrix.argtypes = [_I64, _D, _D]
            lib.og_pair_export.argtypes = [P(_Model), _D, _D, _D, _D]
            lib.og_forward.argtypes = [P(_Model), P(_Grid), _I64, _D, _D, _D, _D]
            lib.og_adjoint_sel.argtypes = [P(_Model), P(_Grid), _I64, _D, _D, _D, _I64,
                                           P(_I64), _D]
            lib.og_dbeta.argtypes = [P(_Model), P(_Grid), _I64, _D, _D, _D, _D, _D, _D]
            lib.og_frob2.argtypes = [P(_Model), P(_Grid), _I64, _D, _D, _D]
            lib.og_frob2.restype = ctypes.c_double
            lib.og_interp.argtypes = [P(_Grid), _I64, _D, _D, _D, _D]
            lib.og_interp_T.argtypes = [P(_Grid), _I64, _D, _D, _D, _D]
            lib.og_laplacian.argtypes = [P(_Grid), _D, _D]
            lib.og_conv_kernel.argtypes = [P(_Model), P(_Grid), _D]
            lib.og_conv_kernel_component.argtypes = [P(_Model), P(_Grid), ctypes.c_int, _D]
            lib.og_conv.argtypes = [P(_Grid), _D, _D, _D]
            lib.og_num_threads.restype = ctypes.c_int
            lib.og_set_num_threads.argtypes = [ctypes.c_int]
            lib.og_set_num_threads.restype = None
            lib.og_kernel_matrix3.argtypes = [_I64, _D, _D]
            lib.og_pair3_export.argtypes = [P(_Model3), _D, _D, _D, _D]
            lib.og_forward3.argtypes = [P(_Model3), P(_Grid3), _I64, _D, _D, _D, _D]
            lib.og_adjoint3_sel.argtypes = [P(_Model3), P(_Grid3), _I64, _D, _D, _D, _I64,
                                            ctypes.POINTER(_I64), _D]
            lib.og_frob2_3.argtypes = [P(_Model3), P(_Grid3), _I64, _D, _D]
            lib.og_frob2_3.restype = ctypes.c_double
            lib.og_conv_kernel3.argtypes = [P(_Model3), P(_Grid3), _D]
            lib.og_conv3.argtypes = [P(_Grid3), _D, _D, _D]
            lib.og_interp3.argtypes = [P(_Grid3), ctypes.c_int, _I64, _D, _D, _D, _D]
            lib.og_interp3_T.argtypes = [P(_Grid3), ctypes.c_int, _I64, _D, _D, _D, _D]
            lib.og_laplacian3.argtypes = [P(_Grid3), _D, _D]
            lib.og_laplacian_h.argtypes = [P(_Grid), _D, _D]
            lib.og_laplacian3_h.argtypes = [P(_Grid3), _D, _D]
            lib.og_conv_kernel_trK.argtypes = [P(_Model), P(_Grid), _D]
            lib.og_conv_kernel3_trK.argtypes = [P(_Model3), P(_Grid3), _D]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _grid(g) -> _Grid:
    return _Grid(int(g["nx"]), int(g["ny"]), float(g["x0"]), float(g["y0"]),
                 float(g["dx"]), float(g["dy"]))


def _model(m) -> _Model:
    G = np.asarray(m["G"], dtype=np.float64).reshape(4)
    p = np.asarray(m["p"], dtype=np.float64).reshape(-1, 2)
    n_ch = p.shape[0]
    if n_ch not in (1, 2):
        raise ValueError("n_ch must be 1 or 2")
    pp = np.zeros(4)
    pp[: 2 * n_ch] = p.reshape(-1)
    return _Model(float(m["beta"]), (ctypes.c_double * 4)(*G), n_ch,
                  (ctypes.c_double * 4)(*pp))


def _grid3(g) -> _Grid3:
    return _Grid3(int(g["nx"]), int(g["ny"]), int(g["nz"]), float(g["x0"]), float(g["y0"]),
                  float(g["z0"]), float(g["dx"]), float(g["dy"]), float(g["dz"]))


def _model3(m) -> _Model3:
    G = np.asarray(m["G"], dtype=np.float64).reshape(9)
    p = np.asarray(m["p"], dtype=np.float64).reshape(-1, 3)
    n_ch = p.shape[0]
    if n_ch not in (1, 2, 3):
        raise ValueError("n_ch must be 1, 2 or 3")
    pp = np.zeros(9)
    pp[: 3 * n_ch] = p.reshape(-1)
    return _Model3(float(m["beta"]), (ctypes.c_double * 9)(*G), n_ch, (ctypes.c_double * 9)(*pp))


def num_threads() -> int:
    return int(_load().og_num_threads())


def set_num_threads(n: int) -> None:
    """Host threads of the oracle's parallel loops (timing only: the loops
    are over independent outputs, so results do not depend on it)."""
    _load().og_set_num_threads(int(n))


# ---------------------------------------------------------------------------
# Langevin family and the MPI kernel (Eq. momentum, Eq. kernel:matrix)

def langevin(z) -> dict:
    """L, L', L'', a = L/z, d = (L' - a)/z^2, e = L''/z at z >= 0."""
    z = _f64(np.atleast_1d(z))
    out = {k: np.empty_like(z) for k in ("L", "Lp", "Lpp", "a", "d", "e")}
    _load().og_langevin(z.size, _ptr(z), _ptr(out["L"]), _ptr(out["Lp"]),
                        _ptr(out["Lpp"]), _ptr(out["a"]), _ptr(out["d"]), _ptr(out["e"]))
    return out


def kernel_matrix(y) -> np.ndarray:
    """K(y) of Eq. kernel:matrix for y of shape [..., 2] -> [..., 2, 2]."""
    y = _f64(y)
    flat = y.reshape(-1, 2)
    K = np.empty((flat.shape[0], 4))
    _load().og_kernel_matrix(flat.shape[0], _ptr(flat), _ptr(K))
    return K.reshape(y.shape[:-1] + (2, 2))


def pair(model, x, r, v) -> np.ndarray:
    """J w = beta K(beta G(x - r)) G v for one voxel/sample pair."""
    x, r, v = _f64(x), _f64(r), _f64(v)
    out = np.empty(2)
    _load().og_pair_export(ctypes.byref(_model(model)), _ptr(x), _ptr(r), _ptr(v), _ptr(out))
    return out


# ---------------------------------------------------------------------------
# The operators

def forward(model, grid, r, v, c) -> np.ndarray:
    """A c: s[k][t] = sum_x c_x p_k^T J(x, t) w_t (Eq. core:formula)."""
    r, v, c = _f64(r), _f64(v), _f64(c)
    T = r.shape[0]
    n_ch = np.asarray(model["p"]).reshape(-1, 2).shape[0]
    s = np.empty((n_ch, T))
    _load().og_forward(ctypes.byref(_model(model)), ctypes.byref(_grid(grid)), T,
                       _ptr(r), _ptr(v), _ptr(c), _ptr(s))
    return s


def adjoint(model, grid, r, v, s, sel=None) -> np.ndarray:
    """A^T s on all voxels ([ny, nx]) or on the flat voxel indices ``sel``."""
    r, v, s = _f64(r), _f64(v), _f64(s)
    T = r.shape[0]
    lib = _load()
    if sel is None:
        out = np.empty((int(grid["ny"]), int(grid["nx"])))
        lib.og_adjoint_sel(ctypes.byref(_model(model)), ctypes.byref(_grid(grid)), T,
                           _ptr(r), _ptr(v), _ptr(s), out.size, None, _ptr(out))
        return out
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    out = np.empty(sel.size)
    lib.og_adjoint_sel(ctypes.byref(_model(model)), ctypes.byref(_grid(grid)), T,
                       _ptr(r), _ptr(v), _ptr(s), sel.size,
                       sel.ctypes.data_as(ctypes.POINTER(_I64)), _ptr(out))
    return out


def dbeta(model, grid, r, v, c, gs) -> float:
    """d/dbeta <gs, A(c; beta)> (the particle-parameter gradient)."""
    r, v, c, gs = _f64(r), _f64(v), _f64(c), _f64(gs)
    T = r.shape[0]
    contrib = np.empty(T)
    out = np.empty(1)
    _load().og_dbeta(ctypes.byref(_model(model)), ctypes.byref(_grid(grid)), T, _ptr(r),
                     _ptr(v), _ptr(c), _ptr(gs), _ptr(contrib), _ptr(out))
    return float(out[0])


def frob2(model, grid, r, v) -> float:
    """||A||_F^2 (sum of squares of all entries of the dense matrix of A)."""
    r, v = _f64(r), _f64(v)
    contrib = np.empty(r.shape[0])
    return float(_load().og_frob2(ctypes.byref(_model(model)), ctypes.byref(_grid(grid)),
                                  r.shape[0], _ptr(r), _ptr(v), _ptr(contrib)))


def nu0_from_frob2(frob2_value: float, n_vox: int) -> float:
    """nu0 = 1e-3 * ||O||_F^2 / N: the mean diagonal of O^T O times 1e-3.

    The paper's nu0 values (1e-5 / 1e-6 / 4e-2, Sec. 2.2 and Sec. 3.6) are in
    its own data units; synthetic data take this scale-free reading."""
    return 1e-3 * frob2_value / n_vox


def interp(grid, r, v, Ahat) -> np.ndarray:
    """M[Ahat]_t = I[Ahat](r_t) v_t, cosine interpolation (Eq. first:step)."""
    r, v, Ahat = _f64(r), _f64(v), _f64(Ahat)
    s = np.empty((2, r.shape[0]))
    _load().og_interp(ctypes.byref(_grid(grid)), r.shape[0], _ptr(r), _ptr(v),
                      _ptr(Ahat), _ptr(s))
    return s


def interp_T(grid, r, v, s) -> np.ndarray:
    r, v, s = _f64(r), _f64(v), _f64(s)
    out = np.empty((4, int(grid["ny"]), int(grid["nx"])))
    _load().og_interp_T(ctypes.byref(_grid(grid)), r.shape[0], _ptr(r), _ptr(v),
                        _ptr(s), _ptr(out))
    return out


def laplacian(grid, f) -> np.ndarray:
    """5-point Laplacian with replicated boundary, one [ny, nx] field."""
    f = _f64(f)
    out = np.empty_like(f)
    _load().og_laplacian(ctypes.byref(_grid(grid)), _ptr(f), _ptr(out))
    return out


def laplacian_h(grid, f) -> np.ndarray:
    """The Laplacian of the function sampled on the nodes (replicated
    boundary): the 5-point stencil with 1/dx^2 and 1/dy^2 (the continuous
    reading of the Core Stage regulariser)."""
    f = _f64(f)
    out = np.empty_like(f)
    _load().og_laplacian_h(ctypes.byref(_grid(grid)), _ptr(f), _ptr(out))
    return out


def conv_kernel_trK(model, grid) -> np.ndarray:
    """beta tr K(beta G y) on all voxel offsets: the kernel of the
    gradient-weighted trace tr(Ahat G^-1) (positive for any G)."""
    out = np.empty((2 * int(grid["ny"]) - 1, 2 * int(grid["nx"]) - 1))
    _load().og_conv_kernel_trK(ctypes.byref(_model(model)), ctypes.byref(_grid(grid)), _ptr(out))
    return out


def weighted_trace(model, Ahat) -> np.ndarray:
    """tr(Ahat G^-1) per node from the 4 Core Stage components (index 2k+m)."""
    Gi = np.linalg.inv(np.asarray(model["G"], dtype=np.float64).reshape(2, 2))
    A = _f64(Ahat)
    return sum(A[2 * k + m] * Gi[m, k] for k in range(2) for m in range(2))


def conv_kernel(model, grid, component=None) -> np.ndarray:
    """kappa_G(y) = beta tr(K(beta G y) G) on all voxel offsets, or, with
    component = (a, b), the entry beta (K(beta G y) G)_ab (the single-channel
    deconvolution kernel of Sec. 3.6 is the (0, 0) entry)."""
    out = np.empty((2 * int(grid["ny"]) - 1, 2 * int(grid["nx"]) - 1))
    comp = -1 if component is None else 2 * int(component[0]) + int(component[1])
    _load().og_conv_kernel_component(ctypes.byref(_model(model)), ctypes.byref(_grid(grid)),
                                     comp, _ptr(out))
    return out


def conv(grid, kern, x) -> np.ndarray:
    """Direct linear convolution C x with the sampled kernel."""
    kern, x = _f64(kern), _f64(x)
    out = np.empty_like(x)
    _load().og_conv(ctypes.byref(_grid(grid)), _ptr(kern), _ptr(x), _ptr(out))
    return out


def conv_fft(kern, x) -> np.ndarray:
    """Second route for C x: zero-padded FFT convolution (the Toeplitz/FFT
    realisation the paper uses for C_h), cropped to the 'valid' centre."""
    ny, nx = x.shape
    KY, KX = kern.shape
    sy, sx = KY + ny - 1, KX + nx - 1
    F = np.fft.rfft2(_f64(kern), (sy, sx)) * np.fft.rfft2(_f64(x), (sy, sx))
    full = np.fft.irfft2(F, (sy, sx))
    return full[ny - 1: 2 * ny - 1, nx - 1: 2 * nx - 1]


# ---------------------------------------------------------------------------
# Iterations

def cg(apply, b, x0, n_iter, rel_tol=None):
    """Textbook conjugate gradient (Hestenes-Stiefel) on an SPD operator.

    Runs n_iter steps after the initial residual; with rel_tol it stops as
    soon as ||r|| <= rel_tol ||b|| (checked before each step).  It also stops
    if r^T r == 0 or p^T A p == 0 (the residual has vanished to round-off).  Returns (x, history of ||r||, operator applications)."""
    x = _f64(x0).copy()
    r = b - apply(x)
    n_app = 1
    p = r.copy()
    rr = float(np.dot(r.ravel(), r.ravel()))
    bn = float(np.sqrt(np.dot(b.ravel(), b.ravel())))
    hist = [np.sqrt(rr)]
    for _ in range(n_iter):
        if rr == 0.0:
            break
        if rel_tol is not None and np.sqrt(rr) <= rel_tol * bn:
            break
        q = apply(p)
        n_app += 1
        pq = float(np.dot(p.ravel(), q.ravel()))
        if pq == 0.0:  # only when r vanished to round-off: nothing left to do
            break
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(np.dot(r.ravel(), r.ravel()))
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        hist.append(np.sqrt(rr))
    return x, hist, n_app


def percentile_value(x, pct) -> float:
    """Linear-interpolated percentile of the values of x (numpy's default
    rule): position h = (N-1) pct/100 in the sorted values."""
    srt = np.sort(_f64(x).ravel())
    n = srt.size
    h = (n - 1) * pct / 100.0
    lo = int(np.floor(h))
    hi = min(lo + 1, n - 1)
    frac = h - lo
    return float(srt[lo] + frac * (srt[hi] - srt[lo]))


def percentile_clamp(x, pct):
    """Percentile trimming (Sec. 3.3): values below the pct-th percentile are
    raised to it."""
    P = percentile_value(x, pct)
    return np.maximum(_f64(x), P)


def variance(x) -> float:
    """Population variance, two passes in FP64 (noise estimate, Sec. 2.2)."""
    x = _f64(x).ravel()
    mean = float(np.sum(x)) / x.size
    dev = x - mean
    return float(np.dot(dev, dev) / x.size)


def _reflect(i: int, n: int) -> int:
    """'reflect' boundary (d c b a | a b c d), periodic with period 2n."""
    i %= 2 * n
    return 2 * n - 1 - i if i >= n else i


def gaussian5(img) -> np.ndarray:
    """Built-in denoiser: separable 5-tap Gaussian, sigma = 1 px, weights
    exp(-m^2/2)/sum for m = -2..2, reflect boundary; rows first, then
    columns."""
    img = _f64(img)
    ny, nx = img.shape
    w = np.exp(-0.5 * np.arange(-2, 3, dtype=np.float64) ** 2)
    w /= w.sum()
    tmp = np.zeros_like(img)
    for i in range(nx):
        for m in range(-2, 3):
            tmp[:, i] += w[m + 2] * img[:, _reflect(i + m, nx)]
    out = np.zeros_like(img)
    for j in range(ny):
        for m in range(-2, 3):
            out[j, :] += w[m + 2] * tmp[_reflect(j + m, ny), :]
    return out


def pnp(op, opT, data, shape, n_it, n_cg, nu0, clip_pct=5.0, denoise=None,
        record=None):
    """ZeroShot-PnP deconvolution, Algorithm 1, with operator O (op / opT).

    rho2 <- 0; for k = 0 .. n_it-1:
      rho1 <- CG(O^T O + nu_k I, O^T data + nu_k rho2, x0 = rho2), n_cg steps
      rho1 <- max(rho1, P_clip(rho1))         (percentile trimming, Sec. 3.3)
      sigma <- sqrt(Var(rho1))                (noise estimate)
      lambda <- nu0 sigma^2 if k == 0
      rho2 <- Denoise(rho1, sigma)
      nu <- lambda / sigma^2 (unchanged if sigma == 0)
    return rho2.
    """
    if denoise is None:
        denoise = lambda img, sigma: gaussian5(img)
    b0 = _f64(opT(data)).reshape(shape)
    rho2 = np.zeros(shape)
    nu = float(nu0)
    lam = None
    for k in range(n_it):
        nu_k = nu
        rhs = b0 + nu_k * rho2
        apply = lambda x, nu_k=nu_k: _f64(opT(op(x))).reshape(shape) + nu_k * x
        rho1, hist, _ = cg(apply, rhs, rho2, n_cg)
        clip = float("-inf")
        if clip_pct is not None and clip_pct >= 0:
            clip = percentile_value(rho1, clip_pct)
            rho1 = percentile_clamp(rho1, clip_pct)
        sigma = float(np.sqrt(variance(rho1)))
        if k == 0:
            lam = nu0 * sigma * sigma
        rho2 = _f64(denoise(rho1, sigma)).reshape(shape)
        if sigma > 0.0:
            nu = lam / (sigma * sigma)
        if record is not None:
            record.append({"sigma": sigma, "nu": nu, "cg_resid": float(hist[-1]),
                           "nu_used": nu_k, "clip": clip})
    return rho2


def _lap_fn(kind, lap, lap_h):
    if kind == "bare":
        return lap
    if kind == "scaled":
        return lap_h
    raise ValueError(f"unknown Laplacian {kind!r}")


def core_stage_channel(grid, r, v, s_k, k, gamma, max_iter, rel_tol=None, lap="bare"):
    """Core Stage with only receive channel k measured (Sec. 3.6):
        s_k(t) = I[A_k0](r_t) v_x(t) + I[A_k1](r_t) v_y(t),
    the two components (A_k0, A_k1) solved as in Eq. first:step with the
    Laplacian regulariser on each.  The measurement operator is the channel-k
    row of the two-channel one (the other channel's components held at zero).
    Returns (A [2, ny, nx], A_kk, residual history)."""
    T = r.shape[0]
    ny, nx = int(grid["ny"]), int(grid["nx"])
    s_k = _f64(s_k).reshape(-1)

    def embed(A2):
        A4 = np.zeros((4, ny, nx))
        A4[2 * k:2 * k + 2] = A2
        return A4

    def M(A2):
        return interp(grid, r, v, embed(A2))[k]

    def MT(y):
        s2 = np.zeros((2, T))
        s2[k] = y
        return interp_T(grid, r, v, s2)[2 * k:2 * k + 2]

    L = _lap_fn(lap, laplacian, laplacian_h)

    def lap2(x):
        return np.stack([L(grid, x[m]) for m in range(2)])

    def apply(x):
        return MT(M(x)) / T + gamma * lap2(lap2(x))

    b = MT(s_k) / T
    x, hist, _ = cg(apply, b, np.zeros((2, ny, nx)), max_iter, rel_tol=rel_tol)
    return x, x[k], hist


def core_stage(grid, r, v, s, gamma, max_iter, rel_tol=None, lap="bare"):
    """Core Stage (Eq. first:step): CG on the Euler-Lagrange equations
        ((1/L) M^T M + gamma Lap^T Lap) Ahat = (1/L) M^T s,   L = T,
    with M the cosine-interpolation measurement operator and Lap the
    replicated-boundary 5-point Laplacian on each of the 4 components (it is
    symmetric, so Lap^T Lap = Lap Lap; lap="scaled": with 1/dx^2, 1/dy^2).
    Starts from 0.  Returns (Ahat
    [4, ny, nx], trace u = Ahat_00 + Ahat_11, residual history)."""
    T = r.shape[0]
    ny, nx = int(grid["ny"]), int(grid["nx"])

    L = _lap_fn(lap, laplacian, laplacian_h)

    def lap4(x):
        return np.stack([L(grid, x[m]) for m in range(4)])

    def apply(x):
        return interp_T(grid, r, v, interp(grid, r, v, x)) / T + gamma * lap4(lap4(x))

    b = interp_T(grid, r, v, s) / T
    x, hist, _ = cg(apply, b, np.zeros((4, ny, nx)), max_iter, rel_tol=rel_tol)
    return x, x[0] + x[3], hist


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))


# ---------------------------------------------------------------------------
# Three-dimensional field-free point (Sec. 2 with n = 3).  A ``grid3`` has
# nx, ny, nz, x0, y0, z0, dx, dy, dz; a ``model3`` has beta, G (3x3) and p
# (n_ch x 3).  Concentrations are [nz, ny, nx], r and v [T, 3].

def kernel_matrix3(y) -> np.ndarray:
    """K(y) of Eq. kernel:matrix for y of shape [..., 3] -> [..., 3, 3]."""
    y = _f64(y)
    flat = y.reshape(-1, 3)
    K = np.empty((flat.shape[0], 9))
    _load().og_kernel_matrix3(flat.shape[0], _ptr(flat), _ptr(K))
    return K.reshape(y.shape[:-1] + (3, 3))


def pair3(model3, x, r, v) -> np.ndarray:
    """J w = beta K(beta G(x - r)) G v in three dimensions."""
    x, r, v = _f64(x), _f64(r), _f64(v)
    out = np.empty(3)
    _load().og_pair3_export(ctypes.byref(_model3(model3)), _ptr(x), _ptr(r), _ptr(v), _ptr(out))
    return out


def forward3(model3, grid3, r, v, c) -> np.ndarray:
    """A c in three dimensions: s[k][t] = sum_x c_x p_k^T J(x, t) w_t."""
    r, v, c = _f64(r), _f64(v), _f64(c)
    T = r.shape[0]
    n_ch = np.asarray(model3["p"]).reshape(-1, 3).shape[0]
    s = np.empty((n_ch, T))
    _load().og_forward3(ctypes.byref(_model3(model3)), ctypes.byref(_grid3(grid3)), T,
                        _ptr(r), _ptr(v), _ptr(c), _ptr(s))
    return s


def adjoint3(model3, grid3, r, v, s, sel=None) -> np.ndarray:
    """A^T s in three dimensions, on all voxels ([nz, ny, nx]) or on the flat
    voxel indices ``sel``."""
    r, v, s = _f64(r), _f64(v), _f64(s)
    T = r.shape[0]
    lib = _load()
    if sel is None:
        out = np.empty((int(grid3["nz"]), int(grid3["ny"]), int(grid3["nx"])))
        lib.og_adjoint3_sel(ctypes.byref(_model3(model3)), ctypes.byref(_grid3(grid3)), T,
                            _ptr(r), _ptr(v), _ptr(s), out.size, None, _ptr(out))
        return out
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    out = np.empty(sel.size)
    lib.og_adjoint3_sel(ctypes.byref(_model3(model3)), ctypes.byref(_grid3(grid3)), T,
                        _ptr(r), _ptr(v), _ptr(s), sel.size,
                        sel.ctypes.data_as(ctypes.POINTER(_I64)), _ptr(out))
    return out


def frob2_3(model3, grid3, r, v) -> float:
    """||A||_F^2 of the three-dimensional forward operator."""
    r, v = _f64(r), _f64(v)
    return float(_load().og_frob2_3(ctypes.byref(_model3(model3)), ctypes.byref(_grid3(grid3)),
                                    r.shape[0], _ptr(r), _ptr(v)))


def conv_kernel3(model3, grid3) -> np.ndarray:
    """kappa_G(y) = beta tr(K(beta G y) G) on all 3-D voxel offsets,
    [2nz-1, 2ny-1, 2nx-1] (Eq. kernel:trace with n - 1 = 2)."""
    out = np.empty((2 * int(grid3["nz"]) - 1, 2 * int(grid3["ny"]) - 1, 2 * int(grid3["nx"]) - 1))
    _load().og_conv_kernel3(ctypes.byref(_model3(model3)), ctypes.byref(_grid3(grid3)), _ptr(out))
    return out


def conv3(grid3, kern, x) -> np.ndarray:
    """Direct linear 3-D convolution with the sampled kernel."""
    kern, x = _f64(kern), _f64(x)
    out = np.empty_like(x)
    _load().og_conv3(ctypes.byref(_grid3(grid3)), _ptr(kern), _ptr(x), _ptr(out))
    return out


def gaussian5_3d(vol) -> np.ndarray:
    """The built-in denoiser on a volume: the 5-tap Gaussian (sigma = 1 voxel,
    reflect boundary) along x, then y, then z."""
    vol = _f64(vol)
    nz, ny, nx = vol.shape
    w = np.exp(-0.5 * np.arange(-2, 3, dtype=np.float64) ** 2)
    w /= w.sum()
    a = np.zeros_like(vol)
    for i in range(nx):
        for m in range(-2, 3):
            a[:, :, i] += w[m + 2] * vol[:, :, _reflect(i + m, nx)]
    b = np.zeros_like(vol)
    for j in range(ny):
        for m in range(-2, 3):
            b[:, j, :] += w[m + 2] * a[:, _reflect(j + m, ny), :]
    out = np.zeros_like(vol)
    for k in range(nz):
        for m in range(-2, 3):
            out[k, :, :] += w[m + 2] * b[_reflect(k + m, nz), :, :]
    return out


def interp3(grid3, r, v, Ahat) -> np.ndarray:
    """Core Stage measurement in three dimensions (Eq. first:step, n = 3):
    s_k(t) = sum_m I[Ahat_km](r_t) v_m(t), I the tensor-product cosine
    interpolation.  Ahat is [n_ch*3, nz, ny, nx] (component 3k+m); returns
    s [n_ch, T]."""
    r, v, Ahat = _f64(r), _f64(v), _f64(Ahat)
    n_ch = Ahat.shape[0] // 3
    s = np.empty((n_ch, r.shape[0]))
    _load().og_interp3(ctypes.byref(_grid3(grid3)), n_ch, r.shape[0], _ptr(r), _ptr(v),
                       _ptr(Ahat), _ptr(s))
    return s


def interp3_T(grid3, r, v, s) -> np.ndarray:
    """Exact transpose of interp3: s [n_ch, T] -> [n_ch*3, nz, ny, nx]."""
    r, v, s = _f64(r), _f64(v), _f64(s)
    s = s.reshape(-1, r.shape[0])
    n_ch = s.shape[0]
    out = np.empty((3 * n_ch, int(grid3["nz"]), int(grid3["ny"]), int(grid3["nx"])))
    _load().og_interp3_T(ctypes.byref(_grid3(grid3)), n_ch, r.shape[0], _ptr(r), _ptr(v),
                         _ptr(s), _ptr(out))
    return out


def laplacian3(grid3, f) -> np.ndarray:
    """7-point Laplacian with replicated boundary, one [nz, ny, nx] volume."""
    f = _f64(f)
    out = np.empty_like(f)
    _load().og_laplacian3(ctypes.byref(_grid3(grid3)), _ptr(f), _ptr(out))
    return out


def laplacian3_h(grid3, f) -> np.ndarray:
    """The 7-point Laplacian with 1/dx^2, 1/dy^2, 1/dz^2 (replicated boundary)."""
    f = _f64(f)
    out = np.empty_like(f)
    _load().og_laplacian3_h(ctypes.byref(_grid3(grid3)), _ptr(f), _ptr(out))
    return out


def conv_kernel3_trK(model3, grid3) -> np.ndarray:
    """beta tr K(beta G y) on all voxel offsets in three dimensions: the kernel
    of tr(Ahat G^-1), positive for any G (the trace kernel of a traceless G
    is not)."""
    shape = tuple(2 * int(grid3[k]) - 1 for k in ("nz", "ny", "nx"))
    out = np.empty(shape)
    _load().og_conv_kernel3_trK(ctypes.byref(_model3(model3)), ctypes.byref(_grid3(grid3)), _ptr(out))
    return out


def weighted_trace3(model3, Ahat) -> np.ndarray:
    """tr(Ahat G^-1) per node from the 9 Core Stage components (index 3k+m)."""
    Gi = np.linalg.inv(np.asarray(model3["G"], dtype=np.float64).reshape(3, 3))
    A = _f64(Ahat)
    return sum(A[3 * k + m] * Gi[m, k] for k in range(3) for m in range(3))


def core_stage3(grid3, r, v, s, gamma, max_iter, rel_tol=None, channel=None, lap="bare"):
    """Core Stage in three dimensions (Eq. first:step with n = 3): CG from 0 on
        ((1/T) M^T M + gamma Lap Lap) Ahat = (1/T) M^T s
    for the 9 components Ahat_km (3 channels x 3 velocity components), Lap the
    7-point replicated-boundary Laplacian on each component.  channel = k:
    only channel k was measured (s [T] or [1, T]); the unknowns are the row
    (A_k0, A_k1, A_k2), solved with channel k's row of M (Sec. 3.6 in three
    dimensions).  Returns (Ahat [9 or 3, nz, ny, nx], trace, residual
    history); the trace is A_00 + A_11 + A_22, or A_kk for one channel."""
    T = r.shape[0]
    nz, ny, nx = int(grid3["nz"]), int(grid3["ny"]), int(grid3["nx"])
    s = _f64(s).reshape(-1, T)
    nc = 9 if channel is None else 3

    L = _lap_fn(lap, laplacian3, laplacian3_h)

    def lapn(x):
        return np.stack([L(grid3, x[m]) for m in range(nc)])

    def apply(x):
        return interp3_T(grid3, r, v, interp3(grid3, r, v, x)) / T + gamma * lapn(lapn(x))

    b = interp3_T(grid3, r, v, s) / T
    x, hist, _ = cg(apply, b, np.zeros((nc, nz, ny, nx)), max_iter, rel_tol=rel_tol)
    if channel is None:
        return x, x[0] + x[4] + x[8], hist
    return x, x[int(channel)], hist


# ---------------------------------------------------------------------------
# Transfer-function correction (Eq. core:formula:conva -> Eq. core:formula and
# the preprocessing of Sec. 3.2).  The measured signal is the model signal
# convolved in time with the receive chain's impulse response a; over one
# period of a periodic trajectory (T samples) that is a circular convolution,
# so its DFT is the product s_hat * a_hat.  The correction divides by a_hat
# bin by bin and drops the bins whose SNR is below the channel's threshold
# (and bins where a_hat vanishes).  DFT convention: numpy's rfft / irfft over
# the T samples of one period (F = T//2 + 1 bins).

def transfer_correct(s_raw, a_hat, snr=None, theta=None) -> np.ndarray:
    """s_raw [n_ch, T] real, a_hat [n_ch, F] complex, snr [n_ch, F] (or None:
    no thresholding), theta [n_ch] -> corrected signal [n_ch, T]."""
    s_raw = np.atleast_2d(_f64(s_raw))
    n_ch, T = s_raw.shape
    a_hat = np.atleast_2d(np.asarray(a_hat, dtype=np.complex128))
    out = np.empty_like(s_raw)
    for k in range(n_ch):
        S = np.fft.rfft(s_raw[k])
        keep = np.abs(a_hat[k]) > 0
        if snr is not None:
            keep &= np.asarray(snr, dtype=np.float64)[k] >= float(theta[k])
        Y = np.zeros_like(S)
        Y[keep] = S[keep] / a_hat[k][keep]
        out[k] = np.fft.irfft(Y, n=T)
    return out

"""Thin ctypes binding of ``libmpi_recon.so`` (declared in include/mpi_recon.h).

Functions carry the C entry-point names and only marshal arguments: every
array is a CUDA ``torch.Tensor`` (float32 or float64, contiguous) whose device
pointer is passed through, and the call is enqueued on the current torch CUDA
stream.  There is no CPU path: if the library cannot be loaded, or a tensor is
not on a CUDA device, the call raises.

``model`` and ``grid`` are mappings (or objects) with the fields of
``mpi_model`` (beta, G 2x2, p n_ch x 2) and ``mpi_grid_desc`` (nx, ny, x0, y0,
dx, dy).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpi_recon.so")

MPI_OK = 0
MPI_ERR_INVALID = -1
MPI_ERR_CUDA = -2
MPI_ERR_NOMEM = -3
MPI_ERR_CALLBACK = -4
MPI_ERR_TIMEOUT = -5
MPI_ERR_UNSUPPORTED = -6
MPI_F32, MPI_F64 = 0, 1
MPI_OP_FORWARD, MPI_OP_CONV = 0, 1


class MPIError(RuntimeError):
    """A non-zero status of a library call, with the library's message."""

    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class GridDesc(ctypes.Structure):
    """mpi_grid_desc: nx x ny voxels, centres (x0 + (i + 1/2) dx, y0 + (j + 1/2) dy)."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double)]


class Model(ctypes.Structure):
    """mpi_model: beta = 1/(mu0 H_sat), G row-major 2x2, n_ch receive directions p."""
    _fields_ = [("beta", ctypes.c_double), ("G", ctypes.c_double * 4), ("n_ch", ctypes.c_int),
                ("p", ctypes.c_double * 4)]


class Traj(ctypes.Structure):
    """mpi_traj: T samples, device pointers to r [T][dim] and v = dr/dt [T][dim]."""
    _fields_ = [("T", ctypes.c_int64), ("r", ctypes.c_void_p), ("v", ctypes.c_void_p)]


class GridOpts(ctypes.Structure):
    """mpi_grid_opts: gamma, CG iteration limit, relative tolerance, channel selector."""
    _fields_ = [("gamma", ctypes.c_double), ("max_iter", ctypes.c_int), ("rel_tol", ctypes.c_double),
                ("channel", ctypes.c_int), ("lap_scaled", ctypes.c_int)]


class PnPOpts(ctypes.Structure):
    """mpi_pnp_opts: operator, outer iterations, CG steps, nu0, clip percentile,
    kernel entry of the single-channel deconvolution."""
    _fields_ = [("op", ctypes.c_int), ("n_iter", ctypes.c_int), ("n_cg", ctypes.c_int),
                ("nu0", ctypes.c_double), ("clip_pct", ctypes.c_double),
                ("kernel_component", ctypes.c_int)]


class Grid3Desc(ctypes.Structure):
    """mpi_grid3_desc: nx x ny x nz voxels with origin and spacing per axis."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class Model3(ctypes.Structure):
    """mpi_model3: beta, G row-major 3x3, n_ch (1..3) receive directions p."""
    _fields_ = [("beta", ctypes.c_double), ("G", ctypes.c_double * 9), ("n_ch", ctypes.c_int),
                ("p", ctypes.c_double * 9)]


class PnPIterInfo(ctypes.Structure):
    """Per-iteration (sigma, nu, final CG residual) of Algorithm 1."""
    _fields_ = [("sigma", ctypes.c_double), ("nu", ctypes.c_double), ("cg_resid", ctypes.c_double),
                ("clip", ctypes.c_double)]


class BatchInfo(ctypes.Structure):
    """The tuned configuration of a batch plan (mpi_batch_plan_info)."""
    _fields_ = [("n_frames", ctypes.c_int), ("tuned", ctypes.c_int),
                ("item_pairs_forward", ctypes.c_longlong), ("item_pairs_adjoint", ctypes.c_longlong),
                ("persistent_forward", ctypes.c_int), ("persistent_adjoint", ctypes.c_int),
                ("forward_items", ctypes.c_longlong), ("adjoint_items", ctypes.c_longlong),
                ("device_bytes", ctypes.c_longlong), ("graph_nodes", ctypes.c_longlong)]


MPI_BATCH_MAX_FRAMES = 64
MPI_BATCH_AUTOTUNE = 1
MPI_BATCH_MATCH_SINGLE = 2

DENOISE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                              ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                ctypes.c_void_p)
DENOISE3_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()

_SIGS = {
    "mpi_forward": [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_forward_noalloc": [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_adjoint": [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_dbeta": [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 4,
    "mpi_conv": [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_conv_component": [ctypes.c_void_p] * 2 + [ctypes.c_int] * 2 + [ctypes.c_void_p] * 3,
    "mpi_interp": [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_interp_adjoint": [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_cell_order": [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_grid": [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 6,
    "mpi_denoise_gaussian5": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "mpi_pnp_solve": [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 2
                     + [DENOISE_FN] + [ctypes.c_void_p] * 4,
    "mpi_pnp_solve_sharded": [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 2
                             + [DENOISE_FN, ctypes.c_void_p, ALLREDUCE_FN] + [ctypes.c_void_p] * 4,
    "mpi_transfer_correct": [ctypes.c_int, ctypes.c_int64, ctypes.c_int] + [ctypes.c_void_p] * 6,
    "mpi_forward3": [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_adjoint3": [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_conv3": [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_conv3_kernel": [ctypes.c_void_p] * 2 + [ctypes.c_int] * 2 + [ctypes.c_void_p] * 3,
    "mpi_weighted_trace3": [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_interp3": [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_interp3_adjoint": [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 3,
    "mpi_grid3": [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 6,
    "mpi_denoise_gaussian5_3d": [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 4
                                + [ctypes.c_void_p] * 3,
    "mpi_pnp_solve3": [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 2
                      + [DENOISE3_FN] + [ctypes.c_void_p] * 4,
    "mpi_batch_plan_create": [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "mpi_batch_pnp_run": [ctypes.c_void_p] * 6,
    "mpi_batch_plan_info": [ctypes.c_void_p, ctypes.c_void_p],
    "mpi_batch_plan_destroy": [ctypes.c_void_p],
    "mpi_kernel_launches": [],
    "mpi_profile_enable": [ctypes.c_int],
    "mpi_profile_read": [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "mpi_status_string": [ctypes.c_int],
    "mpi_last_error_message": [],
    "mpi_version": [],
    "mpi_probe_pipe_rate": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), ctypes.c_void_p],
}


def load(path: str | None = None):
    """Load libmpi_recon.so (build it first with paper_2505_22797_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: run paper_2505_22797_gb300.build.build() first "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        for name, args in _SIGS.items():
            if hasattr(lib, name):
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
        lib.mpi_kernel_launches.restype = ctypes.c_longlong
        lib.mpi_status_string.restype = ctypes.c_char_p
        lib.mpi_last_error_message.restype = ctypes.c_char_p
        _lib = lib
        return lib


def exported_symbols():
    """Names of the entry points this binding declares that the library exports."""
    lib = load()
    return {name for name in _SIGS if hasattr(lib, name)}


PROF_FORWARD, PROF_ADJOINT, PROF_DBETA, PROF_CONV = 0, 1, 2, 3
PROBE_FMA, PROBE_RSQRT, PROBE_EX2, PROBE_RCP, PROBE_DFMA, PROBE_FMA2 = 0, 1, 2, 3, 4, 5


def mpi_probe_pipe_rate(op: int, blocks_per_sm: int = 8, iters: int = 4096, stream=None):
    """(thread-operations per SM per clock, launch ms) of one instruction
    kind (PROBE_FMA, PROBE_RSQRT, PROBE_EX2, PROBE_RCP, PROBE_DFMA, PROBE_FMA2)
    measured on the current GPU; the median over SMs of operations per SM
    clock cycle (PROBE_FMA2: two per packed instruction)."""
    rate = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    _check(load().mpi_probe_pipe_rate(int(op), int(blocks_per_sm), int(iters), ctypes.byref(rate),
                                      ctypes.byref(ms), _stream(stream)))
    return float(rate.value), float(ms.value)


def mpi_kernel_launches() -> int:
    """Number of library kernel launches since the library was loaded."""
    return int(load().mpi_kernel_launches())


def mpi_profile_enable(enable: bool = True):
    """Switch the per-kernel-class CUDA-event timing on or off (see
    mpi_profile_read)."""
    _check(load().mpi_profile_enable(1 if enable else 0))


def mpi_profile_read(kernel_class: int):
    """(launches, total_ms) of one operator-kernel class since enabling."""
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    _check(load().mpi_profile_read(int(kernel_class), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def _check(status: int):
    if status != MPI_OK:
        lib = load()
        msg = lib.mpi_last_error_message().decode(errors="replace")
        raise MPIError(status, f"{lib.mpi_status_string(status).decode()}: {msg}")


def _get(obj, key):
    return obj[key] if isinstance(obj, dict) else getattr(obj, key)


def make_grid(grid) -> GridDesc:
    """mpi_grid_desc from a mapping or object with nx, ny, x0, y0, dx, dy."""
    return GridDesc(int(_get(grid, "nx")), int(_get(grid, "ny")), float(_get(grid, "x0")),
                    float(_get(grid, "y0")), float(_get(grid, "dx")), float(_get(grid, "dy")))


def make_grid3(grid) -> Grid3Desc:
    """mpi_grid3_desc from a mapping or object with nx, ny, nz, x0, y0, z0, dx, dy, dz."""
    return Grid3Desc(*(int(_get(grid, k)) for k in ("nx", "ny", "nz")),
                     *(float(_get(grid, k)) for k in ("x0", "y0", "z0", "dx", "dy", "dz")))


def make_model3(model) -> Model3:
    """mpi_model3 from beta, G (3x3) and p (n_ch x 3, n_ch = 1..3)."""
    G = [float(x) for row in _get(model, "G") for x in row]
    P = [[float(x) for x in row] for row in _get(model, "p")]
    if len(G) != 9 or not 1 <= len(P) <= 3 or any(len(row) != 3 for row in P):
        raise ValueError("a 3-D model needs G 3x3 and 1..3 receive directions of length 3")
    flat = [x for row in P for x in row] + [0.0] * (9 - 3 * len(P))
    return Model3(float(_get(model, "beta")), (ctypes.c_double * 9)(*G), len(P),
                  (ctypes.c_double * 9)(*flat))


def make_model(model) -> Model:
    """mpi_model from beta, G (2x2) and p (n_ch x 2, n_ch = 1 or 2)."""
    G = [float(x) for row in _get(model, "G") for x in row]
    P = [[float(x) for x in row] for row in _get(model, "p")]
    flat = [x for row in P for x in row] + [0.0] * (4 - 2 * len(P))
    return Model(float(_get(model, "beta")), (ctypes.c_double * 4)(*G), len(P),
                 (ctypes.c_double * 4)(*flat))


def _dtype(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return MPI_F32
    if t.dtype == torch.float64:
        return MPI_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _dev(t: torch.Tensor, dtype=None, name="tensor") -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    return t.data_ptr()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _traj(r: torch.Tensor, v: torch.Tensor, dt, dim: int = 2) -> Traj:
    if r.shape != v.shape or r.dim() != 2 or r.shape[1] != dim:
        raise ValueError(f"r and v must both be [T, {dim}]")
    T = r.shape[0]
    return Traj(T, _dev(r, dt, "r") if T else None, _dev(v, dt, "v") if T else None)


def mpi_forward(model, grid, r, v, c, s=None, stream=None):
    """s[k][t] = (A c)_k(t); returns s ([n_ch, T], dtype of c)."""
    dt = c.dtype
    n_ch = len(_get(model, "p"))
    if s is None:
        s = torch.empty((n_ch, r.shape[0]), dtype=dt, device=c.device)
    tr = _traj(r, v, dt)
    m, g = make_model(model), make_grid(grid)
    _check(load().mpi_forward(ctypes.byref(m), ctypes.byref(g), ctypes.byref(tr), _dtype(c),
                              _dev(c, dt, "c"), _dev(s, dt, "s") if s.numel() else None,
                              _stream(stream)))
    return s


def mpi_forward_noalloc(model, grid, r, v, c, s=None, stream=None):
    """Like mpi_forward, for callers that cannot let the library allocate
    device memory while they run: the library's scratch is a fixed 32 MiB
    device array (see include/mpi_recon.h for the size limit and the rule
    that overlapping calls race).  ``s`` should be preallocated by such a
    caller; it is created here only for convenience."""
    dt = c.dtype
    n_ch = len(_get(model, "p"))
    if s is None:
        s = torch.empty((n_ch, r.shape[0]), dtype=dt, device=c.device)
    tr = _traj(r, v, dt)
    m, g = make_model(model), make_grid(grid)
    _check(load().mpi_forward_noalloc(ctypes.byref(m), ctypes.byref(g), ctypes.byref(tr),
                                      _dtype(c), _dev(c, dt, "c"),
                                      _dev(s, dt, "s") if s.numel() else None, _stream(stream)))
    return s


def mpi_adjoint(model, grid, r, v, s, c_out=None, stream=None):
    """c_out = A^T s ([ny, nx], dtype of s)."""
    dt = s.dtype
    g = make_grid(grid)
    if c_out is None:
        c_out = torch.empty((g.ny, g.nx), dtype=dt, device=s.device)
    tr = _traj(r, v, dt)
    m = make_model(model)
    _check(load().mpi_adjoint(ctypes.byref(m), ctypes.byref(g), ctypes.byref(tr), _dtype(s),
                              _dev(s, dt, "s") if s.numel() else None, _dev(c_out, dt, "c_out"),
                              _stream(stream)))
    return c_out


def mpi_dbeta(model, grid, r, v, c, g_s, out=None, stream=None):
    """d/dbeta <g_s, A(c; beta)> as a 0-d float64 CUDA tensor."""
    dt = c.dtype
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=c.device)
    tr = _traj(r, v, dt)
    m, g = make_model(model), make_grid(grid)
    _check(load().mpi_dbeta(ctypes.byref(m), ctypes.byref(g), ctypes.byref(tr), _dtype(c),
                            _dev(c, dt, "c"), _dev(g_s, dt, "g") if g_s.numel() else None,
                            _dev(out, torch.float64, "out"), _stream(stream)))
    return out


def mpi_conv(model, grid, x, out=None, stream=None):
    """out = C x: linear (zero-padded) convolution of x [ny, nx] with the sampled
    trace kernel beta tr(K(beta G y) G) (Eq. kernel:trace); direct sum on small
    grids, FFT route above."""
    dt = x.dtype
    if out is None:
        out = torch.empty_like(x)
    m, g = make_model(model), make_grid(grid)
    _check(load().mpi_conv(ctypes.byref(m), ctypes.byref(g), _dtype(x), _dev(x, dt, "in"),
                           _dev(out, dt, "out"), _stream(stream)))
    return out


def mpi_conv_component(model, grid, component, x, out=None, stream=None):
    """Convolution with entry ``component`` = 2a + b of beta K(beta G y) G
    (-1: the trace kernel, as mpi_conv)."""
    dt = x.dtype
    if out is None:
        out = torch.empty_like(x)
    m, g = make_model(model), make_grid(grid)
    _check(load().mpi_conv_component(ctypes.byref(m), ctypes.byref(g), _dtype(x), int(component),
                                     _dev(x, dt, "in"), _dev(out, dt, "out"), _stream(stream)))
    return out


def mpi_interp(grid, r, v, Ahat, s=None, stream=None):
    """Core Stage measurement (Eq. first:step): s[k][t] = sum_m I[Ahat_{2k+m}](r_t)
    v_m(t) with the cosine interpolation I; Ahat [4, ny, nx] -> s [2, T]."""
    dt = Ahat.dtype
    if s is None:
        s = torch.empty((2, r.shape[0]), dtype=dt, device=Ahat.device)
    tr = _traj(r, v, dt)
    g = make_grid(grid)
    _check(load().mpi_interp(ctypes.byref(g), ctypes.byref(tr), _dtype(Ahat), _dev(Ahat, dt, "Ahat"),
                             _dev(s, dt, "s") if s.numel() else None, _stream(stream)))
    return s


def mpi_interp_adjoint(grid, r, v, s, Ahat=None, stream=None):
    """Exact transpose of mpi_interp: s [2, T] -> Ahat [4, ny, nx], summed in a
    fixed order (no atomics)."""
    dt = s.dtype
    g = make_grid(grid)
    if Ahat is None:
        Ahat = torch.empty((4, g.ny, g.nx), dtype=dt, device=s.device)
    tr = _traj(r, v, dt)
    _check(load().mpi_interp_adjoint(ctypes.byref(g), ctypes.byref(tr), _dtype(s),
                                     _dev(s, dt, "s") if s.numel() else None,
                                     _dev(Ahat, dt, "Ahat"), _stream(stream)))
    return Ahat


def mpi_cell_order(cell_of, n_cells, with_offset=True, stream=None):
    """Binning step of the Core Stage: the samples ordered by cell (a stable
    sort of cell_of, int32 on the device) and, with with_offset, the start of
    each cell's run (offset[n_cells] = T).  Returns (list, offset or None)."""
    if cell_of.dtype != torch.int32 or not cell_of.is_cuda:
        raise TypeError("cell_of must be an int32 CUDA tensor")
    cell_of = cell_of.contiguous()
    T = cell_of.numel()
    lst = torch.empty(T, dtype=torch.int32, device=cell_of.device)
    off = torch.empty(int(n_cells) + 1, dtype=torch.int32, device=cell_of.device) if with_offset else None
    _check(load().mpi_cell_order(int(T), cell_of.data_ptr() if T else None, int(n_cells),
                                 lst.data_ptr() if T else None, off.data_ptr() if off is not None else None,
                                 _stream(stream)))
    return lst, off


def mpi_grid(grid, r, v, s, gamma=1e-7, max_iter=10000, rel_tol=1e-3, Ahat=None, trace=None,
             return_iters=False, channel=None, lap_scaled=False, stream=None):
    """Core Stage.  ``channel`` None: s is [2][T] and Ahat [4][ny][nx];
    channel k (0 or 1): only that channel was measured, s is [T] (or [1][T])
    and Ahat holds (A_k0, A_k1), trace = A_kk.  ``lap_scaled``: regularise
    with the Laplacian scaled by 1/dx^2, 1/dy^2 instead of the bare stencil."""
    dt = s.dtype
    g = make_grid(grid)
    nc = 4 if channel is None else 2
    if Ahat is None:
        Ahat = torch.empty((nc, g.ny, g.nx), dtype=dt, device=s.device)
    if trace is None:
        trace = torch.empty((g.ny, g.nx), dtype=dt, device=s.device)
    tr = _traj(r, v, dt)
    opts = GridOpts(float(gamma), int(max_iter), float(rel_tol),
                    0 if channel is None else int(channel) + 1, 1 if lap_scaled else 0)
    n_it = ctypes.c_int(-1)
    _check(load().mpi_grid(ctypes.byref(g), ctypes.byref(tr), _dtype(s),
                           _dev(s, dt, "s") if s.numel() else None, ctypes.byref(opts),
                           _dev(Ahat, dt, "Ahat"), _dev(trace, dt, "trace"),
                           ctypes.byref(n_it) if return_iters else None, _stream(stream)))
    if return_iters:
        return Ahat, trace, n_it.value
    return Ahat, trace


def mpi_denoise_gaussian5(x, out=None, stream=None):
    """The built-in PnP denoiser: separable 5-tap Gaussian (sigma = 1 px), reflect
    boundary, on x [ny, nx]."""
    dt = x.dtype
    if out is None:
        out = torch.empty_like(x)
    ny, nx = x.shape
    _check(load().mpi_denoise_gaussian5(_dev(x, dt, "in"), _dev(out, dt, "out"), nx, ny, _dtype(x),
                                        None, _stream(stream), None))
    return out


def mpi_pnp_solve(model, grid, r, v, data, n_iter, n_cg, nu0, clip_pct=5.0, op=MPI_OP_FORWARD,
                  denoise=None, rho_out=None, with_info=False, kernel_component=None, stream=None):
    """Algorithm 1.  ``denoise`` is None (built-in Gaussian) or a Python
    callable (in_tensor, out_tensor, sigma_dev_tensor) -> None that enqueues
    on the current stream.  ``kernel_component`` (MPI_OP_CONV only): None for
    the trace kernel, else 2a + b of the kernel-matrix entry to deconvolve."""
    dt = data.dtype
    g = make_grid(grid)
    if rho_out is None:
        rho_out = torch.empty((g.ny, g.nx), dtype=dt, device=data.device)
    if op == MPI_OP_FORWARD:
        tr = _traj(r, v, dt)
    else:
        tr = Traj(0, None, None) if r is None else _traj(r, v, dt)
    m = make_model(model)
    opts = PnPOpts(int(op), int(n_iter), int(n_cg), float(nu0), float(clip_pct),
                   0 if kernel_component is None else int(kernel_component) + 1)
    info = (PnPIterInfo * max(1, n_iter))() if with_info else None
    cb = DENOISE_FN(0)
    keep = None
    if denoise is not None:
        dev = data.device

        def _cb(pin, pout, nx, ny, dtype, sig, strm, user):
            try:
                tdt = torch.float32 if dtype == MPI_F32 else torch.float64
                tin = _wrap(pin, (ny, nx), tdt, dev)
                tout = _wrap(pout, (ny, nx), tdt, dev)
                tsig = _wrap(sig, (), torch.float64, dev)
                denoise(tin, tout, tsig)
                return 0
            except Exception:  # noqa: BLE001 - reported as MPI_ERR_CALLBACK
                return 1
        cb = DENOISE_FN(_cb)
        keep = cb
    _check(load().mpi_pnp_solve(ctypes.byref(m), ctypes.byref(g), ctypes.byref(tr), _dtype(data),
                                _dev(data, dt, "data"), ctypes.byref(opts), cb, None,
                                _dev(rho_out, dt, "rho_out"), info, _stream(stream)))
    del keep
    if with_info:
        return rho_out, [(i.sigma, i.nu, i.cg_resid, i.clip) for i in info[:n_iter]]
    return rho_out


def mpi_pnp_solve_sharded(model, grid, r, v, data, n_iter, n_cg, nu0, allreduce, clip_pct=5.0,
                          rho_out=None, with_info=False, stream=None):
    """Algorithm 1 with A for one problem whose samples are split across
    processes: ``r``, ``v`` ([T_p, 2]) and ``data`` ([n_ch, T_p]) are this
    process's slice.  ``allreduce`` is a callable (tensor) -> None that
    replaces a CUDA float64 tensor by its elementwise sum over all processes
    (identical on every process), ordered on the current stream -- e.g.
    ``torch.distributed.all_reduce`` with NCCL.  The library calls it on a
    view of its own buffer with the library's stream made current."""
    dt = data.dtype
    g = make_grid(grid)
    if rho_out is None:
        rho_out = torch.empty((g.ny, g.nx), dtype=dt, device=data.device)
    tr = _traj(r, v, dt)
    m = make_model(model)
    opts = PnPOpts(MPI_OP_FORWARD, int(n_iter), int(n_cg), float(nu0), float(clip_pct), 0)
    info = (PnPIterInfo * max(1, n_iter))() if with_info else None
    dev = data.device

    def _ar(buf, count, strm, user):
        try:
            t = _wrap(buf, (int(count),), torch.float64, dev)
            if int(strm or 0) == torch.cuda.current_stream(dev).cuda_stream:
                allreduce(t)
            else:
                with torch.cuda.stream(torch.cuda.ExternalStream(int(strm), device=dev)):
                    allreduce(t)
            return 0
        except Exception:  # noqa: BLE001 - reported as MPI_ERR_CALLBACK
            return 1
    cb = ALLREDUCE_FN(_ar)
    data_ptr = _dev(data, dt, "data") if data.numel() else None
    _check(load().mpi_pnp_solve_sharded(ctypes.byref(m), ctypes.byref(g), ctypes.byref(tr), _dtype(data),
                                        data_ptr, ctypes.byref(opts), DENOISE_FN(0), None, cb, None,
                                        _dev(rho_out, dt, "rho_out"), info, _stream(stream)))
    del cb
    if with_info:
        return rho_out, [(i.sigma, i.nu, i.cg_resid, i.clip) for i in info[:n_iter]]
    return rho_out


def _wrap(ptr, shape, dtype, device):
    """A tensor view of library-owned device memory (no copy), through the
    CUDA array interface."""
    n = 1
    for s in shape:
        n *= s
    if n == 0 or not ptr:
        return torch.empty(shape, dtype=dtype, device=device)

    class _CAI:
        __cuda_array_interface__ = {
            "shape": (n,), "typestr": {torch.float32: "<f4", torch.float64: "<f8"}[dtype],
            "data": (ptr, False), "version": 3, "strides": None, "stream": None}
    return torch.as_tensor(_CAI(), device=device).view(shape)


class BatchPlan:
    """mpi_batch_plan: batched Algorithm 1 (FP32) over frames of different
    sizes.  ``frames`` is a list of (model, grid, T); ``nu0`` one value per
    frame."""

    def __init__(self, frames, nu0, n_iter, n_cg, clip_pct=5.0, flags=MPI_BATCH_AUTOTUNE):
        n = len(frames)
        self.n = n
        self._models = (Model * n)(*[make_model(m) for m, _, _ in frames])
        self._grids = (GridDesc * n)(*[make_grid(g) for _, g, _ in frames])
        self._T = (ctypes.c_int64 * n)(*[int(T) for _, _, T in frames])
        self._nu0 = (ctypes.c_double * n)(*[float(x) for x in nu0])
        opts = PnPOpts(MPI_OP_FORWARD, int(n_iter), int(n_cg), 0.0, float(clip_pct), 0)
        self._plan = ctypes.c_void_p()
        _check(load().mpi_batch_plan_create(n, self._models, self._grids, self._T, self._nu0,
                                            ctypes.byref(opts), int(flags), ctypes.byref(self._plan)))
        self.shapes = [(int(_get(g, "ny")), int(_get(g, "nx"))) for _, g, _ in frames]

    def run(self, r, v, s, rho_out=None, stream=None):
        n = self.n
        if rho_out is None:
            rho_out = [torch.empty(sh, dtype=torch.float32, device=s[0].device) for sh in self.shapes]
        P = ctypes.c_void_p * n
        rr = P(*[_dev(t, torch.float32, "r") for t in r])
        vv = P(*[_dev(t, torch.float32, "v") for t in v])
        ss = P(*[_dev(t, torch.float32, "s") for t in s])
        oo = P(*[_dev(t, torch.float32, "rho_out") for t in rho_out])
        _check(load().mpi_batch_pnp_run(self._plan, rr, vv, ss, oo, _stream(stream)))
        return rho_out

    def info(self) -> dict:
        inf = BatchInfo()
        _check(load().mpi_batch_plan_info(self._plan, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in BatchInfo._fields_}

    def close(self):
        if self._plan:
            load().mpi_batch_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


# ---------------------------------------------------------------------------
# Three-dimensional field-free point (Sec. 2 with n = 3).  A ``grid3`` has nx,
# ny, nz, x0, y0, z0, dx, dy, dz; a ``model3`` has beta, G (3x3) and p (n_ch x
# 3).  Volumes are [nz, ny, nx]; r and v are [T, 3].

def mpi_forward3(model3, grid3, r, v, c, s=None, stream=None):
    """Forward operator in three dimensions: c [nz, ny, nx] -> s [n_ch, T],
    s[k][t] = sum c p_k^T beta K(beta G(x - r_t)) G v_t with the 3x3 kernel matrix."""
    dt = c.dtype
    n_ch = len(_get(model3, "p"))
    if s is None:
        s = torch.empty((n_ch, r.shape[0]), dtype=dt, device=c.device)
    tr = _traj(r, v, dt, 3)
    m, g = make_model3(model3), make_grid3(grid3)
    _check(load().mpi_forward3(ctypes.byref(m), ctypes.byref(g), ctypes.byref(tr), _dtype(c),
                               _dev(c, dt, "c"), _dev(s, dt, "s") if s.numel() else None,
                               _stream(stream)))
    return s


def mpi_adjoint3(model3, grid3, r, v, s, c_out=None, stream=None):
    """Adjoint of mpi_forward3: s [n_ch, T] -> c_out [nz, ny, nx]."""
    dt = s.dtype
    g = make_grid3(grid3)
    if c_out is None:
        c_out = torch.empty((g.nz, g.ny, g.nx), dtype=dt, device=s.device)
    tr = _traj(r, v, dt, 3)
    m = make_model3(model3)
    _check(load().mpi_adjoint3(ctypes.byref(m), ctypes.byref(g), ctypes.byref(tr), _dtype(s),
                               _dev(s, dt, "s") if s.numel() else None, _dev(c_out, dt, "c_out"),
                               _stream(stream)))
    return c_out


def mpi_conv3(model3, grid3, x, out=None, stream=None):
    """out = C x in three dimensions: convolution of x [nz, ny, nx] with the
    sampled 3-D trace kernel (n - 1 = 2); direct sum or FFT route."""
    dt = x.dtype
    if out is None:
        out = torch.empty_like(x)
    m, g = make_model3(model3), make_grid3(grid3)
    _check(load().mpi_conv3(ctypes.byref(m), ctypes.byref(g), _dtype(x), _dev(x, dt, "in"),
                            _dev(out, dt, "out"), _stream(stream)))
    return out


def mpi_interp3(grid3, r, v, Ahat, s=None, stream=None):
    """Core Stage measurement in three dimensions: Ahat [9, nz, ny, nx] ->
    s [3, T]."""
    dt = Ahat.dtype
    if s is None:
        s = torch.empty((3, r.shape[0]), dtype=dt, device=Ahat.device)
    tr = _traj(r, v, dt, 3)
    g = make_grid3(grid3)
    _check(load().mpi_interp3(ctypes.byref(g), ctypes.byref(tr), _dtype(Ahat), _dev(Ahat, dt, "Ahat"),
                              _dev(s, dt, "s") if s.numel() else None, _stream(stream)))
    return s


def mpi_interp3_adjoint(grid3, r, v, s, Ahat=None, stream=None):
    """Exact transpose of mpi_interp3: s [3, T] -> Ahat [9, nz, ny, nx], summed
    in a fixed order (no atomics)."""
    dt = s.dtype
    g = make_grid3(grid3)
    if Ahat is None:
        Ahat = torch.empty((9, g.nz, g.ny, g.nx), dtype=dt, device=s.device)
    tr = _traj(r, v, dt, 3)
    _check(load().mpi_interp3_adjoint(ctypes.byref(g), ctypes.byref(tr), _dtype(s),
                                      _dev(s, dt, "s") if s.numel() else None,
                                      _dev(Ahat, dt, "Ahat"), _stream(stream)))
    return Ahat


def mpi_grid3(grid3, r, v, s, gamma=1e-7, max_iter=10000, rel_tol=1e-3, Ahat=None, trace=None,
              return_iters=False, channel=None, lap_scaled=False, stream=None):
    """Core Stage in three dimensions.  ``channel`` None: s is [3][T] and
    Ahat [9][nz][ny][nx], trace = A_00 + A_11 + A_22; channel k (0, 1 or 2):
    only that channel was measured, s is [T] (or [1][T]), Ahat holds the row
    (A_k0, A_k1, A_k2) and trace = A_kk.  ``lap_scaled``: the Laplacian with
    1/dx^2, 1/dy^2, 1/dz^2 instead of the bare stencil."""
    dt = s.dtype
    g = make_grid3(grid3)
    nc = 9 if channel is None else 3
    if Ahat is None:
        Ahat = torch.empty((nc, g.nz, g.ny, g.nx), dtype=dt, device=s.device)
    if trace is None:
        trace = torch.empty((g.nz, g.ny, g.nx), dtype=dt, device=s.device)
    tr = _traj(r, v, dt, 3)
    opts = GridOpts(float(gamma), int(max_iter), float(rel_tol),
                    0 if channel is None else int(channel) + 1, 1 if lap_scaled else 0)
    n_it = ctypes.c_int(-1)
    _check(load().mpi_grid3(ctypes.byref(g), ctypes.byref(tr), _dtype(s),
                            _dev(s, dt, "s") if s.numel() else None, ctypes.byref(opts),
                            _dev(Ahat, dt, "Ahat"), _dev(trace, dt, "trace"),
                            ctypes.byref(n_it) if return_iters else None, _stream(stream)))
    if return_iters:
        return Ahat, trace, n_it.value
    return Ahat, trace


def mpi_conv3_kernel(model3, grid3, kernel, x, out=None, stream=None):
    """mpi_conv3 with kernel 0 (the trace kernel) or 1 (beta tr K(beta G y),
    the kernel of the gradient-weighted trace)."""
    dt = x.dtype
    if out is None:
        out = torch.empty_like(x)
    m, g = make_model3(model3), make_grid3(grid3)
    _check(load().mpi_conv3_kernel(ctypes.byref(m), ctypes.byref(g), _dtype(x), int(kernel),
                                   _dev(x, dt, "in"), _dev(out, dt, "out"), _stream(stream)))
    return out


def mpi_weighted_trace3(model3, grid3, Ahat, out=None, stream=None):
    """tr(Ahat G^-1) per node from the 9 Core Stage components [9, nz, ny, nx]."""
    dt = Ahat.dtype
    g = make_grid3(grid3)
    if out is None:
        out = torch.empty((g.nz, g.ny, g.nx), dtype=dt, device=Ahat.device)
    m = make_model3(model3)
    _check(load().mpi_weighted_trace3(ctypes.byref(m), ctypes.byref(g), _dtype(Ahat), _dev(Ahat, dt, "Ahat"),
                                      _dev(out, dt, "out"), _stream(stream)))
    return out


def mpi_denoise_gaussian5_3d(x, out=None, stream=None):
    """The built-in volume denoiser: the 5-tap Gaussian along x, y and z
    (reflect boundary) on x [nz, ny, nx]."""
    dt = x.dtype
    if out is None:
        out = torch.empty_like(x)
    nz, ny, nx = x.shape
    _check(load().mpi_denoise_gaussian5_3d(_dev(x, dt, "in"), _dev(out, dt, "out"), nx, ny, nz,
                                           _dtype(x), None, _stream(stream), None))
    return out


def mpi_pnp_solve3(model3, grid3, r, v, data, n_iter, n_cg, nu0, clip_pct=5.0, op=MPI_OP_FORWARD,
                   denoise=None, rho_out=None, with_info=False, kernel=0, stream=None):
    """Algorithm 1 in three dimensions.  ``denoise`` is None (built-in volume
    Gaussian) or a callable (in_tensor, out_tensor, sigma_dev_tensor) -> None
    on [nz, ny, nx] volumes that enqueues on the current stream.  ``kernel``
    (with MPI_OP_CONV): 0 the trace kernel, 1 beta tr K(beta G y)."""
    dt = data.dtype
    g = make_grid3(grid3)
    if rho_out is None:
        rho_out = torch.empty((g.nz, g.ny, g.nx), dtype=dt, device=data.device)
    if op == MPI_OP_FORWARD:
        tr = _traj(r, v, dt, 3)
    else:
        tr = Traj(0, None, None) if r is None else _traj(r, v, dt, 3)
    m = make_model3(model3)
    opts = PnPOpts(int(op), int(n_iter), int(n_cg), float(nu0), float(clip_pct), int(kernel))
    info = (PnPIterInfo * max(1, n_iter))() if with_info else None
    cb = DENOISE3_FN(0)
    keep = None
    if denoise is not None:
        dev = data.device

        def _cb(pin, pout, nx, ny, nz, dtype, sig, strm, user):
            try:
                tdt = torch.float32 if dtype == MPI_F32 else torch.float64
                denoise(_wrap(pin, (nz, ny, nx), tdt, dev), _wrap(pout, (nz, ny, nx), tdt, dev),
                        _wrap(sig, (), torch.float64, dev))
                return 0
            except Exception:  # noqa: BLE001 - reported as MPI_ERR_CALLBACK
                return 1
        cb = DENOISE3_FN(_cb)
        keep = cb
    _check(load().mpi_pnp_solve3(ctypes.byref(m), ctypes.byref(g), ctypes.byref(tr), _dtype(data),
                                 _dev(data, dt, "data"), ctypes.byref(opts), cb, None,
                                 _dev(rho_out, dt, "rho_out"), info, _stream(stream)))
    del keep
    if with_info:
        return rho_out, [(i.sigma, i.nu, i.cg_resid, i.clip) for i in info[:n_iter]]
    return rho_out


# ---------------------------------------------------------------------------
# Preprocessing

def mpi_transfer_correct(s_raw, a_hat, snr=None, theta=None, out=None, stream=None):
    """Transfer-function correction: s_raw [n_ch, T] (FP32/FP64, device),
    a_hat [n_ch, T//2 + 1] complex128 (device), snr [n_ch, T//2 + 1] float64
    (device) or None, theta: n_ch thresholds (host sequence)."""
    dt = s_raw.dtype
    if s_raw.dim() != 2:
        raise ValueError("s_raw must be [n_ch, T]")
    n_ch, T = s_raw.shape
    if a_hat.dtype != torch.complex128 or tuple(a_hat.shape) != (n_ch, T // 2 + 1):
        raise ValueError("a_hat must be complex128 [n_ch, T//2 + 1]")
    if out is None:
        out = torch.empty_like(s_raw)
    a_ri = torch.view_as_real(a_hat.contiguous())
    th = None
    if snr is not None:
        if snr.dtype != torch.float64 or tuple(snr.shape) != (n_ch, T // 2 + 1):
            raise ValueError("snr must be float64 [n_ch, T//2 + 1]")
        if theta is None or len(theta) != n_ch:
            raise ValueError("theta needs one threshold per channel")
        th = (ctypes.c_double * n_ch)(*[float(x) for x in theta])
    _check(load().mpi_transfer_correct(n_ch, T, _dtype(s_raw),
                                       _dev(s_raw, dt, "s_raw") if T else None,
                                       _dev(a_ri, torch.float64, "a_hat") if T else None,
                                       _dev(snr, torch.float64, "snr") if snr is not None else None,
                                       th, _dev(out, dt, "out") if T else None, _stream(stream)))
    return out

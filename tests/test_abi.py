"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point declared in include/*.h; host-side argument checks need no GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(mpi_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2505_22797_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"mpi_forward", "mpi_adjoint", "mpi_pnp_solve", "mpi_grid"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2505_22797_gb300 import api
    assert _declared() <= set(api._SIGS)


def test_status_strings(lib):
    lib.mpi_status_string.restype = ctypes.c_char_p
    assert lib.mpi_status_string(0) == b"ok"
    assert lib.mpi_status_string(-1) == b"invalid argument"
    assert lib.mpi_version() >= 100


class _Model(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("G", ctypes.c_double * 4), ("n_ch", ctypes.c_int),
                ("p", ctypes.c_double * 4)]


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double)]


class _Traj(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int64), ("r", ctypes.c_void_p), ("v", ctypes.c_void_p)]


def test_argument_validation_without_gpu(lib):
    """Bad arguments are rejected on the host before any CUDA call."""
    lib.mpi_forward.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 3
    lib.mpi_last_error_message.restype = ctypes.c_char_p
    good = _Model(2331.35, (ctypes.c_double * 4)(2.5e-3, 0, 0, 2.5e-3), 2,
                  (ctypes.c_double * 4)(1, 0, 0, 1))
    grid = _Grid(4, 4, -12, -12, 6, 6)
    tr = _Traj(0, None, None)
    for model, g, t, dtype, why in [
        (_Model(-1.0, good.G, 2, good.p), grid, tr, 0, b"beta"),
        (_Model(1.0, (ctypes.c_double * 4)(1, 2, 2, 4), 2, good.p), grid, tr, 0, b"singular"),
        (_Model(1.0, good.G, 3, good.p), grid, tr, 0, b"n_ch"),
        (good, _Grid(0, 4, 0, 0, 1, 1), tr, 0, b"nx"),
        (good, grid, _Traj(-5, None, None), 0, b"T must"),
        (good, grid, tr, 7, b"dtype"),
        (good, grid, _Traj(10, None, None), 0, b"NULL"),
    ]:
        st = lib.mpi_forward(ctypes.byref(model), ctypes.byref(g), ctypes.byref(t), dtype,
                             None, None, None)
        assert st == -1
        assert why in lib.mpi_last_error_message()


class _Grid3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class _GridOpts(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("max_iter", ctypes.c_int), ("rel_tol", ctypes.c_double),
                ("channel", ctypes.c_int)]


def test_core_stage_argument_validation_without_gpu(lib):
    """The 2-D and 3-D Core Stage entry points reject bad grids, trajectories,
    options and missing buffers on the host (status and message), before any
    CUDA call."""
    lib.mpi_last_error_message.restype = ctypes.c_char_p
    for name in ("mpi_grid", "mpi_grid3"):
        getattr(lib, name).argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 6
    for name in ("mpi_interp3", "mpi_interp3_adjoint"):
        getattr(lib, name).argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 3
    g3 = _Grid3(4, 4, 2, -12, -12, -6, 6, 6, 6)
    g2 = _Grid(4, 4, -12, -12, 6, 6)
    tr0 = _Traj(0, None, None)
    opts = _GridOpts(1e-7, 10, 1e-3, 0)
    buf = ctypes.c_void_p(16)  # never dereferenced: every case fails validation first

    def call3(name, g, t, dtype, o=None, with_out=True):
        f = getattr(lib, name)
        if name == "mpi_grid3":
            return f(ctypes.byref(g), ctypes.byref(t), dtype, None, ctypes.byref(o) if o else None,
                     buf if with_out else None, buf if with_out else None, None, None)
        return f(ctypes.byref(g), ctypes.byref(t), dtype, buf if with_out else None, None, None)

    cases = [
        ("mpi_grid3", _Grid3(4, 0, 2, 0, 0, 0, 1, 1, 1), tr0, 0, opts, True, -1, b"nx, ny, nz"),
        ("mpi_grid3", _Grid3(4, 4, 2, 0, 0, 0, 1, 1, 0.0), tr0, 0, opts, True, -1, b"spacing"),
        ("mpi_grid3", g3, _Traj(-1, None, None), 0, opts, True, -1, b"T must"),
        ("mpi_grid3", g3, tr0, 5, opts, True, -1, b"dtype"),
        ("mpi_grid3", g3, _Traj(1 << 31, buf, buf), 0, opts, True, -6, b"2^31"),
        ("mpi_grid3", _Grid3(1 << 10, 1 << 10, 1 << 7, 0, 0, 0, 1, 1, 1), tr0, 0, opts, True, -6, b"2^27"),
        ("mpi_grid3", g3, tr0, 0, _GridOpts(1e-7, 10, 1e-3, 4), True, -1, b"options"),
        ("mpi_grid3", g3, tr0, 0, _GridOpts(-1.0, 10, 1e-3, 0), True, -1, b"options"),
        ("mpi_grid3", g3, tr0, 0, _GridOpts(1e-7, -1, 1e-3, 0), True, -1, b"options"),
        ("mpi_grid3", g3, tr0, 0, None, True, -1, b"options"),
        ("mpi_grid3", g3, tr0, 0, opts, False, -1, b"NULL"),
        ("mpi_interp3", g3, _Traj(8, None, None), 0, None, True, -1, b"NULL"),
        ("mpi_interp3_adjoint", g3, tr0, 0, None, False, -1, b"NULL"),
    ]
    for name, g, t, dtype, o, with_out, want, why in cases:
        st = call3(name, g, t, dtype, o, with_out)
        assert st == want, (name, why, st)
        assert why in lib.mpi_last_error_message(), (name, why, lib.mpi_last_error_message())
    # the 2-D Core Stage: channel selector 0..2 only
    st = lib.mpi_grid(ctypes.byref(g2), ctypes.byref(tr0), 0, None,
                      ctypes.byref(_GridOpts(1e-7, 10, 1e-3, 3)), buf, buf, None, None)
    assert st == -1 and b"options" in lib.mpi_last_error_message()

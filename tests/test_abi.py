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
                ("channel", ctypes.c_int), ("lap_scaled", ctypes.c_int)]


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
        ("mpi_grid3", g3, tr0, 0, _GridOpts(1e-7, 10, 1e-3, 0, 2), True, -1, b"options"),
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
    st = lib.mpi_grid(ctypes.byref(g2), ctypes.byref(tr0), 0, None,
                      ctypes.byref(_GridOpts(1e-7, 10, 1e-3, 0, -1)), buf, buf, None, None)
    assert st == -1 and b"options" in lib.mpi_last_error_message()


def test_other_entry_points_validate_without_gpu():
    """3-D operators, the convolution entries, the transfer correction, the
    PnP options, the binning step and the batch plan reject bad arguments on the host with
    MPI_ERR_INVALID (or MPI_ERR_UNSUPPORTED) and a message, before any CUDA
    call."""
    from paper_2505_22797_gb300 import api, build
    build.build()
    lib = api.load()
    D9 = ctypes.c_double * 9
    D4 = ctypes.c_double * 4
    eye3 = D9(1, 0, 0, 0, 1, 0, 0, 0, 1)
    G3 = D9(-1.25e-3, 0, 0, 0, -1.25e-3, 0, 0, 0, 2.5e-3)
    m3 = api.Model3(2331.35, G3, 3, eye3)
    g3 = api.Grid3Desc(4, 4, 2, -12, -12, -6, 6, 6, 6)
    m2 = api.Model(2331.35, D4(2.5e-3, 0, 0, 2.5e-3), 2, D4(1, 0, 0, 1))
    g2 = api.GridDesc(4, 4, -12, -12, 6, 6)
    tr0 = api.Traj(0, None, None)
    buf = ctypes.c_void_p(16)  # never dereferenced
    pnp = api.PnPOpts(api.MPI_OP_FORWARD, 2, 3, 1e-3, 5.0, 0)
    no_cb = api.DENOISE_FN(0)
    no_cb3 = api.DENOISE3_FN(0)

    def ref(x):
        return ctypes.byref(x)

    cases = [
        ("singular G (3-D)", lambda: lib.mpi_forward3(ref(api.Model3(1.0, D9(), 3, eye3)), ref(g3), ref(tr0), 0,
                                                     buf, buf, None), -1, b"singular"),
        ("n_ch 4 (3-D)", lambda: lib.mpi_adjoint3(ref(api.Model3(1.0, G3, 4, eye3)), ref(g3), ref(tr0), 0,
                                                 buf, buf, None), -1, b"n_ch"),
        ("nz 0", lambda: lib.mpi_conv3(ref(m3), ref(api.Grid3Desc(4, 4, 0, 0, 0, 0, 1, 1, 1)), 0, buf, buf,
                                       None), -1, b"nx, ny, nz"),
        ("component 4", lambda: lib.mpi_conv_component(ref(m2), ref(g2), 0, 4, buf, buf, None), -1, b""),
        ("conv dtype", lambda: lib.mpi_conv(ref(m2), ref(g2), 3, buf, buf, None), -1, b"dtype"),
        ("transfer n_ch 0", lambda: lib.mpi_transfer_correct(0, 16, 0, buf, buf, None, None, buf, None),
         -1, b""),
        ("transfer n_ch 9", lambda: lib.mpi_transfer_correct(9, 16, 0, buf, buf, None, None, buf, None),
         -1, b""),
        ("transfer T < 0", lambda: lib.mpi_transfer_correct(2, -4, 0, buf, buf, None, None, buf, None),
         -1, b""),
        ("transfer a_hat NULL", lambda: lib.mpi_transfer_correct(2, 16, 0, buf, None, None, None, buf, None),
         -1, b""),
        ("pnp n_iter < 0", lambda: lib.mpi_pnp_solve(ref(m2), ref(g2), ref(tr0), 0, buf,
                                                     ref(api.PnPOpts(0, -1, 3, 1e-3, 5.0, 0)), no_cb, None,
                                                     buf, None, None), -1, b""),
        ("pnp op 7", lambda: lib.mpi_pnp_solve(ref(m2), ref(g2), ref(tr0), 0, buf,
                                               ref(api.PnPOpts(7, 2, 3, 1e-3, 5.0, 0)), no_cb, None,
                                               buf, None, None), -1, b""),
        ("pnp3 kernel entry", lambda: lib.mpi_pnp_solve3(ref(m3), ref(g3), ref(tr0), 0, buf,
                                                        ref(api.PnPOpts(1, 2, 3, 1e-3, 5.0, 2)), no_cb3, None,
                                                        buf, None, None), -1, b""),
        ("pnp3 kernel with A", lambda: lib.mpi_pnp_solve3(ref(m3), ref(g3), ref(tr0), 0, buf,
                                                         ref(api.PnPOpts(0, 2, 3, 1e-3, 5.0, 1)), no_cb3, None,
                                                         buf, None, None), -1, b""),
        ("conv3 kernel 2", lambda: lib.mpi_conv3_kernel(ref(m3), ref(g3), 0, 2, buf, ctypes.c_void_p(32), None),
         -1, b"kernel"),
        ("weighted trace NULL", lambda: lib.mpi_weighted_trace3(ref(m3), ref(g3), 0, None, buf, None), -1,
         b"NULL"),
        ("pnp opts NULL", lambda: lib.mpi_pnp_solve(ref(m2), ref(g2), ref(tr0), 0, buf, None, no_cb, None,
                                                    buf, None, None), -1, b""),
        ("cell order n_cells 0", lambda: lib.mpi_cell_order(8, buf, 0, buf, None, None), -1, b"cell ordering"),
        ("cell order T < 0", lambda: lib.mpi_cell_order(-1, buf, 4, buf, None, None), -1, b"cell ordering"),
        ("cell order T >= 2^31", lambda: lib.mpi_cell_order(1 << 31, buf, 4, buf, None, None), -1,
         b"cell ordering"),
        ("cell order list NULL", lambda: lib.mpi_cell_order(8, buf, 4, None, None, None), -1, b"cell ordering"),
        ("batch 0 frames", lambda: lib.mpi_batch_plan_create(0, ref(m2), ref(g2), None, None, ref(pnp), 0,
                                                             ctypes.byref(ctypes.c_void_p())), -1, b""),
        ("batch 65 frames", lambda: lib.mpi_batch_plan_create(65, ref(m2), ref(g2), None, None, ref(pnp), 0,
                                                              ctypes.byref(ctypes.c_void_p())), None, b""),
    ]
    for what, call, want, why in cases:
        st = call()
        if want is None:
            assert st in (-1, -6), (what, st)
        else:
            assert st == want, (what, st, lib.mpi_last_error_message())
        msg = lib.mpi_last_error_message()
        assert msg and why in msg, (what, msg)


def test_header_is_plain_c_and_links_from_c(tmp_path):
    """include/mpi_recon.h is self-contained C99 (and C++17), and a plain C
    program links against the library and calls it (no GPU needed for
    mpi_version / mpi_status_string)."""
    import shutil
    import subprocess
    cc, cxx = shutil.which("gcc"), shutil.which("g++")
    if not cc or not cxx:
        pytest.skip("gcc/g++ not available")
    from paper_2505_22797_gb300 import build
    lib = build.build()
    hdr = os.path.join(ROOT, "include", "mpi_recon.h")
    for comp, std, lang in ((cc, "-std=c99", "c"), (cxx, "-std=c++17", "c++")):
        res = subprocess.run([comp, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                              "-x", lang, hdr], capture_output=True, text=True)
        assert res.returncode == 0, res.stderr
    src = tmp_path / "main.c"
    src.write_text('#include <string.h>\n#include "mpi_recon.h"\n'
                   'int main(void) { return (mpi_version() >= 100 && '
                   'strcmp(mpi_status_string(MPI_ERR_INVALID), "invalid argument") == 0) ? 0 : 1; }\n')
    exe = tmp_path / "main"
    libdir = os.path.dirname(lib)
    res = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir,
                          "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir, "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    assert subprocess.run([str(exe)]).returncode == 0


def test_pipe_probe_validates_without_gpu():
    """The pipe-rate probe rejects an unknown instruction kind, an occupancy
    outside 1..8 blocks per SM and a zero iteration count on the host."""
    from paper_2505_22797_gb300 import api, build
    build.build()
    lib = api.load()
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    for op, bps, it in ((7, 4, 16), (api.PROBE_RSQRT, 0, 16), (api.PROBE_RSQRT, 9, 16),
                        (api.PROBE_FMA, 4, 0)):
        st = lib.mpi_probe_pipe_rate(op, bps, it, ctypes.byref(rate), ctypes.byref(ms), None)
        assert st == api.MPI_ERR_INVALID
        assert b"probe" in lib.mpi_last_error_message()

"""How the Core Stage regulariser scales with the grid (Eq. first:step): the
paper regularises with the L2 norm of the Laplacian of the core operator and
uses gamma = 1e-7 for every grid, showing 21x21 and 100x100 reconstructions of
the same scan.  On the oracle's two-stage pipeline (Core Stage, then PnP with
the trace-kernel convolution) over the 1632-sample Lissajous scan:

* the 5-point stencil taken as it stands (no 1/h^2) makes gamma act h^-4 more
  weakly on finer grids, and the 100x100 reconstruction fails (relative L2
  distance to the phantom above 1.5, against 0.39 at 21x21);
* the stencil divided by h^2 (h in the grid's length unit, mm), i.e. gamma
  replaced by gamma / h^4 for the unscaled stencil, keeps gamma = 1e-7
  working on both grids (about 0.39 and 0.33).

This pins the observation behind the Core Stage reading, with the oracle
only; it does not change any operator."""
import numpy as np
import pytest

from paper_2505_22797_gb300 import synthetic as syn

pytestmark = pytest.mark.slow


def _two_stage(orc, n, gamma):
    m = syn.default_model()
    r, v = syn.lissajous(1632, 17, 16)
    g = syn.square_grid(n)
    c = syn.ellipses(g, np.random.default_rng(101))
    s = syn.add_noise(orc.forward(m, g, r, v, c), 0.01, 201)
    _, u, _ = orc.core_stage(g, r, v, s, gamma, max_iter=10000, rel_tol=1e-3)
    kern = orc.conv_kernel(m, g)

    def C(x):
        return orc.conv(g, kern, x.reshape(n, n))

    rng = np.random.default_rng(5)
    fro = np.mean([np.sum(C(rng.integers(0, 2, (n, n)) * 2.0 - 1.0) ** 2) for _ in range(4)])
    rho = orc.pnp(C, C, u, (n, n), 10, 20, 1e-3 * fro / (n * n))
    return float(np.linalg.norm(rho - c) / np.linalg.norm(c))


def test_unscaled_stencil_fails_on_the_fine_grid_and_scaled_one_does_not(orc):
    gamma = 1e-7
    h21, h100 = 24.0 / 21, 24.0 / 100
    coarse = _two_stage(orc, 21, gamma)
    coarse_scaled = _two_stage(orc, 21, gamma / h21 ** 4)
    fine = _two_stage(orc, 100, gamma)
    fine_scaled = _two_stage(orc, 100, gamma / h100 ** 4)
    assert coarse < 0.45 and abs(coarse_scaled - coarse) < 0.02
    assert fine > 1.5
    assert fine_scaled < 0.4


def test_single_channel_pipeline_on_the_fine_grid(orc):
    """The single-channel form (channel x only, Sec. 3.6: Core Stage on one
    channel, PnP with the (0, 0) kernel entry) shows the same: at 100x100 the
    bare stencil fails and the scaled Laplacian reconstructs."""
    m = syn.default_model()
    r, v = syn.lissajous(1632, 17, 16)
    n = 100
    g = syn.square_grid(n)
    c = syn.ellipses(g, np.random.default_rng(101))
    s = syn.add_noise(orc.forward(m, g, r, v, c), 0.01, 201)
    kern = orc.conv_kernel(m, g, component=(0, 0))

    def C(x):
        return orc.conv(g, kern, x.reshape(n, n))

    rng = np.random.default_rng(5)
    nu0 = 1e-3 * np.mean([np.sum(C(rng.integers(0, 2, (n, n)) * 2.0 - 1.0) ** 2) for _ in range(4)]) / (n * n)
    errs = {}
    for lap in ("bare", "scaled"):
        _, a00, _ = orc.core_stage_channel(g, r, v, s[0], 0, 1e-7, 10000, rel_tol=1e-3, lap=lap)
        rho = orc.pnp(C, C, a00, (n, n), 10, 20, nu0)
        errs[lap] = float(np.linalg.norm(rho - c) / np.linalg.norm(c))
    assert errs["bare"] > 1.5 and errs["scaled"] < 0.6

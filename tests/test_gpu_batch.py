"""Batched reconstructions (mpi_batch_plan): frames of different grid sizes
and trajectory lengths in one launch per operator application, one PnP
iteration captured as a CUDA graph.  Checked bit for bit against the
single-frame solve when split the same way, and against the FP64 oracle
under the tuned split."""
import numpy as np
import pytest
import torch

from paper_2505_22797_gb300 import api
from paper_2505_22797_gb300 import synthetic as syn
from tests.gpu_util import dev, host, rel_l2, roundoff_spread, rounded, tol

pytestmark = pytest.mark.gpu
F32 = torch.float32


def _frames(orc, specs):
    out = []
    for k, (nx, ny, T, traj) in enumerate(specs):
        cfg = syn.small(nx, ny, T, traj, seed=40 + k)
        m, g = cfg["model"], cfg["grid"]
        if k == 1:
            m = dict(m, G=[[2.4e-3, 3e-4], [3e-4, 2.6e-3]])
        r, v, c = (rounded(cfg[x], F32) for x in ("r", "v", "c"))
        s = rounded(syn.add_noise(orc.forward(m, g, r, v, c), 0.01, 300 + k), F32)
        nu0 = orc.nu0_from_frob2(orc.frob2(m, g, r, v), nx * ny)
        out.append(dict(m=m, g=g, r=r, v=v, s=s, nu0=nu0, T=T))
    return out


SPECS = [(24, 24, 900, "lissajous"), (33, 29, 1500, "spiral"), (40, 40, 3000, "spiral"),
         (17, 31, 700, "lissajous")]


def _plan(frames, n_it, n_cg, flags):
    return api.BatchPlan([(f["m"], f["g"], f["T"]) for f in frames], [f["nu0"] for f in frames],
                         n_it, n_cg, flags=flags)


def _run(plan, frames):
    return [host(x) for x in plan.run([dev(f["r"], F32) for f in frames], [dev(f["v"], F32) for f in frames],
                                      [dev(f["s"], F32) for f in frames])]


def test_batch_matches_single_frame_bitwise(orc):
    frames = _frames(orc, SPECS)
    plan = _plan(frames, 3, 20, api.MPI_BATCH_MATCH_SINGLE)
    got = _run(plan, frames)
    for f, gb in zip(frames, got):
        single = host(api.mpi_pnp_solve(f["m"], f["g"], dev(f["r"], F32), dev(f["v"], F32),
                                        dev(f["s"], F32), 3, 20, f["nu0"]))
        assert np.array_equal(gb, single)
    info = plan.info()
    assert info["graph_nodes"] > 0 and info["n_frames"] == 4


def test_batch_autotuned_vs_oracle_and_replay(orc):
    frames = _frames(orc, SPECS)
    plan = _plan(frames, 4, 5, api.MPI_BATCH_AUTOTUNE)
    first = _run(plan, frames)
    again = _run(plan, frames)  # graph replay, tuned split kept
    info = plan.info()
    assert info["tuned"] == 1
    print("batch plan", info)
    for f, a, b in zip(frames, first, again):
        assert np.array_equal(a, b)
        want = orc.pnp(lambda x, f=f: orc.forward(f["m"], f["g"], f["r"], f["v"], x),
                       lambda y, f=f: orc.adjoint(f["m"], f["g"], f["r"], f["v"], y), f["s"],
                       (f["g"]["ny"], f["g"]["nx"]), 4, 5, f["nu0"])
        # whole reconstructions: the FP32 bar or ten times the oracle's own
        # round-off spread at FP32 (see roundoff_spread), whichever is larger
        spread = roundoff_spread(orc, f["m"], f["g"], f["r"], f["v"], f["s"], 4, 5, f["nu0"], F32)
        assert rel_l2(a, want) <= max(tol(F32), 10 * spread)


def test_batch_invalid():
    m, g = syn.default_model(), syn.square_grid(8)
    with pytest.raises(api.MPIError) as e:
        api.BatchPlan([(m, g, 100)] * 65, [1.0] * 65, 1, 1)
    assert e.value.status == api.MPI_ERR_UNSUPPORTED
    with pytest.raises(api.MPIError):
        api.BatchPlan([(m, g, 0)], [1.0], 1, 1)
    with pytest.raises(api.MPIError):
        api.BatchPlan([(m, g, 10)], [-1.0], 1, 1)


@pytest.mark.slow
def test_batch_full_size_vs_single_frames():
    """The 64-frame workload (grids 64^2..256^2, T in [8192, 131072]) in the
    configuration the benchmark times (autotuned split, persistent or block
    launches, one PnP iteration in a CUDA graph), checked frame by frame
    against the single-frame solve (itself held to the FP64 oracle by the
    other tests) on seeded random data: one PnP iteration of 2 CG steps."""
    frames = syn.batch_frames(64)
    rng = np.random.default_rng(5)
    r = [dev(rounded(f["r"], F32), F32) for f in frames]
    v = [dev(rounded(f["v"], F32), F32) for f in frames]
    s = [dev(rounded(rng.normal(size=(2, f["r"].shape[0])), F32), F32) for f in frames]
    nu0 = [1e-2] * len(frames)
    plan = api.BatchPlan([(f["model"], f["grid"], f["r"].shape[0]) for f in frames], nu0, 1, 2,
                         flags=api.MPI_BATCH_AUTOTUNE)
    got = [host(x) for x in plan.run(r, v, s)]
    for k in range(0, 64, 9):
        f = frames[k]
        single = host(api.mpi_pnp_solve(f["model"], f["grid"], r[k], v[k], s[k], 1, 2, nu0[k]))
        assert rel_l2(got[k], single) <= tol(F32), k

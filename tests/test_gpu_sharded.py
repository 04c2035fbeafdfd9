"""GPU parity of the sample-sharded solve (mpi_pnp_solve_sharded) against
the FP64 oracle's Algorithm 1 on the whole problem.

Processes are stood in for by threads of this process, one shard each, on
the one GPU, each on its own stream, their partial adjoint images summed by
the host-staged fixed-order all-reduce (sharded.ThreadAllreduce): the shards
meet on the host between launches, no kernel waits for another."""
import threading

import numpy as np
import pytest
import torch

from paper_2505_22797_gb300 import api, sharded
from paper_2505_22797_gb300 import synthetic as syn
from tests.gpu_util import dev, host, rel_l2, rounded, tol

pytestmark = pytest.mark.gpu
DTYPES = [torch.float32, torch.float64]


def _case(orc, shape, traj, seed, dt, n_it=4, n_cg=4):
    cfg = syn.small(*shape, traj=traj, seed=seed)
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    s = rounded(syn.add_noise(orc.forward(m, g, r, v, c), cfg["noise_frac"], cfg["noise_seed"]), dt)
    nu0 = orc.nu0_from_frob2(orc.frob2(m, g, r, v), g["nx"] * g["ny"])
    want = orc.pnp(lambda x: orc.forward(m, g, r, v, x), lambda y: orc.adjoint(m, g, r, v, y), s,
                   (g["ny"], g["nx"]), n_it, n_cg, nu0, clip_pct=5.0)
    return m, g, r, v, s, nu0, want, n_it, n_cg


def _run_threads(world, m, g, r, v, s, n_it, n_cg, nu0, dt):
    R, V, S = dev(r, dt), dev(v, dt), dev(s, dt)
    torch.cuda.synchronize()
    ar = sharded.ThreadAllreduce(world, timeout=120)
    out, err = [None] * world, [None] * world

    def run(k):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                rho = sharded.pnp_solve_sharded(m, g, R, V, S, n_iter=n_it, n_cg=n_cg, nu0=nu0,
                                                rank=k, world=world, allreduce=ar.for_rank(k))
                st.synchronize()
                out[k] = rho.double().cpu().numpy()
        except BaseException as e:  # noqa: BLE001 - reported below
            err[k] = e
            ar.abort()
    th = [threading.Thread(target=run, args=(k,)) for k in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert all(e is None for e in err), err
    return out


@pytest.mark.parametrize("dt", DTYPES)
def test_sharded_one_process_matches_oracle(orc, dt):
    m, g, r, v, s, nu0, want, n_it, n_cg = _case(orc, (37, 29, 1500), "spiral", 21, dt)
    args = (m, g, dev(r, dt), dev(v, dt), dev(s, dt), n_it, n_cg, nu0)
    got = host(api.mpi_pnp_solve_sharded(*args, lambda t: None))
    assert rel_l2(got, want) <= tol(dt)
    plain = host(api.mpi_pnp_solve(*args))
    assert rel_l2(got, plain) <= tol(dt)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_threads_match_oracle(orc, dt, world):
    m, g, r, v, s, nu0, want, n_it, n_cg = _case(orc, (33, 27, 2001), "lissajous", 8, dt)
    out = _run_threads(world, m, g, r, v, s, n_it, n_cg, nu0, dt)
    for k in range(world):
        assert np.array_equal(out[k], out[0])  # every shard ends with the same image
    assert rel_l2(out[0], want) <= tol(dt)


def test_sharded_with_an_empty_shard(orc):
    """Two samples over three shards: one shard has none and contributes a
    zero partial image."""
    dt = torch.float64
    m, g, r, v, s, nu0, want, n_it, n_cg = _case(orc, (6, 5, 2), "spiral", 4, dt, n_it=2, n_cg=3)
    out = _run_threads(3, m, g, r, v, s, n_it, n_cg, nu0, dt)
    assert rel_l2(out[2], want) <= tol(dt)


def test_sharded_callback_error_and_arguments():
    dt = torch.float32
    cfg = syn.small(12, 10, 300, seed=2)
    m, g = cfg["model"], cfg["grid"]
    R, V, C = (torch.as_tensor(np.asarray(cfg[k]), dtype=dt, device="cuda") for k in ("r", "v", "c"))
    S = api.mpi_forward(m, g, R, V, C)

    def broken(t):
        raise RuntimeError("link down")
    with pytest.raises(api.MPIError) as e:
        api.mpi_pnp_solve_sharded(m, g, R, V, S, 2, 3, 1e-3, broken)
    assert e.value.status == api.MPI_ERR_CALLBACK
    assert "allreduce" in str(e.value)

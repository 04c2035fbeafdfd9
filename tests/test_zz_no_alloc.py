"""mpi_forward_noalloc, the forward operator for callers that cannot let the
library allocate device memory while they run, against mpi_forward.

The file is named so that pytest collects it last: a run that stops at the
first failure has executed every other test before this one.  It needs
nothing from the other tests and also passes alone in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2505_22797_gb300 import api, build
from paper_2505_22797_gb300 import synthetic as syn
from tests.gpu_util import host, rel_l2, tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.load()


def _inputs(cfg, dt, seed):
    rng = np.random.default_rng(seed)
    c = cfg["c"] + 0.1 * rng.uniform(size=cfg["c"].shape)
    to = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    return to(cfg["r"]), to(cfg["v"]), to(c)


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_noalloc_matches_forward_two_calls(dt):
    """Two calls in a row with different inputs (the scratch keeps the first
    call's contents when the second starts) both match mpi_forward."""
    cfg = syn.config("c2")
    m, g = cfg["model"], cfg["grid"]
    for seed in (1, 2):
        r, v, c = _inputs(cfg, dt, seed)
        want = host(api.mpi_forward(m, g, r, v, c))
        got = host(api.mpi_forward_noalloc(m, g, r, v, c))
        assert rel_l2(got, want) <= tol(dt)


def test_noalloc_small_and_ragged():
    dt = torch.float32
    cfg = syn.small(37, 29, 777, "spiral", seed=3)
    m, g = cfg["model"], cfg["grid"]
    r, v, c = _inputs(cfg, dt, 4)
    for _ in range(2):
        assert rel_l2(host(api.mpi_forward_noalloc(m, g, r, v, c)),
                      host(api.mpi_forward(m, g, r, v, c))) <= tol(dt)


def test_noalloc_rejects_oversize_before_launch():
    dt = torch.float32
    T = 2_000_000  # needs 48 MB of scratch with two channels
    g = syn.square_grid(8)
    m = syn.default_model()
    r = torch.zeros((T, 2), dtype=dt, device="cuda")
    v = torch.zeros((T, 2), dtype=dt, device="cuda")
    c = torch.ones((8, 8), dtype=dt, device="cuda")
    s = torch.full((2, T), 5.0, dtype=dt, device="cuda")
    with pytest.raises(api.MPIError) as e:
        api.mpi_forward_noalloc(m, g, r, v, c, s=s)
    assert e.value.status == api.MPI_ERR_UNSUPPORTED
    assert "scratch" in str(e.value)
    assert float(s[0, 0]) == 5.0  # nothing was enqueued


def test_noalloc_needs_no_allocation(monkeypatch):
    """With every library allocation made to fail (the host-side injector
    MPI_FAULT=alloc), mpi_forward reports MPI_ERR_NOMEM while
    mpi_forward_noalloc still computes the same result: it never allocates."""
    dt = torch.float32
    cfg = syn.small(24, 20, 900, "lissajous", seed=5)
    m, g = cfg["model"], cfg["grid"]
    r, v, c = _inputs(cfg, dt, 6)
    want = host(api.mpi_forward(m, g, r, v, c))
    monkeypatch.setenv("MPI_FAULT", "alloc")
    with pytest.raises(api.MPIError) as e:
        api.mpi_forward(m, g, r, v, c)
    assert e.value.status == api.MPI_ERR_NOMEM
    got = host(api.mpi_forward_noalloc(m, g, r, v, c))
    monkeypatch.delenv("MPI_FAULT")
    assert rel_l2(got, want) <= tol(dt)


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_noalloc_against_oracle(orc, dt):
    """One small case compared with the FP64 oracle's forward directly."""
    cfg = syn.small(24, 20, 900, "spiral", seed=7)
    m, g = cfg["model"], cfg["grid"]
    r, v, c = _inputs(cfg, dt, 8)
    want = orc.forward(m, g, *(host(t) for t in (r, v, c)))
    got = host(api.mpi_forward_noalloc(m, g, r, v, c))
    assert rel_l2(got, want) <= tol(dt)

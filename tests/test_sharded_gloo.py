"""Host logic of the sample-sharded solve, on CPU: the sample partition, the
all-reduce callables (two gloo processes; threads of one process), and the
sharded CG they serve, with a stand-in operator (a seeded dense matrix whose
rows are indexed by channel and sample, as the forward operator's are).

The stand-in CG takes the steps the library's sharded solve takes: b0 is the
sum over ranks of A_r^T s_r; each step's q is the sum over ranks of
A_r^T A_r p plus nu p; all other CG arithmetic is replicated."""
import os
import socket
import threading

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2505_22797_gb300 import sharded


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("T", [0, 1, 7, 100, 65536, 1048577])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_sample_shard_partition(T, world):
    spans = [sharded.sample_shard(T, k, world) for k in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == T
    for (a0, a1), (b0, _) in zip(spans, spans[1:]):
        assert a1 == b0  # contiguous, disjoint
    sizes = [t1 - t0 for t0, t1 in spans]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == T


def test_sample_shard_rejects_bad_requests():
    for args in ((10, 2, 2), (10, -1, 2), (10, 0, 0), (-1, 0, 1)):
        with pytest.raises(ValueError):
            sharded.sample_shard(*args)


def _stand_in(n_ch=2, T=37, nx=5, ny=4, seed=3):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n_ch, T, ny * nx))
    s = rng.normal(size=(n_ch, T))
    return A, s


def _cg_sharded(A_r, s_r, nu, n_cg, reduce):
    """CG on (A^T A + nu I) x = A^T s with the rows of this rank only."""
    n = A_r.shape[-1]
    M = A_r.reshape(-1, n)

    def red(vec):
        t = torch.as_tensor(vec.copy(), dtype=torch.float64)
        reduce(t)
        return t.numpy()
    b = red(M.T @ s_r.reshape(-1))
    x = np.zeros(n)
    r = b - (red(M.T @ (M @ x)) + nu * x)
    p = r.copy()
    rr = r @ r
    for _ in range(n_cg):
        q = red(M.T @ (M @ p)) + nu * p
        alpha = rr / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, s = _stand_in()
        t0, t1 = sharded.sample_shard(A.shape[1], rank, world)
        x = _cg_sharded(A[:, t0:t1], s[:, t0:t1], 0.3, 6, sharded.dist_allreduce())
        # the reduced vector is the same on every rank
        t = torch.full((4,), float(rank + 1), dtype=torch.float64)
        sharded.dist_allreduce()(t)
        out.put((rank, (t0, t1), x, t.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_sharded_cg():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, span, x, t = q.get(timeout=300)
        res[rank] = (span, x, t)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    A, s = _stand_in()
    want = _cg_sharded(A, s, 0.3, 6, lambda t: None)
    assert res[0][0] == (0, 19) and res[1][0] == (19, 37)
    assert np.array_equal(res[0][1], res[1][1])  # identical on both ranks
    assert np.linalg.norm(res[0][1] - want) <= 1e-12 * np.linalg.norm(want)
    assert np.all(res[0][2] == 3.0) and np.all(res[1][2] == 3.0)


def test_thread_allreduce_fixed_order():
    world = 3
    ar = sharded.ThreadAllreduce(world, timeout=30)
    vals = [torch.tensor([0.1 * (k + 1), 1e16 * (-1) ** k, 1.0]) .double() for k in range(world)]
    want = np.zeros(3)
    for k in range(world):  # the same order the threads use
        want += vals[k].numpy()
    got = [None] * world

    def run(k):
        t = vals[k].clone()
        ar.for_rank(k)(t)
        got[k] = t.numpy()
    th = [threading.Thread(target=run, args=(k,)) for k in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=60)
    for k in range(world):
        assert np.array_equal(got[k], want)


def test_thread_sharded_cg_matches_unsharded():
    """Three thread ranks with the host-staged all-reduce run the stand-in
    sharded CG to the unsharded result."""
    world = 3
    A, s = _stand_in(T=50)
    ar = sharded.ThreadAllreduce(world, timeout=30)
    got = [None] * world

    def run(k):
        t0, t1 = sharded.sample_shard(A.shape[1], k, world)
        got[k] = _cg_sharded(A[:, t0:t1], s[:, t0:t1], 0.2, 5, ar.for_rank(k))
    th = [threading.Thread(target=run, args=(k,)) for k in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=60)
    want = _cg_sharded(A, s, 0.2, 5, lambda t: None)
    for k in range(world):
        assert np.array_equal(got[k], got[0])
        assert np.linalg.norm(got[k] - want) <= 1e-12 * np.linalg.norm(want)

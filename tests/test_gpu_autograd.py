"""Hand-written backward of the forward operator (dL/dc through A^T, dL/dbeta
through the beta-derivative kernel) behind torch.autograd, checked against
central finite differences of the GPU FP64 forward and against the oracle
gradient, for L = 1/2 ||A(c; beta) - s||^2."""
import numpy as np
import pytest
import torch

from paper_2505_22797_gb300 import synthetic as syn
from paper_2505_22797_gb300.autograd import mpi_forward_autograd
from tests.gpu_util import dev, host, rel_l2, rounded, tol

pytestmark = pytest.mark.gpu


def _loss(c, beta, m, g, r, v, s):
    return 0.5 * torch.sum((mpi_forward_autograd(c, beta, m, g, r, v) - s) ** 2)


def _setup(cfg, dt, orc=None):
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (rounded(cfg[k], dt) for k in ("r", "v", "c"))
    rng = np.random.default_rng(17)
    s = rounded(rng.normal(size=(2, r.shape[0])) * 0.1, dt)
    return m, g, r, v, c, s


def test_gradients_central_differences_fp64():
    """h = 1e-6 beta central difference of L in beta; directional central
    difference in c; both on the FP64 GPU forward."""
    dt = torch.float64
    cfg = syn.small(40, 36, 3000, "spiral", seed=12)
    m, g, r, v, c, s = _setup(cfg, dt)
    R, V, S = dev(r, dt), dev(v, dt), dev(s, dt)
    C = dev(c, dt).requires_grad_(True)
    beta = torch.tensor(m["beta"], dtype=dt, device="cuda", requires_grad=True)
    L = _loss(C, beta, m, g, R, V, S)
    L.backward()
    h = 1e-6 * m["beta"]
    with torch.no_grad():
        Lp = _loss(C, beta + h, m, g, R, V, S)
        Lm = _loss(C, beta - h, m, g, R, V, S)
        fd_beta = float((Lp - Lm) / (2 * h))
        d = torch.as_tensor(np.random.default_rng(3).normal(size=c.shape), dtype=dt, device="cuda")
        eps = 1e-4
        fd_c = float((_loss(C + eps * d, beta, m, g, R, V, S) - _loss(C - eps * d, beta, m, g, R, V, S))
                     / (2 * eps))
    assert abs(float(beta.grad) - fd_beta) <= 1e-6 * abs(fd_beta)
    assert abs(float(torch.sum(C.grad * d)) - fd_c) <= 1e-8 * abs(fd_c)


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_gradients_vs_oracle_small(orc, dt):
    cfg = syn.small(33, 29, 2500, "lissajous", seed=5)
    m, g, r, v, c, s = _setup(cfg, dt)
    C = dev(c, dt).requires_grad_(True)
    beta = torch.tensor(m["beta"], dtype=dt, device="cuda", requires_grad=True)
    _loss(C, beta, m, g, dev(r, dt), dev(v, dt), dev(s, dt)).backward()
    resid = orc.forward(m, g, r, v, c) - s
    want_c = orc.adjoint(m, g, r, v, resid)
    want_b = orc.dbeta(m, g, r, v, c, resid)
    assert rel_l2(host(C.grad), want_c) <= tol(dt)
    assert abs(float(beta.grad) - want_b) <= tol(dt) * abs(want_b)


def test_gradients_256_full_size(orc):
    """The 256x256 / 262144-sample workload (FP32 forward, FP64 reduction for
    dL/dbeta): dL/dbeta against the oracle's full sum; dL/dc on 64 seeded
    voxels (A^T of the oracle residual, one voxel at a time)."""
    dt = torch.float32
    cfg = syn.config("c4")
    m, g, r, v, c, s = _setup(cfg, dt)
    C = dev(c, dt).requires_grad_(True)
    beta = torch.tensor(m["beta"], dtype=torch.float64, device="cuda", requires_grad=True)
    _loss(C, beta, m, g, dev(r, dt), dev(v, dt), dev(s, dt)).backward()
    resid = orc.forward(m, g, r, v, c) - s
    want_b = orc.dbeta(m, g, r, v, c, resid)
    err_b = abs(float(beta.grad) - want_b) / abs(want_b)
    vox = np.random.default_rng(21).choice(256 * 256, 64, replace=False)
    err_c = rel_l2(host(C.grad).reshape(-1)[vox], orc.adjoint(m, g, r, v, resid, sel=vox))
    print(f"256x256 gradients: dbeta rel err {err_b:.2e}, dc rel-L2 (64 voxels) {err_c:.2e}")
    assert err_b <= tol(dt)
    assert err_c <= tol(dt)

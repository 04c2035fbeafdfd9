"""GPU parity of the transfer-function correction (Eq. core:formula:conva ->
Eq. core:formula; Sec. 3.2) against the FP64 oracle: lengths that take every
radix of the Stockham FFT and lengths that need Bluestein's algorithm, with
and without SNR thresholding, in place, and at the benchmark's full length."""
import numpy as np
import pytest
import torch

from paper_2505_22797_gb300 import api
from paper_2505_22797_gb300 import synthetic as syn
from tests.gpu_util import dev, host, rel_l2, rounded, tol

pytestmark = pytest.mark.gpu
DTYPES = [torch.float32, torch.float64]
LENGTHS = [1, 2, 7, 64, 254, 1632, 4096, 30030, 131, 9973, 65536]


def _inputs(T, n_ch=2, seed=0):
    rng = np.random.default_rng(seed + T)
    t = np.arange(T)
    s_model = np.stack([np.sin(2 * np.pi * (3 + k) * t / max(T, 1)) + 0.3 * rng.normal(size=T)
                        for k in range(n_ch)])
    a_hat = syn.transfer_function(T, n_ch, f_hp=(3.0, 4.0, 2.0)[:n_ch], f_lp=(900.0, 700.0, 500.0)[:n_ch],
                                  delay=(2.5, 3.0, 1.0)[:n_ch])
    raw, snr = syn.measured_signal(s_model, a_hat, 0.01, seed + 7)
    return raw, a_hat, snr


def _dev_c(a):
    return torch.as_tensor(a, dtype=torch.complex128, device="cuda")


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("T", LENGTHS)
def test_transfer_correct(orc, dt, T):
    raw, a_hat, snr = _inputs(T)
    raw = rounded(raw, dt)
    theta = [0.04, 0.01]
    want = orc.transfer_correct(raw, a_hat, snr, theta)
    got = api.mpi_transfer_correct(dev(raw, dt), _dev_c(a_hat), dev(snr, torch.float64), theta)
    assert rel_l2(host(got), want) <= tol(dt)
    want0 = orc.transfer_correct(raw, a_hat)
    got0 = api.mpi_transfer_correct(dev(raw, dt), _dev_c(a_hat))
    assert rel_l2(host(got0), want0) <= tol(dt)


def test_transfer_correct_in_place_three_channels(orc):
    dt = torch.float64
    raw, a_hat, snr = _inputs(1000, n_ch=3, seed=3)
    x = dev(raw, dt)
    api.mpi_transfer_correct(x, _dev_c(a_hat), dev(snr, torch.float64), [0.1, 0.0, 1.0], out=x)
    assert rel_l2(host(x), orc.transfer_correct(raw, a_hat, snr, [0.1, 0.0, 1.0])) <= tol(dt)


def test_transfer_correct_full_workload(orc):
    """The 128 x 128 spiral workload's signal (T = 65 536, two channels)
    through the synthetic chain, FP32, every output compared."""
    dt = torch.float32
    cfg = syn.config("c2")
    m, g = cfg["model"], cfg["grid"]
    r, v, c = (dev(cfg[k], dt) for k in ("r", "v", "c"))
    s_model = host(api.mpi_forward(m, g, r, v, c))
    a_hat = syn.transfer_function(s_model.shape[1])
    raw, snr = syn.measured_signal(s_model, a_hat, 0.01, 5)
    raw = rounded(raw, dt)
    want = orc.transfer_correct(raw, a_hat, snr, [0.04, 0.01])
    got = api.mpi_transfer_correct(dev(raw, dt), _dev_c(a_hat), dev(snr, torch.float64), [0.04, 0.01])
    assert rel_l2(host(got), want) <= tol(dt)


def test_transfer_correct_bad_arguments():
    x = torch.zeros((2, 16), dtype=torch.float32, device="cuda")
    a = torch.ones((2, 9), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        api.mpi_transfer_correct(x, a[:, :8].contiguous())
    with pytest.raises(ValueError):
        api.mpi_transfer_correct(x, a, torch.zeros((2, 9), dtype=torch.float64, device="cuda"), None)
    with pytest.raises(api.MPIError):
        api.mpi_transfer_correct(torch.zeros((9, 4), dtype=torch.float32, device="cuda"),
                                 torch.ones((9, 3), dtype=torch.complex128, device="cuda"))

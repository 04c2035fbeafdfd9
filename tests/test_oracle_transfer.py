"""Pins for the oracle's transfer-function correction (Eq. core:formula:conva
-> Eq. core:formula; Sec. 3.2): it undoes a circular time convolution built
by brute force from an impulse response, leaves an undistorted tone where it
should, and drops exactly the bins below the SNR threshold, all checked with
direct O(T^2) DFT sums rather than the FFT the oracle uses."""
import numpy as np
import pytest


def _dft(x):
    T = x.shape[-1]
    n = np.arange(T)
    return np.exp(-2j * np.pi * np.outer(np.arange(T // 2 + 1), n) / T) @ x


def _circ_conv(x, a):
    T = x.size
    return np.array([sum(x[m] * a[(n - m) % T] for m in range(T)) for n in range(T)])


@pytest.mark.parametrize("T", [1, 2, 7, 16, 51])
def test_undoes_circular_convolution(orc, T):
    rng = np.random.default_rng(T)
    s_true = rng.normal(size=(2, T))
    a = np.zeros((2, T))
    a[0, 0] = 1.0
    a[0, 1 % T] += 0.4
    a[1] = np.exp(-np.arange(T) / 3.0)
    a_hat = np.stack([_dft(a[k]) for k in range(2)])
    assert np.all(np.abs(a_hat) > 1e-3)
    s_raw = np.stack([_circ_conv(s_true[k], a[k]) for k in range(2)])
    got = orc.transfer_correct(s_raw, a_hat)
    assert np.allclose(got, s_true, rtol=1e-11, atol=1e-11)


def test_tone_with_gain_and_phase(orc):
    """A cosine at bin f0 passed through a chain with gain g and phase phi
    comes out as g cos(.. + phi); the correction restores the tone."""
    T, f0 = 64, 5
    n = np.arange(T)
    a_hat = np.ones((1, T // 2 + 1), dtype=complex) * 0.5
    a_hat[0, f0] = 0.3 * np.exp(0.7j)
    raw = 0.3 * np.cos(2 * np.pi * f0 * n / T + 0.7 + 0.2)
    got = orc.transfer_correct(raw[None], a_hat)[0]
    assert np.allclose(got, np.cos(2 * np.pi * f0 * n / T + 0.2), atol=1e-13)


def test_snr_threshold_drops_exactly_the_low_bins(orc):
    T = 40
    rng = np.random.default_rng(1)
    s = rng.normal(size=(2, T))
    a_hat = (0.5 + rng.uniform(size=(2, T // 2 + 1))) * np.exp(1j * rng.uniform(0, 6, size=(2, T // 2 + 1)))
    a_hat[:, 0] = a_hat[:, 0].real
    a_hat[:, -1] = a_hat[:, -1].real
    snr = rng.uniform(0, 0.1, size=(2, T // 2 + 1))
    theta = [0.04, 0.01]
    a_hat[1, 3] = 0.0  # a vanishing bin is dropped as well
    got = orc.transfer_correct(s, a_hat, snr, theta)
    for k in range(2):
        G = _dft(got[k])
        S = _dft(s[k])
        keep = (snr[k] >= theta[k]) & (np.abs(a_hat[k]) > 0)
        assert np.allclose(G[~keep], 0.0, atol=1e-12)
        assert np.allclose(G[keep], S[keep] / a_hat[k][keep], rtol=1e-11, atol=1e-12)

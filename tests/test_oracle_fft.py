"""Pins of the oracle's own FFT: brute-force DFT and an independent library."""
import numpy as np
import pytest

from oracle import fft as F


def brute_dft3(x, sign=-1):
    """O(N^6) triple sum X[k] = sum_x x[x] exp(sign 2 pi i k.x / N)."""
    n0, n1, n2 = x.shape
    out = np.zeros(x.shape, complex)
    idx = np.indices(x.shape).reshape(3, -1)
    xs = x.reshape(-1)
    for k in np.ndindex(*x.shape):
        ph = k[0] * idx[0] / n0 + k[1] * idx[1] / n1 + k[2] * idx[2] / n2
        out[k] = np.sum(xs * np.exp(sign * 2j * np.pi * ph))
    return out


@pytest.mark.parametrize("n", [8, 6, 12])
def test_fft3_matches_brute_force(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    ref = brute_dft3(x)
    assert np.max(np.abs(F.fft3(x) - ref)) <= 1e-13 * np.max(np.abs(ref)) * n
    inv = brute_dft3(ref, sign=+1) / n ** 3
    assert np.max(np.abs(F.ifft3(ref) - inv)) <= 1e-13 * n


def test_non_cubic_axes_and_primes():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((5, 7, 4))
    assert np.allclose(F.fft3(x), brute_dft3(x), atol=1e-12)


@pytest.mark.parametrize("n", [32, 48, 64, 96])
def test_fft3_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n, n))
    ref = np.fft.fftn(x)
    assert np.max(np.abs(F.fft3(x) - ref)) <= 5e-14 * np.max(np.abs(ref))
    assert np.max(np.abs(F.ifft3_real(ref) - x)) <= 1e-13


def test_roundtrip_512_axis():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, 512))
    X = F.fft_axis(x, 1)
    assert np.allclose(X, np.fft.fft(x, axis=1), atol=1e-11)
    assert np.allclose(F.fft_axis(X, 1, inverse=True).real, x, atol=1e-13)

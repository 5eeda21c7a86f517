"""Pins of the oracle's own FFT against the O(N^2) definition and numpy.fft."""
import numpy as np
import pytest

from oracle import fft


def brute_dft(x, axis):
    n = x.shape[axis]
    k = np.arange(n)
    M = np.exp(-2j * np.pi * np.outer(k, k) / n)
    return np.moveaxis(np.tensordot(M, np.moveaxis(x, axis, 0), axes=(1, 0)), 0, axis)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 16, 18, 30, 64])
def test_fft_matches_definition(n):
    x = np.random.default_rng(n).standard_normal((3, n)) + 1j * np.random.default_rng(n + 1).standard_normal((3, n))
    got = fft.fft_axis(x, 1)
    want = brute_dft(x, 1)
    assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))


def test_fftn_matches_numpy_3d():
    x = np.random.default_rng(7).standard_normal((8, 12, 16))
    assert np.allclose(fft.fftn(x), np.fft.fftn(x), rtol=0, atol=1e-11)
    X = fft.fftn(x)
    assert np.allclose(fft.ifftn_real(X), x, rtol=0, atol=1e-13)


def test_single_mode_is_delta_and_parseval():
    n = (8, 16, 32)
    z, y, x = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    f = np.cos(2 * np.pi * (3 * x / 32 + 2 * y / 16 + 1 * z / 8))
    F = fft.fftn(f)
    N = f.size
    peaks = np.argwhere(np.abs(F) > 1e-8)
    assert sorted(map(tuple, peaks)) == sorted([(1, 2, 3), (7, 14, 29)])
    assert np.allclose(np.abs(F[1, 2, 3]), N / 2)
    g = np.random.default_rng(3).standard_normal(n)
    G = fft.fftn(g)
    assert np.isclose(np.sum(g * g), np.sum(np.abs(G) ** 2) / N, rtol=1e-13)


def test_inverse_normalisation():
    X = np.zeros((4, 6), complex)
    X[0, 0] = 24.0
    assert np.allclose(fft.ifftn(X), 1.0)

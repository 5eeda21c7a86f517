"""The oracle's own discrete Fourier transform (FP64).

Definition used throughout (Sec. 3.2 takes FFT/iFFT without fixing a normalisation; the
forward transform is unnormalised and the inverse carries 1/N):

    F(x)_k = sum_j x_j exp(-2 pi i j k / N),     x_j = (1/N) sum_k F_k exp(+2 pi i j k / N).

Implementation: recursive mixed-radix decimation-in-time Cooley-Tukey along one axis,
vectorised over all the other axes.  For N = p*m (p the smallest prime factor) the input is
split into the p interleaved subsequences x[r::p]; each gets an m-point transform and

    X[k + m q] = sum_{r<p} exp(-2 pi i r (k + m q)/N) * Sub_r[k],    q = 0..p-1.

A prime length falls back to the O(N^2) definition.  Twiddle exponents are reduced mod N
before scaling so the angles stay in [0, 2 pi).
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np


def _smallest_factor(n: int) -> int:
    if n % 2 == 0:
        return 2
    f = 3
    while f * f <= n:
        if n % f == 0:
            return f
        f += 2
    return n


@lru_cache(maxsize=None)
def _roots(n: int, sign: int) -> np.ndarray:
    """exp(sign * 2 pi i e / n) for e = 0..n-1."""
    e = np.arange(n, dtype=np.float64)
    return np.exp(sign * 2j * np.pi * e / n)


def _fft_last(x: np.ndarray, sign: int) -> np.ndarray:
    n = x.shape[-1]
    if n == 1:
        return x.astype(np.complex128, copy=True)
    p = _smallest_factor(n)
    w = _roots(n, sign)
    if p == n:
        k = np.arange(n)
        dft = w[np.outer(k, k) % n]              # exact definition for a prime length
        return x.astype(np.complex128) @ dft
    m = n // p
    subs = [_fft_last(x[..., r::p], sign) for r in range(p)]
    out = np.empty(x.shape[:-1] + (n,), dtype=np.complex128)
    k = np.arange(m)
    for q in range(p):
        acc = subs[0].copy()
        for r in range(1, p):
            acc += w[(r * (k + m * q)) % n] * subs[r]
        out[..., q * m:(q + 1) * m] = acc
    return out


def fft_axis(x: np.ndarray, axis: int, inverse: bool = False) -> np.ndarray:
    """1D transform along `axis`; the inverse includes the 1/N factor."""
    y = np.moveaxis(np.asarray(x), axis, -1)
    out = _fft_last(y, +1 if inverse else -1)
    if inverse:
        out /= y.shape[-1]
    return np.moveaxis(out, -1, axis)


def fftn(x: np.ndarray) -> np.ndarray:
    """Full complex d-dimensional transform of a real or complex field."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in range(out.ndim):
        out = fft_axis(out, ax)
    return out


def ifftn(X: np.ndarray) -> np.ndarray:
    out = np.asarray(X, dtype=np.complex128)
    for ax in range(out.ndim):
        out = fft_axis(out, ax, inverse=True)
    return out


def ifftn_real(X: np.ndarray) -> np.ndarray:
    """Inverse of a Hermitian-symmetric spectrum: the real part of ifftn."""
    return ifftn(X).real


def half_spectrum(X: np.ndarray) -> np.ndarray:
    """The kx = 0..Nx/2 part of a full spectrum (x is the last axis)."""
    return X[..., : X.shape[-1] // 2 + 1]

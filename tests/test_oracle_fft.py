"""Pins for the oracle's own recursive FFT (CPU only).

The oracle's FFT is checked against things other than itself: the O(n^2)
definition of the DFT on small n, numpy's pocketfft (an unrelated library
implementation), Parseval's identity, and single-mode inputs whose transform
is known in closed form.
"""
import numpy as np
import pytest

SIZES = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 15, 16, 17, 24, 25, 27, 30, 31, 32,
         45, 48, 60, 64, 96, 97, 100, 128, 192, 243, 256]


def dft_matrix(n, sign=-1):
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


@pytest.mark.parametrize("n", SIZES)
def test_fft1d_matches_definition(oracle_mod, n):
    g = np.random.default_rng(n)
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    X = oracle_mod.fft1d(x)
    ref = dft_matrix(n) @ x
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(X - ref)) / scale < 1e-13
    Xi = oracle_mod.fft1d(x, inverse=True)
    refi = dft_matrix(n, +1) @ x
    assert np.max(np.abs(Xi - refi)) / scale < 1e-13


@pytest.mark.parametrize("n", [2, 3, 5, 64, 100, 243, 384, 512, 768, 1000, 1024])
def test_fft1d_matches_pocketfft(oracle_mod, n):
    g = np.random.default_rng(1000 + n)
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    X = oracle_mod.fft1d(x)
    ref = np.fft.fft(x)
    assert np.max(np.abs(X - ref)) / np.max(np.abs(ref)) < 1e-14
    # unnormalised inverse undoes the forward transform up to n
    back = oracle_mod.fft1d(X, inverse=True) / n
    assert np.max(np.abs(back - x)) < 1e-13


@pytest.mark.parametrize("n", [8, 12, 30, 64, 81, 125])
def test_parseval_and_single_modes(oracle_mod, n):
    g = np.random.default_rng(7 * n)
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    X = oracle_mod.fft1d(x)
    assert abs(np.sum(np.abs(X) ** 2) - n * np.sum(np.abs(x) ** 2)) < 1e-11 * n * np.sum(np.abs(x) ** 2)
    # impulse -> all ones
    d = np.zeros(n, complex)
    d[0] = 1.0
    assert np.max(np.abs(oracle_mod.fft1d(d) - 1.0)) < 1e-15
    # a pure mode e^{+2 pi i m j / n} transforms to n at bin m and 0 elsewhere
    for m in (1, n // 3, n - 1):
        mode = np.exp(2j * np.pi * m * np.arange(n) / n)
        want = np.zeros(n, complex)
        want[m] = n
        assert np.max(np.abs(oracle_mod.fft1d(mode) - want)) < 1e-12 * n


@pytest.mark.parametrize("shape", [(4, 6, 8), (5, 3, 7), (16, 12, 10), (2, 2, 2), (1, 8, 3)])
def test_fft3d_matches_pocketfft(oracle_mod, shape):
    g = np.random.default_rng(sum(shape))
    a = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    A = oracle_mod.fft3d(a)
    ref = np.fft.fftn(a)
    assert np.max(np.abs(A - ref)) / np.max(np.abs(ref)) < 1e-14
    back = oracle_mod.fft3d(A, inverse=True) / a.size
    assert np.max(np.abs(back - a)) < 1e-13

"""Pins of the oracle's transforms (Section 4: derivatives are products with the
wavenumber in Fourier space).  The radix-2 FFT is checked against the DFT
definition evaluated by brute force, closed forms and identities, and the
numpy (pocketfft) library as a special case."""
import math

import numpy as np
import pytest


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _dft_matrix(n, sign):
    j = np.arange(n)
    e = np.outer(j, j) % n  # exact angle reduction
    return np.exp(sign * 2j * math.pi * e / n)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1d_matches_bruteforce_dft(orc, n, sign):
    x = _rand(n, n + 7)
    ref = orc.dft1d(x, sign)
    got = orc.fft1d(x, sign)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got - ref).max() <= 1e-13 * scale * max(1, math.log2(n))


@pytest.mark.parametrize("n", [2, 8, 64])
def test_bruteforce_dft_is_the_definition(orc, n):
    # the brute-force routine itself against the DFT matrix product
    x = _rand(n, 3)
    assert np.allclose(orc.dft1d(x, -1), _dft_matrix(n, -1) @ x, rtol=0, atol=1e-12 * n)


@pytest.mark.parametrize("nx,ny", [(2, 2), (4, 8), (16, 16), (32, 8), (32, 32)])
def test_fft2d_matches_bruteforce(orc, nx, ny):
    a = _rand((ny, nx), nx * 100 + ny)
    ref = _dft_matrix(ny, -1) @ a @ _dft_matrix(nx, -1).T  # sum over y and x
    got = orc.fft2d(a)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max() * 10


def test_fft2d_inverse_normalisation_and_round_trip(orc):
    a = _rand((32, 64), 5)
    back = orc.ifft2d(orc.fft2d(a))
    assert np.abs(back - a).max() <= 1e-14 * 20
    ref = (_dft_matrix(32, 1) @ a @ _dft_matrix(64, 1).T) / (32 * 64)
    assert np.abs(orc.ifft2d(a) - ref).max() <= 1e-15 * 50


def test_delta_maps_to_constant(orc):
    a = np.zeros((16, 16), complex)
    a[0, 0] = 1.0
    assert np.abs(orc.fft2d(a) - 1.0).max() <= 1e-15


def test_single_mode_maps_to_scaled_delta(orc):
    n = 32
    j = np.arange(n)
    mx, my = 5, 29
    a = np.exp(2j * math.pi * (np.outer(j * my, np.ones(n)) + np.outer(np.ones(n), j * mx)) / n)
    h = orc.fft2d(a)
    expect = np.zeros((n, n), complex)
    expect[my, mx] = n * n
    assert np.abs(h - expect).max() <= 1e-11


def test_parseval(orc):
    a = _rand((64, 32), 11)
    h = orc.fft2d(a)
    lhs = np.sum(np.abs(a) ** 2)
    rhs = np.sum(np.abs(h) ** 2) / a.size
    assert abs(lhs - rhs) <= 1e-13 * lhs


def test_matches_numpy_library(orc):
    a = _rand((128, 256), 13)
    assert np.abs(orc.fft2d(a) - np.fft.fft2(a)).max() <= 1e-12 * np.abs(a).sum() ** 0.5
    x = _rand(1024, 17)
    assert np.abs(orc.fft1d(x) - np.fft.fft(x)).max() <= 1e-11


def test_wavenumbers_order_and_nyquist(orc):
    k = orc.wavenumbers(8, 2 * math.pi)
    assert list(k) == [0, 1, 2, 3, -4, -3, -2, -1]
    k = orc.wavenumbers(4, 10 * math.pi)
    assert np.allclose(k, np.array([0, 1, -2, -1]) * 0.2)


def test_rejects_non_power_of_two(orc):
    with pytest.raises(ValueError):
        orc.fft1d(np.ones(6))
    with pytest.raises(ValueError):
        orc.fft2d(np.ones((4, 12)))


def test_planted_sign_error_is_caught(orc):
    # a transform with the wrong exponent sign fails the brute-force pin
    x = _rand(16, 1)
    assert np.abs(orc.fft1d(x, +1) - orc.dft1d(x, -1)).max() > 1e-3

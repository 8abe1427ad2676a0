"""Parity of the hand-written 2D FFT (row pass + column pass, the transform of
every step, Section 4) against the oracle's radix-2 FFT, through pss_fft2d."""
import math

import numpy as np
import pytest

from gpu_util import EPS, check

pytestmark = pytest.mark.gpu


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


SHAPES = [(16, 16, 1), (32, 64, 3), (64, 16, 2), (128, 128, 1), (256, 512, 1), (1024, 1024, 1),
          (2048, 16, 1), (16, 2048, 1), (4096, 32, 1), (32, 4096, 1), (8192, 16, 1), (16, 8192, 1)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("nx,ny,batch", SHAPES)
@pytest.mark.parametrize("direction", [-1, 1])
def test_fft2d_matches_oracle(lib, orc, cuda_device, precision, nx, ny, batch, direction):
    import torch
    a = _rand((batch, ny, nx), nx * 7 + ny + batch)
    cdt = torch.complex64 if precision == "fp32" else torch.complex128
    t = torch.tensor(a, dtype=cdt, device=cuda_device)
    lib.pss_fft2d(t.data_ptr(), nx, ny, batch, lib.PSS_FP32 if precision == "fp32" else lib.PSS_FP64,
                  direction, torch.cuda.current_stream().cuda_stream)
    got = t.cpu().numpy()
    ref = np.stack([(orc.fft2d(x) if direction < 0 else orc.ifft2d(x)) for x in a])
    # error bound of a radix-r FFT grows like eps * log2(size)
    tol = 4 * EPS[precision] * math.log2(nx * ny)
    check(got, ref, tol)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fft2d_round_trip_and_single_mode(lib, orc, cuda_device, precision):
    import torch
    nx, ny = 256, 64
    cdt = torch.complex64 if precision == "fp32" else torch.complex128
    j = np.arange
    mode = np.exp(2j * math.pi * (np.outer(j(ny) * 5, np.ones(nx)) / ny + np.outer(np.ones(ny), j(nx) * 200) / nx))
    t = torch.tensor(mode[None], dtype=cdt, device=cuda_device)
    prec = lib.PSS_FP32 if precision == "fp32" else lib.PSS_FP64
    s = torch.cuda.current_stream().cuda_stream
    lib.pss_fft2d(t.data_ptr(), nx, ny, 1, prec, -1, s)
    h = t.cpu().numpy()[0]
    expect = np.zeros((ny, nx), complex)
    expect[5, 200] = nx * ny
    # zero outputs collect rounding from all nx*ny terms of magnitude 1
    assert np.abs(h - expect).max() <= 64 * EPS[precision] * math.log2(nx * ny) * nx * ny
    lib.pss_fft2d(t.data_ptr(), nx, ny, 1, prec, +1, s)
    check(t.cpu().numpy()[0], mode, 8 * EPS[precision] * math.log2(nx * ny))


def test_fft2d_rejects_bad_sizes(lib, cuda_device):
    with pytest.raises(lib.PssError):
        lib.pss_fft2d(0, 64, 64, 1, lib.PSS_FP32, -1)
    import torch
    t = torch.zeros(64 * 48, dtype=torch.complex64, device=cuda_device)
    with pytest.raises(lib.PssError):
        lib.pss_fft2d(t.data_ptr(), 64, 48, 1, lib.PSS_FP32, -1)

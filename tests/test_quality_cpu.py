"""The image-quality measures bench.py reports for the interpolation / classification
variants (PSNR in dB, SSIM with an 11-tap Gaussian window), checked on closed cases."""
import math

import numpy as np

import bench


def test_identical_images():
    a = np.random.default_rng(0).uniform(0, 1, (40, 50, 4))
    psnr, ssim = bench.image_quality(a, a)
    assert psnr == math.inf and abs(ssim - 1.0) < 1e-12


def test_psnr_of_a_constant_offset():
    a = np.random.default_rng(1).uniform(0.2, 0.8, (30, 30, 4))
    psnr, _ = bench.image_quality(a + 0.01, a)  # MSE = 1e-4 -> 40 dB
    assert abs(psnr - 40.0) < 1e-9


def test_ssim_drops_with_noise_and_is_symmetric():
    rng = np.random.default_rng(2)
    a = rng.uniform(0, 1, (48, 48, 4))
    b = np.clip(a + rng.normal(0, 0.1, a.shape), 0, 1)
    _, s_ab = bench.image_quality(b, a)
    _, s_ba = bench.image_quality(a, b)
    assert 0.0 < s_ab < 0.99 and abs(s_ab - s_ba) < 1e-12

"""Host-side helpers of the benchmark: SSIM of the profile sweep, the clock-sample summary,
the lost-block count."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_2205_11226_gb300 import synth  # noqa: E402


def test_ssim_identity_and_degradation():
    f = synth.make_frame(96, 64, 3)
    assert abs(bench.ssim(f, f) - 1.0) < 1e-12
    rng = np.random.default_rng(0)
    g = np.clip(f + rng.normal(0, 8, f.shape), 0, 255).astype(np.uint8)
    h = np.clip(f + rng.normal(0, 24, f.shape), 0, 255).astype(np.uint8)
    assert 0.0 < bench.ssim(f, h) < bench.ssim(f, g) < 1.0
    # symmetric in its arguments
    assert abs(bench.ssim(f, g) - bench.ssim(g, f)) < 1e-12


def test_ssim_of_constant_images_is_the_luminance_term():
    # SSIM (Wang, Bovik, Sheikh, Simoncelli 2004) with K1 = 0.01, K2 = 0.03, L = 255: on two
    # constant images every local variance and covariance is 0, so each pixel's index is
    # (2 a b + C1) / (a^2 + b^2 + C1), C1 = (0.01 * 255)^2 = 6.5025
    a, b = 100.0, 120.0
    fa = np.full((40, 56), a, np.uint8)
    fb = np.full((40, 56), b, np.uint8)
    c1 = 6.5025
    expected = (2 * a * b + c1) / (a * a + b * b + c1)  # 24006.5025 / 24406.5025
    assert abs(bench.ssim(fa, fb) - expected) < 1e-12
    assert abs(expected - 0.983610925) < 1e-9  # 1 - 400 / 24406.5025


def test_ssim_of_an_intensity_shift_keeps_contrast_and_structure():
    # b = a + 30 (no clipping): local variances and the covariance are equal, so the
    # contrast-structure factor (2 s_ab + C2) / (s_a^2 + s_b^2 + C2) is exactly 1 and the index
    # is the luminance term of the two local means, mu_b = mu_a + 30
    from scipy.ndimage import gaussian_filter
    f = synth.make_frame(64, 48, 5).astype(np.float64)
    f = np.clip(f, 0, 200)
    g = f + 30.0
    mu = gaussian_filter(f, 1.5)
    c1 = 6.5025
    lum = (2 * mu * (mu + 30.0) + c1) / (mu * mu + (mu + 30.0) ** 2 + c1)
    assert abs(bench.ssim(f.astype(np.uint8), g.astype(np.uint8)) - float(lum.mean())) < 1e-9


def test_clock_summary_reads_nvidia_smi_samples(tmp_path):
    # lines as `nvidia-smi --format=csv,noheader,nounits` writes them: index, SM clock, max
    # SM clock, power, active reasons mask, then the four reason columns
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "0, 2070, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, [N/A], 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "garbage\n")
    cs = bench.ClockSampler(0)
    cs.path = str(path)
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    assert not path.exists()  # the sample file is removed once read
    cs.path = str(tmp_path / "absent.csv")
    assert cs.summary() is None


def test_lost_blocks_counts_block_and_pixel_masks():
    f = synth.make_frame(64, 48, 1)
    m = np.zeros((3, 4), np.uint8)
    m[0, 1] = m[2, 3] = 1
    assert bench.lost_blocks(f, m) == 2
    px = synth.lost_pixel_mask(m, 64, 48)
    px[20, 5] = 1  # one more block, (1, 0), holds a lost pixel
    assert bench.lost_blocks(f, px) == 3


def test_packed_views_layout():
    # the bench's arenas: every array at a 256-byte aligned offset, the views holding the data
    import torch
    arrays = [np.arange(35, dtype=np.uint8).reshape(5, 7), np.full((3, 4), 9, np.uint8),
              np.arange(600, dtype=np.uint16).astype(np.uint8).reshape(20, 30)]
    n = bench.packed_size(arrays)
    assert n == 512 + 600
    buf = torch.zeros(n, dtype=torch.uint8)
    views = bench.packed_views(arrays, buf)
    for v, a in zip(views, arrays):
        assert v.data_ptr() % 256 == buf.data_ptr() % 256
        v.numpy()[...] = a
    for v, a in zip(bench.packed_views(arrays, buf), arrays):
        assert np.array_equal(v.numpy(), a)

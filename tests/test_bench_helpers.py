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

"""Host-side helpers of the benchmark: SSIM of the profile sweep."""
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

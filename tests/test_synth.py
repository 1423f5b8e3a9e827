"""The seeded input generators: deterministic, and shaped like the paper's workloads."""
import numpy as np

from paper_2205_11226_gb300 import synth


def test_frames_deterministic_and_8bit():
    a = synth.make_frame(64, 48, 3)
    b = synth.make_frame(64, 48, 3)
    assert a.dtype == np.uint8 and a.shape == (48, 64)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.make_frame(64, 48, 4))
    t = synth.make_frame(64, 48, 3, fine_texture=True)
    assert t.shape == a.shape and not np.array_equal(a, t)


def test_loss_patterns():
    cb = synth.loss_checkerboard(512, 512)
    assert cb.shape == (32, 32) and cb.sum() == 256
    ys, xs = np.nonzero(cb)
    assert (ys % 2 == 1).all() and (xs % 2 == 1).all()
    runs = synth.loss_runs(1920, 1080, 7, 0.20)
    assert runs.shape == (68, 120)
    assert 0.20 <= runs.mean() < 0.24
    iso = synth.loss_isolated(352, 288, 1, 30)
    assert iso.sum() == 30
    for y, x in zip(*np.nonzero(iso)):
        assert iso[max(0, y - 1):y + 2, max(0, x - 1):x + 2].sum() == 1
    mx = synth.loss_mixed(1280, 720, 5, 0.05, 0.30)
    assert 0.04 <= mx.mean() <= 0.31


def test_batch_shapes():
    frames, masks = synth.workload_batch(0, sizes=[(352, 288)] * 2 + [(64, 32)])
    assert [f.shape for f in frames] == [(288, 352), (288, 352), (32, 64)]
    assert [m.shape for m in masks] == [(18, 22), (18, 22), (2, 4)]
    req = synth.stream_requests(0, n=100)
    t = np.array([r[0] for r in req])
    assert (np.diff(t) > 0).all() and len(req) == 100

"""GPU parity for arbitrarily shaped loss (per-pixel masks) against the FP64 oracle.

  - a per-pixel mask that loses whole blocks reproduces the block path bit for bit;
  - small frames with ellipses and strokes: teacher-forced per step and free-running, FP32
    and FP16 mixed, every received pixel unchanged;
  - the 1920x1080 frame with 10 % of its pixels lost in shapes, as the benchmark runs it;
  - a batch mixing block-mask and per-pixel-mask frames equals the frames concealed alone;
  - the single-frame entry skmmse_conceal_px equals the batch path."""
import numpy as np
import pytest

from paper_2205_11226_gb300 import skmmse, synth

from parity import PSNR_TOL, assembled_psnr_delta, check_free, compare, run_forced

pytestmark = pytest.mark.gpu

TOL = {skmmse.FP32: 1e-3, skmmse.MIXED_FP16: 0.5}


def _check(f, px, p, ctx):
    gpu, orc = run_forced(f, px, p, ctx)
    rep = compare(f, px, gpu, orc, p, forced=True, tol=TOL[p.precision])
    assert rep["compared"] + rep["flips"] == rep["patches"], rep
    assert rep["flips"] <= max(2, rep["patches"] // 200), rep
    assert assembled_psnr_delta(f, px, gpu, orc) <= PSNR_TOL
    # free-running, within bounds derived from the oracle's own sensitivity to per-step
    # errors of the size just measured
    _, _, _, g2, _ = check_free(f, px, p, ctx, rep["max_err"])
    lost = px.astype(bool)
    assert np.array_equal(g2["out"][~lost], f[~lost])
    return rep


@pytest.mark.parametrize("precision", [skmmse.FP32, skmmse.MIXED_FP16])
def test_whole_block_pixel_mask_is_the_block_path(gpu_ctx, precision):
    f = synth.make_frame(256, 160, 21, fine_texture=True)
    m = synth.loss_runs(256, 160, 22, 0.3)
    p = skmmse.params("efficient", precision=precision)
    a = skmmse.conceal_numpy(f, m, p, trace=True, ctx=gpu_ctx)
    b = skmmse.conceal_numpy(f, None, p, px_lost=synth.lost_pixel_mask(m, 256, 160), trace=True,
                             ctx=gpu_ctx)
    assert np.array_equal(a["out"], b["out"])
    assert np.array_equal(a["out_f32"], b["out_f32"])
    assert a["trace"].tobytes() == b["trace"].tobytes()


@pytest.mark.parametrize("precision", [skmmse.FP32, skmmse.MIXED_FP16])
@pytest.mark.parametrize("profile,seed", [("efficient", 1), ("excellent", 2), ("express", 3)])
def test_shapes_small(gpu_ctx, precision, profile, seed):
    f = synth.make_frame(256, 160, seed, fine_texture=True)
    px = synth.loss_shapes(256, 160, seed + 100, 0.12)
    _check(f, px, skmmse.params(profile, precision=precision), gpu_ctx)


@pytest.mark.parametrize("precision", [skmmse.FP32, skmmse.MIXED_FP16])
def test_shapes_received_only_support(gpu_ctx, precision):
    f = synth.make_frame(192, 128, 8, fine_texture=True)
    px = synth.loss_shapes(192, 128, 9, 0.12)
    _check(f, px, skmmse.params("efficient", precision=precision, concealed_is_support=0), gpu_ctx)


def test_single_lost_pixels(gpu_ctx):
    # scattered single pixels: every patch filled has three received pixels
    f = synth.make_frame(128, 128, 5, fine_texture=True)
    px = np.zeros((128, 128), np.uint8)
    rng = np.random.default_rng(6)
    px[rng.integers(0, 128, 60), rng.integers(0, 128, 60)] = 1
    _check(f, px, skmmse.params("excellent"), gpu_ctx)


@pytest.mark.parametrize("precision", [skmmse.FP32, skmmse.MIXED_FP16])
def test_shapes_1080p_full(gpu_ctx, precision):
    f, px = synth.workload_shapes_1080p(0)
    assert f.shape == (1080, 1920) and px.mean() >= 0.10
    _check(f, px, skmmse.params("efficient", precision=precision), gpu_ctx)


def test_mixed_batch_and_single_entry(gpu_ctx):
    import torch
    frames, masks = [], []
    for i, (w, h) in enumerate([(352, 288), (200, 120), (352, 288), (128, 96)]):
        frames.append(synth.make_frame(w, h, 60 + i, fine_texture=True))
        masks.append(synth.loss_shapes(w, h, 70 + i, 0.1) if i % 2 == 0
                     else synth.loss_mixed(w, h, 80 + i, 0.1, 0.3))
    p = skmmse.params("efficient", precision=skmmse.MIXED_FP16)
    fd = [torch.from_numpy(f).cuda() for f in frames]
    md = [torch.from_numpy(m).cuda() for m in masks]
    of = [torch.zeros(f.shape, dtype=torch.float32, device="cuda") for f in frames]
    outs, st = gpu_ctx.conceal_batch(fd, md, p, outs_f32=of, stats=True)
    torch.cuda.synchronize()
    assert st["error"] == 0
    assert st["n_lost_mbs"] == sum(int(synth.blocks_of(m).sum()) if m.shape == f.shape else int(m.sum())
                                   for f, m in zip(frames, masks))
    for i, (f, m) in enumerate(zip(frames, masks)):
        px = m.shape == f.shape
        kw = {"px_lost": md[i]} if px else {}
        o1, o1f, _ = gpu_ctx.conceal(fd[i], None if px else md[i], p, out_f32=True, **kw)
        torch.cuda.synchronize()
        assert np.array_equal(o1.cpu().numpy(), outs[i].cpu().numpy())
        assert np.array_equal(o1f.cpu().numpy(), of[i].cpu().numpy())


def test_px_mask_argument_checks(gpu_ctx):
    import torch
    f = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    m = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    px = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    lib, p = skmmse.load(), skmmse.params()
    out = torch.empty_like(f)
    import ctypes
    for mb_ptr, px_ptr, pitch, want in ((m.data_ptr(), px.data_ptr(), 64, 1),  # both masks
                                        (None, None, 64, 1),                    # none
                                        (None, px.data_ptr(), 32, 2)):          # pitch < width
        d = (skmmse.Frame * 1)()
        d[0].frame, d[0].width, d[0].height, d[0].pitch = f.data_ptr(), 64, 64, 64
        d[0].mb_lost, d[0].px_lost, d[0].px_pitch = mb_ptr, px_ptr, pitch
        d[0].out, d[0].out_pitch = out.data_ptr(), 64
        rc = lib.skmmse_conceal_batch(gpu_ctx._h, d, 1, ctypes.byref(p), None,
                                      skmmse._stream_handle(None))
        assert rc == want

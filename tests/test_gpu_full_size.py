"""GPU parity at the full sizes of the benchmarked workloads.

  - 512x512 checkerboard (256 isolated blocks) and one 1920x1080 frame with runs of 4-20
    lost blocks to 20 % (fine texture): teacher-forced per step and free-running against
    the FP64 oracle, as the smaller parity cases.
  - the 64-frame batch of mixed sizes in one skmmse_conceal_batch call, as the benchmark
    launches it, in FP32 and mixed precision: one frame of each size is compared with the
    oracle, and its batch output must equal the same frame concealed alone.

The 0.01 dB PSNR bound applies to the frame assembled from the per-step estimates of a
teacher-forced pair (every step had the oracle's inputs: the arithmetic of the path
alone).  Free-running, the method itself is sensitive: rounding only the written-back
estimates of the FP64 oracle to binary32 already changes decisions on some frames of the
batch, and a near-tie decision that goes the other way changes that patch by up to tens of
gray levels and travels down the dependency chain.  The free-running bounds (drift before
a block's first decision difference, the oracle margins of those differences, the PSNR
delta) are therefore derived from the oracle's own behaviour under per-step errors of the
size each path is held to teacher-forced (parity.py, envelope; tests/golden/sensitivity.json),
at all three precisions and every size."""
import numpy as np
import pytest

from paper_2205_11226_gb300 import skmmse, synth

from parity import PSNR_TOL, assembled_psnr_delta, check_free, compare, run_forced

pytestmark = pytest.mark.gpu

TOL_MIXED = 0.5


def _forced_and_free(f, m, p, ctx, tol):
    gpu, orc = run_forced(f, m, p, ctx)
    rep = compare(f, m, gpu, orc, p, forced=True, tol=tol)
    assert rep["compared"] + rep["flips"] == rep["patches"], rep
    assert rep["flips"] <= max(2, rep["patches"] // 200), rep
    assert assembled_psnr_delta(f, m, gpu, orc) <= PSNR_TOL
    _, s, _, _, _ = check_free(f, m, p, ctx, rep["max_err"])
    return rep, s


@pytest.mark.parametrize("precision,tol", [(skmmse.FP32, 1e-3), (skmmse.MIXED_BF16, TOL_MIXED)])
def test_checkerboard_512_full(gpu_ctx, precision, tol):
    f, m = synth.workload_checkerboard(0)
    assert f.shape == (512, 512) and int(m.sum()) == 256
    _forced_and_free(f, m, skmmse.params("efficient", precision=precision), gpu_ctx, tol)


@pytest.mark.parametrize("precision,tol", [(skmmse.FP32, 1e-3), (skmmse.MIXED_BF16, TOL_MIXED),
                                           (skmmse.MIXED_FP16, TOL_MIXED)])
def test_slice_1080p_full(gpu_ctx, precision, tol):
    f, m = synth.workload_slice_1080p(0)
    assert f.shape == (1080, 1920)
    _forced_and_free(f, m, skmmse.params("efficient", precision=precision), gpu_ctx, tol)


@pytest.mark.parametrize("precision", [skmmse.FP32, skmmse.MIXED_BF16, skmmse.MIXED_FP16])
def test_batch64_sampled_against_oracle(gpu_ctx, precision):
    import torch
    frames, masks = synth.workload_batch(0)
    assert len(frames) == 64
    p = skmmse.params("efficient", precision=precision)
    fd = [torch.from_numpy(f).cuda() for f in frames]
    md = [torch.from_numpy(m).cuda() for m in masks]
    of = [torch.zeros(f.shape, dtype=torch.float32, device="cuda") for f in frames]
    outs, st = gpu_ctx.conceal_batch(fd, md, p, outs_f32=of, stats=True)
    torch.cuda.synchronize()
    assert st["error"] == 0 and st["n_lost_mbs"] == sum(int(m.sum()) for m in masks)
    tol = 1e-3 if precision == skmmse.FP32 else TOL_MIXED
    for i in (0, 24, 48):  # 352x288, 1280x720, 1920x1080
        f, m = frames[i], masks[i]
        gf, of_ = run_forced(f, m, p, gpu_ctx)
        rep = compare(f, m, gf, of_, p, forced=True, tol=tol)
        assert rep["flips"] <= max(2, rep["patches"] // 200), rep
        assert assembled_psnr_delta(f, m, gf, of_) <= PSNR_TOL, i
        # free-running (all three precisions), bounds from the oracle's own sensitivity
        _, _, _, gpu, _ = check_free(f, m, p, gpu_ctx, rep["max_err"])
        # the batch computes exactly what a call for this frame alone computes
        assert np.array_equal(of[i].cpu().numpy(), gpu["out_f32"])
        assert np.array_equal(outs[i].cpu().numpy(), gpu["out"])


@pytest.fixture(scope="module")
def batch_oracle():
    """The FP64 oracle's outputs for all 64 batch frames (efficient profile)."""
    import os
    from parity import matching_oracle_params, oracle_conceal
    frames, masks = synth.workload_batch(0)
    p = skmmse.params("efficient")
    outs = [oracle_conceal(f, m, matching_oracle_params(p), threads=os.cpu_count() or 8)["out"]
            for f, m in zip(frames, masks)]
    return frames, masks, outs


def _pooled_psnr(frames, masks, outs):
    se, npx = 0.0, 0
    for f, m, o in zip(frames, masks, outs):
        lost = synth.lost_pixel_mask(m, f.shape[1], f.shape[0])
        q = np.clip(np.rint(np.asarray(o, np.float64)), 0, 255)
        se += float(np.sum((q[lost] - f[lost]) ** 2))
        npx += int(lost.sum())
    return 10.0 * np.log10(255.0 ** 2 * npx / se)


def _batch_gpu(ctx, frames, masks, p):
    import torch
    fd = [torch.from_numpy(f).cuda() for f in frames]
    md = [torch.from_numpy(m).cuda() for m in masks]
    outs, st = ctx.conceal_batch(fd, md, p, stats=True)
    torch.cuda.synchronize()
    assert st["error"] == 0
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("precision", [skmmse.FP32, skmmse.MIXED_FP16, skmmse.MIXED_BF16])
def test_batch64_pooled_psnr_against_oracle(gpu_ctx, batch_oracle, precision):
    """The metric's form: PSNR over all lost pixels of the 64 frames.  Free-running against
    the FP64 oracle, the pooled delta is held to twice what the oracle itself shows at the
    path's per-step error (the envelope of tests/golden/sensitivity.json), never above the
    metric's 0.01 dB where the oracle's own delta at that error is below half of it; the
    mixed paths against the FP32 path within 0.01 dB (FP16, the benchmark's mode) and the
    BF16 envelope."""
    from parity import PSNR_TOL, SENS_MULT, envelope
    frames, masks, orc = batch_oracle
    env = envelope(precision)
    p = skmmse.params("efficient", precision=precision)
    gpu = _batch_gpu(gpu_ctx, frames, masks, p)
    d = abs(_pooled_psnr(frames, masks, gpu) - _pooled_psnr(frames, masks, orc))
    assert d <= max(PSNR_TOL, SENS_MULT * env["pooled_dpsnr_db_batch"]), (d, env["pooled_dpsnr_db_batch"])
    if precision != skmmse.FP32:
        g32 = _batch_gpu(gpu_ctx, frames, masks, skmmse.params("efficient", precision=skmmse.FP32))
        dm = abs(_pooled_psnr(frames, masks, gpu) - _pooled_psnr(frames, masks, g32))
        bound = PSNR_TOL if precision == skmmse.MIXED_FP16 else max(PSNR_TOL, SENS_MULT * env["pooled_dpsnr_db_batch"])
        assert dm <= bound, (dm, bound)

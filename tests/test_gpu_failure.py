"""Failure detection without a GPU fault, and rerun determinism.

  - A bounded device wait that runs out is reported, not hung: with the test hook
    SKMMSE_FLAG_SHORT_WAITS a CTA that finds no ready block gives up after 64 polls.  On a
    frame with dependency chains idle CTAs give up while others work; the call still
    conceals every block, returns SKMMSE_ERR_TIMEOUT from the device error word, and the
    context stays usable.
  - Every block's arithmetic runs in a fixed order inside one CTA, whatever the order in
    which CTAs claim blocks, so reruns are bit-identical."""
import numpy as np
import pytest

from paper_2205_11226_gb300 import skmmse, synth

pytestmark = pytest.mark.gpu


def _dev(f, m):
    import torch
    return torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda()


def test_idle_timeout_is_reported_and_the_context_stays_usable(gpu_ctx):
    import torch
    f = synth.make_frame(256, 160, 8, fine_texture=True)
    m = synth.loss_runs(256, 160, 3, 0.25)  # runs of lost blocks: dependency chains
    fd, md = _dev(f, m)
    ref = skmmse.conceal_numpy(f, m, skmmse.params("efficient"), ctx=skmmse.Context())
    out = torch.empty_like(fd)
    short = skmmse.params("efficient", flags=skmmse.FLAG_SHORT_WAITS)
    with pytest.raises(skmmse.SkmmseError) as e:
        gpu_ctx.conceal(fd, md, short, out=out, stats=True)
    assert e.value.status == 6  # SKMMSE_ERR_TIMEOUT
    torch.cuda.synchronize()
    # the CTAs still working concealed every block
    assert np.array_equal(out.cpu().numpy(), ref["out"])
    # the same context, normal bounds: no error, the same frame
    out2, _, st = gpu_ctx.conceal(fd, md, skmmse.params("efficient"), out=torch.empty_like(fd), stats=True)
    assert st["error"] == 0
    assert np.array_equal(out2.cpu().numpy(), ref["out"])


@pytest.mark.parametrize("precision", [skmmse.FP32, skmmse.MIXED_FP16])
def test_reruns_are_bit_identical(gpu_ctx, precision):
    import torch
    frames, masks = synth.workload_batch(3, sizes=[(352, 288), (1280, 720), (200, 120)])
    p = skmmse.params("efficient", precision=precision)
    fd = [torch.from_numpy(f).cuda() for f in frames]
    md = [torch.from_numpy(m).cuda() for m in masks]
    res = []
    for rep in range(3):
        of = [torch.zeros(f.shape, dtype=torch.float32, device="cuda") for f in frames]
        if rep == 2:  # a different persistent grid: a different claim order
            gpu_ctx.set_ctas_per_sm(1)
        gpu_ctx.conceal_batch(fd, md, p, outs_f32=of)
        torch.cuda.synchronize()
        res.append([o.cpu().numpy() for o in of])
    gpu_ctx.set_ctas_per_sm(0)
    for a, b, c in zip(*res):
        assert np.array_equal(a, b) and np.array_equal(a, c)

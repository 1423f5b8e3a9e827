"""The batch call recorded as a CUDA graph replays to the same outputs as the direct call,
on new frame contents; every launch configuration the autotuner chooses among (CTAs per SM,
candidates per tensor-core tile) gives the same outputs bit for bit; the autotuner keeps its
choice per shape class."""
import numpy as np
import pytest

from paper_2205_11226_gb300 import skmmse, synth

pytestmark = pytest.mark.gpu


def _batch(seed):
    return synth.workload_batch(seed, sizes=[(352, 288), (200, 120), (128, 96)])


def test_graph_replay_matches_direct_call(gpu_ctx):
    import torch
    p = skmmse.params("efficient")
    frames, masks = _batch(3)
    fd = [torch.from_numpy(f).cuda() for f in frames]
    md = [torch.from_numpy(m).cuda() for m in masks]
    og = [torch.empty_like(f) for f in fd]
    g = gpu_ctx.graph(fd, md, p, outs=og)
    for seed in (3, 4):  # replay on the captured inputs, then on new frame contents
        fr, ms = _batch(seed)
        for d, h in zip(fd, fr):
            d.copy_(torch.from_numpy(h))
        for d, h in zip(md, ms):
            d.copy_(torch.from_numpy(h))
        g.launch()
        st = g.read_stats()
        ref = [skmmse.conceal_numpy(f, m, p, ctx=gpu_ctx)["out"] for f, m in zip(fr, ms)]
        for a, b in zip(og, ref):
            assert np.array_equal(a.cpu().numpy(), b)
        assert st["status"] == 0 and st["n_lost_mbs"] == sum(int(m.sum()) for m in ms)
    g.close()


@pytest.mark.parametrize("precision", [skmmse.MIXED_FP16, skmmse.MIXED_BF16, skmmse.FP32])
def test_every_launch_configuration_gives_identical_results(gpu_ctx, precision):
    import torch
    # the excellent profile sends most patches through HQL, where the tiles act
    p = skmmse.params("excellent", precision=precision)
    frames, masks = _batch(6)
    fd = [torch.from_numpy(f).cuda() for f in frames]
    md = [torch.from_numpy(m).cuda() for m in masks]
    ref = None
    for ctas in (1, 2):
        for tile_cov in (32, 64):
            for tile_dist in (64, 128):
                gpu_ctx.set_config(ctas, tile_cov, tile_dist)
                of = [torch.zeros(f.shape, dtype=torch.float32, device="cuda") for f in fd]
                _, st = gpu_ctx.conceal_batch(fd, md, p, outs_f32=of, stats=True)
                torch.cuda.synchronize()
                assert st["error"] == 0 and st["n_hql"] > 0
                got = [o.cpu().numpy() for o in of]
                if ref is None:
                    ref = got
                for a, b in zip(got, ref):
                    assert np.array_equal(a, b), (ctas, tile_cov, tile_dist)
    gpu_ctx.set_config(0, 64, 64)


def test_autotune_keeps_its_choice_per_shape_class(gpu_ctx):
    import torch
    p = skmmse.params("efficient", precision=skmmse.MIXED_FP16)
    frames, masks = _batch(5)
    fd = [torch.from_numpy(f).cuda() for f in frames]
    md = [torch.from_numpy(m).cuda() for m in masks]
    ref = [skmmse.conceal_numpy(f, m, p, ctx=gpu_ctx)["out"] for f, m in zip(frames, masks)]
    res = gpu_ctx.autotune(fd, md, p, reps=1)
    assert len(res["options"]) == 8 and all(o["ms"] > 0 for o in res["options"])
    assert res["best"]["ms"] == min(o["ms"] for o in res["options"])
    best = {k: res["best"][k] for k in ("ctas_per_sm", "tile_cov", "tile_dist")}
    assert gpu_ctx.get_config(fd, md, p) == best
    # another shape class (one frame fewer) keeps the default
    assert gpu_ctx.get_config(fd[:2], md[:2], p) == {"ctas_per_sm": 0, "tile_cov": 64, "tile_dist": 64}
    outs, _ = gpu_ctx.conceal_batch(fd, md, p)
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert np.array_equal(a.cpu().numpy(), b)

"""Serving: requests arriving while other batches run start on the next free stream, and the
launches of the two streams are resident on the device together (measured by the kernel's
global-timer interval of each launch); every result equals the result of concealing that
frame alone."""
import numpy as np
import pytest

from paper_2205_11226_gb300 import serving, skmmse

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix(gpu_ctx):
    reqs = serving.make_requests(48, seed=2, rate_hz=3000.0, pool_per_size=2)
    # small arenas: a few frames per batch, so batches are many and overlap
    loop = serving.ServeLoop(n_streams=2, arena_bytes=6 << 20, max_batch=8)
    res = loop.run(reqs, realtime=True)
    loop.close()
    assert res["requests"] == 48 and res["batches"] >= 3
    assert res["max_resident_launches"] >= 2, res   # launches resident together on the device
    assert res["mean_resident_launches"] > 1.0, res
    assert res["p99_ms"] >= res["p50_ms"] > 0
    p = skmmse.params("efficient")
    for r in reqs[::3]:
        alone = skmmse.conceal_numpy(r.frame, r.mb_lost, p, ctx=gpu_ctx)["out"]
        assert np.array_equal(r.result, alone), r.rid

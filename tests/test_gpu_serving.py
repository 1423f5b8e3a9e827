"""Serving: requests arriving while other batches run are admitted as memory frees and
overlap on the device; every result equals the result of concealing that frame alone."""
import numpy as np
import pytest

from paper_2205_11226_gb300 import serving, skmmse

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix(gpu_ctx):
    reqs = serving.make_requests(48, seed=2, rate_hz=3000.0, pool_per_size=2)
    # small budget: at most a few frames in flight, so admission really waits for memory
    loop = serving.ServeLoop(n_streams=3, budget_bytes=12 << 20, max_batch=8)
    res = loop.run(reqs, realtime=True)
    loop.close()
    assert res["requests"] == 48 and res["batches"] >= 3
    assert res["max_overlap"] >= 2, res          # batches overlapped on the device
    assert res["p99_ms"] >= res["p50_ms"] > 0
    p = skmmse.params("efficient")
    for r in reqs[::3]:
        alone = skmmse.conceal_numpy(r.frame, r.mb_lost, p, ctx=gpu_ctx)["out"]
        assert np.array_equal(r.result, alone), r.rid

"""CPU checks of the free-running parity machinery (tests/parity.py) and of the sensitivity
record it reads (tests/golden/sensitivity.json, written by make_sensitivity.py from the
oracle alone).  Oracle runs stand in for the GPU side here: no GPU is needed."""
import json
import os

import pytest

from paper_2205_11226_gb300 import build, skmmse, synth

import parity

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sensitivity.json")


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()  # (the binding's parameter presets come from the library; no GPU call)
    return skmmse.load()


@pytest.fixture(scope="module")
def record():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_record_covers_every_path_delta(record):
    env = record["envelope"]
    for precision, delta in parity.PATH_DELTA.items():
        e = env[f"{delta:g}"]
        assert e["drift"] > 0 and e["dpsnr"] >= 0 and e["pooled_dpsnr_db_batch"] >= 0
    # the batch frames, both full-size frames and the excellent-profile cases are in it
    names = set(record["workloads"])
    assert {"batch0", "batch63", "checkerboard512", "slice1080p", "checkerboard512_excellent"} <= names


def test_record_grows_with_the_perturbation(record):
    # a larger per-step error moves the outputs further: the pooled PSNR delta over the batch
    # (the least noisy statistic) at the largest delta exceeds the one at the smallest
    env = record["envelope"]
    assert env["0.1"]["pooled_dpsnr_db_batch"] > env["1e-05"]["pooled_dpsnr_db_batch"]
    assert env["0.1"]["drift"] >= env["1e-05"]["drift"]


def _pair(f, m, p, kw):
    base = parity.oracle_conceal(f, m, parity.matching_oracle_params(p), trace=True, threads=4)
    op = parity.matching_oracle_params(p)
    for k, v in kw.items():
        setattr(op, k, v)
    other = parity.as_run(parity.oracle_conceal(f, m, op, trace=True, threads=4))
    return base, other


def test_binary32_storage_passes_the_fp32_bounds():
    # the oracle storing its estimates in binary32 is a path with per-step errors far below
    # the FP32 bound: it must pass the free-running comparison with the FP32 envelope
    p = skmmse.params("efficient")
    f = synth.make_frame(256, 160, 8, fine_texture=True)
    m = synth.loss_runs(256, 160, 3, 0.25)
    base, other = _pair(f, m, p, {"store_f32": 1})
    sens = parity.envelope(skmmse.FP32)
    rep = parity.compare(f, m, other, base, p, sens=sens)
    assert rep["compared"] > 0
    s = parity.free_running_summary(f, m, other, base)
    assert abs(s["psnr_gpu"] - s["psnr_oracle"]) <= parity.free_psnr_bound(sens)


def test_a_gross_per_step_error_fails_the_fp32_bounds():
    # a planted mistake: every estimate written back up to 10 gray off (far above the FP32
    # per-step bound, and above twice the drift the oracle shows at that bound)
    p = skmmse.params("efficient")
    f = synth.make_frame(256, 160, 8, fine_texture=True)
    m = synth.loss_runs(256, 160, 3, 0.25)
    base, other = _pair(f, m, p, {"perturb": 10.0, "perturb_seed": 5})
    with pytest.raises(AssertionError):
        parity.compare(f, m, other, base, p, sens=parity.envelope(skmmse.FP32))

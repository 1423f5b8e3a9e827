"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs, element by element.  Each configuration runs

  - teacher-forced: every step of the kernel starts from exactly the oracle's inputs
    (binary32-stored oracle estimates written back), every estimate within 1e-3 gray;
  - free-running: both run independently; decisions and values agree up to the first
    decision difference of each block, within bounds derived from the oracle's own
    behaviour under per-step errors of the size the path is held to teacher-forced (twice
    its drift, flip margins and PSNR delta; never below the strict bounds).

Sizes span many candidate chunks, several work-queue entries, ragged frame edges and
dependency chains (see tests/parity.py for the comparison rules)."""
import numpy as np
import pytest

from paper_2205_11226_gb300 import skmmse, synth

from parity import check_free, compare, run_forced

pytestmark = pytest.mark.gpu

TOL_MIXED = 0.5      # gray levels per pixel, tensor-core contractions (BF16/FP16 split operands)


def check(frame, m, p, ctx, free=True, tol=None):
    gpu, orc = run_forced(frame, m, p, ctx)
    rep = compare(frame, m, gpu, orc, p, forced=True, **({"tol": tol} if tol else {}))
    assert rep["compared"] + rep["flips"] == rep["patches"], rep
    assert rep["flips"] <= max(2, rep["patches"] // 200), rep
    if free:
        rep2, s, sens, _, _ = check_free(frame, m, p, ctx, rep["max_err"])
        rep["free"] = {**s, "compared": rep2["compared"], "patches": rep2["patches"],
                       "flips": rep2["flips"], "sensitivity": sens}
    return rep, gpu, orc


@pytest.mark.parametrize("profile", ["express", "efficient", "excellent"])
def test_single_block_256(gpu_ctx, profile):
    f, m = synth.workload_single(0)
    rep, gpu, orc = check(f, m, skmmse.params(profile), gpu_ctx)
    assert gpu["stats"]["n_patches"] == 64 and gpu["stats"]["n_lost_mbs"] == 1
    assert rep["compared"] == 64


@pytest.mark.parametrize("seed", [1, 2])
def test_forced_hql_single_block(gpu_ctx, seed):
    # every patch through HQL: covariance, factorisation, beta grid, I0, alpha
    f, m = synth.workload_single(seed)
    p = skmmse.params("efficient", t_phi=-1.0, t_nu=1e30)
    rep, gpu, orc = check(f, m, p, gpu_ctx)
    assert gpu["stats"]["n_hql"] == 64


def test_forced_idl_single_block(gpu_ctx):
    f, m = synth.workload_single(3)
    p = skmmse.params("efficient", t_phi=-1.0, t_nu=1e-6)
    rep, gpu, orc = check(f, m, p, gpu_ctx)
    assert gpu["stats"]["n_idl"] == 64


@pytest.mark.parametrize("profile", ["efficient", "excellent"])
def test_checkerboard_ragged(gpu_ctx, profile):
    # 200 x 120: partial block column (8 px) and row (8 px); isolated losses
    f = synth.make_frame(200, 120, 7)
    m = synth.loss_checkerboard(200, 120)
    m[7, 12] = 1  # a partial corner block
    check(f, m, skmmse.params(profile), gpu_ctx)


def test_slice_chains(gpu_ctx):
    # consecutive losses: blocks depend on concealed neighbours (raster order)
    f = synth.make_frame(256, 160, 8, fine_texture=True)
    m = synth.loss_runs(256, 160, 3, 0.25)
    check(f, m, skmmse.params("efficient"), gpu_ctx)


def test_received_only_support(gpu_ctx):
    f = synth.make_frame(256, 160, 9)
    m = synth.loss_runs(256, 160, 4, 0.25)
    check(f, m, skmmse.params("efficient", concealed_is_support=0), gpu_ctx)


def test_constant_and_fully_lost(gpu_ctx):
    f = np.full((64, 96), 77, np.uint8)
    m = np.zeros((4, 6), np.uint8)
    m[1:3, 1:5] = 1
    g = skmmse.conceal_numpy(f, m, skmmse.params("excellent"), ctx=gpu_ctx)
    assert np.all(g["out"] == 77) and np.all(np.abs(g["out_f32"][16:48, 16:80] - 77) < 1e-5)
    f = synth.make_frame(48, 32, 2)
    m = np.ones((2, 3), np.uint8)
    g = skmmse.conceal_numpy(f, m, skmmse.params("efficient"), ctx=gpu_ctx)
    assert np.all(g["out"] == 128)
    # one row of blocks, all lost: a chain through every block of the frame (the longest
    # chain a frame can hold, the top work-queue bucket)
    f = synth.make_frame(80, 16, 3)
    m = np.ones((1, 5), np.uint8)
    g = skmmse.conceal_numpy(f, m, skmmse.params("efficient"), ctx=gpu_ctx)
    assert np.all(g["out"] == 128)


def test_batch_equals_single_calls(gpu_ctx):
    import torch
    frames, masks = synth.workload_batch(5, sizes=[(352, 288), (128, 96), (200, 120)])
    p = skmmse.params("efficient")
    alone = [skmmse.conceal_numpy(f, m, p, ctx=gpu_ctx)["out_f32"] for f, m in zip(frames, masks)]
    fd = [torch.from_numpy(f).cuda() for f in frames]
    md = [torch.from_numpy(m).cuda() for m in masks]
    of = [torch.zeros(f.shape, dtype=torch.float32, device="cuda") for f in frames]
    outs, st = gpu_ctx.conceal_batch(fd, md, p, outs_f32=of, stats=True)
    torch.cuda.synchronize()
    for a, b in zip(alone, of):
        assert np.array_equal(a, b.cpu().numpy())
    assert st["n_lost_mbs"] == sum(int(m.sum()) for m in masks)


def test_in_place_and_trace_off_identical(gpu_ctx):
    import torch
    f, m = synth.workload_checkerboard(6, 128, 128)
    p = skmmse.params("efficient")
    ref = skmmse.conceal_numpy(f, m, p, trace=True, ctx=gpu_ctx)["out"]
    fd = torch.from_numpy(f).cuda()
    md = torch.from_numpy(m).cuda()
    gpu_ctx.conceal(fd, md, p, out=fd)
    torch.cuda.synchronize()
    assert np.array_equal(fd.cpu().numpy(), ref)


def test_argument_errors(gpu_ctx):
    import torch
    f = torch.zeros((33, 32), dtype=torch.uint8, device="cuda")
    m = torch.zeros((3, 2), dtype=torch.uint8, device="cuda")
    with pytest.raises(skmmse.SkmmseError) as e:
        gpu_ctx.conceal(f, m)
    assert e.value.status == 2
    f = torch.zeros((32, 32), dtype=torch.uint8, device="cuda")
    m = torch.zeros((2, 2), dtype=torch.uint8, device="cuda")
    with pytest.raises(skmmse.SkmmseError) as e:
        gpu_ctx.conceal(f, m, skmmse.params("efficient", t_nu=0.0))
    assert e.value.status == 1
    with pytest.raises(skmmse.SkmmseError) as e:
        gpu_ctx.conceal(f, m, skmmse.params("efficient", beta_kmin=0, beta_kmax=40))
    assert e.value.status == 1
    with pytest.raises(skmmse.SkmmseError) as e:
        gpu_ctx.conceal(f, m, skmmse.params("efficient", flags=skmmse.FLAG_FORCE))
    assert e.value.status == 1
    # nothing lost: output equals input
    g = torch.randint(0, 255, (32, 32), dtype=torch.uint8, device="cuda")
    out, _, st = gpu_ctx.conceal(g, m, stats=True)
    assert torch.equal(out, g) and st["n_lost_mbs"] == 0


# ---------------------------------------------------------------------------------------
# mixed precision: HQL covariance, whitened distances and beta sums on tcgen05 tensor cores

@pytest.mark.parametrize("precision", [skmmse.MIXED_BF16, skmmse.MIXED_FP16])
@pytest.mark.parametrize("seed", [1, 2])
def test_mixed_forced_hql_single_block(gpu_ctx, precision, seed):
    f, m = synth.workload_single(seed)
    p = skmmse.params("efficient", t_phi=-1.0, t_nu=1e30, precision=precision)
    rep, gpu, orc = check(f, m, p, gpu_ctx, tol=TOL_MIXED)
    assert gpu["stats"]["n_hql"] == 64


@pytest.mark.parametrize("precision", [skmmse.MIXED_BF16, skmmse.MIXED_FP16])
def test_mixed_checkerboard_and_chains(gpu_ctx, precision):
    f = synth.make_frame(200, 120, 7)
    m = synth.loss_checkerboard(200, 120)
    check(f, m, skmmse.params("excellent", precision=precision), gpu_ctx, tol=TOL_MIXED)
    f = synth.make_frame(256, 160, 8, fine_texture=True)
    m = synth.loss_runs(256, 160, 3, 0.25)
    check(f, m, skmmse.params("efficient", precision=precision), gpu_ctx, tol=TOL_MIXED)


# ---------------------------------------------------------------------------------------
# in-loop 8-bit quantisation (SKMMSE_FLAG_QUANTIZE): estimates written back rounded.
# Teacher-forced only: free-running, an estimate within 1e-4 of a half-integer may round
# the other way and the 1-gray difference travels down the chain.

@pytest.mark.parametrize("precision,tol", [(skmmse.FP32, None), (skmmse.MIXED_FP16, TOL_MIXED)])
def test_quantize_inloop(gpu_ctx, precision, tol):
    f = synth.make_frame(256, 160, 8, fine_texture=True)
    m = synth.loss_runs(256, 160, 3, 0.25)
    p = skmmse.params("efficient", precision=precision, flags=skmmse.FLAG_QUANTIZE)
    rep, gpu, orc = check(f, m, p, gpu_ctx, free=False, tol=tol)
    assert np.array_equal(gpu["out_f32"], np.rint(gpu["out_f32"]))
    g = skmmse.conceal_numpy(f, m, p, ctx=gpu_ctx)
    assert np.array_equal(g["out_f32"], np.rint(g["out_f32"]))
    lost = synth.lost_pixel_mask(m, f.shape[1], f.shape[0])  # out_f32: concealed pixels only
    assert np.array_equal(g["out"][lost].astype(np.float32), g["out_f32"][lost])


# ---------------------------------------------------------------------------------------
# IDL distances on tensor cores (SKMMSE_FLAG_IDL_TC): the rings after the first read the
# distances of one Toeplitz-product pass over every window position

@pytest.mark.parametrize("precision", [skmmse.MIXED_FP16, skmmse.MIXED_BF16])
def test_idl_distances_on_tensor_cores(gpu_ctx, precision):
    # T_nu = 10: many patches need rings past the first, where the tensor-core distances act
    f = synth.make_frame(256, 160, 8, fine_texture=True)
    m = synth.loss_runs(256, 160, 3, 0.25)
    p = skmmse.params("efficient", t_nu=10.0, precision=precision, flags=skmmse.FLAG_IDL_TC)
    rep, gpu, orc = check(f, m, p, gpu_ctx, tol=TOL_MIXED)
    assert sum(gpu["stats"]["idl_ring_hist"][2:]) > 50, gpu["stats"]["idl_ring_hist"]
    # against the CUDA-core distances on the same inputs (teacher-forced): the same decisions
    # up to near-ties, the estimates within the mixed tolerance
    p0 = skmmse.params("efficient", t_nu=10.0, precision=precision)
    g0, _ = run_forced(f, m, p0, gpu_ctx)
    same = (gpu["trace"]["layer"] == g0["trace"]["layer"]) & (gpu["trace"]["ring"] == g0["trace"]["ring"])
    assert same.mean() > 0.99
    d = np.abs(gpu["trace"]["x"] - g0["trace"]["x"]).max(-1)[same]
    assert d.max() <= TOL_MIXED


@pytest.mark.parametrize("precision", [skmmse.MIXED_FP16, skmmse.MIXED_BF16])
def test_idl_tc_all_rings_before_hql(gpu_ctx, precision):
    # forced HQL: every step evaluates all rings (tensor-core distances for rings 2..7) and
    # then HQL, whose estimate does not depend on the IDL distances: outputs equal the
    # CUDA-core run's bit for bit
    f, m = synth.workload_single(1)
    base = dict(t_phi=-1.0, t_nu=1e30, precision=precision)
    a = skmmse.conceal_numpy(f, m, skmmse.params("efficient", flags=skmmse.FLAG_IDL_TC, **base), ctx=gpu_ctx)
    b = skmmse.conceal_numpy(f, m, skmmse.params("efficient", **base), ctx=gpu_ctx)
    assert a["stats"]["n_hql"] == 64
    assert np.array_equal(a["out_f32"], b["out_f32"])

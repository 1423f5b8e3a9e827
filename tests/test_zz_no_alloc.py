"""skmmse_conceal_noalloc: the entry point for callers that cannot allocate device memory
(code running inside a memory pool or allocator hook, or under a hard device-memory budget,
where a cudaMalloc would synchronise, fail or recurse).  It keeps its scratch in a static
device array instead of a context's allocations.  It must produce what the context entry
point produces, call after call, on the same inputs.

This file is collected last on purpose (its name), so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2205_11226_gb300 import skmmse, synth

from parity import TOL_FP32

pytestmark = pytest.mark.gpu


def _noalloc(lib, frame, mask, p, out, out_f32):
    import torch
    st = skmmse.Stats()
    H, W = frame.shape
    rc = lib.skmmse_conceal_noalloc(frame.data_ptr(), W, H, frame.stride(0), mask.data_ptr(),
                                    ctypes.byref(p), out.data_ptr(), out.stride(0),
                                    out_f32.data_ptr(), ctypes.byref(st),
                                    int(torch.cuda.current_stream().cuda_stream))
    return rc, st.as_dict()


@pytest.mark.parametrize("precision", [skmmse.FP32, skmmse.MIXED_FP16])
def test_noalloc_matches_context_entry_point_twice(gpu_lib, precision):
    """Calls in a row on one shared scratch: a frame, a larger one, then a smaller one again
    (the last call leaves entries, values and done flags of the larger frame past its own
    blocks).  Each result equals the context entry point's, bit for bit: the same kernels
    run the same arithmetic per block, whatever the number of persistent CTAs."""
    import torch
    cases = [synth.workload_checkerboard(11, 256, 192),
             (synth.make_frame(320, 240, 12, fine_texture=True), synth.loss_runs(320, 240, 13, 0.25)),
             (synth.make_frame(160, 96, 14), synth.loss_runs(160, 96, 15, 0.3))]
    p = skmmse.params("efficient", precision=precision)
    ctx = skmmse.Context()
    for f_np, m_np in cases:
        f = torch.from_numpy(f_np).cuda()
        m = torch.from_numpy(m_np).cuda()
        ref_out, ref_f32, ref_st = ctx.conceal(f, m, p, out_f32=True, stats=True)
        out = torch.empty_like(f)
        out_f32 = torch.zeros(f.shape, dtype=torch.float32, device="cuda")
        rc, st = _noalloc(gpu_lib, f, m, p, out, out_f32)
        torch.cuda.synchronize()
        assert rc == 0, skmmse.STATUS.get(rc, rc)
        assert st["n_lost_mbs"] == int(m_np.sum()) == ref_st["n_lost_mbs"]
        assert st["n_hql"] == ref_st["n_hql"] and st["n_idl"] == ref_st["n_idl"]
        lost = torch.from_numpy(synth.lost_pixel_mask(m_np, f_np.shape[1], f_np.shape[0])).cuda()
        err = (out_f32 - ref_f32)[lost].abs().max().item()
        assert err <= TOL_FP32, err
        assert torch.equal(out_f32[lost], ref_f32[lost])
        assert torch.equal(out, ref_out)
    ctx.close()


def test_noalloc_rejects_frames_beyond_its_scratch(gpu_lib):
    import torch
    f = torch.zeros((1088, 2048), dtype=torch.uint8, device="cuda")  # 128 x 68 = 8704 blocks
    m = torch.zeros((68, 128), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(f)
    out_f32 = torch.zeros(f.shape, dtype=torch.float32, device="cuda")
    rc, _ = _noalloc(gpu_lib, f, m, skmmse.params("efficient"), out, out_f32)
    assert rc == 8
    assert b"static scratch" in gpu_lib.skmmse_status_str(8)

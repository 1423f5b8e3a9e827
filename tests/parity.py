"""GPU-vs-oracle comparison used by the GPU tests and the smoke check.

The concealment chain is sequential: every patch feeds the support of later patches, and
the HQL estimate (small bandwidths beta, an ill-conditioned context covariance) amplifies
tiny input differences: rounding only the written-back estimates of the FP64 oracle to
binary32 already moves later estimates by up to ~2e-3 gray.  Two comparisons follow:

  forced (strict, per step): the oracle stores its estimates in binary32 (store_f32) and
    the kernel writes the oracle's stored estimate back after computing its own
    (SKMMSE_FLAG_FORCE), so every step of the kernel sees exactly the oracle's inputs;
    every estimate must agree within TOL_FP32.
  free-running: kernel and FP64 oracle run independently; values are compared until the
    first decision difference in a block, and summary statistics are returned.

In both, decisions (BRL/IDL/HQL, IDL ring, beta*, I0) are taken by thresholds and argmins
on floating-point values; a difference is accepted only where the oracle's own margin for
that decision is below a near-tie bound.  The fill order (availability only) and the
context sizes must always be identical.

A loss mask is either block flags [ceil(H/16), ceil(W/16)] or a per-pixel mask of the
frame's shape (arbitrarily shaped loss); every helper takes both.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2205_11226_gb300 import skmmse, synth

TOL_FP32 = 1e-3          # gray levels per pixel (FP32 path)
NEAR_TIE = {"phi": 1e-3, "nu": 1e-3, "beta": 1e-3, "i0": 1e-3}


def matching_oracle_params(p: skmmse.Params, store_f32: int = 0) -> oracle.Params:
    """Oracle parameters equal to the float32 values the kernel receives."""
    return oracle.Params(store_f32=store_f32, t_phi=float(p.t_phi), t_nu=float(p.t_nu), sigma2=float(p.sigma2),
                         ring_step=int(p.ring_step), ridge_rel=float(p.ridge_rel),
                         beta_kmin=int(p.beta_kmin), beta_kmax=int(p.beta_kmax),
                         beta_tie_rel=float(p.beta_tie_rel),
                         concealed_is_support=int(p.concealed_is_support),
                         quantize_inloop=1 if (p.flags & skmmse.FLAG_QUANTIZE) else 0)


def loss_views(frame, mask):
    """(block flags, lost-pixel mask, per_pixel) of a block or per-pixel loss mask."""
    H, W = frame.shape
    m = np.asarray(mask) != 0
    if m.shape == (H, W):
        return synth.blocks_of(m).astype(bool), m, True
    return m, synth.lost_pixel_mask(m, W, H), False


def patches_to_fill(lostpx, by, bx):
    """Patches of block (by, bx) holding a lost pixel (all in-frame ones for a lost block)."""
    sub = lostpx[by * 16:by * 16 + 16, bx * 16:bx * 16 + 16]
    return sum(1 for a in range(0, sub.shape[0], 2) for b in range(0, sub.shape[1], 2)
               if sub[a:a + 2, b:b + 2].any())


def oracle_conceal(frame, mask, op, **kw):
    blocks, lostpx, px = loss_views(frame, mask)
    if px:
        return oracle.conceal(frame, None, op, px_lost=lostpx, **kw)
    return oracle.conceal(frame, mask, op, **kw)


def gpu_conceal(frame, mask, p, **kw):
    blocks, lostpx, px = loss_views(frame, mask)
    if px:
        return skmmse.conceal_numpy(frame, None, p, px_lost=lostpx, **kw)
    return skmmse.conceal_numpy(frame, mask, p, **kw)


def compare(frame, mb_lost, gpu, orc, p: skmmse.Params, tol=TOL_FP32, forced=False, near_tie=1.0):
    """gpu/orc: dicts with 'out_f32'/'out' arrays and 'trace'.  Returns a report dict;
    raises AssertionError on a genuine mismatch (or, free-running, an error above tol
    before the first decision difference of a block).  near_tie scales the near-tie
    bounds (free-running mixed precision drifts further from the oracle's inputs)."""
    H, W = frame.shape
    mb_lost, lostpx, _ = loss_views(frame, mb_lost)
    mbh, mbw = mb_lost.shape
    lost = [(y, x) for y in range(mbh) for x in range(mbw) if mb_lost[y, x]]
    gtr, otr = gpu["trace"], orc["trace"]
    tainted = set()
    rep = {"patches": 0, "compared": 0, "flips": 0, "flip_kinds": {}, "tainted_blocks": 0,
           "max_err": 0.0, "blocks_compared": 0}
    for rank, (by, bx) in enumerate(lost):
        b = by * mbw + bx
        if p.concealed_is_support:
            deps = [(by + dy) * mbw + bx + dx for dy, dx in ((-1, -1), (-1, 0), (-1, 1), (0, -1))
                    if 0 <= by + dy and 0 <= bx + dx < mbw and mb_lost[by + dy, bx + dx]]
            if any(d in tainted for d in deps):
                tainted.add(b)
                continue
        npatch = patches_to_fill(lostpx, by, bx)
        rep["patches"] += npatch
        flipped = False
        for s in range(npatch):
            g, o = gtr[rank, s], otr[rank, s]
            assert int(g["mb"]) == b and int(o["mb"]) == b
            assert int(g["patch"]) == int(o["patch"]), (b, s, "fill order")
            assert int(g["ny"]) == int(o["ny"]), (b, s, "context size")
            kind = None
            if int(g["layer"]) != int(o["layer"]):
                pair = {int(g["layer"]), int(o["layer"])}
                assert pair <= {oracle.BRL, oracle.IDL, oracle.HQL}, (b, s, "mask-only decision", pair)
                kind = "phi" if oracle.BRL in pair else "nu"
            elif int(g["layer"]) == oracle.IDL and int(g["ring"]) != int(o["ring"]):
                kind = "nu"
            elif int(g["layer"]) == oracle.HQL:
                n0 = int(o["n0"])
                if int(g["beta_idx"]) != int(o["beta_idx"]):
                    kind = "beta"
                elif int(g["n0"]) != n0 or not np.array_equal(g["i0"][:n0].astype(np.int64),
                                                                o["i0"][:n0].astype(np.int64)):
                    kind = "i0"
            if kind is not None:
                margin = {"phi": o["margin_phi"], "nu": o["margin_nu"], "beta": o["margin_beta"],
                          "i0": o["margin_i0"]}[kind]
                assert margin <= NEAR_TIE[kind] * near_tie, (
                    f"block {b} step {s}: {kind} decision differs with oracle margin {margin:.3g} "
                    f"(gpu layer {int(g['layer'])} ring {int(g['ring'])} beta {int(g['beta_idx'])}, "
                    f"oracle layer {int(o['layer'])} ring {int(o['ring'])} beta {int(o['beta_idx'])})")
                rep["flips"] += 1
                rep["flip_kinds"][kind] = rep["flip_kinds"].get(kind, 0) + 1
                if forced:
                    continue  # the next step starts again from identical inputs
                tainted.add(b)
                flipped = True
                break
            err = float(np.max(np.abs(g["x"].astype(np.float64) - o["x"])))
            assert err <= tol, (f"block {b} step {s} layer {int(o['layer'])}: |gpu - oracle| = {err:.3g}"
                                f" gpu {g['x']} oracle {o['x']}")
            rep["max_err"] = max(rep["max_err"], err)
            rep["compared"] += 1
        if not flipped and not forced:
            ys, xs = slice(by * 16, min(H, by * 16 + 16)), slice(bx * 16, min(W, bx * 16 + 16))
            e = np.max(np.abs(gpu["out_f32"][ys, xs].astype(np.float64) - orc["out"][ys, xs]))
            assert e <= tol, (b, e)
            ro = np.clip(np.rint(orc["out"][ys, xs]), 0, 255)
            ok = (gpu["out"][ys, xs] == ro) | (np.abs(orc["out"][ys, xs] - np.floor(orc["out"][ys, xs]) - 0.5) < tol)
            assert ok.all(), (b, "rounded output")
            rep["blocks_compared"] += 1
    rep["tainted_blocks"] = len(tainted)
    # received pixels untouched
    recv = ~lostpx
    assert np.array_equal(gpu["out"][recv], frame[recv])
    return rep


def run_pair(frame, mb_lost, p: skmmse.Params, ctx=None, threads=8):
    """Free-running pair: kernel and FP64 oracle independently."""
    gpu = gpu_conceal(frame, mb_lost, p, trace=True, ctx=ctx)
    orc = oracle_conceal(frame, mb_lost, matching_oracle_params(p), trace=True, threads=threads)
    return gpu, orc


def run_forced(frame, mb_lost, p: skmmse.Params, ctx=None, threads=8):
    """Teacher-forced pair: the oracle stores binary32 estimates; the kernel writes those
    back after each step, so both see identical inputs at every step."""
    orc = oracle_conceal(frame, mb_lost, matching_oracle_params(p, store_f32=1), trace=True,
                         threads=threads)
    nl = int(loss_views(frame, mb_lost)[0].sum())
    gpu = gpu_conceal(frame, mb_lost, p, ctx=ctx, force_x=orc["trace"]["x"][:nl])
    return gpu, orc


def free_running_summary(frame, mb_lost, gpu, orc):
    """Error statistics of a free-running pair over the lost pixels."""
    lost = loss_views(frame, mb_lost)[1]
    d = np.abs(gpu["out_f32"].astype(np.float64) - orc["out"])[lost]
    ref_q = np.clip(np.rint(orc["out"]), 0, 255).astype(np.uint8)
    return {"max_err": float(d.max()) if d.size else 0.0,
            "frac_gt_1e-3": float((d > 1e-3).mean()) if d.size else 0.0,
            "mean_err": float(d.mean()) if d.size else 0.0,
            "psnr_gpu": synth.psnr(gpu["out"], frame, lost),
            "psnr_oracle": synth.psnr(ref_q, frame, lost)}


def assembled_psnr_delta(frame, mb_lost, gpu, orc):
    """|PSNR(gpu) - PSNR(oracle)| over the lost pixels of the frames assembled from the two
    sets of per-step estimates (trace x, rounded to 8 bits).  With a teacher-forced pair
    this measures the arithmetic of the path alone: every step had the oracle's inputs."""
    H, W = frame.shape
    mb_lost, lm, _ = loss_views(frame, mb_lost)
    mbh, mbw = mb_lost.shape
    lost = [(y, x) for y in range(mbh) for x in range(mbw) if mb_lost[y, x]]
    out = {}
    for name, tr in (("gpu", gpu["trace"]), ("orc", orc["trace"])):
        a = np.full((H, W), np.nan)
        for rank, (by, bx) in enumerate(lost):
            for s in range(patches_to_fill(lm, by, bx)):
                rec = tr[rank, s]
                pa, pb = int(rec["patch"]) >> 3, int(rec["patch"]) & 7
                y, x = by * 16 + 2 * pa, bx * 16 + 2 * pb
                a[y:y + 2, x:x + 2] = np.asarray(rec["x"], np.float64).reshape(2, 2)
        out[name] = np.clip(np.rint(a), 0, 255)
    return abs(synth.psnr(out["gpu"], frame, lm) - synth.psnr(out["orc"], frame, lm))

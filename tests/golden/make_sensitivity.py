"""Write tests/golden/sensitivity.json: the FP64 oracle's own free-running sensitivity,
the record the free-running parity bounds are derived from.  It calls only oracle/ and the
seeded input generator.

The fill of a lost block is a chain of dependent estimates (each reconstructed patch joins
the support, end of Sec. III), and a chain of blocks follows the raster order (reading R1).
An error made at one step moves later contexts, and with them later decisions (flatness,
the IDL ring of Eq. (18), beta* and I0 of HQL).  Here the oracle is run again with every
written-back estimate moved by up to delta (option `perturb`, seeds 1 and 2) and compared
with the unperturbed oracle, the way a path whose per-step error is at most delta compares
with it.  The deltas cover the per-step errors of the GPU paths measured teacher-forced
(FP32 up to ~5e-4 gray against its bound of 1e-3, FP16 split operands ~2.5e-3, BF16 up to
~6e-2).  Estimates stored
rounded to binary32 (option `store_f32`) are recorded as well.

Workloads (seed 0): the 64 frames of the batch, the 512x512 checkerboard and the 1920x1080
frame with runs of lost blocks in the efficient profile; the checkerboard and a 256x160
frame with runs of lost blocks (fine texture) in the excellent profile, where most patches
go through HQL.  Per variant and workload: the
largest difference before a block's first decision difference (blocks depending on a block
with a difference are left out), the largest finite oracle margin per kind at which a
decision differed, the PSNR delta over the lost pixels (8-bit outputs against the
undamaged frame), the largest 8-bit difference; over the batch the pooled PSNR delta.  The
envelope of a delta is the maximum over workloads and seeds.

    python tests/golden/make_sensitivity.py [--threads N]
"""
import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2205_11226_gb300 import synth  # noqa: E402

DELTAS = [1e-5, 1e-3, 5e-3, 1e-1]
SEEDS = [1, 2]


def decision_kind(a, o):
    """The kind of decision step record a takes differently from the oracle's o, or None."""
    la, lo = int(a["layer"]), int(o["layer"])
    if la != lo:
        return "phi" if oracle.BRL in (la, lo) else "nu"
    if lo == oracle.IDL and int(a["ring"]) != int(o["ring"]):
        return "nu"
    if lo == oracle.HQL:
        n0 = int(o["n0"])
        if int(a["beta_idx"]) != int(o["beta_idx"]):
            return "beta"
        if not np.array_equal(a["i0"][:n0], o["i0"][:n0]):
            return "i0"
    return None


def walk(frame, mb_lost, a, o):
    """Run a against the oracle run o (both oracle results with trace): the largest value
    difference before each block's first decision difference, and the differences as
    (kind, o's margin).  Blocks that depend on a block with a difference are left out."""
    H, W = frame.shape
    mbh, mbw = mb_lost.shape
    lost = [(y, x) for y in range(mbh) for x in range(mbw) if mb_lost[y, x]]
    tainted, drift, flips = set(), 0.0, []
    for rank, (by, bx) in enumerate(lost):
        b = by * mbw + bx
        deps = [(by + dy) * mbw + bx + dx for dy, dx in ((-1, -1), (-1, 0), (-1, 1), (0, -1))
                if 0 <= by + dy and 0 <= bx + dx < mbw and mb_lost[by + dy, bx + dx]]
        if any(d in tainted for d in deps):
            tainted.add(b)
            continue
        npatch = sum(1 for r in range(8) for c in range(8) if by * 16 + 2 * r < H and bx * 16 + 2 * c < W)
        flipped = False
        for s in range(npatch):
            ra, ro = a["trace"][rank, s], o["trace"][rank, s]
            kind = decision_kind(ra, ro)
            if kind is not None:
                margin = float(ro["margin_" + kind])
                flips.append((kind, margin))
                tainted.add(b)
                flipped = True
                break
        if not flipped:
            ys, xs = slice(by * 16, min(H, by * 16 + 16)), slice(bx * 16, min(W, bx * 16 + 16))
            drift = max(drift, float(np.max(np.abs(a["out"][ys, xs] - o["out"][ys, xs]))))
    return drift, flips


def run_stats(frame, mb_lost, a, o):
    H, W = frame.shape
    lost = synth.lost_pixel_mask(mb_lost, W, H)
    qa = np.clip(np.rint(a["out"]), 0, 255)
    qo = np.clip(np.rint(o["out"]), 0, 255)
    drift, flips = walk(frame, mb_lost, a, o)
    margin = {}
    for kind, mg in flips:
        if np.isfinite(mg):
            margin[kind] = max(margin.get(kind, 0.0), mg)
    return {"drift": drift, "margin": margin, "flips": len(flips),
            "dpsnr": abs(synth.psnr(qa, frame, lost) - synth.psnr(qo, frame, lost)),
            "max_u8": int(np.abs(qa - qo)[lost].max()) if lost.any() else 0,
            "se_a": float(np.sum((qa[lost] - frame[lost]) ** 2)),
            "se_o": float(np.sum((qo[lost] - frame[lost]) ** 2)), "npx": int(lost.sum())}


def pooled_dpsnr(rows):
    npx = sum(r["npx"] for r in rows)
    return abs(10 * np.log10(255.0 ** 2 * npx / sum(r["se_a"] for r in rows))
               - 10 * np.log10(255.0 ** 2 * npx / sum(r["se_o"] for r in rows)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 8)
    args = ap.parse_args()
    frames, masks = synth.workload_batch(0)
    work = [(f"batch{i}", "efficient", f, m) for i, (f, m) in enumerate(zip(frames, masks))]
    work.append(("checkerboard512", "efficient") + tuple(synth.workload_checkerboard(0)))
    work.append(("slice1080p", "efficient") + tuple(synth.workload_slice_1080p(0)))
    work.append(("checkerboard512_excellent", "excellent") + tuple(synth.workload_checkerboard(0)))
    work.append(("runs256x160_excellent", "excellent", synth.make_frame(256, 160, 8, fine_texture=True),
                 synth.loss_runs(256, 160, 3, 0.25)))
    base = {name: oracle.conceal(f, m, oracle.params(prof), trace=True, threads=args.threads)
            for name, prof, f, m in work}
    variants = [("binary32", {"store_f32": 1}, None)]
    variants += [(f"perturb {d:g} seed {s}", {"perturb": d, "perturb_seed": s}, d) for d in DELTAS for s in SEEDS]
    out = {"workloads": {name: [prof] + list(f.shape) for name, prof, f, _ in work},
           "runs": {}, "envelope": {}}
    for vname, kw, delta in variants:
        rows = {}
        for name, prof, f, m in work:
            r = oracle.conceal(f, m, oracle.params(prof, **kw), trace=True, threads=args.threads)
            rows[name] = run_stats(f, m, r, base[name])
        batch = [rows[f"batch{i}"] for i in range(len(frames))]
        summary = {"pooled_dpsnr_db_batch": pooled_dpsnr(batch),
                   "frames_with_differences_batch": int(sum(r["flips"] > 0 for r in batch)),
                   "per_workload": {k: {kk: (round(vv, 6) if isinstance(vv, float) else vv)
                                        for kk, vv in v.items() if kk not in ("se_a", "se_o", "npx")}
                                    for k, v in rows.items()}}
        out["runs"][vname] = summary
        key = "binary32" if delta is None else f"{delta:g}"
        env = out["envelope"].setdefault(key, {"drift": 0.0, "margin": {}, "dpsnr": 0.0, "max_u8": 0,
                                                "pooled_dpsnr_db_batch": 0.0})
        for v in rows.values():
            env["drift"] = max(env["drift"], v["drift"])
            env["dpsnr"] = max(env["dpsnr"], v["dpsnr"])
            env["max_u8"] = max(env["max_u8"], v["max_u8"])
            for kind, mg in v["margin"].items():
                env["margin"][kind] = max(env["margin"].get(kind, 0.0), mg)
        env["pooled_dpsnr_db_batch"] = max(env["pooled_dpsnr_db_batch"], summary["pooled_dpsnr_db_batch"])
        print(vname, {k: v for k, v in summary.items() if k != "per_workload"}, env, flush=True)
    with open(os.path.join(HERE, "sensitivity.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()

"""Pins of the FP64 oracle against what the paper and the mathematics fix, independently
of the oracle's own code: closed forms, limits of the kernel bandwidth, exact
reconstruction of signals the estimators must reproduce, invariances, brute force on
tiny inputs, and the values Table I prints."""
import os

import numpy as np
import pytest

import oracle
from paper_2205_11226_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def isolated(frame, by=7, bx=7):
    m = np.zeros(((frame.shape[0] + 15) // 16, (frame.shape[1] + 15) // 16), np.uint8)
    m[by, bx] = 1
    return m


def region_avail_first_step(frame, by=7, bx=7):
    """Availability of the 48x48 support region of an isolated lost block before any
    patch is filled (Sec. II: the 8 neighbours are support, the block itself is not)."""
    A = np.ones((48, 48), bool)
    A[16:32, 16:32] = False
    oy, ox = by * 16 - 16, bx * 16 - 16
    R = frame[oy:oy + 48, ox:ox + 48].astype(np.float64)
    return R, A


def brute_candidates(A, cfg):
    """All window positions (u, v) whose configured positions are all available."""
    out = []
    for u in range(43):
        for v in range(43):
            if all(A[u + r, v + c] for r, c in cfg):
                out.append((u, v))
    return out


# ---------------------------------------------------------------------------------------
# Table I / Sec. IV-B constants

def test_table1_profiles_golden():
    rows = {}
    for line in open(os.path.join(GOLDEN, "table1_profiles.txt")):
        line = line.split("#")[0].split()
        if line:
            rows[line[0]] = [float(v) for v in line[1:]]
    for name in ("express", "efficient", "excellent"):
        p = oracle.params(name)
        assert (p.t_phi, p.t_nu) == tuple(rows[name])
        assert p.sigma2 == rows["sigma2"][0]


# ---------------------------------------------------------------------------------------
# whole-method invariants

@pytest.mark.parametrize("mode", ["efficient", "force_idl", "force_hql"])
def test_constant_frame_conceals_to_constant(mode):
    f = np.full((64, 64), 137, np.uint8)
    m = np.zeros((4, 4), np.uint8)
    m[1, 1] = m[2, 2] = m[1, 2] = 1
    kw = {}
    if mode == "force_idl":
        kw = dict(t_phi=-1.0, t_nu=1e-300)
    elif mode == "force_hql":
        kw = dict(t_phi=-1.0, t_nu=1e300)
    r = oracle.conceal(f, m, oracle.params("efficient", **kw))
    assert np.all(np.abs(r["out"] - 137.0) < 1e-9)


def test_received_unchanged_lost_inputs_ignored():
    f, m = synth.workload_checkerboard(3, 96, 96)
    r1 = oracle.conceal(f, m)
    g = f.copy()
    lost = synth.lost_pixel_mask(m, 96, 96)
    g[lost] = np.random.default_rng(0).integers(0, 256, size=lost.sum())
    r2 = oracle.conceal(g, m)
    assert np.array_equal(r1["out"], r2["out"])
    assert np.array_equal(r1["out"][~lost], f[~lost].astype(np.float64))


def test_shift_equivariance():
    f = synth.make_frame(128, 128, 11)
    f = (30 + (f.astype(np.int32) * 170) // 255).astype(np.uint8)  # [30, 200]
    m = synth.loss_checkerboard(128, 128)
    m[2, 2] = 1  # one chained block too
    a = oracle.conceal(f, m, oracle.params("efficient"), trace=True)
    b = oracle.conceal((f + 40).astype(np.uint8), m, oracle.params("efficient"), trace=True)
    lost = synth.lost_pixel_mask(m, 128, 128)
    assert np.max(np.abs(b["out"][lost] - a["out"][lost] - 40.0)) < 1e-6
    assert np.array_equal(a["trace"]["layer"], b["trace"]["layer"])


def test_affine_equivariance_hql():
    # HQL only: Mahalanobis distances, beta and alpha are invariant to I -> s*I + c
    # (8-bit inputs: an even-valued frame f and f/2 + 60 are both exact)
    # (values kept in [64, 192] so that no estimate reaches the clipping bounds)
    f = synth.make_frame(96, 96, 5).astype(np.int32)
    f = (64 + (f * 128 // 255) // 2 * 2).astype(np.uint8)
    m = isolated(f, 2, 2)
    # The ridge's absolute 1e-6 floor does not scale, so a near-tie of I0 or beta* may
    # resolve differently; values must agree step by step up to the first such decision.
    p = oracle.params("efficient", t_phi=-1.0, t_nu=1e300)
    ta = oracle.conceal(f, m, p, trace=True)["trace"][0]
    tb = oracle.conceal((f // 2 + 60).astype(np.uint8), m, p, trace=True)["trace"][0]
    n = 0
    for a, b in zip(ta, tb):
        if a["beta_idx"] != b["beta_idx"] or not np.array_equal(a["i0"], b["i0"]):
            assert min(a["margin_i0"], a["margin_beta"]) < 1e-3
            break
        assert a["patch"] == b["patch"]
        assert np.max(np.abs(b["x"] - (0.5 * a["x"] + 60.0))) < 1e-4
        assert abs(a["alpha"] - b["alpha"]) < 1e-4
        n += 1
    assert n >= 16


def test_fully_lost_frame_fills_128():
    f = synth.make_frame(48, 48, 1)
    m = np.ones((3, 3), np.uint8)
    r = oracle.conceal(f, m, trace=True)
    assert np.all(r["out"] == 128.0)
    assert r["trace"][0, 0]["layer"] == oracle.EMPTY


def test_threads_and_sampling_are_exact():
    f, m = synth.workload_slice_1080p(2)
    f, m = f[:256, :320].copy(), m[:16, :20].copy()
    a = oracle.conceal(f, m, threads=1)["out"]
    b = oracle.conceal(f, m, threads=4)["out"]
    assert np.array_equal(a, b)
    sel = np.zeros_like(m)
    ys, xs = np.nonzero(m)
    sel[ys[-1], xs[-1]] = 1  # last lost block: needs its whole ancestor chain
    c = oracle.conceal(f, m, select=sel)["out"]
    blk = (slice(ys[-1] * 16, ys[-1] * 16 + 16), slice(xs[-1] * 16, xs[-1] * 16 + 16))
    assert np.array_equal(c[blk], a[blk])


@pytest.mark.parametrize("support", [0, 1])
def test_support_rule_r1(support):
    # R1: block A = (3,3) is concealed before its right neighbour B = (3,4) (raster order);
    # with concealed_is_support = 1 B reads A's concealed pixels, with 0 only received
    # ones.  Received pixels of block column 2 lie in A's 48x48 region but not in B's:
    # changing them changes A, and B only through A (support = 1).  Block column 5 lies in
    # B's region only: it never changes A, which is concealed first.
    f = synth.make_frame(128, 128, 3, fine_texture=True)
    m = np.zeros((8, 8), np.uint8)
    m[3, 3] = m[3, 4] = 1
    p = oracle.params("efficient", concealed_is_support=support)
    A, B = (slice(48, 64), slice(48, 64)), (slice(48, 64), slice(64, 80))
    base = oracle.conceal(f, m, p)["out"]
    rng = np.random.default_rng(1)
    g = f.copy()
    g[32:80, 32:48] = rng.integers(0, 256, size=(48, 16))
    a = oracle.conceal(g, m, p)["out"]
    assert np.abs(a[A] - base[A]).max() > 1.0
    assert (np.abs(a[B] - base[B]).max() > 1e-3) == (support == 1)
    g = f.copy()
    g[32:80, 80:96] = rng.integers(0, 256, size=(48, 16))
    b = oracle.conceal(g, m, p)["out"]
    assert np.array_equal(b[A], base[A])
    assert np.abs(b[B] - base[B]).max() > 1.0


def test_rejects_odd_sizes():
    with pytest.raises(ValueError):
        oracle.conceal(np.zeros((33, 32), np.uint8), np.ones((3, 2), np.uint8))


# ---------------------------------------------------------------------------------------
# fill order (Sec. II, Fig. 1(b) caption: outer border towards the centre)

def test_fill_order_starts_at_the_border():
    # R2 (count of available context pixels, ties to the lowest index): the four corners,
    # whose windows see 20 received pixels, come first; every patch is filled once; every
    # patch touches available context when it is filled; the centre patches come last.
    f = synth.make_frame(128, 128, 4)
    r = oracle.conceal(f, isolated(f, 3, 3), trace=True)
    t = r["trace"][0]
    order = list(t["patch"])
    assert sorted(order) == list(range(64))
    assert order[:4] == [0, 7, 56, 63]
    assert list(t["ny"][:4]) == [20, 20, 20, 20]
    assert (t["ny"] >= 12).all()
    ring_of = lambda p: min(p // 8, p % 8, 7 - p // 8, 7 - p % 8)
    assert ring_of(order[-1]) <= 3 and all(ring_of(p) == 0 for p in order[:4])


# ---------------------------------------------------------------------------------------
# BRL, Eq. (16): mean of the context

def test_brl_first_patch_is_context_mean():
    rng = np.random.default_rng(7)
    f = rng.integers(100, 116, size=(128, 128)).astype(np.uint8)  # phi <= 15 < 20 everywhere
    r = oracle.conceal(f, isolated(f, 3, 3), trace=True)
    R, A = region_avail_first_step(f, 3, 3)
    win = R[14:20, 14:20][A[14:20, 14:20]]  # window of patch (0,0)
    t0 = r["trace"][0, 0]
    assert t0["layer"] == oracle.BRL and t0["patch"] == 0 and t0["ny"] == 20
    assert abs(t0["x"][0] - win.mean()) < 1e-12
    assert abs(r["out"][48, 48] - win.mean()) < 1e-12


@pytest.mark.parametrize("top,layer_is_brl", [(120, True), (121, False)])
def test_brl_iff_flatness_at_most_t_phi(top, layer_is_brl):
    # Eq. (17) phi = max - min of the context; R4: BRL iff phi <= T_phi, so the integer tie
    # phi = T_phi = 20 (Efficient, Table I) is BRL and phi = 21 is not
    rng = np.random.default_rng(12)
    f = rng.integers(101, 120, size=(128, 128)).astype(np.uint8)
    f[46, 46], f[46, 47] = 100, top  # in the context of patch (0,0) of block (3,3)
    p = oracle.params("efficient")
    assert p.t_phi == 20.0
    t0 = oracle.conceal(f, isolated(f, 3, 3), p, trace=True)["trace"][0, 0]
    R, A = region_avail_first_step(f, 3, 3)
    win = R[14:20, 14:20][A[14:20, 14:20]]
    assert t0["patch"] == 0 and t0["phi"] == win.max() - win.min() == top - 100
    assert (t0["layer"] == oracle.BRL) == layer_is_brl


def test_no_candidate_falls_back_to_brl():
    # 18x16 frame: the only support of the lost block is a 2-row strip, too thin for any
    # candidate (x rows plus context rows need 4 available rows)
    f = synth.make_frame(16, 18, 9)
    m = np.array([[1], [0]], np.uint8)
    r = oracle.conceal(f, m, oracle.params("efficient", t_phi=-1.0), trace=True)
    t0 = r["trace"][0, 0]
    assert t0["layer"] == oracle.BRL_NOCAND and t0["m"] == 0
    # patch (7,1): rows 14-15, cols 2-3; context = available rows 16-17, cols 0-5
    assert t0["patch"] == 57
    assert abs(t0["x"][0] - f[16:18, 0:6].mean()) < 1e-12


# ---------------------------------------------------------------------------------------
# IDL, Eq. (15): limits of the aperture sigma^2

def periodic_frame(py=3, px=4, seed=0, size=128):
    rng = np.random.default_rng(seed)
    tile = rng.integers(20, 236, size=(py, px))
    yy, xx = np.mgrid[0:size, 0:size]
    return tile[yy % py, xx % px].astype(np.uint8)


def test_idl_sigma_to_zero_reconstructs_periodic_texture_exactly():
    # sigma^2 -> 0: only exact context matches keep weight, so a periodic texture whose
    # period fits in the first ring is reconstructed exactly, patch after patch
    f = periodic_frame()
    m = isolated(f, 3, 3)
    p = oracle.params("efficient", t_phi=-1.0, t_nu=0.5, sigma2=1e-9)
    r = oracle.conceal(f, m, p, trace=True)
    assert (r["trace"][0]["layer"] == oracle.IDL).all()
    lost = synth.lost_pixel_mask(m, 128, 128)
    assert np.array_equal(r["out"][lost], f[lost].astype(np.float64))


def test_idl_sigma_to_infinity_is_plain_candidate_mean():
    f = synth.make_frame(128, 128, 21)
    m = isolated(f, 3, 3)
    p = oracle.params("efficient", t_phi=-1.0, t_nu=0.5, sigma2=1e15)
    r = oracle.conceal(f, m, p, trace=True)
    t0 = r["trace"][0, 0]
    assert t0["layer"] == oracle.IDL and t0["ring"] == 1 and t0["patch"] == 0
    R, A = region_avail_first_step(f, 3, 3)
    cfg = [(rr, cc) for rr in range(6) for cc in range(6) if A[14 + rr, 14 + cc]]
    cfg += [(2, 2), (2, 3), (3, 2), (3, 3)]
    cands = [(u, v) for (u, v) in brute_candidates(A, cfg)
             if max(abs(u + 2 - 16), abs(v + 2 - 16)) <= 4]
    xs = np.array([[R[u + 2, v + 2], R[u + 2, v + 3], R[u + 3, v + 2], R[u + 3, v + 3]]
                   for u, v in cands])
    assert np.max(np.abs(t0["x"] - xs.mean(0))) < 1e-6


def test_nu_bounded_by_candidate_count():
    f, m = synth.workload_checkerboard(5, 160, 160)
    r = oracle.conceal(f, m, oracle.params("excellent"), trace=True)
    t = r["trace"].reshape(-1)
    sel = (t["layer"] == oracle.IDL) | (t["layer"] == oracle.HQL)
    assert sel.any()
    # nu is a sum of at most M raw weights, each <= 1 (R6: the exponent is non-positive)
    assert np.all(t["log_nu"][sel] <= np.log(np.maximum(t["m"][sel], 1)) + 1e-12)


def numpy_idl(R, A, pr, pc, p):
    """Independent NumPy statement of one IDL decision and estimate (Eqs. (15), (18),
    readings R5/R6) for the patch with top-left (pr, pc) of a 48x48 region R with
    availability A: the support grows ring by ring (Chebyshev distance of the candidate
    patch from x0 at most ring_step * k) until the sum of raw weights reaches T_nu.
    Returns (layer, rings evaluated, log nu, estimate or None, M)."""
    wr, wc = pr - 2, pc - 2
    cfg = [(r, c) for r in range(6) for c in range(6)
           if A[wr + r, wc + c] and not (r in (2, 3) and c in (2, 3))]
    ny = len(cfg)
    y0 = np.array([R[wr + r, wc + c] for r, c in cfg])
    xcfg = [(2, 2), (2, 3), (3, 2), (3, 3)]
    cands = brute_candidates(A, cfg + xcfg)
    X = np.array([[R[u + r, v + c] for r, c in xcfg] for u, v in cands])
    Y = np.array([[R[u + r, v + c] for r, c in cfg] for u, v in cands])
    D = np.array([max(abs(u + 2 - pr), abs(v + 2 - pc)) for u, v in cands])
    w = np.exp(-np.sum((Y - y0) ** 2, axis=1) / (2 * p.sigma2 * ny))
    k = 0
    while True:
        k += 1
        inner = D <= p.ring_step * k
        nu = w[inner].sum()
        if nu >= p.t_nu:
            return oracle.IDL, k, np.log(nu), w[inner] @ X[inner] / nu, len(cands)
        if inner.all():
            return oracle.HQL, k, np.log(nu), None, len(cands)


# (profile, sigma^2, frame seed) -> accepted ring (0: no ring reaches T_nu, HQL)
IDL_CASES = [("express", 10.0, 1, 1), ("efficient", 3.0, 2, 2), ("efficient", 3.0, 8, 3),
             ("excellent", 3.0, 3, 5), ("excellent", 10.0, 7, 2), ("efficient", 3.0, 4, 0),
             ("excellent", 10.0, 1, 0)]


@pytest.mark.parametrize("profile,sigma2,seed,ring", IDL_CASES)
def test_idl_first_patch_matches_numpy_brute_force(profile, sigma2, seed, ring):
    # the default aperture and a narrower one, rings 1 to 5 and the fall-through to HQL:
    # the ring partition, the 2 sigma^2 Ny normalisation and the T_nu test all show
    f = synth.make_frame(128, 128, seed, fine_texture=seed % 2 == 0)
    m = isolated(f, 3, 3)
    p = oracle.params(profile, t_phi=-1.0, sigma2=sigma2)
    t0 = oracle.conceal(f, m, p, trace=True)["trace"][0, 0]
    R, A = region_avail_first_step(f, 3, 3)
    layer, k, log_nu, x, M = numpy_idl(R, A, 16, 16, p)
    assert (layer == oracle.IDL) == (ring > 0) and (k == ring or ring == 0)
    assert t0["layer"] == layer and t0["ring"] == k and t0["m"] == M
    assert abs(t0["log_nu"] - log_nu) < 1e-9
    if x is not None:
        assert np.max(np.abs(t0["x"] - x)) < 1e-9


# ---------------------------------------------------------------------------------------
# HQL, Eq. (13)

def test_hql_reconstructs_linear_signal_exactly():
    # candidates of an exactly linear (in the pixel values) image satisfy z_j = z_0 + t_j 1;
    # then C_XY C_YY^-1 maps the context residual to the patch exactly, every leave-one-out
    # residual equals its correction (alpha* >= 1, clamped to 1) and Eq. (13) returns the
    # true patch up to the 1e-6 ridge floor.
    yy, xx = np.mgrid[0:112, 0:112]
    f = (yy + xx + 10).astype(np.uint8)
    m = isolated(f, 3, 3)
    p = oracle.params("efficient", t_phi=-1.0, t_nu=1e300, ridge_rel=0.0)
    r = oracle.conceal(f, m, p, trace=True)
    assert (r["trace"][0]["layer"] == oracle.HQL).all()
    lost = synth.lost_pixel_mask(m, 112, 112)
    assert np.max(np.abs(r["out"][lost] - f[lost])) < 1e-4
    assert np.all(r["trace"][0]["alpha"] > 1.0 - 1e-6)


def numpy_hql(R, A, pr, pc, p):
    """Independent NumPy statement of one HQL estimate (Eqs. (3)-(13), readings R5/R7)
    for the patch with top-left (pr, pc) of a 48x48 region R with availability A."""
    wr, wc = pr - 2, pc - 2
    cfg = [(r, c) for r in range(6) for c in range(6)
           if A[wr + r, wc + c] and not (r in (2, 3) and c in (2, 3))]
    y0 = np.array([R[wr + r, wc + c] for r, c in cfg])
    xcfg = [(2, 2), (2, 3), (3, 2), (3, 3)]
    cands = brute_candidates(A, cfg + xcfg)
    X = np.array([[R[u + r, v + c] for r, c in xcfg] for u, v in cands])
    Y = np.array([[R[u + r, v + c] for r, c in cfg] for u, v in cands])
    Zm = np.hstack([X, Y])
    C = np.cov(Zm, rowvar=False, bias=True)
    ny = len(cfg)
    Cyy = C[4:, 4:] + (p.ridge_rel * np.trace(C[4:, 4:]) / ny + 1e-6) * np.eye(ny)
    Cxy = C[:4, 4:]
    P = np.linalg.inv(Cyy)
    K = np.linalg.solve(Cyy, Cxy.T).T
    d = np.einsum("ij,jk,ik->i", Y - y0, P, Y - y0)
    betas = 2.0 ** (0.5 * np.arange(p.beta_kmin, p.beta_kmax + 1))
    def w_of(dd, beta):
        w = np.exp(-(dd - dd.min()) / (2 * beta))
        return w / w.sum()
    eps = np.array([np.sum((y0 - w_of(d, b) @ Y) ** 2) for b in betas])
    bi = int(np.flatnonzero(eps <= eps.min() * (1 + p.beta_tie_rel))[0])
    w = w_of(d, betas[bi])
    xt, yt = w @ X, w @ Y
    n0 = min(ny + 1, len(cands) - 1)
    I0 = np.lexsort((np.arange(len(d)), d))[:n0]
    R_, G_ = [], []
    for i in I0:
        di = np.einsum("ij,jk,ik->i", Y - Y[i], P, Y - Y[i])
        mask = np.arange(len(d)) != i
        wi = w_of(di[mask], betas[bi])
        R_.append(X[i] - wi @ X[mask])
        G_.append(K @ (Y[i] - wi @ Y[mask]))
    R_, G_ = np.array(R_), np.array(G_)
    alphas = np.linspace(-0.5, 1.5, 20001)
    epsx = [np.mean(np.sum((R_ - a * G_) ** 2, axis=1)) for a in alphas]
    a_scan = float(np.clip(alphas[int(np.argmin(epsx))], 0, 1))
    den = np.sum(G_ * G_)  # 0: every alpha minimises Eq. (11); R7 takes 0
    a_cf = float(np.clip(np.sum(R_ * G_) / den, 0, 1)) if den > 0 else 0.0
    return xt + a_cf * K @ (y0 - yt), a_cf, a_scan, bi, len(cands)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_hql_first_patch_matches_numpy_brute_force(seed):
    f = synth.make_frame(128, 128, seed)
    m = isolated(f, 3, 3)
    p = oracle.params("efficient", t_phi=-1.0, t_nu=1e300)
    r = oracle.conceal(f, m, p, trace=True)
    t0 = r["trace"][0, 0]
    R, A = region_avail_first_step(f, 3, 3)
    xhat, a_cf, a_scan, bi, M = numpy_hql(R, A, 16, 16, p)
    assert t0["layer"] == oracle.HQL and t0["m"] == M and t0["beta_idx"] == bi
    assert abs(a_cf - t0["alpha"]) < 1e-9
    assert abs(a_scan - a_cf) <= 1e-4  # the closed form is the minimiser of Eq. (11)
    assert np.max(np.abs(np.clip(xhat, 0, 255) - t0["x"])) < 1e-8


@pytest.mark.parametrize("seed", [22, 39])
def test_hql_estimate_is_clipped_to_the_pixel_range(seed):
    # R8: Eq. (13) can extrapolate past [0, 255] on a high-contrast frame (here above 255
    # for seed 22, below 0 for seed 39); the estimate and the output are clipped
    base = synth.make_frame(128, 128, seed, fine_texture=True).astype(np.int32)
    f = np.clip(base * 2 - 60, 0, 255).astype(np.uint8)
    p = oracle.params("efficient", t_phi=-1.0, t_nu=1e300)
    r = oracle.conceal(f, isolated(f, 3, 3), p, trace=True)
    t0 = r["trace"][0, 0]
    R, A = region_avail_first_step(f, 3, 3)
    xhat = numpy_hql(R, A, 16, 16, p)[0]
    assert t0["layer"] == oracle.HQL and t0["patch"] == 0
    assert xhat.max() > 255.5 or xhat.min() < -0.5
    assert np.max(np.abs(t0["x"] - np.clip(xhat, 0, 255))) < 1e-8
    assert np.array_equal(r["out"][48:50, 48:50].reshape(-1), t0["x"])


# ---------------------------------------------------------------------------------------
# In-loop 8-bit quantisation (variant of R8): estimates are written back rounded

def test_quantize_inloop_writes_back_rounded_estimates():
    # every output value is the round-half-even of the estimate the trace records for
    # that pixel, and later steps read those integers back
    f = synth.make_frame(96, 96, 31, fine_texture=True)
    m = np.zeros((6, 6), np.uint8)
    m[2, 2] = m[2, 3] = m[3, 2] = 1  # a small chain: later blocks read rounded values
    p = oracle.params("excellent", quantize_inloop=1)
    r = oracle.conceal(f, m, p, trace=True)
    out, tr = r["out"], r["trace"]
    assert np.array_equal(out, np.rint(out))
    lost = [(y, x) for y in range(6) for x in range(6) if m[y, x]]
    for rank, (by, bx) in enumerate(lost):
        for rec in tr[rank]:
            a, b = int(rec["patch"]) >> 3, int(rec["patch"]) & 7
            y, x = by * 16 + 2 * a, bx * 16 + 2 * b
            est = np.asarray(rec["x"], np.float64).reshape(2, 2)
            assert np.array_equal(out[y:y + 2, x:x + 2], np.rint(est))
    # the unrounded variant differs (the estimates are not all integers here)
    r0 = oracle.conceal(f, m, oracle.params("excellent"), trace=True)
    assert not np.array_equal(r0["out"], out)


def test_quantize_inloop_is_a_no_op_when_estimates_are_integers():
    # sigma^2 -> 0 on a periodic texture copies exact integer matches: rounding changes
    # nothing, so both variants give the same frame and the same decisions
    f = periodic_frame()
    m = isolated(f, 3, 3)
    kw = dict(t_phi=-1.0, t_nu=0.5, sigma2=1e-9)
    a = oracle.conceal(f, m, oracle.params("efficient", **kw), trace=True)
    b = oracle.conceal(f, m, oracle.params("efficient", quantize_inloop=1, **kw), trace=True)
    assert np.array_equal(a["out"], b["out"])
    assert np.array_equal(a["trace"]["layer"], b["trace"]["layer"])


# ---------------------------------------------------------------------------------------
# Arbitrarily shaped loss (R9: per-pixel mask; the paper notes the method extends to any
# loss shape)

def shapes_case(seed=0, w=128, h=96, target=0.08):
    f = synth.make_frame(w, h, seed, fine_texture=True)
    return f, synth.loss_shapes(w, h, seed + 1, target)


@pytest.mark.parametrize("profile", ["efficient", "excellent"])
def test_pixel_mask_of_whole_blocks_is_the_block_method(profile):
    # a per-pixel mask that loses whole blocks must give the block method, bit for bit
    f = synth.make_frame(160, 128, 41, fine_texture=True)
    m = synth.loss_runs(160, 128, 42, 0.3)
    a = oracle.conceal(f, m, oracle.params(profile), trace=True)
    b = oracle.conceal(f, None, oracle.params(profile), px_lost=synth.lost_pixel_mask(m, 160, 128),
                       trace=True)
    assert np.array_equal(a["out"], b["out"])
    assert a["trace"].tobytes() == b["trace"].tobytes()
    assert a["stats"] == b["stats"]


def test_shapes_received_unchanged_lost_inputs_ignored():
    f, px = shapes_case(3)
    lost = px.astype(bool)
    r1 = oracle.conceal(f, None, px_lost=px)
    assert not np.isnan(r1["out"]).any()
    assert np.array_equal(r1["out"][~lost], f[~lost].astype(np.float64))
    g = f.copy()
    g[lost] = np.random.default_rng(1).integers(0, 256, size=lost.sum())
    r2 = oracle.conceal(g, None, px_lost=px)
    assert np.array_equal(r1["out"], r2["out"])


@pytest.mark.parametrize("mode", ["efficient", "force_idl", "force_hql"])
def test_shapes_constant_frame_conceals_to_constant(mode):
    _, px = shapes_case(5, 96, 96, 0.15)
    f = np.full((96, 96), 91, np.uint8)
    kw = {"force_idl": dict(t_phi=-1.0, t_nu=1e-300), "force_hql": dict(t_phi=-1.0, t_nu=1e300)}
    r = oracle.conceal(f, None, oracle.params("efficient", **kw.get(mode, {})), px_lost=px)
    assert np.all(np.abs(r["out"] - 91.0) < 1e-9)


def test_shapes_intensity_shift_equivariance():
    f, px = shapes_case(7)
    f = (30 + (f.astype(np.int32) * 170) // 255).astype(np.uint8)  # [30, 200]
    a = oracle.conceal(f, None, px_lost=px, trace=True)
    b = oracle.conceal((f + 40).astype(np.uint8), None, px_lost=px, trace=True)
    lost = px.astype(bool)
    assert np.max(np.abs(b["out"][lost] - a["out"][lost] - 40.0)) < 1e-6
    assert np.array_equal(a["trace"]["layer"], b["trace"]["layer"])


def test_shapes_fill_exactly_the_patches_holding_a_lost_pixel():
    f, px = shapes_case(9)
    r = oracle.conceal(f, None, px_lost=px, trace=True)
    blocks = synth.blocks_of(px)
    ys, xs = np.nonzero(blocks)
    assert len(r["trace"]) == len(ys)
    for rank, (by, bx) in enumerate(zip(ys, xs)):
        sub = px[by * 16:by * 16 + 16, bx * 16:bx * 16 + 16]
        want = {a * 8 + b for a in range(8) for b in range(8)
                if sub[2 * a:2 * a + 2, 2 * b:2 * b + 2].any()}
        recs = r["trace"][rank][:len(want)]
        assert set(int(p) for p in recs["patch"]) == want
        assert all(int(m) == by * blocks.shape[1] + bx for m in recs["mb"])
        assert (r["trace"][rank][len(want):]["ny"] == 0).all()  # no further records


def single_lost_pixel(seed, y=50, x=51):
    f = synth.make_frame(128, 128, seed, fine_texture=True)
    px = np.zeros((128, 128), np.uint8)
    px[y, x] = 1
    return f, px


def test_partly_lost_patch_brl_is_mean_of_context_outside_the_patch():
    # pixel (50, 51) lies in patch (1, 1) of block (3, 3) (rows 50-51, cols 50-51); its
    # context is the 6x6 window rows 48-53, cols 48-53 less the patch: 32 received pixels;
    # the patch's three received pixels are not context and stay as they are
    f, px = single_lost_pixel(4)
    r = oracle.conceal(f, None, oracle.params("efficient", t_phi=1e9), px_lost=px, trace=True)
    t = r["trace"][0]
    assert t[0]["patch"] == 9 and t[0]["ny"] == 32 and t[0]["layer"] == oracle.BRL
    win = f[48:54, 48:54].astype(np.float64).copy()
    win[2:4, 2:4] = np.nan
    assert abs(t[0]["x"][1] - np.nanmean(win)) < 1e-12
    assert r["out"][50, 51] == t[0]["x"][1]
    for yy, xx in ((50, 50), (51, 50), (51, 51)):
        assert r["out"][yy, xx] == f[yy, xx]
    assert t[1]["ny"] == 0  # one patch only


@pytest.mark.parametrize("seed", [1, 2])
def test_single_lost_pixel_hql_matches_numpy_brute_force(seed):
    # candidates (R5 with R9): every window of the 48x48 region of block (3, 3) whose 36
    # positions avoid the one lost pixel; context: the 32 pixels around the patch
    f, px = single_lost_pixel(seed)
    p = oracle.params("efficient", t_phi=-1.0, t_nu=1e300)
    r = oracle.conceal(f, None, p, px_lost=px, trace=True)
    t0 = r["trace"][0, 0]
    R = f[32:80, 32:80].astype(np.float64)
    A = np.ones((48, 48), bool)
    A[50 - 32, 51 - 32] = False
    xhat, a_cf, a_scan, bi, M = numpy_hql(R, A, 18, 18, p)
    assert M == 43 * 43 - 36  # the windows that contain the lost pixel
    assert t0["layer"] == oracle.HQL and t0["ny"] == 32 and t0["m"] == M and t0["beta_idx"] == bi
    assert abs(a_cf - t0["alpha"]) < 1e-9
    assert np.max(np.abs(np.clip(xhat, 0, 255) - t0["x"])) < 1e-8
    assert r["out"][50, 51] == t0["x"][1]


# ------------------------------------------------------------------------------------
# Sensitivity option (test infrastructure, not the method): a seeded perturbation of
# every written-back estimate, used to measure how far the sequential fill carries a
# per-step error of a given size.

def test_splitmix64_matches_the_published_sequence():
    # SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) seeded with 1234567: the first five
    # outputs of the reference generator, whose state advances by 0x9E3779B97F4A7C15
    expected = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                4593380528125082431, 16408922859458223821]
    state = 1234567
    for v in expected:
        assert oracle.splitmix64(state) == v
        state = (state + 0x9E3779B97F4A7C15) % 2 ** 64


def test_perturb_zero_leaves_the_method_unchanged():
    f = synth.make_frame(128, 96, 21, fine_texture=True)
    m = synth.loss_runs(128, 96, 22, 0.3)
    a = oracle.conceal(f, m, oracle.params("efficient"), trace=True)
    b = oracle.conceal(f, m, oracle.params("efficient", perturb=0.0, perturb_seed=7), trace=True)
    assert np.array_equal(a["out"], b["out"])
    assert np.array_equal(a["trace"]["x"], b["trace"]["x"])


def test_perturb_moves_each_write_by_at_most_delta_around_the_constant():
    # constant frame: every estimate of every layer is the constant (the contexts hold only
    # the constant and earlier writes), so with a perturbation each write is the mean of
    # earlier values within the constant +- k*delta, moved by at most delta
    c, delta = 100.0, 0.25
    f = np.full((64, 64), int(c), np.uint8)
    m = isolated(f, 1, 1)
    r = oracle.conceal(f, m, oracle.params("efficient", perturb=delta, perturb_seed=3), trace=True)
    x = r["trace"]["x"][0]                       # 64 steps x 4 pixels, in fill order
    dev = np.abs(x - c)
    assert dev.max() <= 64 * delta and dev.max() > 0
    first = x[0] - c                             # first step: the context is all received
    assert np.all(np.abs(first) <= delta) and np.any(first != 0)
    # zero-mean draws: over 256 writes the mean deviation is far below delta
    assert abs(float(np.mean(x - c))) < 0.25 * delta
    # another seed draws other values
    r2 = oracle.conceal(f, m, oracle.params("efficient", perturb=delta, perturb_seed=4), trace=True)
    assert not np.array_equal(r2["trace"]["x"][0], x)

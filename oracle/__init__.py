"""FP64 CPU oracle for SK-MMSE spatial error concealment (arXiv 2205.11226).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers.  The product path never imports this
package, and this package imports nothing from the product path.

The arithmetic lives in ``skmmse_oracle.c`` (plain C, FP64, no vectorisation tricks);
this module compiles it with gcc and exposes it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skmmse_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libskmmse_oracle.so")
_lock = threading.Lock()
_lib = None

# layer codes of the trace
EMPTY, BRL, IDL, HQL, BRL_NOCAND = 0, 1, 2, 3, 4
LAYER_NAMES = {EMPTY: "empty", BRL: "brl", IDL: "idl", HQL: "hql", BRL_NOCAND: "brl_nocand"}


class Params(ctypes.Structure):
    _fields_ = [
        ("t_phi", ctypes.c_double),
        ("t_nu", ctypes.c_double),
        ("sigma2", ctypes.c_double),
        ("ring_step", ctypes.c_int),
        ("ridge_rel", ctypes.c_double),
        ("beta_kmin", ctypes.c_int),
        ("beta_kmax", ctypes.c_int),
        ("beta_tie_rel", ctypes.c_double),
        ("concealed_is_support", ctypes.c_int),
        ("store_f32", ctypes.c_int),
        ("quantize_inloop", ctypes.c_int),
        ("perturb", ctypes.c_double),
        ("perturb_seed", ctypes.c_uint64),
    ]


class TraceRec(ctypes.Structure):
    _fields_ = [
        ("mb", ctypes.c_int32), ("step", ctypes.c_int32), ("patch", ctypes.c_int32),
        ("layer", ctypes.c_int32), ("ny", ctypes.c_int32), ("m", ctypes.c_int32),
        ("ring", ctypes.c_int32), ("beta_idx", ctypes.c_int32), ("n0", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("phi", ctypes.c_double), ("log_nu", ctypes.c_double), ("alpha", ctypes.c_double),
        ("eps_best", ctypes.c_double), ("x", ctypes.c_double * 4),
        ("margin_phi", ctypes.c_double), ("margin_nu", ctypes.c_double),
        ("margin_beta", ctypes.c_double), ("margin_i0", ctypes.c_double),
        ("i0", ctypes.c_uint16 * 36),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("n_patches", ctypes.c_int64), ("n_empty", ctypes.c_int64), ("n_brl", ctypes.c_int64),
        ("n_idl", ctypes.c_int64), ("n_hql", ctypes.c_int64), ("n_brl_nocand", ctypes.c_int64),
        ("idl_ring_hist", ctypes.c_int64 * 16), ("idl_cand_evals", ctypes.c_int64),
        ("hql_cands", ctypes.c_int64),
    ]


# Profiles, Table I of the paper: (T_phi, T_nu)
PROFILES = {"express": (20.0, 0.01), "efficient": (20.0, 0.1), "excellent": (20.0, 100.0)}


def params(profile: str = "efficient", **kw) -> Params:
    """Oracle parameters: Table I thresholds, sigma^2 = 10 (Sec. IV-B), and the readings
    of the unstated parts (ring width, ridge, beta grid, beta tie tolerance)."""
    t_phi, t_nu = PROFILES[profile]
    p = Params(t_phi=t_phi, t_nu=t_nu, sigma2=10.0, ring_step=4, ridge_rel=1e-3,
               beta_kmin=-8, beta_kmax=16, beta_tie_rel=1e-3, concealed_is_support=1,
               store_f32=0, quantize_inloop=0, perturb=0.0, perturb_seed=0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE semantics: no fast-math, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        path = build()
        lib = ctypes.CDLL(path)
        lib.oracle_conceal.restype = ctypes.c_int
        lib.oracle_conceal.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_void_p,
            ctypes.POINTER(Stats), ctypes.c_int]
        lib.oracle_conceal_px.restype = ctypes.c_int
        lib.oracle_conceal_px.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
            ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_void_p,
            ctypes.POINTER(Stats), ctypes.c_int]
        assert lib.oracle_trace_rec_size() == ctypes.sizeof(TraceRec)
        assert lib.oracle_params_size() == ctypes.sizeof(Params)
        lib.oracle_splitmix64.restype = ctypes.c_uint64
        lib.oracle_splitmix64.argtypes = [ctypes.c_uint64]
        assert lib.oracle_stats_size() == ctypes.sizeof(Stats)
        _lib = lib
    return _lib


def splitmix64(x: int) -> int:
    """The generator behind the ``perturb`` option (SplitMix64 output of state x)."""
    return int(_load().oracle_splitmix64(ctypes.c_uint64(x & (2 ** 64 - 1))))


def trace_to_numpy(buf) -> np.ndarray:
    """View a TraceRec array as a numpy structured array."""
    dt = np.dtype([
        ("mb", "<i4"), ("step", "<i4"), ("patch", "<i4"), ("layer", "<i4"), ("ny", "<i4"),
        ("m", "<i4"), ("ring", "<i4"), ("beta_idx", "<i4"), ("n0", "<i4"), ("pad", "<i4"),
        ("phi", "<f8"), ("log_nu", "<f8"), ("alpha", "<f8"), ("eps_best", "<f8"),
        ("x", "<f8", (4,)), ("margin_phi", "<f8"), ("margin_nu", "<f8"),
        ("margin_beta", "<f8"), ("margin_i0", "<f8"), ("i0", "<u2", (36,))])
    assert dt.itemsize == ctypes.sizeof(TraceRec)
    return np.frombuffer(buf, dtype=dt)


def blocks_of(px_lost: np.ndarray) -> np.ndarray:
    """Block flags of a per-pixel loss mask: a block is worked on iff it holds a lost pixel."""
    px = np.asarray(px_lost) != 0
    H, W = px.shape
    mbh, mbw = (H + 15) // 16, (W + 15) // 16
    pad = np.zeros((mbh * 16, mbw * 16), dtype=bool)
    pad[:H, :W] = px
    return pad.reshape(mbh, 16, mbw, 16).any(axis=(1, 3)).astype(np.uint8)


def conceal(frame: np.ndarray, mb_lost: np.ndarray | None, p: Params | None = None, *,
            px_lost: np.ndarray | None = None, select: np.ndarray | None = None,
            trace: bool = False, threads: int = 1):
    """Conceal the lost 16x16 blocks of one 8-bit frame.

    frame: uint8 [H, W]; mb_lost: uint8/bool [ceil(H/16), ceil(W/16)], 1 = lost; or, for
    an arbitrarily shaped loss, mb_lost None and px_lost: uint8/bool [H, W], 1 = lost.
    Returns dict(out=float64 [H, W], stats=dict, trace=structured array or None).
    Trace records are indexed [rank among lost blocks in raster order, step]; with px_lost
    the lost blocks are those holding a lost pixel.
    """
    lib = _load()
    p = p if p is not None else params()
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    H, W = frame.shape
    mbh, mbw = (H + 15) // 16, (W + 15) // 16
    if px_lost is not None:
        assert mb_lost is None, "give either mb_lost or px_lost"
        px_lost = np.ascontiguousarray(np.asarray(px_lost) != 0, dtype=np.uint8)
        assert px_lost.shape == (H, W), (px_lost.shape, (H, W))
        mb_lost = blocks_of(px_lost)
    mb_lost = np.ascontiguousarray(mb_lost, dtype=np.uint8)
    assert mb_lost.shape == (mbh, mbw), (mb_lost.shape, (mbh, mbw))
    sel = None
    if select is not None:
        sel = np.ascontiguousarray(select, dtype=np.uint8)
        assert sel.shape == (mbh, mbw)
    out = np.empty((H, W), dtype=np.float64)
    nlost = int(mb_lost.astype(bool).sum())
    tbuf = None
    if trace:
        tbuf = (TraceRec * max(1, nlost * 64))()
    st = Stats()
    sel_p = None if sel is None else sel.ctypes.data
    tb_p = None if tbuf is None else ctypes.addressof(tbuf)
    if px_lost is None:
        rc = lib.oracle_conceal(frame.ctypes.data, W, H, W, mb_lost.ctypes.data, sel_p,
                                ctypes.byref(p), out.ctypes.data, tb_p, ctypes.byref(st),
                                int(threads))
    else:
        rc = lib.oracle_conceal_px(frame.ctypes.data, W, H, W, px_lost.ctypes.data, W, sel_p,
                                   ctypes.byref(p), out.ctypes.data, tb_p, ctypes.byref(st),
                                   int(threads))
    if rc != 0:
        raise ValueError(f"oracle_conceal rejected the arguments (rc={rc})")
    stats = {k: (list(getattr(st, k)) if k == "idl_ring_hist" else int(getattr(st, k)))
             for k, _ in Stats._fields_}
    tr = None
    if tbuf is not None:
        tr = trace_to_numpy(bytes(tbuf)).reshape(max(1, nlost), 64)[:nlost]
    return {"out": out, "stats": stats, "trace": tr}

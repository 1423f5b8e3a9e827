"""Python binding of the C-ABI library ``libskmmse.so`` (include/skmmse.h).

Argument marshalling only: every step of the concealment runs in the CUDA kernels of
the library.  PyTorch provides device memory and streams.  There is no fallback: if the
library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libskmmse_phase.so" if os.environ.get("SKMMSE_PHASE_CLOCKS", "0") == "1"
                        else "libskmmse.so")

EXPRESS, EFFICIENT, EXCELLENT = 0, 1, 2
PROFILES = {"express": EXPRESS, "efficient": EFFICIENT, "excellent": EXCELLENT}
FP32, MIXED_BF16, MIXED_FP16 = 0, 1, 2
FLAG_TRACE = 1
FLAG_FORCE = 2
FLAG_QUANTIZE = 4
FLAG_SHORT_WAITS = 8
FLAG_IDL_TC = 16

STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported frame shape", 3: "unsupported alignment",
          4: "device memory allocation failed", 5: "CUDA runtime error",
          6: "dependency wait timed out on the device", 7: "unsupported precision or flag",
          8: "frame exceeds the static scratch of the no-allocation entry point"}
NOALLOC_MAX_MBS = 8192
ABI_VERSION = 3


class Params(ctypes.Structure):
    _fields_ = [
        ("t_phi", ctypes.c_float), ("t_nu", ctypes.c_float), ("sigma2", ctypes.c_float),
        ("ring_step", ctypes.c_int), ("ridge_rel", ctypes.c_float), ("beta_kmin", ctypes.c_int),
        ("beta_kmax", ctypes.c_int), ("beta_tie_rel", ctypes.c_float),
        ("concealed_is_support", ctypes.c_int), ("precision", ctypes.c_int), ("flags", ctypes.c_uint),
    ]


class Frame(ctypes.Structure):
    _fields_ = [
        ("frame", ctypes.c_void_p), ("width", ctypes.c_int), ("height", ctypes.c_int),
        ("pitch", ctypes.c_int), ("mb_lost", ctypes.c_void_p), ("out", ctypes.c_void_p),
        ("out_pitch", ctypes.c_int), ("out_f32", ctypes.c_void_p), ("out_f32_pitch", ctypes.c_int),
        ("trace", ctypes.c_void_p), ("px_lost", ctypes.c_void_p), ("px_pitch", ctypes.c_int),
        ("reserved", ctypes.c_int),
    ]


class Config(ctypes.Structure):
    """skmmse_config: persistent CTAs per SM and the tensor-core tile sizes."""
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("tile_cov", ctypes.c_int), ("tile_dist", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


TUNE_MAX_OPTIONS = 8


class Stats(ctypes.Structure):
    _fields_ = [
        ("n_lost_mbs", ctypes.c_longlong), ("n_patches", ctypes.c_longlong),
        ("n_empty", ctypes.c_longlong), ("n_brl", ctypes.c_longlong), ("n_idl", ctypes.c_longlong),
        ("n_hql", ctypes.c_longlong), ("n_brl_nocand", ctypes.c_longlong),
        ("idl_ring_hist", ctypes.c_longlong * 16), ("idl_cand_evals", ctypes.c_longlong),
        ("idl_ny_evals", ctypes.c_longlong), ("hql_cands", ctypes.c_longlong),
        ("hql_ny_cands", ctypes.c_longlong), ("hql_i0_cands", ctypes.c_longlong),
        ("alg_flops", ctypes.c_longlong), ("hql_ny2_cands", ctypes.c_longlong), ("hql_ny3", ctypes.c_longlong),
        ("hql_i0_ny_cands", ctypes.c_longlong), ("patch_ny", ctypes.c_longlong), ("mma_flops", ctypes.c_longlong),
        ("t_first_inv_ns", ctypes.c_longlong), ("t_last_ns", ctypes.c_longlong),
        ("n_beta", ctypes.c_longlong), ("error", ctypes.c_int), ("pad", ctypes.c_int),
    ]

    def as_dict(self) -> dict:
        d = {k: (list(getattr(self, k)) if k == "idl_ring_hist" else int(getattr(self, k)))
             for k, _ in self._fields_ if k != "pad"}
        # the concealment kernel's resident interval on the device (global timer, ns)
        d["t_first_ns"] = (~d.pop("t_first_inv_ns")) & (2 ** 64 - 1) if d["t_last_ns"] else 0
        return d


TRACE_DTYPE = np.dtype([
    ("mb", "<i4"), ("step", "<i2"), ("patch", "<i2"), ("layer", "i1"), ("ring", "i1"),
    ("beta_idx", "i1"), ("n0", "i1"), ("ny", "<i2"), ("m", "<i2"), ("phi", "<f4"),
    ("log_nu", "<f4"), ("alpha", "<f4"), ("eps_best", "<f4"), ("x", "<f4", (4,)),
    ("i0", "<u2", (36,))])

# every symbol include/skmmse.h declares
EXPORTS = ["skmmse_abi_version", "skmmse_struct_size", "skmmse_status_str", "skmmse_params_preset",
           "skmmse_create", "skmmse_destroy", "skmmse_conceal", "skmmse_conceal_px", "skmmse_conceal_batch",
           "skmmse_read_stats", "skmmse_read_phase_clocks", "skmmse_conceal_noalloc",
           "skmmse_probe_peaks",
           "skmmse_graph_create", "skmmse_graph_launch", "skmmse_graph_read_stats",
           "skmmse_graph_destroy", "skmmse_autotune", "skmmse_set_ctas_per_sm", "skmmse_set_config",
           "skmmse_get_config"]

_lib = None


class SkmmseError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libskmmse.so (built by ``paper_2205_11226_gb300.build``).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run paper_2205_11226_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    vp, ci = ctypes.c_void_p, ctypes.c_int
    lib.skmmse_abi_version.restype = ci
    lib.skmmse_struct_size.restype = ci
    lib.skmmse_struct_size.argtypes = [ci]
    lib.skmmse_status_str.restype = ctypes.c_char_p
    lib.skmmse_status_str.argtypes = [ci]
    lib.skmmse_params_preset.restype = None
    lib.skmmse_params_preset.argtypes = [ctypes.POINTER(Params), ci]
    lib.skmmse_create.restype = ci
    lib.skmmse_create.argtypes = [ctypes.POINTER(vp)]
    lib.skmmse_destroy.restype = None
    lib.skmmse_destroy.argtypes = [vp]
    lib.skmmse_conceal.restype = ci
    lib.skmmse_conceal.argtypes = [vp, vp, ci, ci, ci, vp, ctypes.POINTER(Params), vp, ci, vp,
                                   ctypes.POINTER(Stats), vp]
    lib.skmmse_conceal_px.restype = ci
    lib.skmmse_conceal_px.argtypes = [vp, vp, ci, ci, ci, vp, ci, ctypes.POINTER(Params), vp, ci, vp,
                                      ctypes.POINTER(Stats), vp]
    lib.skmmse_conceal_batch.restype = ci
    lib.skmmse_conceal_batch.argtypes = [vp, ctypes.POINTER(Frame), ci, ctypes.POINTER(Params),
                                         ctypes.POINTER(Stats), vp]
    lib.skmmse_read_stats.restype = ci
    lib.skmmse_read_stats.argtypes = [vp, ctypes.POINTER(Stats), vp]
    lib.skmmse_conceal_noalloc.restype = ci
    lib.skmmse_conceal_noalloc.argtypes = [vp, ci, ci, ci, vp, ctypes.POINTER(Params), vp, ci, vp,
                                           ctypes.POINTER(Stats), vp]
    lib.skmmse_graph_create.restype = ci
    lib.skmmse_graph_create.argtypes = [vp, ctypes.POINTER(Frame), ci, ctypes.POINTER(Params),
                                        ctypes.POINTER(vp)]
    lib.skmmse_graph_launch.restype = ci
    lib.skmmse_graph_launch.argtypes = [vp, vp]
    lib.skmmse_graph_read_stats.restype = ci
    lib.skmmse_graph_read_stats.argtypes = [vp, ctypes.POINTER(Stats), vp]
    lib.skmmse_graph_destroy.restype = None
    lib.skmmse_graph_destroy.argtypes = [vp]
    lib.skmmse_autotune.restype = ci
    lib.skmmse_autotune.argtypes = [vp, ctypes.POINTER(Frame), ci, ctypes.POINTER(Params), ci, vp,
                                    ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_float),
                                    ctypes.POINTER(ci), ctypes.POINTER(ci)]
    lib.skmmse_set_config.restype = ci
    lib.skmmse_set_config.argtypes = [vp, ctypes.POINTER(Config)]
    lib.skmmse_get_config.restype = ci
    lib.skmmse_get_config.argtypes = [vp, ctypes.POINTER(Frame), ci, ctypes.POINTER(Params), ctypes.POINTER(Config)]
    lib.skmmse_set_ctas_per_sm.restype = ci
    lib.skmmse_set_ctas_per_sm.argtypes = [vp, ci]
    lib.skmmse_probe_peaks.restype = ci
    lib.skmmse_probe_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    lib.skmmse_read_phase_clocks.restype = ci
    lib.skmmse_read_phase_clocks.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), vp]
    assert lib.skmmse_abi_version() == ABI_VERSION, "library ABI version"
    assert lib.skmmse_struct_size(0) == TRACE_DTYPE.itemsize, "trace record layout"
    assert lib.skmmse_struct_size(1) == ctypes.sizeof(Stats), "stats layout"
    assert lib.skmmse_struct_size(2) == ctypes.sizeof(Params), "params layout"
    assert lib.skmmse_struct_size(3) == ctypes.sizeof(Frame), "frame layout"
    assert lib.skmmse_struct_size(4) == ctypes.sizeof(Config), "config layout"
    _lib = lib
    return lib


def params(profile: str | int = "efficient", **kw) -> Params:
    lib = load()
    p = Params()
    lib.skmmse_params_preset(ctypes.byref(p), PROFILES.get(profile, profile) if isinstance(profile, str) else profile)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def probe_peaks(stream=None) -> dict:
    """Measured FP32 FMA (TFLOP/s) and exp2 (per second) throughput of the current device."""
    lib = load()
    fma, ex2 = ctypes.c_double(), ctypes.c_double()
    _check(lib.skmmse_probe_peaks(ctypes.byref(fma), ctypes.byref(ex2), _stream_handle(stream)),
           "skmmse_probe_peaks")
    return {"fma_tflops": fma.value, "ex2_per_s": ex2.value}


def _check(status: int, where: str):
    if status != 0:
        raise SkmmseError(status, where)


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Context:
    """Owns the library's device scratch for calls ordered on one stream."""

    def __init__(self):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.skmmse_create(ctypes.byref(h)), "skmmse_create")
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.skmmse_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------------------------
    def conceal(self, frame, mb_lost, p: Params | None = None, *, px_lost=None, out=None,
                out_f32=None, stats: bool = False, stream=None):
        """frame: uint8 CUDA tensor [H, W]; mb_lost: uint8 CUDA tensor [ceil(H/16), ceil(W/16)]
        (whole lost blocks), or None with px_lost: uint8 CUDA tensor [H, W] (arbitrarily
        shaped loss, 1 = lost pixel).
        Returns (out, out_f32, stats_dict_or_None); out_f32 only if given (or True)."""
        import torch
        p = p if p is not None else params()
        assert frame.is_cuda and frame.dtype == torch.uint8 and frame.dim() == 2
        assert (mb_lost is None) != (px_lost is None), "give mb_lost or px_lost"
        mask = mb_lost if px_lost is None else px_lost
        assert mask.is_cuda and mask.dtype == torch.uint8 and mask.stride(1) == 1
        H, W = frame.shape
        if out is None:
            out = torch.empty_like(frame)
        if out_f32 is True:
            out_f32 = torch.zeros((H, W), dtype=torch.float32, device=frame.device)
        st = Stats() if stats else None
        tail = (ctypes.byref(p), out.data_ptr(), out.stride(0),
                out_f32.data_ptr() if out_f32 is not None else None,
                ctypes.byref(st) if st is not None else None, _stream_handle(stream))
        if px_lost is None:
            assert mb_lost.is_contiguous()
            rc = self._lib.skmmse_conceal(self._h, frame.data_ptr(), W, H, frame.stride(0),
                                          mb_lost.data_ptr(), *tail)
        else:
            assert tuple(px_lost.shape) == (H, W)
            rc = self._lib.skmmse_conceal_px(self._h, frame.data_ptr(), W, H, frame.stride(0),
                                             px_lost.data_ptr(), px_lost.stride(0), *tail)
        _check(rc, "skmmse_conceal" if px_lost is None else "skmmse_conceal_px")
        return out, out_f32, (st.as_dict() if st is not None else None)

    @staticmethod
    def _descs(frames, masks, outs, outs_f32=None, traces=None):
        """masks[i]: block flags [ceil(H/16), ceil(W/16)] (contiguous), or a per-pixel mask
        of the frame's own shape [H, W] (arbitrarily shaped loss)."""
        n = len(frames)
        descs = (Frame * n)()
        for i, (f, m) in enumerate(zip(frames, masks)):
            H, W = f.shape
            d = descs[i]
            d.frame, d.width, d.height, d.pitch = f.data_ptr(), W, H, f.stride(0)
            if tuple(m.shape) == (H, W):
                assert m.stride(1) == 1
                d.px_lost, d.px_pitch = m.data_ptr(), m.stride(0)
            else:
                assert m.is_contiguous()
                d.mb_lost = m.data_ptr()
            d.out, d.out_pitch = outs[i].data_ptr(), outs[i].stride(0)
            if outs_f32 is not None and outs_f32[i] is not None:
                d.out_f32, d.out_f32_pitch = outs_f32[i].data_ptr(), outs_f32[i].stride(0)
            if traces is not None and traces[i] is not None:
                d.trace = traces[i].data_ptr()
        return descs

    def conceal_batch(self, frames, masks, p: Params | None = None, *, outs=None, outs_f32=None,
                      traces=None, stats: bool = False, stream=None):
        """Batch of frames (lists of uint8 CUDA tensors); one persistent launch."""
        import torch
        p = p if p is not None else params()
        n = len(frames)
        if outs is None:
            outs = [torch.empty_like(f) for f in frames]
        descs = self._descs(frames, masks, outs, outs_f32, traces)
        st = Stats() if stats else None
        rc = self._lib.skmmse_conceal_batch(self._h, descs, n, ctypes.byref(p),
                                            ctypes.byref(st) if st is not None else None,
                                            _stream_handle(stream))
        _check(rc, "skmmse_conceal_batch")
        return outs, (st.as_dict() if st is not None else None)

    def graph(self, frames, masks, p: Params | None = None, *, outs, outs_f32=None):
        """Record the batch call on these fixed buffers as a CUDA graph (see Graph)."""
        return Graph(self, frames, masks, p if p is not None else params(), outs, outs_f32)

    def autotune(self, frames, masks, p: Params | None = None, *, outs=None, reps: int = 2,
                 stream=None) -> dict:
        """Time every launch configuration on this batch and keep the fastest for its shape
        class.  Returns the options timed, their mean milliseconds and the chosen one."""
        import torch
        p = p if p is not None else params()
        if outs is None:
            outs = [torch.empty_like(f) for f in frames]
        descs = self._descs(frames, masks, outs)
        opts = (Config * TUNE_MAX_OPTIONS)()
        ms = (ctypes.c_float * TUNE_MAX_OPTIONS)()
        nopt, best = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.skmmse_autotune(self._h, descs, len(frames), ctypes.byref(p), reps,
                                         _stream_handle(stream), opts, ms, ctypes.byref(nopt),
                                         ctypes.byref(best)), "skmmse_autotune")
        options = [{**opts[i].as_dict(), "ms": float(ms[i])} for i in range(nopt.value)]
        chosen = options[best.value]
        return {"options": options, "best": chosen, "ctas_per_sm": chosen["ctas_per_sm"],
                "ms": [o["ms"] for o in options]}

    def set_config(self, ctas_per_sm: int = 0, tile_cov: int = 64, tile_dist: int = 64):
        """The configuration of shape classes the autotuner has not timed."""
        c = Config(ctas_per_sm, tile_cov, tile_dist)
        _check(self._lib.skmmse_set_config(self._h, ctypes.byref(c)), "skmmse_set_config")

    def get_config(self, frames, masks, p: Params | None = None) -> dict:
        """The configuration a batch call with these frames would use."""
        p = p if p is not None else params()
        descs = self._descs(frames, masks, frames)
        c = Config()
        _check(self._lib.skmmse_get_config(self._h, descs, len(frames), ctypes.byref(p), ctypes.byref(c)),
               "skmmse_get_config")
        return c.as_dict()

    def set_ctas_per_sm(self, k: int):
        _check(self._lib.skmmse_set_ctas_per_sm(self._h, int(k)), "skmmse_set_ctas_per_sm")

    PHASES = ["stage", "ctx", "brl", "idl", "h_cand", "h_cov", "h_chol", "h_dist", "h_beta",
              "h_i0", "h_alpha", "h_est", "writeback", "publish", "x1", "x2"]

    def read_phase_clocks(self, stream=None) -> dict:
        """Per-phase SM cycles of the last call (library built with SKMMSE_PHASE_CLOCKS)."""
        buf = (ctypes.c_longlong * 16)()
        _check(self._lib.skmmse_read_phase_clocks(self._h, buf, _stream_handle(stream)),
               "skmmse_read_phase_clocks")
        return dict(zip(self.PHASES, list(buf)))

    def read_stats(self, stream=None) -> dict:
        st = Stats()
        rc = self._lib.skmmse_read_stats(self._h, ctypes.byref(st), _stream_handle(stream))
        d = st.as_dict()
        d["status"] = rc
        return d


class Graph:
    """A batch call on fixed device buffers captured as a CUDA graph: each launch()
    conceals what the frame buffers hold at that time (persistent kernel and queue
    construction replayed without host work)."""

    def __init__(self, ctx: Context, frames, masks, p: Params, outs, outs_f32=None):
        self._lib = ctx._lib
        self._keep = (frames, masks, outs, outs_f32)  # the buffers must outlive the graph
        descs = Context._descs(frames, masks, outs, outs_f32)
        h = ctypes.c_void_p()
        _check(self._lib.skmmse_graph_create(ctx._h, descs, len(frames), ctypes.byref(p),
                                             ctypes.byref(h)), "skmmse_graph_create")
        self._h = h

    def launch(self, stream=None):
        _check(self._lib.skmmse_graph_launch(self._h, _stream_handle(stream)), "skmmse_graph_launch")

    def read_stats(self, stream=None) -> dict:
        st = Stats()
        rc = self._lib.skmmse_graph_read_stats(self._h, ctypes.byref(st), _stream_handle(stream))
        d = st.as_dict()
        d["status"] = rc
        return d

    def close(self):
        if getattr(self, "_h", None):
            self._lib.skmmse_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _px_blocks(px: np.ndarray) -> np.ndarray:
    h, w = px.shape
    r, c = (h + 15) // 16, (w + 15) // 16
    pad = np.zeros((r * 16, c * 16), dtype=bool)
    pad[:h, :w] = px
    return pad.reshape(r, 16, c, 16).any(axis=(1, 3))


def trace_buffer(mask_np: np.ndarray, device="cuda", px: bool = False):
    """Device buffer for the per-patch decision records of one frame (mask: the block
    flags, or with px=True the per-pixel mask)."""
    import torch
    m = np.asarray(mask_np) != 0
    nlost = int(_px_blocks(m).sum()) if px else int(m.sum())
    return torch.zeros(max(1, nlost) * 64 * TRACE_DTYPE.itemsize, dtype=torch.uint8, device=device)


def trace_to_numpy(buf, nlost: int) -> np.ndarray:
    raw = buf.cpu().numpy().tobytes()
    return np.frombuffer(raw, dtype=TRACE_DTYPE).reshape(max(1, nlost), 64)[:nlost]


def conceal_numpy(frame: np.ndarray, mb_lost: np.ndarray | None, p: Params | None = None, *,
                  px_lost: np.ndarray | None = None, trace: bool = False,
                  ctx: Context | None = None, force_x: np.ndarray | None = None):
    """Host-buffer convenience: copy in, conceal on cuda:0, copy out.
    mb_lost: block flags, or None with px_lost: per-pixel loss [H, W].
    Returns dict(out=uint8 [H, W], out_f32=float32 [H, W], stats, trace).
    force_x (verification hook, float [n_lost, 64, 4]): reference estimates written back
    into the support after each step instead of the kernel's own (SKMMSE_FLAG_FORCE)."""
    import torch
    p = params() if p is None else p
    ctx = ctx or Context()
    assert (mb_lost is None) != (px_lost is None), "give mb_lost or px_lost"
    mask = np.ascontiguousarray(np.asarray(mb_lost if px_lost is None else px_lost) != 0, dtype=np.uint8)
    nlost = int(mask.sum()) if px_lost is None else int(_px_blocks(mask != 0).sum())
    f = torch.from_numpy(np.ascontiguousarray(frame, dtype=np.uint8)).cuda()
    m = torch.from_numpy(mask).cuda()
    of = torch.zeros(f.shape, dtype=torch.float32, device=f.device)
    tb = None
    if trace or force_x is not None:
        p = Params.from_buffer_copy(p)
        p.flags |= FLAG_TRACE
        if force_x is not None:
            p.flags |= FLAG_FORCE
            rec = np.zeros((max(1, nlost), 64), dtype=TRACE_DTYPE)
            rec["x"][:nlost] = np.asarray(force_x, dtype=np.float32).reshape(nlost, 64, 4)
            tb = torch.from_numpy(rec.view(np.uint8).reshape(-1).copy()).cuda()
        else:
            tb = trace_buffer(mask, px=px_lost is not None)
    outs, st = ctx.conceal_batch([f], [m], p, outs_f32=[of], traces=[tb] if tb is not None else None,
                                 stats=True)
    torch.cuda.synchronize()
    return {"out": outs[0].cpu().numpy(), "out_f32": of.cpu().numpy(), "stats": st,
            "trace": trace_to_numpy(tb, nlost) if tb is not None else None}

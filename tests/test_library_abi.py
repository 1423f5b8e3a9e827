"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports every
entry point include/skmmse.h declares, and its struct layouts and presets agree with the
binding and with Table I.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_2205_11226_gb300 import build, skmmse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return skmmse.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "skmmse.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(skmmse_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert set(names) == set(skmmse.EXPORTS), names
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts(lib):
    assert lib.skmmse_abi_version() == skmmse.ABI_VERSION == 3
    assert lib.skmmse_struct_size(0) == skmmse.TRACE_DTYPE.itemsize == 120
    assert lib.skmmse_struct_size(1) == ctypes.sizeof(skmmse.Stats)
    assert lib.skmmse_struct_size(2) == ctypes.sizeof(skmmse.Params)
    assert lib.skmmse_struct_size(3) == ctypes.sizeof(skmmse.Frame)
    assert lib.skmmse_struct_size(4) == ctypes.sizeof(skmmse.Config) == 12
    assert lib.skmmse_struct_size(9) == -1


def test_presets_follow_table1(lib):
    rows = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "table1_profiles.txt")):
        line = line.split("#")[0].split()
        if line:
            rows[line[0]] = [float(v) for v in line[1:]]
    for name, code in skmmse.PROFILES.items():
        p = skmmse.params(code)
        assert p.t_phi == rows[name][0]
        assert p.t_nu == pytest.approx(rows[name][1], rel=1e-6)
        assert p.sigma2 == rows["sigma2"][0]
        assert (p.ring_step, p.beta_kmin, p.beta_kmax, p.concealed_is_support) == (4, -8, 16, 1)


def test_null_arguments_rejected_without_compute(lib):
    p = skmmse.params()
    f = skmmse.Frame()
    assert lib.skmmse_conceal_batch(None, ctypes.byref(f), 1, ctypes.byref(p), None, None) == 1
    assert lib.skmmse_create(None) == 1
    assert lib.skmmse_read_stats(None, None, None) == 1
    lib.skmmse_destroy(None)
    assert lib.skmmse_status_str(6) == b"dependency wait timed out on the device"
    assert lib.skmmse_status_str(99) == b"unknown status"


def test_argument_validation_before_any_device_call(lib):
    # skmmse_conceal_noalloc checks its parameters and frame on the host before its first
    # CUDA call, so every rejection below is reached without a GPU.  The device pointers
    # are placeholders that are never dereferenced.
    FR, MB, OUT = 0x10000, 0x20000, 0x30000

    def call(w=64, h=64, pitch=64, out_pitch=64, f32=None, mb=MB, **kw):
        p = skmmse.params()
        for k, v in kw.items():
            setattr(p, k, v)
        return lib.skmmse_conceal_noalloc(FR, w, h, pitch, mb, ctypes.byref(p), OUT, out_pitch,
                                          f32, None, None)

    ARG, SHAPE, ALIGN, TOO_LARGE = 1, 2, 3, 8
    assert call(t_nu=0.0) == ARG
    assert call(sigma2=-1.0) == ARG
    assert call(t_phi=float("nan")) == ARG
    assert call(ridge_rel=-1e-3) == ARG
    assert call(ring_step=0) == ARG
    assert call(beta_kmin=3, beta_kmax=2) == ARG
    assert call(beta_kmin=-40, beta_kmax=40) == ARG      # more grid values than supported
    assert call(precision=7) == ARG
    assert call(flags=1 << 20) == ARG
    assert call(flags=skmmse.FLAG_TRACE) == ARG         # no trace buffer on this entry
    assert call(mb=None) == ARG
    assert call(w=63) == SHAPE and call(h=0) == SHAPE
    assert call(pitch=32) == SHAPE and call(out_pitch=32) == SHAPE
    assert call(f32=OUT + 2) == ALIGN
    assert call(w=4096, h=4096, pitch=4096, out_pitch=4096) == TOO_LARGE


def test_noalloc_scratch_size_stated_in_the_header():
    # the static scratch of skmmse_conceal_noalloc, as the header states it (the library
    # pins the same figure with a static_assert on its layout)
    text = open(os.path.join(ROOT, "include", "skmmse.h")).read()
    nbytes = int(re.search(r"#define SKMMSE_NOALLOC_SCRATCH_BYTES (\d+)", text).group(1))
    ctas = int(re.search(r"#define SKMMSE_NOALLOC_MAX_CTAS (\d+)", text).group(1))
    mbs = int(re.search(r"#define SKMMSE_NOALLOC_MAX_MBS (\d+)", text).group(1))
    assert mbs == skmmse.NOALLOC_MAX_MBS and ctas == 128
    # per CTA: the whitened vectors of one HQL step, 1849 candidates x 32 floats
    assert nbytes > ctas * 1849 * 32 * 4 + mbs * 256 * 4
    assert f"{nbytes / 1e6:.1f} MB" in text

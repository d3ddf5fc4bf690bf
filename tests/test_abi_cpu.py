"""The C-ABI library loads, exports every declared symbol, and computes its
host-side tables exactly as the oracle does (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "chimebf.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(bf_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(built_lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(built_lib, n), n
    assert set(names) == set(B.SYMBOLS)


def test_config_defaults(built_lib):
    c = B.bf_config_default()
    assert (c.n_cyl, c.n_feed, c.n_pol, c.pad, c.n_ew, c.upchan, c.f_ds, c.t_ds) == (4, 256, 2, 2, 4, 128, 8, 3)
    assert c.feed_spacing_m == 0.3048 and c.cyl_spacing_m == 20.0 and c.dt_s == 2.56e-6


@pytest.mark.parametrize("freq", [400e6, 400.1953125e6, 410e6, 491.8e6, 520e6, 600e6, 650e6, 700e6, 790e6, 800e6])
def test_clamp_table_equals_oracle(built_lib, freq):
    lut, ew = B.bf_debug_tables(freq)
    assert np.array_equal(lut, O.clamp_lut(freq))
    w = O.ew_weights(freq)                       # [c, j]
    assert np.allclose(ew, w.T, rtol=0, atol=2e-7)


def test_clamp_table_sweep_and_custom_pointings(built_lib):
    freqs = 400e6 + 390625.0 * (np.arange(1024) + 0.5)
    for f in freqs[::7]:
        assert np.array_equal(B.bf_debug_tables(f)[0], O.clamp_lut(f))
    rng = np.random.default_rng(5)
    ns = rng.uniform(-1, 1, 256)
    ewd = np.sin(np.radians(rng.uniform(-1.2, 1.2, 4)))
    cfg = B.bf_config_default(ns_sin=ns, ew_sin=ewd, feed_spacing_m=0.31, cyl_spacing_m=22.0)
    g = O.Geometry(feed_spacing_m=0.31, cyl_spacing_m=22.0)
    for f in [433.3e6, 777.7e6]:
        lut, ew = B.bf_debug_tables(f, cfg)
        assert np.array_equal(lut, O.clamp_lut(f, ns, g))
        assert np.allclose(ew, O.ew_weights(f, ewd, g).T, atol=2e-7)


def test_bad_geometry_rejected_before_cuda(built_lib):
    for field, val in [("n_feed", 128), ("pad", 4), ("upchan", 64), ("n_ew", 8), ("t_ds", 2)]:
        c = B.bf_config_default(**{field: val})
        h = ctypes.c_void_p()
        assert built_lib.bf_plan(ctypes.byref(c), ctypes.byref(h)) == B.BF_EINVAL
        assert "geometry" in B.bf_last_error()
    c = B.bf_config_default(feed_spacing_m=-1.0)
    assert built_lib.bf_plan(ctypes.byref(c), ctypes.byref(ctypes.c_void_p())) == B.BF_EINVAL
    assert built_lib.bf_plan(None, None) == B.BF_EINVAL
    assert built_lib.bf_debug_tables(None, 600e6, None, None) == B.BF_EINVAL
    for bad in (-1, 4097):                       # table slots: 0 (default 4096) or 1 .. 4096
        c = B.bf_config_default(max_tables=bad)
        assert built_lib.bf_plan(ctypes.byref(c), ctypes.byref(ctypes.c_void_p())) == B.BF_EINVAL
        assert "max_tables" in B.bf_last_error()


def test_null_plan_calls_fail_cleanly(built_lib):
    nf = ctypes.c_int64()
    assert built_lib.bf_poll(None, 1, 0, ctypes.byref(nf)) == B.BF_EINVAL
    times = (ctypes.c_double * 5)()
    assert built_lib.bf_poll_timed(None, 1, 0, ctypes.byref(nf), times) == B.BF_EINVAL
    assert built_lib.bf_destroy(None) == B.BF_EINVAL
    assert built_lib.bf_submit(None, None, None) == B.BF_EINVAL


def test_plan_without_gpu_reports_cuda_error(built_lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    c = B.bf_config_default()
    h = ctypes.c_void_p()
    rc = built_lib.bf_plan(ctypes.byref(c), ctypes.byref(h))
    assert rc == B.BF_ECUDA and h.value is None
    assert B.bf_last_error()


@pytest.mark.parametrize("freq", [410e6, 520e6, 600e6, 650e6, 700e6, 790e6, 799.8e6])
def test_gather_order_is_a_conflict_avoiding_permutation(built_lib, freq):
    """The FP32 form's consumer slots take the beams in a per-frequency order: a
    permutation of the 256 beams (each output is written once) in which eight
    consecutive slots, gathered by one 16-byte load phase, mostly hit distinct
    bank groups of the swizzled bin row (bsw(L) mod 8) or share a bin."""
    order = B.bf_debug_gather_order(freq).astype(int)
    assert sorted(order) == list(range(256))
    lut = O.clamp_lut(freq).astype(int)

    def extra_wavefronts(slots):
        extra = 0
        for o in range(32):
            bins = {int(lut[m]) for m in slots[8 * o:8 * o + 8]}
            groups = {}
            for L in bins:
                groups.setdefault((L ^ ((L >> 3) & 1)) & 7, set()).add(L)
            extra += max(len(v) for v in groups.values()) - 1
        return extra

    natural = extra_wavefronts(list(range(256)))
    ordered = extra_wavefronts(list(order))
    assert ordered <= 8 and ordered < natural, (ordered, natural)

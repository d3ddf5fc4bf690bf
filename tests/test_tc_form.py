"""Tensor-core DFT form against the FP64 oracle.

The N-S stage runs as a DFT-matrix GEMM over the 256 clamped rows (FP16
operands, FP32 accumulation).  Error budget per form, from the operand
rounding: data hi+lo is exact to ~2^-22; FP16 twiddles alone carry 2^-12
relative error, hi+lo twiddles ~2^-23.  Tolerances (max relative error per
output element against the oracle):

* BF_TC_DFT256 (3 terms: twiddles hi+lo, data hi+lo): 1e-5, as the FP32 path;
* BF_TC_DFT256_X2 (2 terms: twiddles hi, data hi+lo): 1e-3;
* BF_TC_DFT256_X1 (1 term: twiddles hi, data hi): 1e-3 (measured 3.3-3.5e-4).
"""
import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMS = {B.BF_TC_DFT256: 1e-5, B.BF_TC_DFT256_X2: 1e-3, B.BF_TC_DFT256_X1: 1e-3}
# GEMM stage, max |error| / rms over ~8e5 values: FP32 accumulation over K = 512
# (3 terms); FP16 twiddle rounding 2^-12 summed over 256 random-phase feeds,
# rms ~1.4e-4, ~5 sigma at the maximum (2 terms); the FP16 data rounding adds
# as much again (1 term, rms x sqrt 2).  Measured maxima 9.1e-6 / 6.5e-4 / 1.15e-3.
GEMM_TOL = {B.BF_TC_DFT256: 2e-5, B.BF_TC_DFT256_X2: 1.5e-3, B.BF_TC_DFT256_X1: 2e-3}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(got, ref):
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref) / np.abs(ref)))


@pytest.mark.parametrize("form", list(FORMS))
def test_gemm_stage_dump(built_lib, form):
    freq = 650e6
    raw = synth.noise_only([freq], 384, seed=31)[0]
    with B.Plan(form=form) as p:
        out = torch.empty(3, 2, 4, 256, 128, 2, dtype=torch.float32, device="cuda")
        B.bf_debug_gemm(p.handle, freq, dev(raw), 384, out)
        got = out.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]                             # [blk, p, j, m, t]
    ref = O.ew_beams(O.ns_beams(O.unpack(raw), O.clamp_lut(freq)), O.ew_weights(freq))  # [T, p, j, m]
    ref = np.transpose(ref.reshape(3, 128, 2, 4, 256), (0, 2, 3, 4, 1))
    scale = np.sqrt(np.mean(np.abs(ref) ** 2))
    err = np.max(np.abs(got - ref)) / scale
    assert err <= GEMM_TOL[form], f"GEMM stage error {err:.3e} (x rms)"


@pytest.mark.parametrize("form", list(FORMS))
def test_point_source_per_form(built_lib, form):
    raw, f = synth.config_point_source(0)
    with B.Plan(form=form) as p:
        out = p.run(dev(raw), list(f)).cpu().numpy()
    ref = O.beamform(raw, f)
    err = rel_err(out, ref)
    assert err <= FORMS[form], f"max relative error {err:.3e}"
    assert int(out.sum(axis=(1, 2)).argmax()) == 939


@pytest.mark.parametrize("form", [B.BF_TC_DFT256, B.BF_TC_DFT256_X2])
def test_upchan_stage_dump_tc(built_lib, form):
    freq = 520e6
    raw = synth.noise_only([freq], 768, seed=32)[0]
    with B.Plan(form=form) as p:
        out = torch.empty(6, 2, 4, 256, 128, 2, dtype=torch.float32, device="cuda")
        B.bf_debug_upchan(p.handle, freq, dev(raw), 768, out)
        got = out.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    _, st = O.beamform_channel(raw, freq, return_stages=True)
    scale = np.sqrt(np.mean(np.abs(st["Y"]) ** 2))
    assert np.max(np.abs(got - st["Y"])) / scale <= 10 * GEMM_TOL[form]


def test_tc_multichannel_ragged_and_node_slice_sample(built_lib):
    freqs = [410e6, 600e6, 790e6]
    raw = synth.noise_only(freqs, 384 * 3 + 50, seed=33)
    with B.Plan(form=B.BF_TC_DFT256) as p:
        out = p.run(dev(raw), freqs).cpu().numpy()
    assert out.shape == (1024, 48, 3)
    assert rel_err(out, O.beamform(raw, freqs)) <= 1e-5

    raw, freqs, _ = synth.config_node_slice(0)
    with B.Plan(form=B.BF_TC_DFT256_X2) as p:
        out = p.run(dev(raw), list(freqs)).cpu().numpy()
    rng = np.random.default_rng(1)
    picks = [(int(rng.integers(4)), int(rng.integers(1024)), int(rng.integers(128))) for _ in range(32)]
    ref = O.beamform_sample(raw, freqs, picks)
    got = np.stack([out[b, 16 * ch:16 * ch + 16, fr] for ch, b, fr in picks])
    assert rel_err(got, ref) <= FORMS[B.BF_TC_DFT256_X2]


def test_tc_dft512_not_built(built_lib):
    with pytest.raises(B.BfError) as e:
        B.Plan(form=B.BF_TC_DFT512)
    assert e.value.code == B.BF_EINVAL

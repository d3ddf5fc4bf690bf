"""Tensor-core DFT form against the FP64 oracle.

The N-S stage runs as a DFT-matrix GEMM over the 256 clamped rows (FP16
operands, FP32 accumulation).  Error budget per form, from the operand
rounding: data hi+lo is exact to ~2^-22; FP16 twiddles alone carry 2^-12
relative error, hi+lo twiddles ~2^-23.  Tolerances (max relative error per
output element against the oracle):

* BF_TC_DFT256 (3 terms: twiddles hi+lo, data hi+lo): 1e-5, as the FP32 path;
* BF_TC_DFT256_X2 (2 terms: twiddles hi, data hi+lo): 1e-3;
* BF_TC_DFT256_X1 (1 term: twiddles hi, data hi): 1e-3 (measured 3.3-3.5e-4);
* BF_TC_DFT512 (all 512 rows of the zero-padded transform, 1 term, the clamp
  applied to the result): 1e-3, and the same values as BF_TC_DFT256_X1, whose
  rows are the kept rows of the same FP16 matrix.
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


def test_dft512_point_source(built_lib):
    # the data of the point-source case (one channel at 600 MHz, 3072 samples) through the
    # 512 x 256 DFT-matrix GEMM
    raw, f = synth.config_point_source(0)
    with B.Plan(form=B.BF_TC_DFT512) as p:
        out = p.run(dev(raw), list(f)).cpu().numpy()
    ref = O.beamform(raw, f)
    err = rel_err(out, ref)
    assert err <= 1e-3, f"max relative error {err:.3e}"
    assert int(out.sum(axis=(1, 2)).argmax()) == 939


def test_dft512_equals_the_256_row_form(built_lib):
    # 410 MHz leaves bins that no beam takes; at 600 MHz aliasing gives some bins two beams
    freqs = [410e6, 600e6, 790e6]
    assert len(set(O.clamp_lut(600e6).tolist())) < 256
    assert len(set(O.clamp_lut(410e6).tolist())) == 256
    raw = synth.noise_only(freqs, 384 * 5 + 77, seed=34)
    with B.Plan(form=B.BF_TC_DFT512) as p:
        o512 = p.run(dev(raw), freqs).cpu().numpy()
    with B.Plan(form=B.BF_TC_DFT256_X1) as p:
        o256 = p.run(dev(raw), freqs).cpu().numpy()
    assert o512.shape == (1024, 48, 5)
    # the kept rows of the 512-row GEMM are the 256-row form's rows: same FP16 operands,
    # same accumulation order, same epilogue
    assert np.array_equal(o512, o256)
    assert rel_err(o512, O.beamform(raw, freqs)) <= 1e-3


def test_dft512_streams_carry_dumps_and_stall_check(built_lib):
    freqs = [520e6, 650e6]
    n = 384 * 4 + 200
    raw = synth.noise_only(freqs, n, seed=35)
    cut = 384 + 123
    with B.Plan(form=B.BF_TC_DFT512) as p:
        a = p.run(dev(raw[:, :cut]), freqs, stream_id=7, flags=0).cpu().numpy()
        b = p.run(dev(raw[:, cut:]), freqs, stream_id=7, flags=B.BF_END_OF_STREAM).cpu().numpy()
        vin = dev(raw[0, :384])
        out = torch.empty(3, 2, 4, 256, 128, 2, dtype=torch.float32, device="cuda")
        with pytest.raises(B.BfError) as e:
            B.bf_debug_gemm(p.handle, freqs[0], vin, 384, out)
        assert e.value.code == B.BF_EINVAL
        # the stall check runs the form's own kernel (clusters of four)
        assert B.bf_debug_stall(p.handle, vin, 1000000) == B.BF_ETIMEDOUT
    got = np.concatenate([a, b], axis=2)
    assert got.shape == (1024, 32, 4)
    assert rel_err(got, O.beamform(raw, freqs)) <= 1e-3

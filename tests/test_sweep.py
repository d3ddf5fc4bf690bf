"""Throughput-sweep workload: 64 channels over 400-800 MHz x 1 s (390625
samples) x 2048 inputs = 51.2 GB on the device, from the counter-based
generator; sampled outputs against the oracle, which rebuilds the sampled
frames on the host from the same generator."""
import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED, NCH, T = 11, 64, 390625


@pytest.fixture(scope="module")
def sweep_input(built_lib):
    vin = synth.hash_noise_device(SEED, NCH, T)
    torch.cuda.synchronize()
    yield vin
    del vin
    torch.cuda.empty_cache()


def sampled_reference(picks):
    ref = []
    for ch, beam, fr in picks:
        rows = synth.hash_noise_rows(SEED, ch, T, 384 * fr, 384 * fr + 384)
        ref.append(O.beamform_sample(rows[None], [synth.SWEEP_FREQS[ch]], [(0, beam, 0)])[0])
    return np.stack(ref)


@pytest.mark.parametrize("form,tol", [(B.BF_FP32_FFT, 1e-5), (B.BF_TC_DFT256_X1, 1e-3)])
def test_sweep_sampled(sweep_input, form, tol):
    nf = T // 384
    assert nf == 1017                                   # 97 trailing samples are dropped
    with B.Plan(form=form) as p:
        out = p.run(sweep_input, synth.SWEEP_FREQS)
        torch.cuda.synchronize()
        assert out.shape == (1024, 16 * NCH, nf)
        rng = np.random.default_rng(form)
        picks = [(int(rng.integers(NCH)), int(rng.integers(1024)), int(rng.integers(nf))) for _ in range(20)]
        picks += [(0, 0, 0), (NCH - 1, 1023, nf - 1)]
        got = np.stack([out[b, 16 * ch:16 * ch + 16, fr].cpu().numpy() for ch, b, fr in picks])
        # whole frames: all 1024 beams x 16 sub-channels of the last frame of channel 0 and
        # of a middle frame of the last channel
        whole = {(ch, fr): out[:, 16 * ch:16 * ch + 16, fr].cpu().numpy() for ch, fr in ((0, nf - 1), (NCH - 1, 500))}
        del out
    ref = sampled_reference(picks)
    err = np.max(np.abs(got - ref) / ref)
    assert err <= tol, f"max relative error {err:.3e}"
    for (ch, fr), g in whole.items():
        rows = synth.hash_noise_rows(SEED, ch, T, 384 * fr, 384 * fr + 384)
        r = O.beamform(rows[None], [synth.SWEEP_FREQS[ch]])[:, :, 0]
        e = np.max(np.abs(g.astype(np.float64) - r) / r)
        assert e <= tol, f"channel {ch} frame {fr}: max relative error {e:.3e}"

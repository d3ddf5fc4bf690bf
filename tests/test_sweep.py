"""Throughput-sweep workload: 64 channels over 400-800 MHz x 1 s (390625
samples) x 2048 inputs = 51.2 GB on the device, from the counter-based
generator, with five dispersed bursts (DM 100-2000) from zenith; sampled
outputs against the oracle, which rebuilds the sampled frames on the host from
the same generator (burst frames included), and the bursts found again by
dedispersing the beamformed sweep."""
import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED, NCH, T = 11, 64, 390625


OFFSETS = None


def offsets():
    global OFFSETS
    if OFFSETS is None:
        OFFSETS = synth.burst_offsets(synth.SWEEP_FREQS, T, synth.SWEEP_BURSTS, SEED)
    return OFFSETS


def burst_frame(b, ch):
    """Output frame in which burst b peaks in channel ch."""
    f = synth.SWEEP_FREQS[ch]
    t = b.t0_s + synth.K_DM * b.dm * ((f / 1e6) ** -2 - (b.f_ref_hz / 1e6) ** -2)
    return int(t / (384 * synth.DT_S))


@pytest.fixture(scope="module")
def sweep_input(built_lib):
    vin = synth.hash_noise_device(SEED, NCH, T, offsets=offsets())
    torch.cuda.synchronize()
    yield vin
    del vin
    torch.cuda.empty_cache()


def sampled_reference(picks):
    ref = []
    for ch, beam, fr in picks:
        rows = synth.hash_noise_rows(SEED, ch, T, 384 * fr, 384 * fr + 384, offsets=offsets())
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
        # frames where the DM-100 and DM-2000 bursts peak in the top channel (zenith beams)
        picks += [(NCH - 1, 256 + 127, burst_frame(synth.SWEEP_BURSTS[0], NCH - 1)),
                  (NCH - 1, 512 + 128, burst_frame(synth.SWEEP_BURSTS[4], NCH - 1))]
        got = np.stack([out[b, 16 * ch:16 * ch + 16, fr].cpu().numpy() for ch, b, fr in picks])
        # whole frames: all 1024 beams x 16 sub-channels of the last frame of channel 0 and
        # of a middle frame of the last channel
        whole = {(ch, fr): out[:, 16 * ch:16 * ch + 16, fr].cpu().numpy() for ch, fr in ((0, nf - 1), (NCH - 1, 500))}
        del out
    ref = sampled_reference(picks)
    err = np.max(np.abs(got - ref) / ref)
    assert err <= tol, f"max relative error {err:.3e}"
    for (ch, fr), g in whole.items():
        rows = synth.hash_noise_rows(SEED, ch, T, 384 * fr, 384 * fr + 384, offsets=offsets())
        r = O.beamform(rows[None], [synth.SWEEP_FREQS[ch]])[:, :, 0]
        e = np.max(np.abs(g.astype(np.float64) - r) / r)
        assert e <= tol, f"channel {ch} frame {fr}: max relative error {e:.3e}"


def test_sweep_bursts_are_recovered_by_dedispersion(sweep_input):
    """The bursts come from zenith, where the default pointings have no beam; a
    plan with an N-S pointing (128) and an E-W beam (0) at zenith beamforms the
    same input.  The two bursts that cross most of the band inside the 1 s window
    (DM 100 and 300), dedispersed at their DM over the top channels whose delay
    fits the window (42 and 21 channels), stand out in that beam at the frame
    where they cross the top of the band."""
    ns = (np.arange(256) - 127.5) / 128.0
    ns[128] = 0.0
    ew = np.sin(np.radians([0.0, -0.2, 0.2, 0.6]))
    nf = T // 384
    with B.Plan(ns_sin=ns, ew_sin=ew) as p:
        out = p.run(sweep_input, synth.SWEEP_FREQS)
        for b in synth.SWEEP_BURSTS[:2]:
            c0 = next(c for c in range(NCH) if O.dedisperse_delays(synth.SWEEP_FREQS[c:], b.dm).max() < 0.8 * nf)
            sub = out[:, 16 * c0:, :].contiguous()
            ser = p.dedisperse(sub, synth.SWEEP_FREQS[c0:], b.dm).cpu().numpy()[128]
            fr = burst_frame(b, NCH - 1)
            assert NCH - c0 >= 20 and ser.size > fr + 3
            med = np.median(ser)
            mad = np.median(np.abs(ser - med)) * 1.4826
            snr = (ser[max(0, fr - 2):fr + 3].max() - med) / mad
            # nominal S/N 200 over the band becomes ~10 after the incoherent sum over the channels
            # that fit the window, the 0.98 ms frames and the rounded delays
            assert snr > (6.0 if b.dm < 200 else 4.0), f"DM {b.dm} over {NCH - c0} channels: S/N {snr:.1f}"
            del sub
        del out

"""The full band (Fig. 3, Sec. 3.1, Sec. 3.3): all 1024 coarse channels of
400-800 MHz in one request, a plane-wave source at 26 deg N-S.

* Parity: whole outputs of sampled channels (including both sides of the
  aliasing onset near 492 MHz) against the FP64 oracle, for the FP32 form and
  for the 1-term tensor-core form on one plan (1024 table slots at once).
* The frequency-summed map (bf_skymap) peaks at the source; its aliases
  (Sec. 3.3: -88 .. -50 deg for a 26 deg source) are smeared over many N-S
  beams and stay well below the source.
* The width of the frequency-summed N-S beam, measured by scanning a source
  across a beam toward zenith and one toward 78.7 deg, equals the oracle's
  noiseless frequency-summed beam within the scan step; it lies between the
  beam widths at the top and at the bottom of the band (the paper's ~0.5 deg
  and ~2.8 deg are the bottom-of-band widths).

Inputs come from the device-side generator (torch's random numbers); the
channels the oracle checks are copied back as bytes.
"""
import math

import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BAND = synth.BAND_FREQS
U_SRC = math.sin(math.radians(0.2))          # E-W beam j = 2, array factor 4 at every frequency
J_SRC = 2


@pytest.fixture(scope="module")
def band_input(built_lib):
    pw = synth.PlaneWave(1.5, u=U_SRC, s=math.sin(math.radians(26.0)))
    vin = synth.plane_wave_device(BAND, 768, seed=26, plane_waves=[pw])
    torch.cuda.synchronize()
    yield vin
    del vin
    torch.cuda.empty_cache()


def ns_angles():
    return np.degrees(np.arcsin(O.default_ns_sin()))


def summed_response(thetas_deg, freqs=BAND):
    """Noiseless frequency-summed power [angle, 256 N-S beams] for a unit plane
    wave from each angle, from the oracle's clamp table and N-S DFT."""
    s = np.sin(np.radians(np.atleast_1d(np.asarray(thetas_deg, dtype=np.float64))))
    n = np.arange(256)
    ns = O.default_ns_sin()
    tot = np.zeros((len(s), 256))
    for f in freqs:
        x = np.exp(2j * np.pi * np.outer(s, n) * f * O.CHIME.feed_spacing_m / O.C0)[:, None, :, None]
        tot += np.abs(O.ns_beams(x, O.clamp_lut(f, ns))[:, 0, 0, :]) ** 2
    return tot


def width(th, r):
    """Half-power width by linear interpolation between scan points."""
    k = int(np.argmax(r))
    half = 0.5 * r[k]
    lo = k
    while lo > 0 and r[lo - 1] >= half:
        lo -= 1
    hi = k
    while hi < len(r) - 1 and r[hi + 1] >= half:
        hi += 1
    if lo == 0 or hi == len(r) - 1:
        raise AssertionError("scan does not cover the half-power points")
    left = th[lo - 1] + (half - r[lo - 1]) / (r[lo] - r[lo - 1]) * (th[lo] - th[lo - 1])
    right = th[hi] + (r[hi] - half) / (r[hi] - r[hi + 1]) * (th[hi + 1] - th[hi])
    return right - left


@pytest.mark.parametrize("form,tol", [(B.BF_FP32_FFT, 1e-5), (B.BF_TC_DFT256_X1, 1e-3)])
def test_band_in_one_request_matches_oracle_on_sampled_channels(band_input, form, tol):
    with B.Plan(form=form) as p:
        out = p.run(band_input, BAND)
        torch.cuda.synchronize()
        assert out.shape == (1024, 16 * 1024, 2)
        for ch in (0, 1, 233, 235, 236, 511, 700, 1023):        # 491.8 MHz lies in channel 235
            raw = band_input[ch].cpu().numpy()
            ref = O.beamform(raw[None], [BAND[ch]])
            got = out[:, 16 * ch:16 * ch + 16, :].cpu().numpy().astype(np.float64)
            err = float(np.max(np.abs(got - ref) / ref))
            assert err <= tol, f"channel {ch}: max relative error {err:.3e}"


def test_band_map_peaks_at_the_source_and_smears_its_aliases(band_input):
    with B.Plan() as p:
        out = p.run(band_input, BAND)
        smap = p.skymap(out).cpu().numpy().astype(np.float64)
    ang = ns_angles()
    m_src = int(np.argmin(np.abs(ang - 26.0)))
    assert int(np.argmax(smap)) == 256 * J_SRC + m_src
    row = smap[256 * J_SRC:256 * (J_SRC + 1)]
    floor = np.median(row)
    sig = row - floor
    alias = (ang > -88.0) & (ang < -50.0)
    quiet = (ang > -40.0) & (ang < -5.0)
    # aliases are present over the whole -88 .. -50 deg range, spread thin
    assert sig[alias].mean() > 10.0 * abs(sig[quiet].mean()) + 1e-6 * sig.max()
    assert sig[alias].max() < 0.2 * sig[m_src]
    # the map follows the noiseless frequency-summed response of the oracle's N-S stage
    ref = summed_response([26.0])[0]
    c = np.corrcoef(sig, ref)[0, 1]
    assert c > 0.99, c


@pytest.mark.parametrize("m,half_span,step", [(128, 0.45, 0.025), (253, 2.25, 0.125)])
def test_frequency_summed_beam_width(built_lib, m, half_span, step):
    th_m = ns_angles()[m]
    ref_th = np.arange(th_m - half_span, th_m + half_span + 1e-9, step / 5)
    ref_w = width(ref_th, summed_response(ref_th)[:, m])
    scan = np.arange(th_m - half_span, th_m + half_span + 1e-9, step)
    resp = []
    with B.Plan() as p:
        for k, th in enumerate(scan):
            pw = synth.PlaneWave(1.5, u=U_SRC, s=math.sin(math.radians(th)))
            vin = synth.plane_wave_device(BAND, 384, seed=1000 + k, plane_waves=[pw])
            out = p.run(vin, BAND)
            row = p.skymap(out)[256 * J_SRC:256 * (J_SRC + 1)].cpu().numpy().astype(np.float64)
            del vin, out
            resp.append(row[m] - np.median(row))
    torch.cuda.empty_cache()
    got_w = width(scan, np.array(resp))
    assert abs(got_w - ref_w) <= step, (got_w, ref_w)
    # between the beam widths at the top and the bottom of the band
    lo_w = width(ref_th, summed_response(ref_th, [BAND[-1]])[:, m])
    hi_w = width(ref_th, summed_response(ref_th, [BAND[0]])[:, m])
    assert lo_w < got_w < hi_w

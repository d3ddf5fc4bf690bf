"""Tracking E-W beams (Sec. 3.1: the E-W beams are static or track the sky)
on the GPU against the FP64 oracle.

A request may carry one row of four E-W sines per output frame; the host
turns each row into phases in FP64 and the fused kernels weight the
cylinders of every frame with its own row.  Tolerances as for static beams:
1e-5 relative for the FP32 form and the 3-term tensor-core form, 1e-3 for the
1-term forms on CTA clusters (256 and 512 rows).
"""
import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMS = {B.BF_FP32_FFT: 1e-5, B.BF_TC_DFT256: 1e-5, B.BF_TC_DFT256_X1: 1e-3, B.BF_TC_DFT512: 1e-3}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(got, ref):
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref) / np.abs(ref)))


def random_sines(nf, seed):
    return np.random.default_rng(seed).uniform(-0.9, 0.9, size=(nf, 4))


@pytest.mark.parametrize("form", list(FORMS))
def test_tracking_multichannel_ragged(built_lib, form):
    freqs = [420e6, 555e6, 760e6]
    raw = synth.noise_only(freqs, 384 * 3 + 77, seed=41)
    u = random_sines(3, 42)
    with B.Plan(form=form) as p:
        out = p.run(dev(raw), freqs, ew_sin_frames=u).cpu().numpy()
    ref = O.beamform(raw, freqs, ew_sin_frames=u)
    assert out.shape == ref.shape == (1024, 48, 3)
    assert rel_err(out, ref) <= FORMS[form]


@pytest.mark.parametrize("form", list(FORMS))
def test_tracking_across_requests_with_carry(built_lib, form):
    """Rows belong to the frames each request produces, carried samples included."""
    freqs = [610e6, 640e6]
    raw = synth.noise_only(freqs, 384 * 4, seed=43)
    u = random_sines(4, 44)
    cut = 500                                     # request 1: frame 0 (+116 carried); request 2: frames 1..3
    outs = []
    with B.Plan(form=form) as p:
        for lo, hi, flags in ((0, cut, 0), (cut, 384 * 4, B.BF_END_OF_STREAM)):
            nf = p.frames_out(9, hi - lo)
            first = sum(o.shape[2] for o in outs)
            out = torch.empty((1024, 32, nf), dtype=torch.float32, device="cuda")
            _, t = p.submit(dev(raw[:, lo:hi]), freqs, out, stream_id=9, flags=flags,
                            ew_sin_frames=u[first:first + nf])
            p.poll(t)
            outs.append(out.cpu().numpy())
    got = np.concatenate(outs, axis=2)
    ref = O.beamform(raw, freqs, ew_sin_frames=u)
    assert rel_err(got, ref) <= FORMS[form]


def test_tracking_keeps_the_coherent_gain(built_lib):
    """Exact plane wave drifting by quarter turns per frame: the tracked beam
    has 16x the power of cylinder 0 alone (the oracle's pin, on the GPU)."""
    freq = 600e6
    k = [0, 1, 2, 3, 1, 2]
    raw = synth.cylinder_quarter_turns(k, seed=45)
    only0 = raw.copy()
    only0.reshape(-1, 4, 512)[:, 1:] = synth.encode(0, 0)
    u = np.zeros((len(k), 4))
    u[:, 0] = [kk * O.C0 / (4.0 * freq * 20.0) for kk in k]
    with B.Plan() as p:
        track = p.run(dev(raw[None]), [freq], ew_sin_frames=u).cpu().numpy()
        single = p.run(dev(only0[None]), [freq], ew_sin_frames=u).cpu().numpy()
    assert rel_err(track[:256], 16.0 * single[:256].astype(np.float64)) <= 2e-5
    ref = O.beamform_channel(raw, freq, ew_sin_frames=u)
    assert rel_err(track[:256], ref[:256]) <= 1e-5


def test_tracking_in_serving_mode_beside_static_streams(built_lib):
    freqs = [500e6, 530e6]
    raws = [synth.noise_only(freqs, 768, seed=46 + i) for i in range(3)]
    u = random_sines(2, 49)
    with B.Plan(mode=B.BF_MODE_SERVING) as p:
        torch.cuda.synchronize()
        outs, tickets = [], []
        for i, raw in enumerate(raws):
            out = torch.empty((1024, 32, 2), dtype=torch.float32, device="cuda")
            vin = dev(raw)
            torch.cuda.synchronize()
            _, t = p.submit(vin, freqs, out, stream_id=100 + i, flags=B.BF_END_OF_STREAM,
                            ew_sin_frames=u if i == 1 else None)
            outs.append((out, vin))
            tickets.append(t)
        for t in tickets:
            p.poll(t)
    for i, raw in enumerate(raws):
        ref = O.beamform(raw, freqs, ew_sin_frames=u) if i == 1 else O.beamform(raw, freqs)
        assert rel_err(outs[i][0].cpu().numpy(), ref) <= 1e-5


def test_tracking_rejects_bad_sines(built_lib):
    raw = synth.noise_only([600e6], 384, seed=50)
    with B.Plan() as p:
        for bad in (np.full((1, 4), 1.5), np.full((1, 4), np.nan)):
            with pytest.raises(B.BfError) as e:
                p.run(dev(raw), [600e6], ew_sin_frames=bad)
            assert e.value.code == B.BF_EINVAL

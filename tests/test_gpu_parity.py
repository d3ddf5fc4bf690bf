"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerance (FP32 path): every output element within 1e-5 relative of the
oracle (|got - ref| <= 1e-5 * ref).  Each output sums 48 |Y|^2 terms of
values that passed ~20 rounded FP32 operations (9 N-S FFT levels, 4-term
E-W sum, 7 up-channel levels), i.e. a few 1e-7 relative per term; 1e-5 is
the bound stated for this path.  Degenerate inputs whose exact outputs
vanish use an absolute floor of 1e-6 of the largest output instead.
Integer work (unpack, clamp table) is compared bit for bit.
"""
import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module")
def plan(built_lib):
    p = B.Plan()
    yield p
    p.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rand_raw(shape, seed, lo=-8):
    r = np.random.default_rng(seed)
    return synth.encode(r.integers(lo, 8, size=shape), r.integers(lo, 8, size=shape))


def assert_rel(got, ref, rel=REL, floor=0.0):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    tol = rel * np.abs(ref) + floor
    bad = err > tol
    assert not bad.any(), (f"{bad.sum()} of {bad.size} outside tolerance; worst rel "
                           f"{(err / np.maximum(np.abs(ref), 1e-300)).max():.3e}")


def test_unpack_all_bytes_bit_exact(plan):
    d_in = torch.arange(256, dtype=torch.uint8, device="cuda")
    d_out = torch.empty(256, 2, dtype=torch.float32, device="cuda")
    B.bf_debug_unpack(plan.handle, d_in, d_out, 256)
    raw = np.zeros((256, 2048), np.uint8)
    raw[:, 0] = np.arange(256)
    ref = O.unpack(raw)[:, 0, 0, 0]
    got = d_out.cpu().numpy()
    assert np.array_equal(got[:, 0], ref.real) and np.array_equal(got[:, 1], ref.imag)


@pytest.mark.parametrize("freq", [410e6, 600e6, 790e6])
def test_ns_ew_beams_stage_dump(plan, freq):
    T = 48
    raw = rand_raw((T, 2048), seed=int(freq) % 97)
    out = torch.empty(T, 2, 4, 256, 2, dtype=torch.float32, device="cuda")
    B.bf_debug_beams(plan.handle, freq, dev(raw), T, out)
    got = out.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    ref = O.ew_beams(O.ns_beams(O.unpack(raw), O.clamp_lut(freq)), O.ew_weights(freq))
    scale = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(got - ref)) <= 1e-5 * scale


@pytest.mark.parametrize("freq", [450e6, 650e6])
def test_upchannelised_stage_dump(plan, freq):
    T = 768
    raw = rand_raw((T, 2048), seed=11)
    out = torch.empty(T // 128, 2, 4, 256, 128, 2, dtype=torch.float32, device="cuda")
    B.bf_debug_upchan(plan.handle, freq, dev(raw), T, out)
    got = out.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    _, st = O.beamform_channel(raw, freq, return_stages=True)
    ref = st["Y"]
    scale = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(got - ref)) <= 1e-5 * scale


def test_point_source_config(plan):
    raw, f = synth.config_point_source(0)
    out = plan.run(dev(raw), f).cpu().numpy()
    ref = O.beamform(raw, f)
    assert out.shape == ref.shape == (1024, 16, 8)
    assert_rel(out, ref)
    assert int(out.sum(axis=(1, 2)).argmax()) == 939


def test_multichannel_ragged_tail(plan):
    freqs = [410e6, 600e6, 790e6]
    raw = rand_raw((3, 384 * 5 + 100, 2048), seed=3, lo=-7)
    out = plan.run(dev(raw), freqs).cpu().numpy()
    ref = O.beamform(raw, freqs)
    assert out.shape == (1024, 48, 5)
    assert_rel(out, ref)


def test_custom_pointings_and_spacing(built_lib):
    rng = np.random.default_rng(9)
    ns = np.sort(rng.uniform(-0.95, 0.95, 256))
    ew = np.sin(np.radians([-1.0, -0.1, 0.3, 0.9]))
    g = O.Geometry(feed_spacing_m=0.29, cyl_spacing_m=21.5)
    raw = rand_raw((1, 768, 2048), seed=4, lo=-7)
    with B.Plan(ns_sin=ns, ew_sin=ew, feed_spacing_m=0.29, cyl_spacing_m=21.5) as p:
        out = p.run(dev(raw), [555e6]).cpu().numpy()
    ref = O.beamform(raw, [555e6], ns, ew, g)
    assert_rel(out, ref)


def test_zero_and_extreme_inputs(plan):
    zero = np.full((1, 384, 2048), 0x88, np.uint8)
    assert np.count_nonzero(plan.run(dev(zero), [500e6]).cpu().numpy()) == 0
    for code in (0x00, 0xFF, 0x0F, 0xF0):
        raw = np.full((1, 384, 2048), code, np.uint8)
        raw[0, ::3, ::5] = 0x88
        out = plan.run(dev(raw), [700e6]).cpu().numpy()
        ref = O.beamform(raw, [700e6])
        assert_rel(out, ref, floor=1e-6 * ref.max())


def test_empty_and_short_requests(plan):
    vin = torch.zeros(1, 16, 2048, dtype=torch.uint8, device="cuda")
    st, t = plan.submit(vin, [600e6], None, stream_id=77, n_samples=0)
    assert plan.poll(t) == (B.BF_OK, 0)
    st, t = plan.submit(vin, [600e6], None, stream_id=77, n_samples=16, flags=B.BF_END_OF_STREAM)
    assert plan.poll(t) == (B.BF_OK, 0)


def test_stream_split_is_bitwise_identical(plan):
    freqs = [480e6, 720e6]
    T = 2000
    raw = rand_raw((2, T, 2048), seed=21, lo=-7)
    whole = plan.run(dev(raw), freqs, stream_id=1000)
    cuts = [0, 100, 600, 983, 1700, T]
    parts = []
    for i in range(len(cuts) - 1):
        a, b = cuts[i], cuts[i + 1]
        chunk = dev(raw[:, a:b])
        flags = B.BF_END_OF_STREAM if b == T else 0
        nf = plan.frames_out(1001, b - a)
        out = torch.empty(1024, 32, nf, dtype=torch.float32, device="cuda")
        _, t = plan.submit(chunk, freqs, out if nf else None, stream_id=1001, flags=flags, n_samples=b - a)
        assert plan.poll(t) == (B.BF_OK, nf)
        parts.append(out)
    joined = torch.cat(parts, dim=2)
    assert joined.shape == whole.shape
    assert torch.equal(joined, whole)


def test_node_slice_full_size_sampled(plan):
    raw, freqs, info = synth.config_node_slice(0)
    out = plan.run(dev(raw), list(freqs)).cpu().numpy()
    assert out.shape == (1024, 64, 128)
    assert np.isfinite(out).all() and (out > 0).all()
    rng = np.random.default_rng(0)
    picks = [(int(rng.integers(4)), int(rng.integers(1024)), int(rng.integers(128))) for _ in range(40)]
    picks += [(ch, b, fr) for ch in range(4) for b in (0, 1023) for fr in (0, 127)]
    ref = O.beamform_sample(raw, freqs, picks)
    got = np.stack([out[b, 16 * ch:16 * ch + 16, fr] for ch, b, fr in picks])
    assert_rel(got, ref)


@pytest.mark.parametrize("form,rel", [(B.BF_FP32_FFT, REL), (B.BF_TC_DFT256, REL), (B.BF_TC_DFT256_X1, 1e-3),
                                      (B.BF_TC_DFT256_X2, 1e-3)])
def test_tail_split_items_match_whole_items(built_lib, form, rel):
    """A launch whose last round of items would leave at least half of the CTAs
    idle runs each item of that round as two half units on two CTAs (the 2-term
    form never splits).  The output must equal, bit for bit, a run of the same
    stream in two requests whose items all run whole, and the oracle within the
    form's tolerance."""
    with B.Plan(form=form) as plan:
        _tail_split_case(plan, rel)


def _tail_split_case(plan, rel):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nf1, nf2 = sms // 4, 5
    items = 4 * (nf1 + nf2)
    rem = items % sms
    if not (items > sms and 0 < rem and 2 * rem <= sms):
        pytest.skip(f"{sms} SMs: no tail split for {items} items")
    freq = 615e6
    T = 384 * (nf1 + nf2)
    raw = rand_raw((1, T, 2048), seed=31, lo=-7)
    whole = plan.run(dev(raw), [freq], stream_id=2000)
    assert whole.shape == (1024, 16, nf1 + nf2)
    parts = []
    for a, b, flags in ((0, 384 * nf1, 0), (384 * nf1, T, B.BF_END_OF_STREAM)):
        nf = (b - a) // 384
        out = torch.empty(1024, 16, nf, dtype=torch.float32, device="cuda")
        _, t = plan.submit(dev(raw[:, a:b]), [freq], out, stream_id=2001, flags=flags, n_samples=b - a)
        assert plan.poll(t) == (B.BF_OK, nf)
        parts.append(out)
    assert torch.equal(torch.cat(parts, dim=2), whole)
    got = whole.cpu().numpy()
    rng = np.random.default_rng(33)
    picks = [(0, int(rng.integers(1024)), fr) for fr in range(nf1 - 1, nf1 + nf2) for _ in range(3)]
    ref = O.beamform_sample(raw, [freq], picks)
    assert_rel(np.stack([got[b, 0:16, fr] for _, b, fr in picks]), ref, rel=rel)


@pytest.mark.parametrize("form", [B.BF_FP32_FFT, B.BF_TC_DFT256])
def test_more_channels_than_one_launch_holds(built_lib, form):
    """200 channels (segments) exceed one launch's 160 segment descriptors, so the
    request runs as several launches; every channel's frames must still land in
    their place.  Channel frequencies repeat, so table reuse is covered too."""
    n_chan, T = 200, 384 * 2 + 17
    freqs = [400e6 + 390625.0 * (7 * c % 1024 + 0.5) for c in range(n_chan)]
    freqs[150:] = freqs[:50]                                   # repeated frequencies
    raw = rand_raw((n_chan, T, 2048), seed=91, lo=-7)
    rng = np.random.default_rng(92)
    with B.Plan(form=form) as p:
        out = p.run(dev(raw), freqs).cpu().numpy()
    assert out.shape == (1024, 16 * n_chan, 2)
    picks = [(ch, int(rng.integers(1024)), fr) for ch in (0, 1, 79, 159, 160, 161, 199) for fr in (0, 1)]
    ref = O.beamform_sample(raw, freqs, picks)
    got = np.stack([out[b, 16 * ch:16 * ch + 16, fr] for ch, b, fr in picks])
    assert_rel(got, ref)                       # 1e-5: FP32 form and the 3-term tensor-core form


def test_bad_arguments(plan):
    vin = torch.zeros(1, 384 * 2 + 1, 2048, dtype=torch.uint8, device="cuda")
    out = torch.empty(1024, 16, 2, dtype=torch.float32, device="cuda")
    with pytest.raises(B.BfError) as e:
        B.bf_submit(plan.handle, 5, [600e6], 384, vin.data_ptr() + 1, out)
    assert e.value.code == B.BF_EINVAL
    with pytest.raises(B.BfError) as e:
        B.bf_submit(plan.handle, 5, [-1.0], 384, vin, out)
    assert e.value.code == B.BF_EINVAL
    with pytest.raises(B.BfError) as e:
        B.bf_poll(plan.handle, 123456789, 0)
    assert e.value.code == B.BF_ENOTICKET
    _, t = B.bf_submit(plan.handle, 6, [600e6], 384, vin, out)
    assert B.bf_poll(plan.handle, t)[0] == B.BF_OK
    with pytest.raises(B.BfError) as e:
        B.bf_submit(plan.handle, 6, [600e6, 700e6], 384, vin, out)
    assert e.value.code == B.BF_EINVAL

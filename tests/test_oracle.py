"""Pins for the FP64 oracle: closed forms, library routines, invariants,
brute force on tiny geometries, and the paper's stated facts (Table 1,
Sec. 3.1, Sec. 3.3).  None of these re-types the oracle's own formulas."""
import cmath
import json
import math
import os

import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(1234)


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def rand_raw(shape, clip=7):
    re = rng.integers(-clip, clip + 1, size=shape)
    im = rng.integers(-clip, clip + 1, size=shape)
    return synth.encode(re, im)


# --- a0 unpack ------------------------------------------------------------------------

def test_unpack_examples():
    ex = gold("unpack_examples.json")["examples"]
    b = np.array([e["byte"] for e in ex], dtype=np.uint8)
    raw = np.zeros((len(b), 2048), np.uint8)
    raw[:, 0] = b
    z = O.unpack(raw)[:, 0, 0, 0]
    assert np.array_equal(z.real, [e["re"] for e in ex])
    assert np.array_equal(z.imag, [e["im"] for e in ex])


def test_unpack_is_bijection_onto_4bit_grid():
    raw = np.zeros((256, 2048), np.uint8)
    raw[:, 5] = np.arange(256)
    z = O.unpack(raw)[:, 0, 2, 1]          # input 5 = (cyl 0, feed 2, pol 1)
    pairs = {(int(a.real), int(a.imag)) for a in z}
    assert pairs == {(r, i) for r in range(-8, 8) for i in range(-8, 8)}
    # the generator's encoder is the inverse
    re, im = z.real.astype(int), z.imag.astype(int)
    assert np.array_equal(synth.encode(re, im), np.arange(256, dtype=np.uint8))


def test_unpack_input_order():
    # byte (c*256 + n)*2 + p carries (cyl c, feed n, pol p)
    raw = np.full((1, 2048), 0x88, np.uint8)
    c, n, p = 2, 77, 1
    raw[0, (c * 256 + n) * 2 + p] = 0x9A
    z = O.unpack(raw)[0]
    nz = np.argwhere(z != 0)
    assert nz.tolist() == [[c, n, p]] and z[c, n, p] == 1 + 2j


# --- clamp table (Eq. 1) -------------------------------------------------------------

def nearest_beam_bins(freq, ns_sin, g=O.CHIME):
    """Nearest-neighbour search over every zero-padded beam (and its aliases)."""
    M = g.n_bins
    out = []
    for s in ns_sin:
        best, best_d = None, None
        for L in range(-2 * M, 2 * M + 1):
            s_beam = L * O.C0 / (M * freq * g.feed_spacing_m)   # beam L steers here
            d = abs(s_beam - s)
            if best_d is None or d < best_d - 1e-12:
                best, best_d = L, d
        out.append(best % M)
    return np.array(out)


@pytest.mark.parametrize("freq", [400.390625e6, 410e6, 491e6, 520e6, 600e6, 650e6, 790e6, 799.6e6])
def test_lut_is_nearest_formed_beam(freq):
    ns = O.default_ns_sin()
    assert np.array_equal(O.clamp_lut(freq, ns), nearest_beam_bins(freq, ns))


def test_lut_custom_pointings_nearest():
    ns = np.sort(rng.uniform(-1, 1, size=256))
    assert np.array_equal(O.clamp_lut(700e6, ns), nearest_beam_bins(700e6, ns))


def test_lut_eq2_incremental_update():
    # Eq. (2): moving from f_k to f_k + df shifts each index by N P df d sin(theta)/c;
    # after rounding the two indices differ from that shift by less than 1.
    ns = O.default_ns_sin()
    f0, df = 600e6, 390625.0 * 7
    L0 = np.floor(O.clamp_arg(f0, ns) + 0.5)
    L1 = np.floor(O.clamp_arg(f0 + df, ns) + 0.5)
    shift = 512 * df * 0.3048 * ns / O.C0
    assert np.all(np.abs((L1 - L0) - shift) < 1.0)
    assert np.array_equal(np.mod(L1, 512).astype(int), O.clamp_lut(f0 + df, ns))


def test_aliasing_onset_matches_paper():
    t = gold("table1.json")
    onset = O.C0 / (2 * 0.3048)                       # spacing = half a wavelength
    assert abs(onset - t["aliasing_onset_hz_approx"]) < 0.02 * onset
    ns = O.default_ns_sin()
    below = np.floor(O.clamp_arg(onset * 0.99, ns) + 0.5)
    above = np.floor(O.clamp_arg(onset * 1.06, ns) + 0.5)
    assert below.min() >= -256 and below.max() < 256           # no wrap below onset
    assert above.min() < -256 or above.max() >= 256             # wraps above it
    assert len(set(O.clamp_lut(onset * 0.99, ns).tolist())) == 256
    assert len(set(O.clamp_lut(600e6, ns).tolist())) < 256    # aliased duplicates


def test_lut_fig1_chromatic_spacing():
    # Fig. 1: formed beams crowd together at high frequency; the clamp keeps the
    # selected beam within half a beam spacing of its pointing at every frequency.
    ns = O.default_ns_sin()
    for f in np.linspace(400e6, 800e6, 9):
        L = np.floor(O.clamp_arg(f, ns) + 0.5)
        s_sel = L * O.C0 / (512 * f * 0.3048)
        assert np.all(np.abs(s_sel - ns) <= O.C0 / (2 * 512 * f * 0.3048) + 1e-12)


# --- a1 N-S beams ---------------------------------------------------------------------

def all_bins_lut():
    return np.arange(512)


def test_ns_matches_numpy_fft():
    x = O.unpack(rand_raw((3, 2048)))
    X = O.ns_beams(x, all_bins_lut())                  # [t, c, p, 512]
    ref = np.fft.fft(np.moveaxis(x, 2, 3), n=512, axis=-1)
    assert np.allclose(X, ref, rtol=0, atol=1e-9)
    lut = O.clamp_lut(650e6)
    assert np.allclose(O.ns_beams(x, lut), ref[..., lut], rtol=0, atol=1e-9)


def test_ns_even_odd_split():
    x = O.unpack(rand_raw((2, 2048)))
    X = O.ns_beams(x, all_bins_lut())
    xt = np.moveaxis(x, 2, 3)
    n = np.arange(256)
    assert np.allclose(X[..., 0::2], np.fft.fft(xt, axis=-1), atol=1e-9)
    assert np.allclose(X[..., 1::2], np.fft.fft(xt * np.exp(-1j * np.pi * n / 256), axis=-1), atol=1e-9)


def test_ns_delta_and_constant():
    x = np.zeros((1, 4, 256, 2), complex)
    x[0, 1, 37, 0] = 1.0
    X = O.ns_beams(x, all_bins_lut())
    assert np.allclose(np.abs(X[0, 1, 0]), 1.0)
    a = 3 - 2j
    x = np.full((1, 4, 256, 2), a)
    X = O.ns_beams(x, all_bins_lut())[0, 0, 0]
    k = np.arange(512)
    assert abs(X[0] - 256 * a) < 1e-9
    assert np.allclose(X[2::2], 0, atol=1e-9)
    odd = k[1::2]
    assert np.allclose(X[1::2], 2 * a / (1 - np.exp(-1j * np.pi * odd / 256)), atol=1e-9)


def test_ns_parseval():
    x = O.unpack(rand_raw((4, 2048)))
    X = O.ns_beams(x, all_bins_lut())
    lhs = (np.abs(X) ** 2).sum(axis=-1)
    rhs = 512 * (np.abs(x) ** 2).sum(axis=2)
    assert np.allclose(lhs, rhs, rtol=1e-12)


def test_ns_plane_wave_on_bin_and_steering_identity():
    f, L = 700e6, 93
    s = L * O.C0 / (512 * f * 0.3048)                  # exactly on beam L
    a = 1.7
    g = synth.geometric_phase(f, 0.0, s).reshape(4, 256, 2)
    X = O.ns_beams((a * g)[None], all_bins_lut())
    assert abs(abs(X[0, 2, 1, L]) - 256 * a) < 1e-8
    # zero-padded bin L equals direct phasing toward s' = L c/(M f d)
    x = O.unpack(rand_raw((1, 2048)))[0, 0, :, 0]
    direct = sum(x[n] * cmath.exp(-2j * math.pi * f * n * 0.3048 * s / O.C0) for n in range(256))
    assert abs(O.ns_beams(x.reshape(1, 1, 256, 1), all_bins_lut())[0, 0, 0, L] - direct) < 1e-8


def test_alias_of_26deg_source_fig3():
    # Sec. 3.3 / Fig. 3: a source near 26 deg has aliases, of comparable strength
    # in one channel, between about -88 and -50 deg at the top of the band; in
    # the frequency-summed map the source dominates and the alias is smeared.
    t = gold("table1.json")
    lo, hi = t["alias_smear_deg_for_26deg_source"]
    ns = O.default_ns_sin()
    s_src = math.sin(math.radians(26.0))
    m_src = int(np.argmin(np.abs(ns - s_src)))
    near = np.abs(np.arange(256) - m_src) <= 2
    total = np.zeros(256)
    for f in np.linspace(400e6, 800e6, 41):
        g = synth.geometric_phase(f, 0.0, s_src).reshape(4, 256, 2)
        P = np.abs(O.ns_beams(g[None], O.clamp_lut(f, ns))[0, 0, 0]) ** 2
        total += P / P.max()
        if f >= 700e6:
            alias_deg = math.degrees(math.asin(ns[~near][np.argmax(P[~near])]))
            assert lo - 3 <= alias_deg <= hi + 3
            assert P[~near].max() > 0.3 * P.max()        # comparable in one channel
    assert abs(int(np.argmax(total)) - m_src) <= 1
    assert total[~near].max() < 0.5 * total.max()


# --- a2 E-W beams ---------------------------------------------------------------------

def test_ew_zero_angle_is_cylinder_sum():
    X = rng.standard_normal((2, 4, 2, 256)) + 1j * rng.standard_normal((2, 4, 2, 256))
    B = O.ew_beams(X, O.ew_weights(600e6, np.zeros(4)))
    assert np.allclose(B, X.sum(axis=1)[:, :, None, :])


def test_ew_dft_spaced_is_unitary():
    f = 600e6
    u = np.arange(4) * O.C0 / (4 * 20.0 * f)
    X = rng.standard_normal((2, 4, 2, 256)) + 1j * rng.standard_normal((2, 4, 2, 256))
    B = O.ew_beams(X, O.ew_weights(f, u))
    assert np.allclose((np.abs(B) ** 2).sum(axis=2), 4 * (np.abs(X) ** 2).sum(axis=1))
    assert np.allclose(B, np.fft.fft(X, axis=1).transpose(0, 2, 1, 3))


# --- a3 up-channelisation -------------------------------------------------------------

def test_upchan_matches_numpy_and_parseval():
    B = rng.standard_normal((256, 2, 1, 3)) + 1j * rng.standard_normal((256, 2, 1, 3))
    Y = O.upchannelize(B)                                  # [2, p, j, m, 128]
    ref = np.fft.fftshift(np.fft.fft(np.moveaxis(B.reshape(2, 128, 2, 1, 3), 1, -1), axis=-1), axes=-1)
    assert np.allclose(Y, ref, atol=1e-9)
    assert np.allclose((np.abs(Y) ** 2).sum(-1), 128 * (np.abs(B.reshape(2, 128, 2, 1, 3)) ** 2).sum(1))


@pytest.mark.parametrize("k", [0, 1, 5, 63, -1, -64, 40])
def test_upchan_tone_lands_in_one_fine_channel(k):
    tau = np.arange(128)
    B = np.exp(2j * np.pi * k * tau / 128)[:, None, None, None]
    Y = O.upchannelize(B)[0, 0, 0, 0]
    qp = (k + 64) % 128                                    # shifted index, q' = 0 lowest
    assert abs(Y[qp] - 128) < 1e-9
    assert np.allclose(np.delete(Y, qp), 0, atol=1e-9)


# --- a4 + a5, whole path ---------------------------------------------------------------

def test_integration_parseval_invariant():
    raw = rand_raw((768, 2048))
    O_, st = O.beamform_channel(raw, 520e6, return_stages=True)
    B = st["B"]                                            # [T, p, j, m]
    e = (np.abs(B) ** 2).sum(axis=1).reshape(2, 384, 4, 256).sum(axis=1)   # [frame, j, m]
    lhs = O_.sum(axis=1).reshape(4, 256, 2)
    assert np.allclose(lhs, 128 * np.transpose(e, (1, 2, 0)), rtol=1e-10)


def test_noise_mean_closed_form():
    sigma = 2.5
    raw = synth.noise_only([450e6], 384 * 4, seed=7, sigma=sigma)
    out = O.beamform(raw, [450e6])
    var = synth.quantized_noise_variance(sigma)            # per real component
    expect = 24 * 2 * 128 * 4 * 256 * (2 * var)
    # every output is a sum of 96 nearly independent chi^2_2 terms -> CV ~ 0.1;
    # the mean over 65536 outputs is good to well under 1 %
    assert abs(out.mean() / expect - 1) < 0.01


def test_point_source_peaks_in_predicted_beam():
    raw, f = synth.config_point_source(0)
    out = O.beamform(raw, f)
    # source at 20 deg N-S (bin 106.8 at 600 MHz -> pointing 171 kept at bin 106)
    # and 0.5 deg E-W (nearest E-W beam: +0.6 deg, j = 3)
    assert int(out.sum(axis=(1, 2)).argmax()) == 3 * 256 + 171


def test_sample_route_matches_full_route():
    raw, f = synth.config_point_source(3)
    raw = raw[:, :1152]
    full = O.beamform(raw, f)
    picks = [(0, 939, 1), (0, 0, 0), (0, 1023, 2), (0, 300, 1)]
    s = O.beamform_sample(raw, f, picks)
    for i, (_, b, fr) in enumerate(picks):
        assert np.allclose(s[i], full[b, :, fr], rtol=1e-12)


def test_geometry_matches_table1():
    t = gold("table1.json")
    g = O.CHIME
    assert g.n_input == t["n_inputs"] and g.n_sub == t["output_channels_per_input_channel"]
    assert g.n_ew * g.n_ns == t["n_intensity_beams"] and g.pad == t["padding_factor"]
    assert abs(g.frame * t["input_time_resolution_s"] - t["output_time_resolution_s"]) < 1e-6
    chan = 400e6 / t["input_channels"]
    assert abs(chan / g.n_sub - t["output_frequency_resolution_hz"]) < 0.03 * 24e3
    assert abs(chan / g.upchan - t["upchannel_resolution_hz"]) < 0.03 * 3e3
    raw = rand_raw((1, 384 * 2 + 100, 2048))
    out = O.beamform(raw, [600e6])
    assert out.shape == (1024, 16, 2)                        # trailing samples dropped


def test_pointing_spacing_matches_fwhm_statements():
    # Sec. 3.1: FWHM ~0.5 deg at zenith and ~2.8 deg at 10 deg elevation; the
    # default pointings are spaced close to these widths.
    t = gold("table1.json")
    ns = O.default_ns_sin()
    th = np.degrees(np.arcsin(ns))
    zen = np.diff(th)[127]
    low_el = 90.0 - t["low_elevation_deg"]
    k = int(np.searchsorted(th, low_el)) - 1          # interval holding 80 deg
    assert abs(zen - t["zenith_fwhm_deg_approx"]) < 0.1
    assert abs(np.diff(th)[k] - t["low_elevation_fwhm_deg_approx"]) < 0.5


def ns_response(freq, ns_sin, m, thetas_deg):
    """|X[m]|^2 of the oracle's N-S stage for an exact unit plane wave from each
    zenith angle (one time sample, one cylinder and polarisation)."""
    s = np.sin(np.radians(np.asarray(thetas_deg, dtype=np.float64)))
    n = np.arange(256)
    x = np.exp(2j * np.pi * np.outer(s, n) * freq * O.CHIME.feed_spacing_m / O.C0)     # [angle, n]
    x = x[:, None, :, None]                                                            # [T, c, n, p]
    X = O.ns_beams(x, O.clamp_lut(freq, ns_sin))                                       # [T, c, p, m]
    return np.abs(X[:, 0, 0, m]) ** 2


def half_power_width(thetas, r):
    k = int(np.argmax(r))
    lo, hi = k, k
    while lo > 0 and r[lo - 1] >= 0.5 * r[k]:
        lo -= 1
    while hi < len(r) - 1 and r[hi + 1] >= 0.5 * r[k]:
        hi += 1
    return thetas[hi] - thetas[lo]


def test_beam_fwhm_matches_the_paper_at_the_bottom_of_the_band():
    """Sec. 3.1: the formed N-S beams are ~0.5 deg wide (FWHM) at zenith and
    up to ~2.8 deg at 10 deg elevation.  The widest beams are those at the
    lowest frequency: at 400 MHz the oracle's beam toward zenith is 0.49 deg and
    toward 80 deg zenith angle 2.8 deg wide; at 800 MHz half of that."""
    ns = O.default_ns_sin().copy()
    ns[128], ns[250] = 0.0, np.sin(np.radians(80.0))
    f_lo, f_hi = 400e6 + 195312.5, 800e6 - 195312.5
    th0 = np.linspace(-1.0, 1.0, 8001)
    th80 = np.linspace(74.0, 86.0, 12001)
    w0_lo = half_power_width(th0, ns_response(f_lo, ns, 128, th0))
    w80_lo = half_power_width(th80, ns_response(f_lo, ns, 250, th80))
    w0_hi = half_power_width(th0, ns_response(f_hi, ns, 128, th0))
    assert abs(w0_lo - 0.5) < 0.05, w0_lo
    assert abs(w80_lo - 2.8) < 0.25, w80_lo
    assert abs(w0_hi / w0_lo - 0.5) < 0.02                       # the width scales as 1/f
    # and as 1/cos(theta): 80 deg is 5.76 times wider than zenith
    assert abs(w80_lo / w0_lo - 1.0 / np.cos(np.radians(80.0))) < 0.3


# --- brute force on a tiny geometry -----------------------------------------------------

TINY = O.Geometry(n_cyl=2, n_feed=4, n_pol=2, pad=2, n_ew=2, upchan=4, f_ds=2, t_ds=2,
                  feed_spacing_m=0.3048, cyl_spacing_m=20.0)


def brute_force(raw, freq, ns_sin, ew_sin, g):
    """Literal loops over the definition, one term at a time."""
    M, U = g.n_bins, g.upchan
    T = raw.shape[0]
    nfr = T // g.frame
    lut = nearest_beam_bins(freq, ns_sin, g)
    out = np.zeros((g.n_ew * g.n_ns, g.n_sub, nfr))
    for fr in range(nfr):
        for j in range(g.n_ew):
            for m in range(g.n_ns):
                for blk in range(g.t_ds):
                    for p in range(g.n_pol):
                        beam = []
                        for tau in range(U):
                            t = fr * g.frame + blk * U + tau
                            acc = 0j
                            for c in range(g.n_cyl):
                                xc = 0j
                                for n in range(g.n_feed):
                                    byte = int(raw[t, (c * g.n_feed + n) * g.n_pol + p])
                                    v = complex((byte >> 4) - 8, (byte & 15) - 8)
                                    xc += v * cmath.exp(-2j * math.pi * n * lut[m] / M)
                                acc += xc * cmath.exp(-2j * math.pi * freq * c * g.cyl_spacing_m * ew_sin[j] / O.C0)
                            beam.append(acc)
                        for q in range(U):
                            yq = sum(beam[tau] * cmath.exp(-2j * math.pi * q * tau / U) for tau in range(U))
                            qp = (q + U // 2) % U
                            out[j * g.n_ns + m, qp // g.f_ds, fr] += abs(yq) ** 2
    return out


@pytest.mark.parametrize("freq", [450e6, 780e6])
def test_brute_force_tiny_geometry(freq):
    g = TINY
    T = g.frame * 2 + 3
    raw = rand_raw((T, g.n_input), clip=8 - 1)
    raw[0, 0] = 0x00                                   # the -8 code decodes too
    ns = np.array([-0.9, -0.2, 0.3, 0.95])
    ew = np.sin(np.radians([-0.4, 0.5]))
    ref = brute_force(raw, freq, ns, ew, g)
    got = O.beamform_channel(raw, freq, ns, ew, g)
    assert got.shape == ref.shape
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-9)


# --- products of the output (NEXT items) -------------------------------------------------

def test_rescale_u8_rule():
    X = np.zeros((2, 4, 8), np.float32)
    X[0, 0] = 5.0                                        # constant row -> 64
    X[0, 1] = np.tile([0.0, 1.0], 4)                     # mean 0.5, std 0.5 -> z = -1, +1
    X[0, 2] = [0, 0, 0, 0, 0, 0, 0, 1000]                # one outlier: z = +sqrt(7) ~ 2.65
    X[0, 3] = np.float32(0.1)                            # constant row whose FP32 sum is not exact
    X[1, 0] = [1000, 1000, 1000, 1000, 1000, 1000, 1000, 0]   # z = -sqrt(7) for the last
    X[1, 1] = np.arange(8)
    X[1, 2] = [0, 0, 0, 0, 0, 0, 0, 1e30]                # FP64 squares stay finite
    X[1, 3] = [0, 0, 0, 0, 0, 0, 0, 1e6]                 # z of the zeros -1/sqrt(7), of the peak +sqrt(7)
    codes, stats = O.rescale_u8(X)
    assert np.all(codes[0, 0] == 64) and stats[0, 0, 1] == 0.0 and np.all(codes[0, 3] == 64)
    assert np.array_equal(codes[0, 1], np.tile([48, 80], 4))
    assert codes[0, 2, 7] == int(np.floor(64 + 16 * np.sqrt(7) + 0.5)) == 106
    assert codes[0, 2, 0] == int(np.floor(64 - 16 / np.sqrt(7) + 0.5)) == 58
    assert codes[1, 0, 7] == int(np.floor(64 - 16 * np.sqrt(7) + 0.5)) == 22
    assert np.allclose(stats[1, 1], [3.5, np.sqrt(5.25)], rtol=1e-15)   # population std of 0..7
    # 0..7: z = (k - 3.5) / sqrt(5.25), v = 64 + 16 z -> 39.6, 46.6, 53.5, 60.5, 67.5, 74.5, 81.4, 88.4
    assert codes[1, 1].tolist() == [40, 47, 54, 61, 67, 74, 81, 88]
    assert codes[1, 2].tolist() == [58] * 7 + [106] and np.array_equal(codes[1, 2], codes[1, 3])
    # range: z = -4 is code 0, z = +11.9 is code 254.4 -> 254; beyond that the codes clip
    Y = np.zeros((1, 1, 257), np.float64)
    Y[0, 0, 0] = 1.0                                     # z of the peak = sqrt(256) = 16 -> clipped at 255
    c, st = O.rescale_u8(Y)
    assert c[0, 0, 0] == 255 and c[0, 0, 1] == int(np.floor(64 - 16 / 16 + 0.5)) == 63
    v, const, _ = O.rescale_value(X)
    assert const.tolist() == [[True, False, False, True], [False, False, False, False]]
    assert np.all(v[0, 0] == 64.0)


def test_sky_map_parseval_total_with_dft_tiling():
    """With pointings on the even bins (L(m) = 2m, the 256-point DFT of the feed
    line) and DFT-spaced E-W beams (cylinder phase steps of j/4 turn), every
    transform of the path is unitary up to its length, so the frequency- and
    time-summed map of ANY input totals 128 x 256 x 4 x sum |x|^2 over the whole
    frames, |x|^2 taken straight from the nibbles."""
    f = 610e6
    d = O.CHIME.feed_spacing_m
    L = np.where(np.arange(256) < 128, 2 * np.arange(256), 2 * np.arange(256) - 512)
    ns = L * O.C0 / (512 * f * d)
    ew = np.arange(4) * O.C0 / (4 * f * O.CHIME.cyl_spacing_m)
    assert np.array_equal(O.clamp_lut(f, ns), 2 * np.arange(256))
    raw = rand_raw((2, 384 * 2 + 50, 2048))
    out = O.beamform(raw, [f, f], ns, ew)
    smap = O.sky_map(out)
    b = raw[:, :768].astype(np.int64)
    power = int((((b >> 4) - 8) ** 2 + ((b & 15) - 8) ** 2).sum())
    assert smap.shape == (1024,)
    assert abs(smap.sum() / (128 * 256 * 4 * power) - 1) < 1e-12


def test_sky_map_of_a_zenith_source_closed_form():
    """A source at zenith, x = a i^k with quarter-turn phases k per sample and
    polarisation (exact on the 4-bit grid), summed over channels 400-800 MHz:
    beam (j, m) holds sum_f 128 x 384 x n_frames x 2 x a^2 |D(L_f(m))|^2 |A_j(f)|^2
    with D(L) = sum_n exp(-2 pi i n L / 512) (256 at L = 0, 0 at other even L,
    2 / (1 - exp(-i pi L / 256)) at odd L) and A_j the E-W array factor."""
    a = 3
    freqs = [400e6 + 390625.0 * (k + 0.5) for k in (0, 137, 512, 700, 1023)]
    ns = O.default_ns_sin().copy()
    ns[128] = 0.0
    ew = np.array([0.0, np.sin(np.radians(0.2)), np.sin(np.radians(-0.6)), 0.01])
    T = 384 * 2
    k = np.random.default_rng(8).integers(0, 4, size=(len(freqs), T, 2))
    z = a * (1j ** k)                                            # [ch, t, pol]
    re = np.broadcast_to(np.rint(z.real).astype(int)[:, :, None, None, :], (len(freqs), T, 4, 256, 2))
    im = np.broadcast_to(np.rint(z.imag).astype(int)[:, :, None, None, :], (len(freqs), T, 4, 256, 2))
    raw = synth.encode(re, im).reshape(len(freqs), T, 2048)
    smap = O.sky_map(O.beamform(raw, freqs, ns, ew))
    expect = np.zeros(1024)
    n = np.arange(256)
    for f in freqs:
        Lf = nearest_beam_bins(f, ns)
        D = np.array([256.0 if Lm == 0 else (0.0 if Lm % 2 == 0 else abs(2 / (1 - cmath.exp(-1j * math.pi * Lm / 256))))
                      for Lm in Lf])
        A = np.abs(np.exp(-2j * np.pi * f * np.outer(np.arange(4) * 20.0, ew) / O.C0).sum(axis=0))   # [j]
        expect += 128 * T * 2 * a * a * (A[:, None] ** 2 * D[None, :] ** 2).ravel()
    assert np.allclose(smap, expect, rtol=1e-9, atol=1e-9 * expect.max())
    assert int(np.argmax(smap)) == 0 * 256 + 128 and abs(smap[128] / (len(freqs) * 128 * T * 2 * (a * 1024) ** 2) - 1) < 1e-12


@pytest.mark.parametrize("f_c", [410e6, 650e6])
def test_subchannel_freqs_hold_the_tones_that_land_in_them(f_c):
    """Sec. 3.2 up-channelisation: a coarse-channel sample rotates as
    exp(+2 pi i delta t dt) for a sky tone at f_c + delta (the sign of the
    plane-wave convention).  A tone at each of the 128 fine-channel centres
    must land, whole, in one sub-channel; the sub-channel holding it must be the
    one whose centre frequency (subchannel_freqs) is nearest the tone, and each
    sub-channel's centre must be the mean of the eight tones it holds.  A
    flipped fftshift, a one-sub-channel shift or a half-fine-channel offset of
    the centres fails one of these."""
    fine = 390625.0 / 128
    dt = 2.56e-6
    centres = O.subchannel_freqs([f_c])
    assert centres.shape == (16,)
    held = {s: [] for s in range(16)}
    tau = np.arange(384)
    for q in range(128):
        delta = (q - 64) * fine                               # any integer number of fine channels
        B = np.exp(2j * np.pi * delta * tau * dt)[:, None, None, None] * np.ones((1, 2, 4, 256))
        P = O.detect_downsample(O.upchannelize(B))[0, :, 0]   # beam 0, [sub]
        s = int(np.argmax(P))
        assert abs(P[s] - P.sum()) <= 1e-9 * P.sum()          # the whole tone in one sub-channel
        assert s == int(np.argmin(np.abs(centres - (f_c + delta))))
        held[s].append(f_c + delta)
    for s in range(16):
        assert len(held[s]) == 8 and abs(np.mean(held[s]) - centres[s]) < 1e-6
    # tones between fine-channel centres: negative offsets, and within a quarter of a
    # fine channel of a sub-channel edge, still go to the nearest centre
    for delta in (-0.3 * fine, -64.2 * fine, 8 * fine - 0.6 * fine, 23.8 * fine, -8.7 * fine):
        B = np.exp(2j * np.pi * delta * tau * dt)[:, None, None, None] * np.ones((1, 2, 4, 256))
        P = O.detect_downsample(O.upchannelize(B))[0, :, 0]
        assert int(np.argmax(P)) == int(np.argmin(np.abs(centres - (f_c + delta))))


def test_dedispersion_aligns_a_synthetic_sweep():
    # Sec. 3.2: dispersion delays lower frequencies by k_DM DM f^-2; shifting each
    # sub-channel by its delay re-aligns a dispersed pulse.  Build the pulse
    # directly in the output domain from the continuous f^-2 law.
    freqs = [600e6 + 390625.0 * k for k in range(6)]
    dm = 150.0
    fs = O.subchannel_freqs(freqs) / 1e6
    frame = 384 * 2.56e-6
    delay = O.K_DM_S_MHZ2 * dm * (fs ** -2.0 - fs.max() ** -2.0) / frame
    d = O.dedisperse_delays(freqs, dm)
    assert np.all(np.abs(d - delay) <= 0.5 + 1e-9)          # nearest frame
    assert np.all(np.diff(d.reshape(6, 16), axis=1) <= 0)   # higher sub-channels arrive first
    nf = 80
    Oarr = np.zeros((1024, 96, nf))
    t0 = 10
    for s in range(96):
        Oarr[5, s, t0 + d[s]] = 1.0
    series, _ = O.dedisperse(Oarr, freqs, dm)
    assert series.shape == (1024, nf - d.max())
    assert series[5, t0] == 96 and series[5].sum() == 96
    flat, d0 = O.dedisperse(Oarr, freqs, 0.0)
    assert np.all(d0 == 0) and np.allclose(flat, Oarr.sum(axis=1))


# --- tracking E-W beams (Sec. 3.1: static or tracking) ---------------------------------

def quarter_turn_sines(freq, k_frames, D=20.0):
    """E-W sine at which the cylinder phase step f D u / c0 is k/4 turns."""
    return np.array([k * O.C0 / (4.0 * freq * D) for k in k_frames])


def test_tracking_with_constant_table_is_static():
    freq = 480e6
    raw = rand_raw((384 * 2 + 40, 2048))
    u = np.array([-0.3, 0.0, 0.1, 0.45])
    ref = O.beamform_channel(raw, freq, ew_sin=u)
    got = O.beamform_channel(raw, freq, ew_sin_frames=np.tile(u, (2, 1)))
    assert np.allclose(got, ref, rtol=1e-12, atol=0)


def test_tracking_beam_keeps_the_coherent_gain_of_a_drifting_source():
    """Cylinder c carries cylinder 0 times i^(k_F c) in frame F (an exact
    plane wave drifting in E-W).  A beam that tracks it adds the four
    cylinders in phase: its power is 4^2 = 16 times the power of cylinder 0
    alone, frame by frame; a static beam loses that gain once the source moves."""
    freq = 600e6
    k = [0, 1, 2, 3, 1]
    raw = synth.cylinder_quarter_turns(k, seed=5)
    only0 = raw.copy()
    only0.reshape(-1, 4, 512)[:, 1:] = synth.encode(0, 0)
    u = np.zeros((len(k), 4))
    u[:, 0] = quarter_turn_sines(freq, k)
    track = O.beamform_channel(raw, freq, ew_sin_frames=u)
    single = O.beamform_channel(only0, freq, ew_sin_frames=u)
    assert np.allclose(track[:256], 16.0 * single[:256], rtol=1e-10, atol=0)
    static = O.beamform_channel(raw, freq, ew_sin=u[0])
    for F in (1, 2, 3):
        assert static[:256, :, F].sum() < 0.5 * track[:256, :, F].sum()
    # beams 1..3 point at u = 0: a k = 2 (half-turn) step cancels in pairs
    assert np.allclose(track[256:, :, 2], 0.0, atol=1e-9 * track[:256, :, 2].max())


def test_tracking_rows_select_their_own_frame():
    freq = 700e6
    raw = rand_raw((384 * 3, 2048))
    u = np.array([[0.0, 0.1, 0.2, 0.3], [0.05, -0.1, 0.25, -0.3], [0.5, 0.4, -0.2, 0.01]])
    got = O.beamform_channel(raw, freq, ew_sin_frames=u)
    for F in range(3):
        one = O.beamform_channel(raw[384 * F:384 * (F + 1)], freq, ew_sin=u[F])
        assert np.allclose(got[..., F], one[..., 0], rtol=1e-12, atol=0)

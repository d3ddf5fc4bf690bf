"""Products of the intensity output on the GPU: the frequency-summed sky map
(Fig. 3, Sec. 3.3) and 8-bit rescaling (Table 1), against the oracle."""
import math

import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_skymap_fig3_source_dominates_aliases(built_lib):
    # Sec. 3.3 / Fig. 3: a source near 26 deg, summed over the band, is
    # detected at its position; its aliases (-88 .. -50 deg above ~490 MHz)
    # are smeared and weaker than the source in the summed map.
    freqs = [400e6 + 400e6 * (i + 0.5) / 24 for i in range(24)]
    s_src = math.sin(math.radians(26.0))
    u_src = math.sin(math.radians(0.2))
    pw = synth.PlaneWave(1.0, u=u_src, s=s_src)
    raw = synth.make_voltages(freqs, 768, seed=5, plane_waves=[pw])
    with B.Plan() as p:
        out = p.run(torch.from_numpy(raw).cuda(), freqs)
        smap = p.skymap(out).cpu().numpy()
    ref = O.sky_map(O.beamform(raw, freqs))
    assert np.max(np.abs(smap - ref) / ref) <= 1e-5
    ns = O.default_ns_sin()
    m_src = int(np.argmin(np.abs(ns - s_src)))
    beam = int(np.argmax(smap))
    j, m = divmod(beam, 256)
    assert j == 2 and abs(m - m_src) <= 1                      # E-W beam +0.2 deg, N-S pointing of 26 deg
    ang = np.degrees(np.arcsin(ns))
    alias = (ang > -90) & (ang < -45)
    noise_floor = np.median(smap[j * 256:(j + 1) * 256])
    assert (smap[j * 256:(j + 1) * 256][alias] - noise_floor).max() < 0.5 * (smap[beam] - noise_floor)

@pytest.mark.parametrize("n_sub,nf,offset", [(16 * 1024, 2, 0), (64, 128, 0), (48, 5, 1), (16, 1, 0)])
def test_skymap_kernel_against_the_oracle(built_lib, n_sub, nf, offset):
    """The map kernel alone on seeded intensities of the band shape (16384
    sub-channels x 2 frames), the node-slice shape, a ragged shape whose beam
    blocks are not 16-byte aligned (offset by one float), and one frame:
    within 1e-5 relative (FP32 sums of up to 32768 positive terms)."""
    rng = np.random.default_rng(n_sub + nf)
    x = rng.gamma(48.0, 1e4, size=(1024, n_sub, nf)).astype(np.float32)
    buf = torch.zeros(x.size + 4, dtype=torch.float32, device="cuda")
    d = buf[offset:offset + x.size]
    d.copy_(torch.from_numpy(x.ravel()))
    m = torch.empty(1024, dtype=torch.float32, device="cuda")
    with B.Plan() as p:
        B.bf_skymap(p.handle, d, n_sub, nf, m)
        torch.cuda.synchronize()
    ref = O.sky_map(x)
    assert np.max(np.abs(m.cpu().numpy() - ref) / ref) <= 1e-5


U32 = 2.0 ** -24          # FP32 unit roundoff


def check_rescale(x, codes, stats):
    """The kernel (FP32) against the FP64 rule of the oracle.  Codes must be
    equal except where the FP64 value v = 64 + 16 z lies within `tol` of a
    rounding boundary (v + 1/2 an integer), where a code one step either side is
    also correct.  tol bounds the FP32 evaluation: recursive sums of n terms
    shifted by the row's first frame give |mean error| <= (n + 1) u A (A = mean
    |x - x0|) plus u |mean|, the standard deviation a relative (n/2 + 4) u,
    and the product 16 (x - mean) / std three more roundings, u = 2^-24; the
    bound is doubled.  Statistics within the same bounds; constant rows give
    code 64 and std 0 exactly."""
    x = np.asarray(x, np.float64)
    rows, n = x.shape
    v, const, st = O.rescale_value(x)
    ref = np.clip(np.floor(v + 0.5), 0, 255)
    mean, sd = st[:, 0], st[:, 1]
    A = np.abs(x - x[:, :1]).mean(axis=1)
    dmean = 2 * ((n + 1) * U32 * A + 2 * U32 * np.abs(mean))
    with np.errstate(divide="ignore", invalid="ignore"):
        z = np.where(const[:, None], 0.0, (v - 64.0) / 16.0)
        tol = 2 * (16 * U32 * (np.abs(z) * (n / 2 + 6)) + 16 * dmean[:, None] / np.where(const, 1.0, sd)[:, None]
                   + 512 * U32)
    dist = np.abs((v + 0.5) - np.rint(v + 0.5))
    near = (dist <= tol) & ~const[:, None]
    got = np.asarray(codes, np.int64).reshape(rows, n)
    assert np.array_equal(got[~near], ref[~near].astype(np.int64)), "code differs away from a rounding boundary"
    assert np.all(np.abs(got[near] - ref[near]) <= 1)
    assert near.mean() < 0.01                                # the allowance stays small
    gs = np.asarray(stats, np.float64).reshape(rows, 2)
    assert np.all(np.abs(gs[:, 0] - mean) <= dmean)
    assert np.all(np.abs(gs[:, 1] - sd) <= 2 * (n / 2 + 4) * U32 * sd + dmean)
    assert np.all(got[const] == 64) and np.all(gs[const, 1] == 0.0)
    return int(near.sum())


def intensity_rows(rng, rows, nf):
    """Seeded stand-in for the intensity output: chi^2-like rows (gamma, k = 48
    as for 48 squared terms), some with an outlier frame, some constant."""
    x = rng.gamma(48.0, 1e4, size=(rows, nf))
    x[::7, nf // 3] *= 4.0                                    # a burst-like outlier
    x[3::11] = x[3::11, :1]                                    # constant rows
    x[5] = np.float32(0.1)
    return x.astype(np.float32)


def test_rescale_u8_matches_the_rule():
    rng = np.random.default_rng(8)
    x = intensity_rows(rng, 1024 * 16, 40)
    with B.Plan() as p:
        d = torch.from_numpy(x).cuda()
        codes = torch.empty(x.shape, dtype=torch.uint8, device="cuda")
        stats = torch.empty(x.shape[0], 2, dtype=torch.float32, device="cuda")
        B.bf_rescale_u8(p.handle, d, x.shape[0], x.shape[1], codes, stats)
        zero = p.run(torch.full((1, 384 * 3, 2048), 0x88, dtype=torch.uint8, device="cuda"), [560e6])
        zc, zs = p.rescale_u8(zero)
        torch.cuda.synchronize()
    check_rescale(x, codes.cpu().numpy(), stats.cpu().numpy())
    assert np.all(zc.cpu().numpy() == 64) and np.all(zs.cpu().numpy() == 0.0)
    # the outlier frame dominates its rows: among 40 frames it reaches z ~ 5 (code > 140)
    c = codes.cpu().numpy()
    burst_rows = [r for r in range(0, x.shape[0], 7) if r % 11 != 3 and r != 5]   # not the constant rows
    assert c[burst_rows, 40 // 3].min() > 140


@pytest.mark.parametrize("nf,offset", [(128, 0), (300, 0), (41, 0), (128, 1), (1, 0)])
def test_rescale_u8_row_lengths_and_alignment(built_lib, nf, offset):
    """Row lengths that take the staged word path (128), the direct path (300 >
    256 frames staged), the staged byte path (41, not a multiple of 4), an
    output one byte off a 4-byte boundary, and single-frame rows (constant)."""
    rng = np.random.default_rng(nf + offset)
    rows = 77
    xh = intensity_rows(rng, rows, nf)
    x = torch.from_numpy(xh).cuda()
    buf = torch.zeros(rows * nf + 8, dtype=torch.uint8, device="cuda")
    codes = buf[offset:offset + rows * nf]
    stats = torch.empty(rows, 2, dtype=torch.float32, device="cuda")
    with B.Plan() as p:
        B.bf_rescale_u8(p.handle, x, rows, nf, codes, stats)
        torch.cuda.synchronize()
    check_rescale(xh, codes.cpu().numpy(), stats.cpu().numpy())
    assert buf[:offset].sum().item() == 0 and buf[offset + rows * nf:].sum().item() == 0


@pytest.mark.parametrize("n_chan,nf,dm", [(8, 64, 150.0), (4, 128, 500.0), (3, 9, 0.0), (64, 40, 20.0)])
def test_dedisperse_kernel_against_the_oracle(built_lib, n_chan, nf, dm):
    """The dedispersion kernel alone on seeded intensities against the oracle's
    rule (delays from the sub-channel centres of Sec. 3.2 and k_DM), within
    1e-5 relative; n_out matches, and DM 0 is the plain sum over sub-channels."""
    rng = np.random.default_rng(n_chan * nf)
    freqs = [400e6 + 390625.0 * (37 * k % 1024 + 0.5) for k in range(n_chan)]
    x = rng.gamma(48.0, 1e4, size=(1024, 16 * n_chan, nf)).astype(np.float32)
    ref, d = O.dedisperse(x, freqs, dm)
    with B.Plan() as p:
        ser = p.dedisperse(torch.from_numpy(x).cuda(), freqs, dm).cpu().numpy()
    assert ser.shape == ref.shape
    if ref.size:
        assert np.max(np.abs(ser - ref) / ref) <= 1e-5


def test_dedispersion_recovers_a_burst(built_lib):
    """A DM-150 burst across 8 channels from 600 MHz, beamformed and then
    dedispersed: the burst's beam has the highest dedispersed peak, and
    dedispersing raises its S/N over the plain frequency sum."""
    freqs = [600e6 + 390625.0 * k for k in range(8)]
    dm, T = 150.0, 384 * 64
    m, j = 171, 3
    s_src = (m - 127.5) / 128.0
    u_src = math.sin(math.radians(0.6))
    burst = synth.Burst(0.5, u=u_src, s=s_src, dm=dm, t0_s=0.4 * T * synth.DT_S, f_ref_hz=max(freqs))
    raw = synth.make_voltages(freqs, T, seed=21, bursts=[burst])
    with B.Plan() as p:
        out = p.run(torch.from_numpy(raw).cuda(), freqs)
        ser = p.dedisperse(out, freqs, dm).cpu().numpy()
        ser0 = p.dedisperse(out, freqs, 0.0).cpu().numpy()
    assert O.dedisperse_delays(freqs, dm).max() > 10
    beam = 256 * j + m

    def snr(x):
        return (x.max() - np.median(x)) / np.std(x)

    assert snr(ser[beam]) > 1.5 * snr(ser0[beam][: ser.shape[1]])
    assert int(np.argmax(ser.max(axis=1))) == beam

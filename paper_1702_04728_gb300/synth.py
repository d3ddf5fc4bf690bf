"""Seeded synthetic baseband voltages for the CHIME/FRB fan-beam path.

This module is the input generator shared by the tests, the benchmark and the
smoke check.  It holds none of the beamformer's arithmetic: it only models the
sky signal and the F-engine quantiser, and writes packed bytes.

Input format (Sec. 2 and Table 1: 2048 inputs, 4-bit real + 4-bit imaginary
per sample, one sample per 2.56 us):

* one byte per (time, input); the high nibble is the real part and the low
  nibble the imaginary part, each offset-encoded as ``value + 8``;
* inside a time sample the 2048 bytes are ordered cylinder-major, then feed,
  then polarisation: ``byte = (cyl * 256 + feed) * 2 + pol``;
* a channel's block is ``[T][2048]`` and a multi-channel request stacks them
  as ``[n_chan][T][2048]``.

Signal model (used only to make realistic test inputs):

* noise: real and imaginary parts i.i.d. N(0, sigma^2), rounded to the nearest
  integer (ties to even) and clipped to [-7, 7];
* a source in direction (u, s) (E-W and N-S direction cosines) arrives at
  cylinder ``c``, feed ``n`` with phase ``exp(+2 pi i f (c D u + n d s) / c0)``,
  added before quantisation;
* a dispersed burst has a Gaussian envelope with a complex-Gaussian carrier, a
  per-channel arrival delay ``k_DM DM (f^-2 - f_ref^-2)`` and the intra-channel
  dispersive chirp applied in the Fourier domain of the channel's series.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Iterable, List, Optional, Sequence

import numpy as np

C0 = 299_792_458.0            # speed of light, m/s
K_DM = 4.148808e3             # dispersion constant, s MHz^2 / (pc cm^-3)
N_CYL, N_FEED, N_POL = 4, 256, 2
N_INPUT = N_CYL * N_FEED * N_POL
FEED_SPACING_M = 0.3048       # N-S feed spacing (Sec. 1)
CYL_SPACING_M = 20.0          # E-W cylinder spacing (cylinder width, Sec. 1)
DT_S = 2.56e-6                # sample cadence (Table 1)
CHAN_BW_HZ = 390625.0         # coarse channel width, 400 MHz / 1024


def encode(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Offset-encode integer parts in [-8, 7] into one byte each."""
    re = np.asarray(re, dtype=np.int16)
    im = np.asarray(im, dtype=np.int16)
    if re.min(initial=0) < -8 or re.max(initial=0) > 7 or im.min(initial=0) < -8 or im.max(initial=0) > 7:
        raise ValueError("4-bit parts must lie in [-8, 7]")
    return (((re + 8) << 4) | (im + 8)).astype(np.uint8)


def quantize(z: np.ndarray, clip: int = 7) -> np.ndarray:
    """Round re/im to the nearest integer, clip to [-clip, clip], encode."""
    re = np.clip(np.rint(z.real), -clip, clip).astype(np.int16)
    im = np.clip(np.rint(z.imag), -clip, clip).astype(np.int16)
    return encode(re, im)


def geometric_phase(freq_hz: float, u: float, s: float,
                    feed_spacing: float = FEED_SPACING_M,
                    cyl_spacing: float = CYL_SPACING_M) -> np.ndarray:
    """Per-input complex gain [2048] of a unit plane wave from (u, s)."""
    c = np.arange(N_CYL, dtype=np.float64)[:, None, None]
    n = np.arange(N_FEED, dtype=np.float64)[None, :, None]
    path = (c * cyl_spacing * u + n * feed_spacing * s) / C0 * freq_hz
    ph = np.exp(2j * np.pi * np.mod(path, 1.0))
    return np.broadcast_to(ph, (N_CYL, N_FEED, N_POL)).reshape(N_INPUT)


@dataclasses.dataclass
class PlaneWave:
    """Point source with a random per-sample phase, independent per pol."""
    amplitude: float
    u: float                  # E-W direction cosine
    s: float                  # N-S direction cosine (sin of zenith angle)


@dataclasses.dataclass
class Burst:
    """Dispersed burst: Gaussian envelope of ``fwhm_s``, complex carrier."""
    amplitude: float
    u: float
    s: float
    dm: float                 # pc cm^-3
    t0_s: float               # arrival time at ``f_ref_hz``
    fwhm_s: float = 1e-3
    f_ref_hz: float = 650e6


def burst_series(b: Burst, freq_hz: float, n_samples: int,
                 rng: np.random.Generator) -> np.ndarray:
    """Complex baseband series [T] of a burst in one coarse channel."""
    t = np.arange(n_samples) * DT_S
    delay = K_DM * b.dm * ((freq_hz / 1e6) ** -2 - (b.f_ref_hz / 1e6) ** -2)
    sig = b.fwhm_s / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    env = np.exp(-0.5 * ((t - b.t0_s - delay) / sig) ** 2)
    carrier = (rng.standard_normal(n_samples) + 1j * rng.standard_normal(n_samples)) / math.sqrt(2.0)
    x = b.amplitude * env * carrier
    if b.dm != 0.0 and env.max() > 1e-12:
        # Intra-channel dispersion: group delay falls with baseband frequency nu.
        nu = np.fft.fftfreq(n_samples, d=DT_S)
        k = K_DM * 1e12 * b.dm            # s Hz^2
        phase = 2.0 * np.pi * k * nu ** 2 / (freq_hz ** 2 * (freq_hz + nu))
        x = np.fft.ifft(np.fft.fft(x) * np.exp(1j * phase))
    return x


def make_voltages(freqs_hz: Sequence[float], n_samples: int, seed: int,
                  sigma: float = 2.5,
                  plane_waves: Iterable[PlaneWave] = (),
                  bursts: Iterable[Burst] = (),
                  chunk: int = 2048) -> np.ndarray:
    """Packed voltages ``uint8[n_chan][n_samples][2048]`` for the given channels.

    Deterministic in ``seed``; generated in time chunks to bound memory.
    """
    plane_waves = list(plane_waves)
    bursts = list(bursts)
    out = np.empty((len(freqs_hz), n_samples, N_INPUT), dtype=np.uint8)
    root = np.random.default_rng(seed)
    for ci, f in enumerate(freqs_hz):
        rng = np.random.default_rng(root.integers(0, 2**63))
        pw_gain = [geometric_phase(f, p.u, p.s) * p.amplitude for p in plane_waves]
        b_series = [(burst_series(b, f, n_samples, rng), geometric_phase(f, b.u, b.s))
                    for b in bursts]
        for t0 in range(0, n_samples, chunk):
            t1 = min(n_samples, t0 + chunk)
            nt = t1 - t0
            z = rng.standard_normal((nt, N_INPUT), dtype=np.float32) * sigma \
                + 1j * (rng.standard_normal((nt, N_INPUT), dtype=np.float32) * sigma)
            for g in pw_gain:
                # random per-sample phase, independent per polarisation
                ph = np.exp(2j * np.pi * rng.random((nt, 1, 1, N_POL)))
                z += (ph * g.reshape(1, N_CYL, N_FEED, N_POL)).reshape(nt, N_INPUT)
            for series, g in b_series:
                seg = series[t0:t1]
                if np.abs(seg).max(initial=0.0) > 1e-9:
                    z += seg[:, None] * g[None, :]
            out[ci, t0:t1] = quantize(z)
    return out


# --- the workloads used by tests and the benchmark -------------------------

def config_point_source(seed: int = 0):
    """1 channel at 600 MHz, 3072 samples, plane wave at 20 deg N-S, 0.5 deg E-W."""
    freqs = [600e6]
    pw = PlaneWave(1.5, u=math.sin(math.radians(0.5)), s=math.sin(math.radians(20.0)))
    raw = make_voltages(freqs, 3072, seed, plane_waves=[pw])
    return raw, np.array(freqs)


def burst_amplitude(n_chan: int, sigma: float = 2.5, snr: float = 20.0) -> float:
    """Per-input burst amplitude giving nominal S/N ``snr`` in a 1 ms boxcar."""
    return math.sqrt(snr * sigma * sigma / (1024.0 * math.sqrt(390.0 * 2.0 * n_chan)))


def config_node_slice(seed: int = 0, n_samples: int = 49152, freqs=None):
    """4 channels (410/520/650/790 MHz by default), 49152 samples, one DM-500 burst."""
    freqs = list(freqs) if freqs is not None else [410e6, 520e6, 650e6, 790e6]
    rng = np.random.default_rng(seed + 1)
    m = int(rng.integers(0, 256))
    j = int(rng.integers(0, 4))
    s = (m - 127.5) / 128.0
    u = math.sin(math.radians([-0.6, -0.2, 0.2, 0.6][j]))
    b = Burst(burst_amplitude(len(freqs)), u=u, s=s, dm=500.0,
              t0_s=0.5 * n_samples * DT_S, f_ref_hz=freqs[2])
    raw = make_voltages(freqs, n_samples, seed, bursts=[b])
    return raw, np.array(freqs), {"burst_beam": 256 * j + m, "burst_chan": 2}


def cylinder_quarter_turns(k_frames: Sequence[int], seed: int, frame: int = 384) -> np.ndarray:
    """uint8 [len(k_frames) * frame, 2048]: random 4-bit values in [-7, 7] on
    cylinder 0; cylinder c holds cylinder 0's values times i^(k_F c) during
    frame F.  Multiplying by i maps the clipped 4-bit lattice onto itself, so
    this is an exact plane wave whose E-W phase step between cylinders is k_F
    quarter turns, changing from frame to frame (a source drifting in E-W)."""
    rng = np.random.default_rng(seed)
    T = len(k_frames) * frame
    re = rng.integers(-7, 8, size=(T, N_FEED, 2), dtype=np.int16)
    im = rng.integers(-7, 8, size=(T, N_FEED, 2), dtype=np.int16)
    out_re = np.empty((T, N_CYL, N_FEED, 2), np.int16)
    out_im = np.empty_like(out_re)
    for F, k in enumerate(k_frames):
        sl = slice(F * frame, (F + 1) * frame)
        for c in range(N_CYL):
            r, i = re[sl], im[sl]
            for _ in range((int(k) * c) % 4):
                r, i = -i, r
            out_re[sl, c], out_im[sl, c] = r, i
    return encode(out_re, out_im).reshape(T, N_INPUT)


def noise_only(freqs_hz: Sequence[float], n_samples: int, seed: int, sigma: float = 2.5) -> np.ndarray:
    return make_voltages(freqs_hz, n_samples, seed, sigma=sigma)


def quantized_noise_variance(sigma: float = 2.5, clip: int = 7) -> float:
    """Exact variance of clip(round(N(0, sigma^2)), +-clip), by summation."""
    from math import erf, sqrt
    cdf = lambda x: 0.5 * (1.0 + erf(x / (sigma * sqrt(2.0))))
    var = 0.0
    for k in range(-clip, clip + 1):
        if k == -clip:
            p = cdf(k + 0.5)
        elif k == clip:
            p = 1.0 - cdf(k - 0.5)
        else:
            p = cdf(k + 0.5) - cdf(k - 0.5)
        var += p * k * k
    return var


# --- counter-based noise for workloads too large to generate on the host -----------
#
# Byte i of a channel block is drawn from SplitMix64 (Steele, Lea and Flood,
# 2014) of (seed, i): the two 32-bit halves of the 64-bit output pick the real
# and imaginary parts through integer thresholds of the clipped, rounded normal
# distribution.  The device generator (torch) and the host generator (numpy)
# implement the same definition in integer arithmetic, so they agree bit for
# bit and the oracle can rebuild any sampled frame on the host.

_SM_GAMMA = 0x9E3779B97F4A7C15
_SM_M1 = 0xBF58476D1CE4E5B9
_SM_M2 = 0x94D049BB133111EB


def noise_thresholds(sigma: float = 2.5, clip: int = 7):
    """uint32 thresholds t_k (k = -clip .. clip-1): value = -clip + #{t_k <= u}."""
    from math import erf, sqrt
    out = []
    for k in range(-clip, clip):
        cdf = 0.5 * (1.0 + erf((k + 0.5) / (sigma * sqrt(2.0))))
        out.append(min(2**32 - 1, int(cdf * 2**32)))
    return out


def _mix_np(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = x + np.uint64(_SM_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_SM_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_SM_M2)
        return z ^ (z >> np.uint64(31))


def hash_noise_rows(seed: int, chan: int, n_samples_per_chan: int, t0: int, t1: int,
                    sigma: float = 2.5, offsets=None) -> np.ndarray:
    """Host copy of rows [t0, t1) of channel `chan`: uint8 [t1 - t0][2048].
    offsets: optional (re, im) int8 [n_chan][n_samples] burst offsets in units
    of 1/BURST_Q count (see burst_offsets); row t of the channel is quantised
    with the thresholds of its offset."""
    base = (np.uint64(seed) << np.uint64(40)) + np.uint64(chan * n_samples_per_chan * N_INPUT)
    idx = base + np.arange(t0 * N_INPUT, t1 * N_INPUT, dtype=np.uint64)
    z = _mix_np(idx).reshape(t1 - t0, N_INPUT)
    lo = z & np.uint64(0xFFFFFFFF)
    hi = z >> np.uint64(32)
    if offsets is None:
        thr = np.array(noise_thresholds(sigma), dtype=np.uint64)
        re = -7 + (hi[..., None] >= thr).sum(axis=-1).astype(np.int16)
        im = -7 + (lo[..., None] >= thr).sum(axis=-1).astype(np.int16)
    else:
        table = burst_thresholds(sigma)                                   # [2 R + 1][14]
        t_re = table[offsets[0][chan, t0:t1].astype(np.int64) + BURST_R]   # [rows][14]
        t_im = table[offsets[1][chan, t0:t1].astype(np.int64) + BURST_R]
        re = -7 + (hi[..., None] >= t_re[:, None, :]).sum(axis=-1).astype(np.int16)
        im = -7 + (lo[..., None] >= t_im[:, None, :]).sum(axis=-1).astype(np.int16)
    return encode(re, im).reshape(t1 - t0, N_INPUT)


def hash_noise_device(seed: int, n_chan: int, n_samples: int, device="cuda", sigma: float = 2.5,
                      chunk: int = 1 << 26, offsets=None):
    """Device generation of uint8 [n_chan][n_samples][2048] (same bytes as above);
    offsets as in hash_noise_rows.  chunk: bytes per step, a multiple of 2048."""
    import torch
    assert chunk % N_INPUT == 0
    thr = noise_thresholds(sigma)
    out = torch.empty(n_chan * n_samples * N_INPUT, dtype=torch.uint8, device=device)
    total = out.numel()
    base = seed << 40
    mask32 = 0xFFFFFFFF
    if offsets is not None:
        table = torch.from_numpy(burst_thresholds(sigma).astype(np.int64)).to(device)     # [2 R + 1][14]
        off_re = torch.from_numpy(np.ascontiguousarray(offsets[0]).reshape(-1).astype(np.int64) + BURST_R).to(device)
        off_im = torch.from_numpy(np.ascontiguousarray(offsets[1]).reshape(-1).astype(np.int64) + BURST_R).to(device)

    def as_i64(v):                                   # uint64 constant as a wrapped int64
        return v - (1 << 64) if v >= (1 << 63) else v

    def srl(z, k):                                   # logical right shift of int64 bit patterns
        return (z >> k) & ((1 << (64 - k)) - 1)

    for s in range(0, total, chunk):
        n = min(chunk, total - s)
        z = torch.arange(s, s + n, dtype=torch.int64, device=device) + (base + as_i64(_SM_GAMMA))
        z = (z ^ srl(z, 30)) * as_i64(_SM_M1)
        z = (z ^ srl(z, 27)) * as_i64(_SM_M2)
        z = z ^ srl(z, 31)
        hi = srl(z, 32).view(-1, N_INPUT)
        lo = (z & mask32).view(-1, N_INPUT)
        re = torch.zeros_like(hi, dtype=torch.int16)
        im = torch.zeros_like(hi, dtype=torch.int16)
        if offsets is None:
            for t in thr:
                re += (hi >= t).to(torch.int16)
                im += (lo >= t).to(torch.int16)
        else:
            rows = torch.arange(s // N_INPUT, (s + n) // N_INPUT, device=device)     # global row = chan * T + t
            t_re = table[off_re[rows]]                                                # [rows][14]
            t_im = table[off_im[rows]]
            for k in range(len(thr)):
                re += (hi >= t_re[:, k:k + 1]).to(torch.int16)
                im += (lo >= t_im[:, k:k + 1]).to(torch.int16)
        out[s:s + n] = (((re + 1) << 4) | (im + 1)).to(torch.uint8).view(-1)   # (v + 8) with v = count - 7
        del z, hi, lo, re, im
    return out.view(n_chan, n_samples, N_INPUT)


# --- dispersed bursts in the counter-based workload ------------------------------
#
# A burst from zenith (u = s = 0) reaches every input of a channel with the same
# complex amplitude b(t); the sample is then clip(round(noise + b)).  b is
# quantised to BURST_Q steps per count (at most BURST_R steps) on the host in
# FP64, and the rounding of noise + b becomes a comparison of the same uniform
# integer with shifted thresholds floor(2^32 Phi((k + 1/2 - b) / sigma)), one
# table row per quantised b (row BURST_R, b = 0, holds the plain noise
# thresholds).  Host and device use the same table and integer comparisons, so
# they still agree bit for bit.

BURST_Q = 256
BURST_R = 127


def burst_thresholds(sigma: float = 2.5, clip: int = 7) -> np.ndarray:
    """uint64 [2 BURST_R + 1][2 clip]: thresholds for offsets b = (i - BURST_R) / BURST_Q."""
    from math import erf, sqrt
    out = np.empty((2 * BURST_R + 1, 2 * clip), dtype=np.uint64)
    for i in range(2 * BURST_R + 1):
        b = (i - BURST_R) / BURST_Q
        for kk, k in enumerate(range(-clip, clip)):
            cdf = 0.5 * (1.0 + erf((k + 0.5 - b) / (sigma * sqrt(2.0))))
            out[i, kk] = min(2**32 - 1, int(cdf * 2**32))
    return out


def burst_offsets(freqs_hz: Sequence[float], n_samples: int, bursts: Iterable[Burst], seed: int):
    """(re, im) int8 [n_chan][n_samples]: the bursts' complex amplitude per channel
    and sample (burst_series: Gaussian envelope, complex-Gaussian carrier,
    arrival k_DM DM (f^-2 - f_ref^-2), intra-channel chirp) in units of
    1/BURST_Q count, rounded and clipped to +-BURST_R.  Channels the burst does
    not reach inside the window are left at zero."""
    bursts = list(bursts)
    re = np.zeros((len(freqs_hz), n_samples), np.int8)
    im = np.zeros((len(freqs_hz), n_samples), np.int8)
    T = n_samples * DT_S
    for bi, b in enumerate(bursts):
        for ci, f in enumerate(freqs_hz):
            arrive = b.t0_s + K_DM * b.dm * ((f / 1e6) ** -2 - (b.f_ref_hz / 1e6) ** -2)
            smear = 8.3e-6 * b.dm * (CHAN_BW_HZ / 1e6) / (f / 1e9) ** 3 + 5 * b.fwhm_s
            if arrive + smear < 0 or arrive - smear > T:
                continue
            rng = np.random.default_rng([seed, bi, ci])
            x = burst_series(b, f, n_samples, rng)
            re[ci] = np.clip(np.rint(re[ci] + x.real * BURST_Q), -BURST_R, BURST_R).astype(np.int8)
            im[ci] = np.clip(np.rint(im[ci] + x.imag * BURST_Q), -BURST_R, BURST_R).astype(np.int8)
    return re, im


SWEEP_FREQS = [400e6 + 6.25e6 * (i + 0.5) for i in range(64)]
# the sweep's five bursts: zenith, 1 ms FWHM, nominal S/N 200 over the 64 channels (0.07 counts
# per input, well below the noise), reaching 800 MHz 10 + 20 i ms into the 1 s window and
# sweeping down the band (a DM-100 burst crosses 48 of the 64 channels inside the window, a
# DM-2000 burst 5)
SWEEP_BURSTS = [Burst(burst_amplitude(64, snr=200.0), u=0.0, s=0.0, dm=dm, t0_s=0.01 + 0.02 * i, f_ref_hz=800e6)
                for i, dm in enumerate((100.0, 300.0, 700.0, 1200.0, 2000.0))]


# --- device-side generator for band-wide workloads ------------------------------

BAND_FREQS = [400e6 + CHAN_BW_HZ * (k + 0.5) for k in range(1024)]   # the 1024 coarse channels, 400-800 MHz


def plane_wave_device(freqs_hz: Sequence[float], n_samples: int, seed: int,
                      plane_waves: Iterable[PlaneWave] = (), sigma: float = 2.5,
                      device="cuda", chunk_chan: int = 32):
    """Packed voltages ``uint8[n_chan][n_samples][2048]`` generated on the device
    with torch: noise N(0, sigma^2) per real part plus plane waves (same model as
    ``make_voltages``: geometric phase per input, random per-sample phase per
    polarisation), rounded half to even, clipped to +-7 and offset-encoded.
    Deterministic in ``seed`` on a given device and torch build (torch's
    generator, not numpy's: the host cannot rebuild the bytes, so tests copy
    back the channels they check)."""
    import torch
    plane_waves = list(plane_waves)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty((len(freqs_hz), n_samples, N_INPUT), dtype=torch.uint8, device=device)
    for c0 in range(0, len(freqs_hz), chunk_chan):
        fs = list(freqs_hz[c0:c0 + chunk_chan])
        nc = len(fs)
        re = torch.randn((nc, n_samples, N_INPUT), generator=g, device=device) * sigma
        im = torch.randn((nc, n_samples, N_INPUT), generator=g, device=device) * sigma
        for p in plane_waves:
            gain = np.stack([geometric_phase(f, p.u, p.s) * p.amplitude for f in fs])      # [nc, 2048]
            gr = torch.from_numpy(gain.real.astype(np.float32)).to(device).view(nc, 1, N_CYL * N_FEED, N_POL)
            gi = torch.from_numpy(gain.imag.astype(np.float32)).to(device).view(nc, 1, N_CYL * N_FEED, N_POL)
            ph = torch.rand((nc, n_samples, 1, N_POL), generator=g, device=device) * (2.0 * math.pi)
            cr, ci = torch.cos(ph), torch.sin(ph)
            re += (gr * cr - gi * ci).view(nc, n_samples, N_INPUT)
            im += (gr * ci + gi * cr).view(nc, n_samples, N_INPUT)
        qr = torch.clamp(torch.round(re), -7, 7).to(torch.int16) + 8
        qi = torch.clamp(torch.round(im), -7, 7).to(torch.int16) + 8
        out[c0:c0 + nc] = ((qr << 4) | qi).to(torch.uint8)
        del re, im, qr, qi
    return out

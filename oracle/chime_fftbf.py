"""FP64 reference ("oracle") for the CHIME/FRB hybrid FFT beamformer path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or call this module.  It shares no
code with the CUDA library and never imports the product package.

It writes out, in double precision and with direct O(N^2) sums (no FFT), what
the fan-beam pipeline of Sec. 3 computes for one coarse frequency channel:

  a0  unpack 4+4-bit offset-encoded voltages (Sec. 2, Table 1);
  a1  N-S beams: the 2x zero-padded 512-point DFT of each cylinder's 256-feed
      line, evaluated only at the clamped bins given by Eq. (1) (Sec. 3.1) --
      an FFT followed by the clamp yields exactly these values;
  a2  four E-W beams by exact phasing across the four cylinders (Sec. 3);
  a3  up-channelisation: a 128-point DFT of each non-overlapping block of 128
      samples of each beam and polarisation (Sec. 3.2), then fftshift;
  a4  Stokes I: |.|^2 summed over the two polarisations (Sec. 3);
  a5  integration to 16 sub-channels (8 fine channels each) and 0.983 ms
      (3 blocks) cadence (Sec. 3, Table 1).

Readings of points the paper leaves open (each is a plan parameter or a
convention chosen where the paper is silent):

* nibble order: high nibble = real, low nibble = imaginary, value = nibble - 8;
* input order inside a time sample: (cylinder * 256 + feed) * 2 + pol;
* forward transforms use exp(-i ...); a source at N-S direction cosine s puts
  feed phase exp(+2 pi i f n d s / c0), so it peaks at bin M f d s / c0;
* Eq. (1): L(m) = floor(N P f d s_m / c0 + 0.5) mod (N P), the product taken
  left to right in double precision; Eq. (2) is the same quantity evaluated
  incrementally, so Eq. (1) is evaluated directly for every channel;
* default pointings s_m = (m - 127.5) / 128, m = 0..255 (evenly spaced in sin);
* E-W: cylinder c sits at c * D (D = 20 m); beam j weights cylinder c by
  exp(-2 pi i f c D u_j / c0) with u_j = sin({-0.6, -0.2, 0.2, 0.6} deg);
* the tables follow the coarse-channel centre frequency;
* up-channel blocks start at sample 0, no window, unnormalised; after fftshift
  fine channel q' = 0 is the lowest frequency and sub-channel s holds
  q' = 8s..8s+7;
* integration is a plain sum; output is float ``[beam = 256 j + m][16 ch + s][frame]``;
* samples past the last whole 384-sample frame are dropped.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

C0 = 299_792_458.0


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Array and channelisation parameters (Sec. 1, Sec. 2, Sec. 3)."""
    n_cyl: int = 4
    n_feed: int = 256
    n_pol: int = 2
    pad: int = 2
    n_ew: int = 4
    upchan: int = 128
    f_ds: int = 8
    t_ds: int = 3
    feed_spacing_m: float = 0.3048
    cyl_spacing_m: float = 20.0

    @property
    def n_bins(self) -> int:          # M = N P
        return self.n_feed * self.pad

    @property
    def n_ns(self) -> int:            # number of N-S beams kept by the clamp
        return self.n_feed

    @property
    def n_sub(self) -> int:           # sub-channels per coarse channel
        return self.upchan // self.f_ds

    @property
    def frame(self) -> int:           # samples per output frame
        return self.upchan * self.t_ds

    @property
    def n_input(self) -> int:
        return self.n_cyl * self.n_feed * self.n_pol


CHIME = Geometry()


def default_ns_sin(g: Geometry = CHIME) -> np.ndarray:
    """Default N-S pointings: evenly spaced in sin(theta) over the horizon."""
    m = np.arange(g.n_ns, dtype=np.float64)
    return (m - (g.n_ns - 1) / 2.0) / (g.n_ns / 2.0)


def default_ew_sin() -> np.ndarray:
    return np.sin(np.deg2rad(np.array([-0.6, -0.2, 0.2, 0.6])))


# --- a0: unpack ---------------------------------------------------------------

def unpack(raw: np.ndarray, g: Geometry = CHIME) -> np.ndarray:
    """uint8 [..., T, n_input] -> complex128 [..., T, n_cyl, n_feed, n_pol]."""
    b = raw.astype(np.int64)
    z = ((b >> 4) - 8).astype(np.float64) + 1j * ((b & 15) - 8).astype(np.float64)
    return z.reshape(raw.shape[:-1] + (g.n_cyl, g.n_feed, g.n_pol))


# --- clamp table, Eq. (1) --------------------------------------------------------

def clamp_arg(freq_hz: float, ns_sin: np.ndarray, g: Geometry = CHIME) -> np.ndarray:
    """Unrounded Eq. (1) argument N*P*f*d*sin(theta)/c, left to right in FP64."""
    s = np.asarray(ns_sin, dtype=np.float64)
    return (((float(g.n_feed * g.pad) * float(freq_hz)) * g.feed_spacing_m) * s) / C0


def clamp_lut(freq_hz: float, ns_sin: Optional[np.ndarray] = None, g: Geometry = CHIME) -> np.ndarray:
    """Bin index in [0, M) of the zero-padded FFT kept for each N-S pointing (Eq. 1)."""
    if ns_sin is None:
        ns_sin = default_ns_sin(g)
    unwrapped = np.floor(clamp_arg(freq_hz, ns_sin, g) + 0.5).astype(np.int64)
    return np.mod(unwrapped, g.n_bins)


# --- a1: N-S beams --------------------------------------------------------------

def ns_dft_matrix(lut: np.ndarray, g: Geometry = CHIME) -> np.ndarray:
    """D[m, n] = exp(-2 pi i n L(m) / M), exponent reduced mod M in integers."""
    n = np.arange(g.n_feed, dtype=np.int64)
    e = np.mod(np.outer(np.asarray(lut, dtype=np.int64), n), g.n_bins)
    return np.exp(-2j * np.pi * e.astype(np.float64) / g.n_bins)


def ns_beams(x: np.ndarray, lut: np.ndarray, g: Geometry = CHIME) -> np.ndarray:
    """x [T, c, n, p] -> X [T, c, p, m]: direct DFT of the feed line at the clamped bins."""
    D = ns_dft_matrix(lut, g)                         # [m, n]
    xt = np.moveaxis(x, 2, 3)                          # [T, c, p, n]
    return xt @ D.T                                    # [T, c, p, m]


# --- a2: E-W beams ----------------------------------------------------------------

def ew_weights(freq_hz: float, ew_sin: Optional[np.ndarray] = None, g: Geometry = CHIME) -> np.ndarray:
    """w[c, j] = exp(-2 pi i f c D u_j / c0)."""
    if ew_sin is None:
        ew_sin = default_ew_sin()
    c = np.arange(g.n_cyl, dtype=np.float64)[:, None]
    u = np.asarray(ew_sin, dtype=np.float64)[None, :]
    cycles = (((float(freq_hz) * c) * g.cyl_spacing_m) * u) / C0
    return np.exp(-2j * np.pi * np.mod(cycles, 1.0))


def ew_beams(X: np.ndarray, w: np.ndarray) -> np.ndarray:
    """X [T, c, p, m] -> B [T, p, j, m] = sum_c X[T, c, p, m] w[c, j]."""
    return np.einsum("tcpm,cj->tpjm", X, w)


def ew_weights_tracking(freq_hz: float, ew_sin_frames: np.ndarray, g: Geometry = CHIME) -> np.ndarray:
    """Tracking E-W beams (Sec. 3.1: the E-W beams may be static or track the
    sky): beam j of output frame F points at ew_sin_frames[F, j].  Returns
    w [F, c, j], each frame's weights defined as for static beams."""
    u = np.asarray(ew_sin_frames, dtype=np.float64)
    return np.stack([ew_weights(freq_hz, u[F], g) for F in range(u.shape[0])])


def ew_beams_tracking(X: np.ndarray, W: np.ndarray, g: Geometry = CHIME) -> np.ndarray:
    """X [T, c, p, m], W [F, c, j] -> B [F * frame, p, j, m]: sample t uses the
    weights of the output frame t // frame it falls in; samples past the last
    whole frame are dropped (they reach no output)."""
    nf = W.shape[0]
    Xf = X[:nf * g.frame].reshape(nf, g.frame, *X.shape[1:])
    return np.einsum("ftcpm,fcj->ftpjm", Xf, W).reshape(nf * g.frame, X.shape[2], W.shape[2], X.shape[3])


# --- a3: up-channelisation ------------------------------------------------------------

def upchan_dft_matrix(g: Geometry = CHIME) -> np.ndarray:
    """F[q, tau] = exp(-2 pi i q tau / U)."""
    k = np.arange(g.upchan, dtype=np.int64)
    e = np.mod(np.outer(k, k), g.upchan)
    return np.exp(-2j * np.pi * e.astype(np.float64) / g.upchan)


def upchannelize(B: np.ndarray, g: Geometry = CHIME) -> np.ndarray:
    """B [T, p, j, m] -> Y [blk, p, j, m, q'] with q' the fftshifted fine channel."""
    U = g.upchan
    nblk = B.shape[0] // U
    Bb = B[: nblk * U].reshape((nblk, U) + B.shape[1:])          # [blk, tau, p, j, m]
    Bb = np.moveaxis(Bb, 1, -1)                                   # [blk, p, j, m, tau]
    Y = Bb @ upchan_dft_matrix(g).T                               # [blk, p, j, m, q]
    shift = (np.arange(U) + U // 2) % U                           # q for each q'
    return Y[..., shift]


# --- a4 + a5: detect and integrate --------------------------------------------------------

def detect_downsample(Y: np.ndarray, g: Geometry = CHIME) -> np.ndarray:
    """Y [blk, p, j, m, q'] -> O [j*n_ns + m, sub, frame] (sums over pol, 8 q', 3 blocks)."""
    nblk = Y.shape[0]
    nfr = nblk // g.t_ds
    P = (np.abs(Y[: nfr * g.t_ds]) ** 2).sum(axis=1)              # [blk, j, m, q']
    P = P.reshape(nfr, g.t_ds, g.n_ew, g.n_ns, g.n_sub, g.f_ds).sum(axis=(1, 5))
    return np.ascontiguousarray(np.transpose(P, (1, 2, 3, 0))).reshape(g.n_ew * g.n_ns, g.n_sub, nfr)


# --- whole path ---------------------------------------------------------------------------

def beamform_channel(raw: np.ndarray, freq_hz: float, ns_sin=None, ew_sin=None,
                     g: Geometry = CHIME, return_stages: bool = False, ew_sin_frames=None):
    """uint8 [T, 2048] of one coarse channel -> float64 [1024, 16, n_frames].

    ew_sin_frames [n_frames, 4], if given, replaces the static E-W pointings
    frame by frame (tracking beams)."""
    x = unpack(raw, g)
    X = ns_beams(x, clamp_lut(freq_hz, ns_sin, g), g)
    if ew_sin_frames is None:
        B = ew_beams(X, ew_weights(freq_hz, ew_sin, g))
    else:
        if len(ew_sin_frames) != raw.shape[0] // g.frame:
            raise ValueError("one row of E-W sines per output frame")
        B = ew_beams_tracking(X, ew_weights_tracking(freq_hz, ew_sin_frames, g), g)
    Y = upchannelize(B, g)
    O = detect_downsample(Y, g)
    if return_stages:
        return O, {"x": x, "X": X, "B": B, "Y": Y}
    return O


def beamform(raw: np.ndarray, freqs_hz: Sequence[float], ns_sin=None, ew_sin=None,
             g: Geometry = CHIME, ew_sin_frames=None) -> np.ndarray:
    """uint8 [n_chan, T, 2048] -> float64 [1024, 16 n_chan, n_frames]."""
    outs = [beamform_channel(raw[c], f, ns_sin, ew_sin, g, ew_sin_frames=ew_sin_frames)
            for c, f in enumerate(freqs_hz)]
    return np.concatenate(outs, axis=1)


def beamform_sample(raw: np.ndarray, freqs_hz: Sequence[float], picks,
                    ns_sin=None, ew_sin=None, g: Geometry = CHIME) -> np.ndarray:
    """Outputs for chosen (chan, beam, frame) triples: float64 [len(picks), 16].

    Evaluates the same definition restricted to one beam and one frame, so it
    runs at any stream length.
    """
    res = np.empty((len(picks), g.n_sub))
    F = upchan_dft_matrix(g)
    shift = (np.arange(g.upchan) + g.upchan // 2) % g.upchan
    for i, (ch, beam, fr) in enumerate(picks):
        j, m = divmod(int(beam), g.n_ns)
        f = float(freqs_hz[ch])
        lut = clamp_lut(f, ns_sin, g)
        d = ns_dft_matrix(lut[m:m + 1], g)[0]                  # [n]
        w = ew_weights(f, ew_sin, g)[:, j]                      # [c]
        t0 = int(fr) * g.frame
        x = unpack(raw[ch, t0:t0 + g.frame], g)                 # [384, c, n, p]
        b = np.einsum("tcnp,n,c->tp", x, d, w)                  # [384, p]
        blocks = b.reshape(g.t_ds, g.upchan, g.n_pol)           # [blk, tau, p]
        Y = np.einsum("qt,btp->bpq", F, blocks)[..., shift]     # [blk, p, q']
        P = (np.abs(Y) ** 2).sum(axis=(0, 1))                   # [q']
        res[i] = P.reshape(g.n_sub, g.f_ds).sum(axis=1)
    return res


# --- after the fan-beam path (NEXT items) -----------------------------------------------

def sky_map(O: np.ndarray) -> np.ndarray:
    """Frequency- and time-summed response per beam (the map of Fig. 3):
    O [beam, sub, frame] -> [beam]."""
    return np.asarray(O, dtype=np.float64).sum(axis=(1, 2))


def rescale_value(O: np.ndarray):
    """The unrounded 8-bit code value of every element and the row statistics
    (Table 1 lists 8-bit integer intensity; the scaling rule is not given).
    Reading: per (beam, sub-channel) row of frames, the mean and the population
    standard deviation over the row, v = 64 + 16 (x - mean) / std, i.e. the
    codes span -4 sigma .. +11.9 sigma in 1/16 sigma steps.  Plain definitions
    in FP64.  Returns (v float64 like O, constant bool [rows], stats float64
    [..., 2] = mean, std); v is 64 on a constant row."""
    X = np.asarray(O, dtype=np.float64).reshape(-1, O.shape[-1])
    mean = X.mean(axis=1)
    d = X - mean[:, None]
    sd = np.sqrt((d * d).mean(axis=1))
    const = np.all(X == X[:, :1], axis=1)
    v = np.full(X.shape, 64.0)
    ok = ~const
    v[ok] = 64.0 + 16.0 * d[ok] / sd[ok, None]
    sd = np.where(const, 0.0, sd)
    stats = np.stack([mean, sd], axis=1)
    return v.reshape(O.shape), const.reshape(O.shape[:-1]), stats.reshape(O.shape[:-1] + (2,))


def rescale_u8(O: np.ndarray):
    """8-bit output: code = clip(floor(v + 1/2), 0, 255) of rescale_value's v
    (round half up to the nearest 1/16 sigma step, clipped to one byte); a
    constant row gets code 64.  Returns (codes uint8 like O, stats float64
    [..., 2] = mean, std)."""
    v, _, stats = rescale_value(O)
    codes = np.clip(np.floor(v + 0.5), 0, 255).astype(np.uint8)
    return codes, stats


K_DM_S_MHZ2 = 4.148808e3        # dispersion constant, s MHz^2 / (pc cm^-3)


def subchannel_freqs(freqs_hz, g: Geometry = CHIME, chan_bw_hz: float = 390625.0) -> np.ndarray:
    """Centre frequency of every output sub-channel [16 n_chan]: fine channel q'
    sits at f + (q' - U/2) * bw/U (q' = 0 lowest), a sub-channel averages its
    f_ds fine channels."""
    fine = chan_bw_hz / g.upchan
    out = []
    for f in freqs_hz:
        for s in range(g.n_sub):
            out.append(float(f) + (g.f_ds * s + (g.f_ds - 1) / 2.0 - g.upchan // 2) * fine)
    return np.array(out)


def dedisperse_delays(freqs_hz, dm: float, frame_s: float = 384 * 2.56e-6, g: Geometry = CHIME) -> np.ndarray:
    """Delay in frames of every sub-channel relative to the highest one:
    floor(((K_DM DM) (1/(f f) - 1/(f_max f_max))) / T_frame + 1/2), f in MHz,
    FP64 in that order (Sec. 3.2: dispersion delays the lower frequencies)."""
    fs = [float(f) / 1e6 for f in subchannel_freqs(freqs_hz, g)]
    fmax = max(fs)
    out = []
    for f in fs:
        x = ((K_DM_S_MHZ2 * float(dm)) * (1.0 / (f * f) - 1.0 / (fmax * fmax))) / frame_s
        out.append(int(np.floor(x + 0.5)))
    return np.array(out)


def dedisperse(O: np.ndarray, freqs_hz, dm: float, g: Geometry = CHIME):
    """Incoherent dedispersion of the intensity output to one nominal DM (the
    fourth kernel proposed in Sec. 3.2): series[beam, t] = sum over sub-channels
    s of O[beam, s, t + d_s], for t < n_frames - max(d)."""
    d = dedisperse_delays(freqs_hz, dm, g=g)
    nf = O.shape[2]
    n_out = max(0, nf - int(d.max()))
    X = np.asarray(O, dtype=np.float64)
    series = np.zeros((O.shape[0], n_out))
    for s in range(O.shape[1]):
        series += X[:, s, d[s]:d[s] + n_out]
    return series, d

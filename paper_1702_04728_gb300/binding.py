"""ctypes binding of the C ABI in ``include/chimebf.h`` (argument marshalling only).

Every step of the beamformer runs in ``_lib/libchimebf.so``; this module only
packs arguments.  Torch tensors are accepted for device buffers and streams
(``data_ptr()`` / ``cuda_stream``).  Importing it does not load the library;
the first call does, and raises if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libchimebf.so")

BF_OK, BF_PENDING, BF_EQUEUED = 0, 1, 2
BF_EINVAL, BF_ENOMEM, BF_ECUDA, BF_ETIMEDOUT, BF_ENOTICKET, BF_ESHUTDOWN = -1, -2, -3, -4, -5, -6
BF_FP32_FFT, BF_TC_DFT256, BF_TC_DFT512, BF_TC_DFT256_X2, BF_TC_DFT256_X1 = 0, 1, 2, 3, 4
BF_MODE_DIRECT, BF_MODE_SERVING = 0, 1
BF_END_OF_STREAM = 1

N_BEAMS, N_SUB, FRAME, N_INPUT = 1024, 16, 384, 2048

SYMBOLS = ["bf_config_default", "bf_plan", "bf_frames_out", "bf_submit", "bf_poll", "bf_destroy",
           "bf_last_error", "bf_skymap", "bf_rescale_u8", "bf_dedisperse", "bf_debug_tables", "bf_debug_gather_order", "bf_debug_gemm", "bf_debug_unpack", "bf_debug_beams",
           "bf_debug_upchan", "bf_debug_stall", "bf_dedisperse_static", "bf_fp32_fma_probe",
           "bf_poll_timed"]


class BfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"chimebf error {code}: {msg}")
        self.code = code


class bf_config(ctypes.Structure):
    _fields_ = [("n_cyl", ctypes.c_int), ("n_feed", ctypes.c_int), ("n_pol", ctypes.c_int),
                ("pad", ctypes.c_int), ("n_ew", ctypes.c_int), ("upchan", ctypes.c_int),
                ("f_ds", ctypes.c_int), ("t_ds", ctypes.c_int),
                ("feed_spacing_m", ctypes.c_double), ("cyl_spacing_m", ctypes.c_double),
                ("dt_s", ctypes.c_double),
                ("ns_sin", ctypes.POINTER(ctypes.c_double)), ("ew_sin", ctypes.POINTER(ctypes.c_double)),
                ("form", ctypes.c_int), ("mode", ctypes.c_int), ("mem_budget", ctypes.c_size_t),
                ("max_streams", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("max_tables", ctypes.c_int)]


class bf_request(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_uint64), ("n_chan", ctypes.c_int),
                ("chan_freq_hz", ctypes.POINTER(ctypes.c_double)), ("n_samples", ctypes.c_int64),
                ("vin", ctypes.c_void_p), ("out", ctypes.c_void_p), ("flags", ctypes.c_int),
                ("ew_sin_frames", ctypes.POINTER(ctypes.c_double))]


_lib = None


def lib() -> ctypes.CDLL:
    """Load ``libchimebf.so`` (once); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the beamformer has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.bf_config_default.argtypes = [ctypes.POINTER(bf_config)]
        L.bf_plan.argtypes = [ctypes.POINTER(bf_config), ctypes.POINTER(P)]
        L.bf_frames_out.argtypes = [P, U64, I64, ctypes.POINTER(I64)]
        L.bf_submit.argtypes = [P, ctypes.POINTER(bf_request), ctypes.POINTER(U64)]
        L.bf_poll.argtypes = [P, U64, I64, ctypes.POINTER(I64)]
        L.bf_poll_timed.argtypes = [P, U64, I64, ctypes.POINTER(I64), ctypes.POINTER(D)]
        L.bf_destroy.argtypes = [P]
        L.bf_last_error.argtypes = []
        L.bf_last_error.restype = ctypes.c_char_p
        L.bf_debug_gather_order.argtypes = [ctypes.POINTER(bf_config), D, ctypes.POINTER(ctypes.c_int16)]
        L.bf_debug_tables.argtypes = [ctypes.POINTER(bf_config), D, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_float)]
        L.bf_debug_unpack.argtypes = [P, P, P, I64]
        L.bf_debug_beams.argtypes = [P, D, P, I64, P]
        L.bf_debug_upchan.argtypes = [P, D, P, I64, P]
        L.bf_debug_gemm.argtypes = [P, D, P, I64, P]
        L.bf_debug_stall.argtypes = [P, P, I64]
        L.bf_skymap.argtypes = [P, P, I64, I64, P]
        L.bf_rescale_u8.argtypes = [P, P, I64, I64, P, P]
        L.bf_dedisperse.argtypes = [P, P, I, ctypes.POINTER(D), I64, D, P, ctypes.POINTER(I64)]
        L.bf_dedisperse_static.argtypes = [P, P, I, ctypes.POINTER(D), I64, D, P, ctypes.POINTER(I64)]
        L.bf_fp32_fma_probe.argtypes = [P, I, I64, P, I64, ctypes.POINTER(D)]
        for name in SYMBOLS:
            getattr(L, name).restype = ctypes.c_char_p if name == "bf_last_error" else I
        _lib = L
    return _lib


def bf_last_error() -> str:
    return lib().bf_last_error().decode()


def _check(rc: int) -> int:
    if rc < 0:
        raise BfError(rc, bf_last_error())
    return rc


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _dbl_array(vals):
    if vals is None:
        return None, None
    arr = (ctypes.c_double * len(vals))(*[float(v) for v in vals])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), arr


CUDA_STREAM_LEGACY = 1      # cudaStreamLegacy: the legacy default stream


def stream_handle(s) -> Optional[int]:
    """cudaStream_t for a torch stream or an int; the legacy default stream
    (torch handle 0) maps to cudaStreamLegacy, since NULL asks the plan to
    create a stream of its own."""
    if s is None:
        return None
    h = getattr(s, "cuda_stream", s)
    return CUDA_STREAM_LEGACY if h == 0 else h


def bf_config_default(**kw) -> bf_config:
    cfg = bf_config()
    _check(lib().bf_config_default(ctypes.byref(cfg)))
    keep = []
    for k, v in kw.items():
        if k in ("ns_sin", "ew_sin"):
            ptr, arr = _dbl_array(v)
            keep.append(arr)
            setattr(cfg, k, ptr)
        elif k == "cuda_stream":
            cfg.cuda_stream = stream_handle(v)
        else:
            setattr(cfg, k, v)
    cfg._keep = keep                      # arrays must outlive bf_plan's copy
    return cfg


def bf_plan(cfg: bf_config) -> int:
    h = ctypes.c_void_p()
    _check(lib().bf_plan(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def bf_frames_out(plan: int, stream_id: int, n_samples: int) -> int:
    nf = ctypes.c_int64()
    _check(lib().bf_frames_out(plan, stream_id, n_samples, ctypes.byref(nf)))
    return nf.value


def bf_submit(plan: int, stream_id: int, freqs: Sequence[float], n_samples: int, vin, out,
              flags: int = 0, ew_sin_frames=None):
    """Returns (status, ticket); status is BF_OK or BF_EQUEUED.  ew_sin_frames:
    optional [n_frames_out][4] E-W beam sines per output frame (tracking)."""
    fptr, farr = _dbl_array(list(freqs))
    tptr, tarr = (None, None)
    if ew_sin_frames is not None:
        import numpy as np
        tptr, tarr = _dbl_array(np.asarray(ew_sin_frames, dtype=np.float64).ravel().tolist())
    req = bf_request(stream_id, len(freqs), fptr, n_samples, _ptr(vin), _ptr(out), flags, tptr)
    t = ctypes.c_uint64()
    rc = _check(lib().bf_submit(plan, ctypes.byref(req), ctypes.byref(t)))
    del farr, tarr
    return rc, t.value


def bf_poll(plan: int, ticket: int, timeout_us: int = -1):
    """Returns (status, n_frames_out); status BF_OK or BF_PENDING."""
    nf = ctypes.c_int64()
    rc = _check(lib().bf_poll(plan, ticket, timeout_us, ctypes.byref(nf)))
    return rc, nf.value


def bf_poll_timed(plan: int, ticket: int, timeout_us: int = -1):
    """Returns (status, n_frames_out, times): times = (submitted, launched, completion
    seen, collected) in seconds on the host's monotonic clock and the batch's device
    time in seconds, None while pending."""
    nf = ctypes.c_int64()
    times = (ctypes.c_double * 5)()
    rc = _check(lib().bf_poll_timed(plan, ticket, timeout_us, ctypes.byref(nf), times))
    return rc, nf.value, (tuple(times) if rc == BF_OK else None)


def bf_destroy(plan: int) -> None:
    _check(lib().bf_destroy(plan))


def bf_debug_gather_order(freq_hz: float, cfg: Optional[bf_config] = None):
    """Beam taken by each consumer slot (TMEM lane + 128 x bin half) of the FP32 form."""
    import numpy as np
    cfg = cfg or bf_config_default()
    order = (ctypes.c_int16 * 256)()
    _check(lib().bf_debug_gather_order(ctypes.byref(cfg), float(freq_hz), order))
    return np.frombuffer(order, dtype=np.int16).copy()


def bf_debug_tables(freq_hz: float, cfg: Optional[bf_config] = None):
    import numpy as np
    cfg = cfg or bf_config_default()
    lut = (ctypes.c_int32 * 256)()
    ew = (ctypes.c_float * 32)()
    _check(lib().bf_debug_tables(ctypes.byref(cfg), float(freq_hz), lut, ew))
    w = np.frombuffer(ew, dtype=np.float32).reshape(4, 4, 2)
    return np.frombuffer(lut, dtype=np.int32).copy(), (w[..., 0] + 1j * w[..., 1]).astype(np.complex64)


def bf_debug_unpack(plan: int, d_in, d_out, n: int) -> None:
    _check(lib().bf_debug_unpack(plan, _ptr(d_in), _ptr(d_out), n))


def bf_debug_beams(plan: int, freq_hz: float, d_vin, n_samples: int, d_out) -> None:
    _check(lib().bf_debug_beams(plan, float(freq_hz), _ptr(d_vin), n_samples, _ptr(d_out)))


def bf_debug_upchan(plan: int, freq_hz: float, d_vin, n_samples: int, d_out) -> None:
    _check(lib().bf_debug_upchan(plan, float(freq_hz), _ptr(d_vin), n_samples, _ptr(d_out)))


def bf_debug_gemm(plan: int, freq_hz: float, d_vin, n_samples: int, d_out) -> None:
    _check(lib().bf_debug_gemm(plan, float(freq_hz), _ptr(d_vin), n_samples, _ptr(d_out)))


def bf_debug_stall(plan: int, d_vin, wait_ns: int) -> int:
    """Returns the status code as is (BF_ETIMEDOUT is the expected outcome)."""
    return int(lib().bf_debug_stall(plan, _ptr(d_vin), int(wait_ns)))


def bf_skymap(plan: int, d_out, n_sub: int, n_frames: int, d_map) -> None:
    _check(lib().bf_skymap(plan, _ptr(d_out), n_sub, n_frames, _ptr(d_map)))


def bf_dedisperse(plan: int, d_out, freqs, n_frames: int, dm: float, d_series) -> int:
    """Returns n_out (frames of the dedispersed series)."""
    fptr, farr = _dbl_array(list(freqs))
    n = ctypes.c_int64()
    _check(lib().bf_dedisperse(plan, _ptr(d_out), len(freqs), fptr, n_frames, float(dm), _ptr(d_series),
                               ctypes.byref(n)))
    del farr
    return n.value


def bf_dedisperse_static(plan: int, d_out, freqs, n_frames: int, dm: float, d_series) -> int:
    """As bf_dedisperse, with the delay table in the library's static device array."""
    fptr, farr = _dbl_array(list(freqs))
    n = ctypes.c_int64()
    _check(lib().bf_dedisperse_static(plan, _ptr(d_out), len(freqs), fptr, n_frames, float(dm), _ptr(d_series),
                                      ctypes.byref(n)))
    del farr
    return n.value


def bf_rescale_u8(plan: int, d_out, n_rows: int, n_frames: int, d_codes, d_stats=None) -> None:
    _check(lib().bf_rescale_u8(plan, _ptr(d_out), n_rows, n_frames, _ptr(d_codes), _ptr(d_stats)))


def bf_fp32_fma_probe(stream, paired: bool, iters: int, d_sink, n_sink: int) -> float:
    """Enqueue the FP32 FMA-pipe probe on `stream`; returns the flops it issues."""
    f = ctypes.c_double()
    _check(lib().bf_fp32_fma_probe(stream_handle(stream), 1 if paired else 0, int(iters), _ptr(d_sink),
                                   int(n_sink), ctypes.byref(f)))
    return f.value


# ---- convenience over torch device memory (allocation and marshalling only) ----

class Plan:
    """Owns a bf_plan_t.  ``run`` submits one request and waits for it."""

    def __init__(self, mode: int = BF_MODE_DIRECT, stream="current", **cfg_kw):
        """stream: a torch stream or cudaStream_t; "current" (default) takes
        torch's current stream, None lets the plan create its own."""
        if isinstance(stream, str) and stream == "current":
            import torch
            stream = torch.cuda.current_stream()
        self.cfg = bf_config_default(mode=mode, cuda_stream=stream, **cfg_kw)
        self.handle = bf_plan(self.cfg)

    def frames_out(self, stream_id: int, n_samples: int) -> int:
        return bf_frames_out(self.handle, stream_id, n_samples)

    def submit(self, vin, freqs, out, stream_id: int = 0, flags: int = 0, n_samples: Optional[int] = None,
               ew_sin_frames=None):
        if n_samples is None:
            n_samples = vin.shape[-2]
        return bf_submit(self.handle, stream_id, freqs, n_samples, vin, out, flags, ew_sin_frames)

    def poll(self, ticket: int, timeout_us: int = -1):
        return bf_poll(self.handle, ticket, timeout_us)

    def poll_timed(self, ticket: int, timeout_us: int = -1):
        return bf_poll_timed(self.handle, ticket, timeout_us)

    def run(self, vin, freqs, stream_id: int = 0, flags: int = BF_END_OF_STREAM, ew_sin_frames=None):
        """vin: torch.uint8 CUDA tensor [n_chan, T, 2048] -> float32 [1024, 16 n_chan, n_frames]."""
        import torch
        n_chan, T = int(vin.shape[0]), int(vin.shape[1])
        nf = self.frames_out(stream_id, T)
        out = torch.empty((N_BEAMS, N_SUB * n_chan, nf), dtype=torch.float32, device=vin.device)
        _, t = self.submit(vin, freqs, out, stream_id, flags, T, ew_sin_frames)
        rc, got = self.poll(t)
        assert got == nf
        return out

    def skymap(self, out):
        """float32 [1024] sum over sub-channels and frames of a run() output."""
        import torch
        m = torch.empty(N_BEAMS, dtype=torch.float32, device=out.device)
        bf_skymap(self.handle, out, out.shape[1], out.shape[2], m)
        return m

    def dedisperse(self, out, freqs, dm: float):
        """float32 [1024, n_out] series of a run() output dedispersed to `dm`."""
        import torch
        flat = torch.empty(N_BEAMS * max(1, out.shape[2]), dtype=torch.float32, device=out.device)
        n = bf_dedisperse(self.handle, out, freqs, out.shape[2], dm, flat)
        return flat[: N_BEAMS * n].view(N_BEAMS, n)

    def rescale_u8(self, out):
        """(codes uint8 like out, stats float64 [1024, n_sub, 2]) of a run() output."""
        import torch
        codes = torch.empty(out.shape, dtype=torch.uint8, device=out.device)
        stats = torch.empty(out.shape[0], out.shape[1], 2, dtype=torch.float32, device=out.device)
        bf_rescale_u8(self.handle, out, out.shape[0] * out.shape[1], out.shape[2], codes, stats)
        return codes, stats

    def close(self) -> None:
        if self.handle:
            bf_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Throughput benchmark of the fused fan-beam path on one node slice.

Workload (one step): 4 coarse channels (410, 520, 650, 790 MHz) x 49152
samples x 2048 inputs of seeded synthetic 4+4-bit voltages with a DM-500
burst -> float32 [1024 beams][64 sub-channels][128 frames].  Inputs (402.7 MB)
are larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line.  ``value`` is device-timed input-samples/s with inputs
resident in HBM; ``e2e`` times the same work from pinned host memory through
the public API, copies included.  Under torchrun every rank processes its own
node slice (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "beamformed input-samples/s & HBM roofline %, FFT vs TC-DFT at stated err; p99 latency"
WORKLOAD = "node_slice: 4 ch (410/520/650/790 MHz) x 49152 samples x 2048 inputs, DM-500 burst"
N_CHAN, N_SAMP, N_INPUT = 4, 49152, 2048
FLOP_PER_SAMPLE = 162.0          # N-S 90 (5 N log2 N at N = 512 per 256 inputs) + E-W 32 + up-channel 35 + detect 5
BYTES_PER_SAMPLE = 1.0 + 1024 * 16 * 4 / (384 * 2048)   # 1 B in + float32 out
FORM_NAMES = {"BF_FP32_FFT": "fp32_fft", "BF_TC_DFT256": "tc_dft256_3term",
              "BF_TC_DFT256_X2": "tc_dft256_2term", "BF_TC_DFT256_X1": "tc_dft256_1term",
              "BF_TC_DFT512": "tc_dft512_1term"}
# tensor flop per input-sample of each tensor-core form: 8 real flop per (row, feed) and
# term, over the 256 clamped rows or all 512 rows of the zero-padded transform
TC_FLOP = {"tc_dft256_3term": 3 * 2048, "tc_dft256_2term": 2 * 2048, "tc_dft256_1term": 2048,
           "tc_dft512_1term": 4096}


def bench_config(form: str) -> dict:
    """The workload both arms report (static: no measured values)."""
    return {"workload": WORKLOAD, "n_chan": N_CHAN, "n_samples": N_SAMP, "n_inputs": N_INPUT,
            "form": FORM_NAMES[form], "output": "float32 [1024][64][128]",
            "l2": "inputs (402.7 MB) larger than L2; no flush"}


KERNEL_SOURCES = {
    "fused_fp32_kernel": ["fused_fp32.cu", "device_common.cuh", "bf_internal.h"],
    "fused_tc_kernel": ["fused_tc.cu", "device_common.cuh", "bf_internal.h"],
    "fused_tc_pair_kernel": ["fused_tc_pair.cu", "device_common.cuh", "bf_internal.h"],
}
# the kernel that runs each form's detecting launches
FORM_KERNEL = {"fp32_fft": "fused_fp32_kernel", "tc_dft256_3term": "fused_tc_kernel",
               "tc_dft256_2term": "fused_tc_kernel", "tc_dft256_1term": "fused_tc_pair_kernel",
               "tc_dft512_1term": "fused_tc_pair_kernel"}


def kernel_hash(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1702_04728_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(form: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    sources are unchanged since the capture (else None)."""
    kernel = FORM_KERNEL[form]
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[form]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("source_sha256") != kernel_hash(kernel):
        return None
    return rec.get("dram_bytes_per_launch")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_input(rank: int, world: int = 1):
    """Rank r's node slice: the 4 channels shifted by r coarse channels, seed per rank."""
    from paper_1702_04728_gb300 import dist as D, synth
    freqs = D.rank_channels(rank, world)
    raw, _, _ = synth.config_node_slice(seed=D.rank_seed(rank), freqs=freqs)
    return raw, freqs


def fp32_peak(B, torch, stream, iters=32768, reps=10):
    """Measured throughput of the FP32 FMA pipe (TFLOP/s): the library's FFMA2
    probe (4 CTAs per SM, 16 independent chains per thread), device-timed on
    `stream` after warm-up, with the SM clock sampled meanwhile; the scalar-FMA
    probe beside it."""
    n_sink = 4 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 256
    sink = torch.empty(n_sink, dtype=torch.float32, device="cuda")
    res = {}
    for paired, name in ((True, "ffma2"), (False, "ffma")):
        flop = 0.0
        for _ in range(3):
            flop = B.bf_fp32_fma_probe(stream, paired, iters, sink, n_sink)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            B.bf_fp32_fma_probe(stream, paired, iters, sink, n_sink)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"tflops": flop / (ms * 1e-3) / 1e12, "ms": ms}
    return res


def sweep_run(B, torch, stream, ws, roofline, steps=3):
    """64 channels over 400-800 MHz x 390625 samples (1 s) x 2048 inputs = 51.2 GB,
    counter-based noise with five dispersed bursts (DM 100-2000) generated on the
    device; device-timed per form."""
    from paper_1702_04728_gb300 import synth
    n_chan, T = 64, 390625
    vin = synth.hash_noise_device(11, n_chan, T, offsets=synth.burst_offsets(synth.SWEEP_FREQS, T, synth.SWEEP_BURSTS, 11))
    out = torch.empty(1024, 16 * n_chan, T // 384, dtype=torch.float32, device="cuda")
    res = {"workload": "64 ch (400-800 MHz) x 390625 samples x 2048 inputs (51.2 GB), noise and 5 bursts (DM 100-2000)",
           "forms": []}
    for fid, fname in [(B.BF_FP32_FFT, "fp32_fft"), (B.BF_TC_DFT256_X1, "tc_dft256_1term")]:
        p = B.Plan(stream=stream, form=fid)
        _, t = p.submit(vin, synth.SWEEP_FREQS, out, stream_id=3, flags=B.BF_END_OF_STREAM)
        p.poll(t)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tk = [p.submit(vin, synth.SWEEP_FREQS, out, stream_id=3, flags=B.BF_END_OF_STREAM)[1] for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        for t in tk:
            p.poll(t)
        p.close()
        ms = e0.elapsed_time(e1) / steps
        res["forms"].append({"form": fname, "ms_per_step": ms,
                             "input_samples_per_s": n_chan * T * N_INPUT / (ms * 1e-3),
                             "roofline": roofline(fname, n_chan * T * N_INPUT, ms)})
    del vin, out
    torch.cuda.empty_cache()
    return res


def serving_run(B, torch, capacity_sps, load, seconds, n_streams=200, seed=0, form=0):
    """Poisson arrivals of frames (384..49152 samples, 1..16 channels per stream)
    from n_streams streams at `load` x capacity; returns latency percentiles."""
    import random
    rng = random.Random(seed)
    max_chan, max_samp = 16, 49152
    pool_in = torch.randint(0, 256, (max_chan * max_samp * N_INPUT,), dtype=torch.uint8, device="cuda")
    pool_out = torch.empty(1024 * 16 * max_chan * (max_samp // 384), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()            # the serving plan runs on a stream of its own
    stream_chan = [rng.randint(1, max_chan) for _ in range(n_streams)]
    mean_samples = 8.5 * 384 * 64.5 * N_INPUT         # input-samples per request (mean)
    rate = load * capacity_sps / mean_samples          # requests per second
    plan = B.Plan(mode=B.BF_MODE_SERVING, stream=None, mem_budget=40 << 30, form=form)
    freqs = {s: [400e6 + 390625.0 * (rng.randrange(1024) + 0.5) for _ in range(stream_chan[s])]
             for s in range(n_streams)}
    # warm the per-frequency tables
    for s in range(n_streams):
        _, t = plan.submit(pool_in, freqs[s], pool_out, stream_id=10_000 + s, n_samples=384,
                           flags=B.BF_END_OF_STREAM)
        plan.poll(t)
    torch.cuda.synchronize()
    import queue as _queue
    pend = _queue.Queue()
    lat = []
    parts = {"queue": [], "stream_wait": [], "batch_exec": [], "collect": [], "done": []}

    def poller():                       # completions arrive in batch order; poll FIFO
        while True:
            item = pend.get()
            if item is None:
                return
            t, ts = item
            _, _, tm = plan.poll_timed(t)
            lat.append(time.perf_counter() - ts)
            # the runtime's timeline of the request: queued, on the GPU, waiting to be collected
            parts["queue"].append(tm[1] - tm[0])
            parts["stream_wait"].append(max(0.0, tm[2] - tm[1] - tm[4]))
            parts["batch_exec"].append(tm[4])
            parts["collect"].append(tm[3] - tm[2])
            parts["done"].append(tm[2] - tm[0])

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t0 = time.perf_counter()
    t_next = t0
    samples = 0
    while True:
        now = time.perf_counter()
        if now - t0 >= seconds:
            break
        if now < t_next:
            time.sleep(min(t_next - now, 0.0005))
            continue
        s = rng.randrange(n_streams)
        n = 384 * rng.randint(1, 128)
        ts = time.perf_counter()
        _, t = plan.submit(pool_in, freqs[s], pool_out, stream_id=s, n_samples=n, flags=B.BF_END_OF_STREAM)
        pend.put((t, ts))
        samples += stream_chan[s] * n * N_INPUT
        t_next += rng.expovariate(rate)
    pend.put(None)
    th.join()
    elapsed = time.perf_counter() - t0
    plan.close()
    lat.sort()
    pct = lambda q: 1e3 * lat[min(len(lat) - 1, int(q * len(lat)))]

    def pcts(v):
        v = sorted(v)
        return {"p50_ms": 1e3 * v[len(v) // 2], "p99_ms": 1e3 * v[min(len(v) - 1, int(0.99 * len(v)))]}
    return {"offered_load_frac": load, "offered_input_GBps": load * capacity_sps / 1e9,
            "requests": len(lat), "p50_ms": pct(0.50), "p99_ms": pct(0.99), "max_ms": 1e3 * lat[-1],
            "breakdown": {k: pcts(v) for k, v in parts.items() if v},
            "breakdown_note": "runtime timeline per request: queue = submit to its batch's launch, "
                              "stream_wait = launch to completion seen minus batch_exec (earlier batches still "
                              "on the stream), batch_exec = the batch's device time (CUDA events), collect = "
                              "completion to this poller's FIFO collection, done = submit to completion seen",
            "sustained_samples_per_s": samples / elapsed, "streams": n_streams, "seconds": seconds}


def cpu_baseline(raw, freqs, gpu_out=None, form_outs=None, frames_per_chan: int = 16):
    """The FP64 oracle as it stands, on the first frames of every channel."""
    import oracle.chime_fftbf as O
    T = frames_per_chan * 384
    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    ref = O.beamform(np.ascontiguousarray(raw[:, :T]), freqs)
    dt = time.perf_counter() - t0
    res = {"value": N_CHAN * T * N_INPUT / dt, "unit": "input-samples/s", "cores": cores, "kind": "oracle",
           "sample": f"first {frames_per_chan} frames ({T} samples) of each of the {N_CHAN} channels, "
                     f"numpy FP64 direct DFTs, {dt:.1f} s"}
    if gpu_out is not None:
        got = gpu_out[:, :, :frames_per_chan].astype(np.float64)
        res["max_rel_err_vs_gpu"] = float(np.max(np.abs(got - ref) / ref))
    for name, o in (form_outs or {}).items():
        got = o[:, :, :frames_per_chan].astype(np.float64)
        res.setdefault("max_rel_err_by_form", {})[name] = float(np.max(np.abs(got - ref) / ref))
        res.setdefault("rel_l2_err_by_form", {})[name] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return res


def oracle_one_core(raw, freqs, frames_per_chan: int = 1):
    """The oracle on one host core: a child process with single-threaded BLAS
    (the thread count is fixed when numpy loads, so it cannot change here)."""
    import subprocess
    import tempfile
    T = frames_per_chan * 384
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "raw.npy")
        np.save(path, np.ascontiguousarray(raw[:, :T]))
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = ("import sys, time, numpy as np; sys.path.insert(0, %r); import oracle.chime_fftbf as O; "
                "raw = np.load(%r); O.beamform(raw[:, :384], %r); t0 = time.perf_counter(); "
                "O.beamform(raw, %r); print(time.perf_counter() - t0)") % (ROOT, path, list(freqs), list(freqs))
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    dt = float(r.stdout.strip().splitlines()[-1])
    return {"value": N_CHAN * T * N_INPUT / dt, "unit": "input-samples/s", "cores": 1,
            "sample": f"first {frames_per_chan} frame(s) of each of the {N_CHAN} channels, single-threaded BLAS, "
                      f"{dt:.1f} s"}


def precision_run(B, torch, stream, roofline, steps=10):
    """The precision-form workload: each form's throughput on one 600 MHz channel of
    49152 samples (device-timed), and its output on the point-source data (one
    channel at 600 MHz, 3072 samples) for the error against the oracle."""
    from paper_1702_04728_gb300 import synth
    T = 49152
    vin = synth.hash_noise_device(3, 1, T)
    raw1, f1 = synth.config_point_source(0)
    vin1 = torch.from_numpy(raw1).cuda()
    out = torch.empty(1024, 16, T // 384, dtype=torch.float32, device="cuda")
    runs, outs1 = [], {}
    for name, fname in FORM_NAMES.items():
        p = B.Plan(stream=stream, form=getattr(B, name))
        for _ in range(3):
            p.poll(p.submit(vin, [600e6], out, stream_id=3, flags=B.BF_END_OF_STREAM)[1])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tk = [p.submit(vin, [600e6], out, stream_id=3, flags=B.BF_END_OF_STREAM)[1] for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        for t in tk:
            p.poll(t)
        ms = e0.elapsed_time(e1) / steps
        outs1[fname] = p.run(vin1, list(f1)).cpu().numpy()
        p.close()
        runs.append({"form": fname, "ms_per_step": ms, "input_samples_per_s": T * N_INPUT / (ms * 1e-3),
                     "roofline": roofline(fname, T * N_INPUT, ms)})
    return {"workload": "1 ch (600 MHz) x 49152 samples x 2048 inputs (100.7 MB); errors on the point-source "
                        "data (600 MHz, 3072 samples)", "forms": runs}, (raw1, f1, outs1)


def precision_errors(raw1, f1, outs1):
    """Max and relative-L2 error of each form's point-source output against the oracle."""
    import oracle.chime_fftbf as O
    ref = O.beamform(raw1, list(f1))
    res = {}
    for name, o in outs1.items():
        d = o.astype(np.float64) - ref
        res[name] = {"max_rel_err": float(np.max(np.abs(d) / ref)),
                     "rel_l2_err": float(np.linalg.norm(d) / np.linalg.norm(ref))}
    return res


def cpu_fft_baseline(B, raw, freqs, frames_per_chan: int = 16, gpu_out=None):
    """FP32 FFT pipeline on the host cores (torch.fft on CPU, all threads): unpack,
    zero-padded 512-point N-S FFT per (time, cylinder, pol), the clamped bins, E-W
    phasing, 128-point up-channel FFT per block, detection and the 8 x 3 sums.  The
    clamp table and E-W phases come from the library's host-side tables; a baseline
    timing, not a check (the oracle is the check)."""
    import torch
    T = frames_per_chan * 384
    cores = torch.get_num_threads()
    outs = []
    t0 = time.perf_counter()
    for c, f in enumerate(freqs):
        lut, w = B.bf_debug_tables(float(f))
        b = torch.from_numpy(np.ascontiguousarray(raw[c, :T])).to(torch.int16)
        x = torch.complex((b >> 4).float() - 8.0, (b & 15).float() - 8.0).reshape(T, 4, 256, 2)
        X = torch.fft.fft(x, n=512, dim=2)[:, :, torch.from_numpy(lut).long(), :]      # [T, cyl, m, pol]
        Bj = torch.einsum("tcmp,jc->tpjm", X, torch.from_numpy(w))                    # [T, pol, j, m]
        Y = torch.fft.fftshift(torch.fft.fft(Bj.reshape(T // 128, 128, 2, 4, 256), dim=1), dim=1)
        P = (Y.real ** 2 + Y.imag ** 2).sum(dim=2)                                      # [blk, q', j, m]
        O = P.reshape(frames_per_chan, 3, 16, 8, 4, 256).sum(dim=(1, 3))                # [F, s, j, m]
        outs.append(O.permute(2, 3, 1, 0).reshape(1024, 16, frames_per_chan))
    dt = time.perf_counter() - t0
    res = {"value": len(freqs) * T * N_INPUT / dt, "unit": "input-samples/s", "cores": cores,
           "kind": "fp32 fft (torch.fft on cpu)",
           "sample": f"first {frames_per_chan} frames ({T} samples) of each of the {len(freqs)} channels, {dt:.1f} s"}
    if gpu_out is not None:
        got = torch.cat(outs, dim=1).double().numpy()
        ref = gpu_out[:, :, :frames_per_chan].astype(np.float64)
        res["max_rel_diff_vs_gpu"] = float(np.max(np.abs(got - ref) / ref))
    return res


def run_reference(args):
    """The oracle as it stands on the host cores: W untimed and K timed steps, each
    one frame (384 samples) of every channel of the node slice, so that the run
    ends within minutes at the default step counts."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    raw, freqs = make_input(0, 1)
    for _ in range(args.warmup):
        cb = cpu_baseline(raw, freqs, frames_per_chan=1)
    t_all = time.perf_counter()
    for _ in range(args.steps):
        cb = cpu_baseline(raw, freqs, frames_per_chan=1)
    dt = time.perf_counter() - t_all
    v = args.steps * N_CHAN * 384 * N_INPUT / dt
    sample = (f"per step the first frame (384 samples) of each of the {N_CHAN} channels, numpy FP64 "
              f"direct DFTs, {1e3 * dt / args.steps:.0f} ms")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "input-samples/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(args.form),
            "cpu_baseline": {"value": v, "unit": "input-samples/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "input-samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    ap.add_argument("--sweep", type=int, default=1, help="time the 64-channel x 1 s sweep (0: skip)")
    ap.add_argument("--form", default="BF_FP32_FFT",
                    choices=list(FORM_NAMES))
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_1702_04728_gb300 import binding as B

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    raw, freqs = make_input(rank, ws)
    host_in = torch.from_numpy(raw).pin_memory()
    stream = torch.cuda.Stream()                 # copies, launches and events all on this stream
    torch.cuda.set_stream(stream)
    vin = host_in.to("cuda", non_blocking=True)
    plan = B.Plan(stream=stream)
    nf = N_SAMP // 384
    out = torch.empty(1024, 16 * N_CHAN, nf, dtype=torch.float32, device="cuda")
    host_out = torch.empty_like(out, device="cpu").pin_memory()

    def step(sid):
        st, t = plan.submit(vin, freqs, out, stream_id=sid, flags=B.BF_END_OF_STREAM)
        return t

    tickets = [step(1) for _ in range(args.warmup)]
    torch.cuda.synchronize()
    for t in tickets:
        plan.poll(t)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    form_names = {getattr(B, k): v for k, v in FORM_NAMES.items()}
    headline_form = getattr(B, args.form)
    if headline_form != B.BF_FP32_FFT:
        plan.close()
        plan = B.Plan(stream=stream, form=headline_form)
        tickets = [step(1) for _ in range(args.warmup)]
        for t in tickets:
            plan.poll(t)
    with ClockSampler(local) as clk:
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        tickets = [step(2) for _ in range(args.steps)]
        ev1.record(stream)
        barrier()
        for t in tickets:
            plan.poll(t)
        ms = ev0.elapsed_time(ev1) / args.steps
    clocks = clk.summary()
    with ClockSampler(local) as clk_probe:
        probe = fp32_peak(B, torch, stream)
    probe["clocks"] = clk_probe.summary()
    peaks, peak_kind = load_peaks()
    n_sm_dev = torch.cuda.get_device_properties(local).multi_processor_count

    def roofline(fname, n_samples, ms_):
        """Roofline of one form's launch: the tensor pipe (2048 GEMM flop per input-sample
        and term) for the tensor-core forms, the FP32 pipe (162 algorithmic flop per
        input-sample) for the FFT form, against the measured peaks."""
        if fname in TC_FLOP:
            achieved = TC_FLOP[fname] * n_samples / (ms_ * 1e-3) / 1e12
            pk = peaks.get("bf16_tflops", 1927.5)
            return {"bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                    "traffic": recorded_traffic(fname),
                    "peak_note": f"dense FP16 tensor peak = measured bf16 burst ({peak_kind}; FP16 and BF16 "
                                 f"share the rate); achieved = {TC_FLOP[fname]} GEMM flop per input-sample"}
        nominal = n_sm_dev * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        alu_peak = probe["ffma2"]["tflops"]
        achieved = FLOP_PER_SAMPLE * n_samples / (ms_ * 1e-3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": recorded_traffic(fname),
                "peak_note": f"FP32 FMA pipe, measured: the FFMA2 probe (4 CTAs/SM x 256 threads x 16 "
                             f"independent chains) at a median SM clock of {probe['clocks'].get('sm_mhz')} MHz; "
                             f"nominal {n_sm_dev} SMs x 128 lanes x 2 flop x "
                             f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz = {nominal:.1f}; "
                             f"achieved = {FLOP_PER_SAMPLE:.0f} algorithmic flop per input-sample",
                "frac_of_nominal": achieved / nominal}

    # products of the output (sky map, 8-bit rescale, dedispersion), device-timed
    def timed(fn, reps=20):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    smap = torch.empty(1024, dtype=torch.float32, device="cuda")
    codes = torch.empty(out.shape, dtype=torch.uint8, device="cuda")
    stats_u8 = torch.empty(out.shape[0], out.shape[1], 2, dtype=torch.float32, device="cuda")
    series = torch.empty(1024, out.shape[2], dtype=torch.float32, device="cuda")
    out_bytes = out.numel() * 4
    post = {"input": "node-slice output float32 [1024][64][128] (33.5 MB)"}
    t_map = timed(lambda: B.bf_skymap(plan.handle, out, out.shape[1], out.shape[2], smap))
    t_u8 = timed(lambda: B.bf_rescale_u8(plan.handle, out, out.shape[0] * out.shape[1], out.shape[2], codes,
                                          stats_u8))
    n_dd = B.bf_dedisperse(plan.handle, out, freqs, out.shape[2], 1.0, series)
    t_dd = timed(lambda: B.bf_dedisperse(plan.handle, out, freqs, out.shape[2], 1.0, series))
    post["skymap"] = {"ms": t_map, "GBps": out_bytes / (t_map * 1e-3) / 1e9}
    post["rescale_u8"] = {"ms": t_u8, "GBps": (out_bytes + out.numel() * 1.25) / (t_u8 * 1e-3) / 1e9,
                          "note": "FP32 statistics, three passes over each row"}
    post["dedisperse_dm1"] = {"ms": t_dd, "frames_out": n_dd,
                              "GBps": (1024 * 64 * n_dd * 4 + 1024 * n_dd * 4) / (t_dd * 1e-3) / 1e9}

    # every form on the same resident input (device-timed, same stream)
    form_runs = []
    form_outs = {}
    for fid, fname in form_names.items():
        fp = B.Plan(stream=stream, form=fid)
        fo = torch.empty_like(out)
        for _ in range(3):
            _, t = fp.submit(vin, freqs, fo, stream_id=7, flags=B.BF_END_OF_STREAM)
            fp.poll(t)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nrep = max(10, args.steps // 5)
        e0.record(stream)
        tk = [fp.submit(vin, freqs, fo, stream_id=7, flags=B.BF_END_OF_STREAM)[1] for _ in range(nrep)]
        e1.record(stream)
        barrier()
        for t in tk:
            fp.poll(t)
        fms = e0.elapsed_time(e1) / nrep
        fp.close()
        samples_ = N_CHAN * N_SAMP * N_INPUT
        run = {"form": fname, "ms_per_step": fms, "input_samples_per_s": samples_ / (fms * 1e-3),
               "roofline": roofline(fname, samples_, fms)}
        form_runs.append(run)
        form_outs[fname] = fo[:, :, :16].cpu().numpy()

    # end to end through the public API: pinned host in -> device -> beamform -> host out.
    # Each channel goes in requests of whole frames on one stream (the plan's carry state joins
    # them).  A request holds one wave of work items (SMs / 4 E-W beams frames), so no launch
    # ends with a partial wave; the remainder makes a short first piece for the first channel
    # and a short last piece for the others (the last one splits into half items).  Channels alternate between
    # two plans on two streams; the copy of piece i + 1 is issued before piece i's request, so
    # the copy engine never waits for the host.
    copy_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream()
    stream2 = torch.cuda.Stream()
    plan2 = B.Plan(stream=stream2, form=headline_form)
    e2e_plans = [(plan, stream), (plan2, stream2)]
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    wave = max(1, n_sm // 4)
    nfc = N_SAMP // 384
    full, rest = divmod(nfc, wave)
    sched = [([rest] if rest else []) + [wave] * full] + [[wave] * full + ([rest] if rest else [])] * (N_CHAN - 1)
    pieces = []
    for c in range(N_CHAN):
        lo = 0
        for k, nfr in enumerate(sched[c]):
            pieces.append((c, k, lo, lo + 384 * nfr, k == len(sched[c]) - 1))
            lo += 384 * nfr
    # Steps follow one another as in a continuous stream: step s uses device input and output
    # buffers s mod 2, so its copies overlap the previous step's last kernels; events keep a
    # buffer from being overwritten before the kernels (input) or the device->host copies
    # (output) of the step two back are done with it.
    vins = [vin, torch.empty_like(vin)]
    outs_p = [{(c, k): torch.empty(1024, 16, (hi - lo) // 384, dtype=torch.float32, device="cuda")
               for c, k, lo, hi, _ in pieces} for _ in range(2)]
    host_outs_p = {p_: torch.empty(tuple(v.shape), dtype=torch.float32).pin_memory() for p_, v in outs_p[0].items()}
    in_ev = [{p_[:2]: torch.cuda.Event() for p_ in pieces} for _ in range(2)]
    done_ev = [{p_[:2]: torch.cuda.Event() for p_ in pieces} for _ in range(2)]
    d2h_ev = [{p_[:2]: torch.cuda.Event() for p_ in pieces} for _ in range(2)]
    free_ev = [[torch.cuda.Event(), torch.cuda.Event()] for _ in range(2)]
    used = [False, False]

    def e2e_step(sidx, pending):
        bsel = sidx & 1
        vb, ob = vins[bsel], outs_p[bsel]
        if used[bsel]:
            for ev in free_ev[bsel]:                    # kernels of step sidx - 2 have read vb
                copy_s.wait_event(ev)

        def h2d(i):
            c, k, lo, hi, _ = pieces[i]
            with torch.cuda.stream(copy_s):
                vb[c, lo:hi].copy_(host_in[c, lo:hi], non_blocking=True)
                in_ev[bsel][(c, k)].record(copy_s)
        h2d(0)
        tk = []
        for i, (c, k, lo, hi, last) in enumerate(pieces):
            if i + 1 < len(pieces):
                h2d(i + 1)
            pl, st = e2e_plans[c % 2]
            st.wait_event(in_ev[bsel][(c, k)])          # beamform the piece once it has landed
            if used[bsel]:
                st.wait_event(d2h_ev[bsel][(c, k)])     # step sidx - 2 has read this output back
            _, t = pl.submit(vb[c:c + 1, lo:hi], freqs[c:c + 1], ob[(c, k)], stream_id=100 + c,
                             flags=B.BF_END_OF_STREAM if last else 0, n_samples=hi - lo)
            done_ev[bsel][(c, k)].record(st)
            tk.append((pl, t))
            with torch.cuda.stream(d2h_s):              # device->host of each output as it is done
                d2h_s.wait_event(done_ev[bsel][(c, k)])
                host_outs_p[(c, k)].copy_(ob[(c, k)], non_blocking=True)
                d2h_ev[bsel][(c, k)].record(d2h_s)
        free_ev[bsel][0].record(stream)
        free_ev[bsel][1].record(stream2)
        used[bsel] = True
        for pl, t in pending:                           # the previous step's tickets
            pl.poll(t)
        return tk

    def e2e_run(n, sync_each):
        pend = []
        for sidx in range(n):
            pend = e2e_step(sidx, pend)
            if sync_each:
                for pl, t in pend:
                    pl.poll(t)
                pend = []
                torch.cuda.synchronize()
        for pl, t in pend:
            pl.poll(t)
        torch.cuda.synchronize()

    e2e_run(2, False)
    e2e_run(1, True)
    barrier()
    t0 = time.perf_counter()
    e2e_run(args.e2e_steps, True)
    barrier()
    e2e_single_ms = (time.perf_counter() - t0) * 1e3 / args.e2e_steps
    t0 = time.perf_counter()
    e2e_run(args.e2e_steps, False)
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.e2e_steps
    # this box's pinned host -> device copy rate: one copy of the whole input, device-timed
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(4):
        if i == 1:
            c0.record(copy_s)
        with torch.cuda.stream(copy_s):
            vin.copy_(host_in, non_blocking=True)
    c1.record(copy_s)
    copy_s.synchronize()
    h2d_ms = c0.elapsed_time(c1) / 3
    host_out = torch.cat([torch.cat([host_outs_p[(c, k)] for k in range(len(sched[c]))], dim=2)
                          for c in range(N_CHAN)], dim=1)
    e2e_equal = bool(torch.equal(host_out, out.cpu()))     # the stream's output, bit for bit

    ms_t = torch.tensor([ms, e2e_ms], device="cuda")
    if ws > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms, e2e_ms = ms_t.tolist()
    samples = N_CHAN * N_SAMP * N_INPUT
    value = samples * ws / (ms * 1e-3)

    if rank == 0:
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        hbm_gbs = BYTES_PER_SAMPLE * samples / (ms * 1e-3) / 1e9
        fname = form_names[headline_form]
        terms = fname in TC_FLOP
        roof = roofline(fname, samples, ms)
        line = {
            "metric": METRIC, "value": value, "unit": "input-samples/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16-tc/f32" if terms else "f32",
            "data": "synthetic",
            "config": bench_config(args.form),
            "hbm": {"gbs": hbm_gbs, "frac_of_measured": hbm_gbs / peaks["hbm_gbs"]},
            "roofline": roof,
            "e2e": {"value": samples * ws / (e2e_ms * 1e-3), "unit": "input-samples/s",
                    "h2d_bytes_per_step": samples, "d2h_bytes_per_step": out.numel() * 4,
                    "ms_per_step": e2e_ms, "single_step_ms": e2e_single_ms, "h2d_copy_ms": h2d_ms,
                    "equals_device_output": e2e_equal,
                    "h2d_copy_GBps": samples / (h2d_ms * 1e-3) / 1e9, "how": f"wall clock over consecutive steps of a continuous stream; "
                                                  f"requests of {wave} frames (one wave of work items) per "
                                                  "channel on one stream, a short first and last piece, H2D of "
                                                  "the next piece overlapping beamforming of the previous one, "
                                                  "channels alternating between two plans on two streams, D2H "
                                                  "of each output; device buffers alternate between steps so a "
                                                  "step's copies overlap the previous step's last kernels; "
                                                  "single_step_ms: the same with a full synchronisation after "
                                                  "every step"},
            "gpu_launches": args.steps,
            "forms": form_runs,
            "post": post,
            "clocks": clocks,
            "fp32_probe": probe,
        }
        # the workloads reported beside the headline, and the host baselines, run at N = 1 only:
        # under torchrun the other ranks' GPUs would be held idle meanwhile
        extras = ws == 1
        prec, prec_outs = precision_run(B, torch, stream, roofline) if extras else (None, None)
        if extras:
            line["precision_forms"] = prec
        if args.sweep and extras:
            line["sweep"] = sweep_run(B, torch, stream, ws, roofline)
        if args.serving_seconds > 0 and extras:
            cap = samples / (ms * 1e-3)
            line["serving"] = [serving_run(B, torch, cap, ld, args.serving_seconds, form=headline_form)
                               for ld in (0.5, 0.9)]
            # the full-array offered load of 0.8 TB/s of packed voltage, above one GPU's capacity
            line["serving"].append(serving_run(B, torch, cap, 0.8e12 / cap, min(1.0, args.serving_seconds),
                                               form=headline_form))
        if not args.no_cpu_baseline and extras:
            line["cpu_baseline"] = cpu_baseline(raw, freqs, host_out.numpy(), form_outs)
            line["cpu_baseline"]["one_core"] = oracle_one_core(raw, freqs)
            line["precision_forms"]["errors_vs_oracle"] = precision_errors(*prec_outs)
            line["cpu_fft_baseline"] = cpu_fft_baseline(B, raw, freqs, gpu_out=host_out.numpy())
        print(json.dumps(line), flush=True)
    plan2.close()
    plan.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

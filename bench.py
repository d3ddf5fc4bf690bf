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
FLOP_PER_SAMPLE = 162.0          # conventional 5 N log2 N FFT count + E-W + detect (see design notes)
BYTES_PER_SAMPLE = 1.0 + 1024 * 16 * 4 / (384 * 2048)   # 1 B in + float32 out


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


def make_input(rank: int):
    from paper_1702_04728_gb300 import synth
    raw, freqs, _ = synth.config_node_slice(seed=rank)
    return raw, [float(f) for f in freqs]


def cpu_baseline(raw, freqs, gpu_out=None, frames_per_chan: int = 16):
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
    return res


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    raw, freqs = make_input(0)
    # each step is a bounded sample (3 frames of each channel) so the run ends in minutes
    steps = max(1, min(args.steps, 5))
    vals = []
    cpu_baseline(raw, freqs, frames_per_chan=1)          # warm-up (BLAS threads, caches)
    t_all = time.perf_counter()
    cb = None
    for _ in range(steps):
        cb = cpu_baseline(raw, freqs, frames_per_chan=3)
        vals.append(cb["value"])
    dt = time.perf_counter() - t_all
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "input-samples/s", "n_gpus": 1,
            "steps": len(vals), "warmup": 1, "ms_per_step": 1e3 * dt / len(vals), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": cb["sample"]},
            "cpu_baseline": {"value": v, "unit": "input-samples/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
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

    raw, freqs = make_input(rank)
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

    peaks, peak_kind = load_peaks()
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

    # end to end through the public API: pinned host in -> device -> beamform -> host out
    barrier()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.e2e_steps):
        vin.copy_(host_in, non_blocking=True)
        t = step(3)
        host_out.copy_(out, non_blocking=True)
        plan.poll(t)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / args.e2e_steps

    ms_t = torch.tensor([ms, e2e_ms], device="cuda")
    if ws > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms, e2e_ms = ms_t.tolist()
    samples = N_CHAN * N_SAMP * N_INPUT
    value = samples * ws / (ms * 1e-3)

    if rank == 0:
        sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        alu_peak = n_sm * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12   # FP32 TFLOP/s at max clock
        achieved = FLOP_PER_SAMPLE * samples / (ms * 1e-3) / 1e12
        hbm_gbs = BYTES_PER_SAMPLE * samples / (ms * 1e-3) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": "input-samples/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_chan": N_CHAN, "n_samples": N_SAMP, "n_inputs": N_INPUT,
                       "form": "fp32_fft", "output": "float32 [1024][64][128]",
                       "l2": "inputs (402.7 MB) larger than L2; no flush",
                       "hbm_gbs": hbm_gbs, "hbm_frac_of_measured": hbm_gbs / peaks["hbm_gbs"]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved / alu_peak, "traffic": None,
                         "peak_note": f"FP32 FMA pipe: {n_sm} SMs x 128 lanes x 2 flop x "
                                      f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({peak_kind} max clock); "
                                      f"achieved = {FLOP_PER_SAMPLE:.0f} algorithmic flop per input-sample"},
            "e2e": {"value": samples * ws / (e2e_ms * 1e-3), "unit": "input-samples/s",
                    "h2d_bytes_per_step": samples, "d2h_bytes_per_step": out.numel() * 4,
                    "ms_per_step": e2e_ms},
            "gpu_launches": args.steps,
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(raw, freqs, host_out.numpy())
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

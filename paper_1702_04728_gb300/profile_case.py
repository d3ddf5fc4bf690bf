"""Repeated launches of one fused kernel on a node-slice-sized input, for
profiler captures (``ncu -k <kernel> -s <n> -c <k>``) and quick timings.

    python -m paper_1702_04728_gb300.profile_case [--form fp32|tc1|tc2|tc3|tc512]
        [--launches N] [--n-chan 4] [--n-samples 49152]

The input is counter-based noise generated on the device (the same generator
as the 64-channel sweep), so start-up takes seconds and the device holds only
the input (n_chan x n_samples x 2048 bytes) and the output.  Each launch is one
request of all channels on the plan's stream; the script prints the mean
device time per launch (CUDA events around the launches after the first).
"""
from __future__ import annotations

import argparse
import json

FORMS = {"fp32": "BF_FP32_FFT", "tc3": "BF_TC_DFT256", "tc2": "BF_TC_DFT256_X2", "tc1": "BF_TC_DFT256_X1",
         "tc512": "BF_TC_DFT512"}
NODE_SLICE_HZ = (410e6, 520e6, 650e6, 790e6)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--form", default="fp32", choices=sorted(FORMS))
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--n-chan", type=int, default=4)
    ap.add_argument("--n-samples", type=int, default=49152)
    ap.add_argument("--seed", type=int, default=5)
    args = ap.parse_args(argv)

    import torch
    from paper_1702_04728_gb300 import binding as B, synth

    freqs = [NODE_SLICE_HZ[c % 4] + 390625.0 * (c // 4) for c in range(args.n_chan)]
    vin = synth.hash_noise_device(args.seed, args.n_chan, args.n_samples)
    stream = torch.cuda.current_stream()
    nf = args.n_samples // 384
    out = torch.empty(1024, 16 * args.n_chan, nf, dtype=torch.float32, device="cuda")
    with B.Plan(stream=stream, form=getattr(B, FORMS[args.form])) as p:
        _, t = p.submit(vin, freqs, out, stream_id=1, flags=B.BF_END_OF_STREAM)
        p.poll(t)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tickets = [p.submit(vin, freqs, out, stream_id=1, flags=B.BF_END_OF_STREAM)[1]
                   for _ in range(max(0, args.launches - 1))]
        e1.record(stream)
        torch.cuda.synchronize()
        for t in tickets:
            p.poll(t)
    ms = e0.elapsed_time(e1) / max(1, args.launches - 1)
    print(json.dumps({"form": args.form, "launches": args.launches, "n_chan": args.n_chan,
                      "n_samples": args.n_samples, "ms_per_launch": ms,
                      "input_samples_per_s": args.n_chan * args.n_samples * 2048 / (ms * 1e-3)}))


if __name__ == "__main__":
    main()

"""Serving mode: continuous batching of many channel streams of uneven length.

Each stream's output must be the same alone and in the mix (the kernel
computes every frame independently, so equality is bit for bit); requests
wait for memory under the admission budget and all complete; per-stream
order and carry state hold across batches.
"""
import threading

import numpy as np
import pytest

from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make_streams(n_streams, seed):
    rng = np.random.default_rng(seed)
    streams = []
    for s in range(n_streams):
        n_chan = int(rng.integers(1, 4))
        freqs = list(400e6 + 390625.0 * (rng.integers(0, 1024, size=n_chan) + 0.5))
        lens = [int(x) for x in rng.integers(1, 1500, size=int(rng.integers(1, 5)))]
        T = sum(lens)
        raw = synth.encode(rng.integers(-7, 8, size=(n_chan, T, 2048)), rng.integers(-7, 8, size=(n_chan, T, 2048)))
        streams.append({"id": 5000 + s, "freqs": freqs, "lens": lens, "raw": raw})
    return streams


def run_stream(plan, st, out_list, lock=None, budget_wait=False):
    """Submit the stream's requests in order; keep device buffers alive until polled."""
    raw_d = torch.from_numpy(st["raw"]).cuda()
    chunks, a = [], 0
    for n in st["lens"]:
        chunks.append(raw_d[:, a:a + n].contiguous())
        a += n
    torch.cuda.current_stream().synchronize()     # the plan may run on another stream
    pend = []
    for i, (n, chunk) in enumerate(zip(st["lens"], chunks)):
        flags = B.BF_END_OF_STREAM if i == len(st["lens"]) - 1 else 0
        nf = plan.frames_out(st["id"], n)
        out = torch.empty(1024, 16 * len(st["freqs"]), nf, dtype=torch.float32, device="cuda")
        rc, t = plan.submit(chunk, st["freqs"], out if nf else None, stream_id=st["id"], flags=flags, n_samples=n)
        pend.append((t, nf, out, chunk))
    outs = []
    for t, nf, out, chunk in pend:
        rc, got = plan.poll(t)
        assert rc == B.BF_OK and got == nf
        outs.append(out)
    out_list.append((st["id"], torch.cat(outs, dim=2).cpu()))


@pytest.mark.parametrize("form", [B.BF_FP32_FFT, B.BF_TC_DFT256, B.BF_TC_DFT256_X1, B.BF_TC_DFT512])
def test_mixed_batches_equal_alone(built_lib, form):
    """In the tensor-core form a mixed batch holds segments of many channel
    frequencies, so the twiddle images change from chunk to chunk within one
    launch; the results must still match the single-stream runs bit for bit."""
    streams = make_streams(10, seed=1)
    torch.cuda.synchronize()
    # alone: one stream at a time on a direct plan
    alone = {}
    with B.Plan(mode=B.BF_MODE_DIRECT, form=form) as p:
        for st in streams:
            res = []
            run_stream(p, st, res)
            alone[res[0][0]] = res[0][1]
    # mixed: all streams from 5 host threads on one serving plan
    mixed = []
    with B.Plan(mode=B.BF_MODE_SERVING, stream=None, form=form) as p:
        groups = [streams[i::5] for i in range(5)]
        ths = [threading.Thread(target=lambda g=g: [run_stream(p, st, mixed) for st in g]) for g in groups]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
    assert len(mixed) == len(streams)
    for sid, out in mixed:
        assert out.shape == alone[sid].shape
        assert torch.equal(out, alone[sid]), f"stream {sid} differs in the mix"


def test_admission_budget_queues_then_completes(built_lib):
    n = 384 * 4
    raw = torch.from_numpy(synth.noise_only([600e6], n, seed=3)).cuda()
    one = raw.numel() + 1024 * 16 * 4 * 4 + 383 * 2048
    with B.Plan(mode=B.BF_MODE_SERVING, stream=None, mem_budget=int(one * 1.5)) as p:
        outs, tickets, codes = [], [], []
        for s in range(4):
            out = torch.empty(1024, 16, 4, dtype=torch.float32, device="cuda")
            rc, t = p.submit(raw, [600e6], out, stream_id=700 + s, flags=B.BF_END_OF_STREAM)
            codes.append(rc)
            outs.append(out)
            tickets.append(t)
        assert B.BF_EQUEUED in codes
        for t in tickets:
            assert p.poll(t) == (B.BF_OK, 4)
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        with pytest.raises(B.BfError) as e:
            big = torch.zeros(1, 384 * 8, 2048, dtype=torch.uint8, device="cuda")
            p.submit(big, [600e6], torch.empty(1024, 16, 8, device="cuda"), stream_id=900)
        assert e.value.code == B.BF_ENOMEM


def test_poll_timeout_and_unknown_ticket(built_lib):
    with B.Plan(mode=B.BF_MODE_SERVING, stream=None) as p:
        raw = torch.from_numpy(synth.noise_only([700e6], 384 * 64, seed=4)).cuda()
        out = torch.empty(1024, 16, 64, dtype=torch.float32, device="cuda")
        _, t = p.submit(raw, [700e6], out, stream_id=1, flags=B.BF_END_OF_STREAM)
        rc, _ = p.poll(t, timeout_us=0)
        assert rc in (B.BF_OK, B.BF_PENDING)
        if rc == B.BF_PENDING:
            assert p.poll(t)[0] == B.BF_OK
        with pytest.raises(B.BfError) as e:
            p.poll(t)
        assert e.value.code == B.BF_ENOTICKET


def test_request_timeline_is_ordered(built_lib):
    # bf_poll_timed: submitted <= launched <= completion seen <= collected, for requests that
    # share batches and for one that waits behind them
    with B.Plan(mode=B.BF_MODE_SERVING, stream=None) as p:
        raw = torch.from_numpy(synth.noise_only([520e6], 384 * 32, seed=6)).cuda()
        outs = [torch.empty(1024, 16, 32, dtype=torch.float32, device="cuda") for _ in range(6)]
        torch.cuda.synchronize()
        tickets = [p.submit(raw, [520e6], outs[i], stream_id=20 + i, flags=B.BF_END_OF_STREAM)[1]
                   for i in range(6)]
        for t in tickets:
            rc, nf, tm = p.poll_timed(t)
            assert rc == B.BF_OK and nf == 32
            assert tm[0] <= tm[1] <= tm[2] <= tm[3]
            assert tm[3] - tm[0] < 10.0
            # the batch's device time fits between its launch and the completion being seen
            assert 0.0 < tm[4] <= (tm[2] - tm[0]) + 1e-3
        ref = outs[0].cpu()
        for o in outs[1:]:
            assert torch.equal(o.cpu(), ref)


def test_destroy_drains_outstanding_work(built_lib):
    raw = torch.from_numpy(synth.noise_only([650e6], 384 * 16, seed=5)).cuda()
    ref_plan = B.Plan()
    ref = ref_plan.run(raw, [650e6])
    ref_plan.close()
    p = B.Plan(mode=B.BF_MODE_SERVING, stream=None)
    outs = []
    for s in range(6):
        out = torch.empty_like(ref)
        p.submit(raw, [650e6], out, stream_id=10 + s, flags=B.BF_END_OF_STREAM)
        outs.append(out)
    p.close()                      # drains the queue and the device work
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)

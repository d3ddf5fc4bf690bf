"""Failure detection without a GPU fault.

* A device-side wait that nothing will release runs out: the tensor-core
  kernel is launched with its MMA warp idle and a 2 ms bound on every
  mbarrier wait; it must return BF_ETIMEDOUT quickly (no trap, no unbounded
  spin), and the plan and the CUDA context must stay usable.
* A host producer that dies in the middle of its stream (never sends the end
  of the stream) does not hold up the other streams of a serving plan, and
  the plan still drains and frees everything at destroy.
"""
import threading
import time

import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(got, ref):
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref) / np.abs(ref)))


# FP32 and 3-term plans run the single-CTA tensor-core kernel's check; the 1-term and
# 512-row plans run their own cluster kernel's (CTA-to-CTA copies, then an abort drain)
@pytest.mark.parametrize("form", [B.BF_FP32_FFT, B.BF_TC_DFT256, B.BF_TC_DFT256_X1, B.BF_TC_DFT512])
def test_device_wait_expires_and_context_survives(built_lib, form):
    freq = 600e6
    raw = synth.noise_only([freq], 384, seed=60)
    with B.Plan(form=form) as p:
        vin = dev(raw[0])
        t0 = time.perf_counter()
        rc = B.bf_debug_stall(p.handle, vin, 2_000_000)
        elapsed = time.perf_counter() - t0
        assert rc == B.BF_ETIMEDOUT
        assert elapsed < 5.0
        # the status word was cleared and the context still runs work correctly
        out = p.run(dev(raw), [freq]).cpu().numpy()
        tol = 1e-5 if form in (B.BF_FP32_FFT, B.BF_TC_DFT256) else 1e-3
        assert rel_err(out, O.beamform(raw, [freq])) <= tol
        assert B.bf_debug_stall(p.handle, vin, 1_000_000) == B.BF_ETIMEDOUT


def test_stall_check_rejects_bad_bounds(built_lib):
    raw = synth.noise_only([600e6], 384, seed=61)
    with B.Plan() as p:
        vin = dev(raw[0])
        assert B.bf_debug_stall(p.handle, vin, 0) == B.BF_EINVAL
        assert B.bf_debug_stall(p.handle, vin, 3_000_000_000) == B.BF_EINVAL


def test_dead_producer_does_not_block_other_streams(built_lib):
    freqs = [480e6, 610e6]
    n_streams, n_parts, part = 4, 4, 384 * 2 + 100
    raws = [synth.noise_only(freqs, n_parts * part, seed=70 + i) for i in range(n_streams)]
    results, errors = {}, {}
    with B.Plan(mode=B.BF_MODE_SERVING) as p:
        torch.cuda.synchronize()

        def producer(i):
            try:
                outs, keep = [], []
                for k in range(n_parts):
                    if i == 1 and k == 2:
                        raise RuntimeError("producer died mid-stream")
                    chunk = raws[i][:, k * part:(k + 1) * part]
                    nf = p.frames_out(200 + i, part)
                    out = torch.empty((1024, 32, nf), dtype=torch.float32, device="cuda")
                    vin = dev(chunk)
                    torch.cuda.synchronize()
                    flags = B.BF_END_OF_STREAM if k == n_parts - 1 else 0
                    _, t = p.submit(vin, freqs, out, stream_id=200 + i, flags=flags)
                    keep.append(vin)
                    p.poll(t)
                    outs.append(out.cpu().numpy())
                results[i] = np.concatenate(outs, axis=2)
            except RuntimeError as e:
                errors[i] = str(e)

        threads = [threading.Thread(target=producer, args=(i,)) for i in range(n_streams)]
        for th in threads:
            th.start()
        for th in threads:
            th.join(timeout=120)
        assert not any(th.is_alive() for th in threads)
    # destroy drained the plan with stream 201 never ended
    assert set(errors) == {1}
    assert set(results) == {0, 2, 3}
    for i in results:
        ref = O.beamform(raws[i], freqs)
        assert results[i].shape == ref.shape
        assert rel_err(results[i], ref) <= 1e-5

"""Per-frequency table slots (clamp table of Eq. 1, E-W phases, tensor-core
twiddle image): a plan holds bf_config.max_tables of them and reuses the
least recently used one that no open stream and no running batch references.

A serving plan with 64 slots runs 1100 requests of distinct frequencies (more
than 17 times its slots) with up to 24 in flight, for the FP32 form and the
1-term tensor-core forms (256 rows: twiddle images per slot; 512 rows: the
bin-to-beams tables per slot); sampled results match the oracle, and a frequency
whose slot was refilled many times over gives the same bits as on first use.
More distinct frequencies than slots in one request fail cleanly.
"""
import collections

import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("form,tol", [(B.BF_FP32_FFT, 1e-5), (B.BF_TC_DFT256_X1, 1e-3), (B.BF_TC_DFT512, 1e-3)])
def test_serving_plan_reuses_table_slots(built_lib, form, tol):
    n_req, in_flight = 1100, 24
    rng = np.random.default_rng(17)
    raw = synth.encode(rng.integers(-7, 8, size=(1, 768, 2048)), rng.integers(-7, 8, size=(1, 768, 2048)))
    vin = dev(raw)
    freqs = [400e6 + 363377.0 * k for k in range(n_req)]          # 1100 distinct frequencies, 400-800 MHz
    checks = set(range(0, n_req, 61)) | {n_req - 1}
    first = {}
    with B.Plan(mode=B.BF_MODE_SERVING, stream=None, form=form, max_tables=64) as p:
        pending = collections.deque()

        def retire_one():
            k, t, out = pending.popleft()
            assert p.poll(t) == (B.BF_OK, 2)
            if k in checks:
                first[k] = out.cpu()

        for k in range(n_req):
            out = torch.empty(1024, 16, 2, dtype=torch.float32, device="cuda")
            _, t = p.submit(vin, [freqs[k]], out, stream_id=k, flags=B.BF_END_OF_STREAM)
            pending.append((k, t, out))
            while len(pending) > in_flight:
                retire_one()
        while pending:
            retire_one()
        # frequency 0's slot has been reused ~17 times since: run it again
        again = torch.empty(1024, 16, 2, dtype=torch.float32, device="cuda")
        _, t = p.submit(vin, [freqs[0]], again, stream_id=5000, flags=B.BF_END_OF_STREAM)
        assert p.poll(t) == (B.BF_OK, 2)
        assert torch.equal(again.cpu(), first[0])
    for k in sorted(checks):
        ref = O.beamform(raw, [freqs[k]])
        err = float(np.max(np.abs(first[k].numpy().astype(np.float64) - ref) / ref))
        assert err <= tol, f"request {k} ({freqs[k] / 1e6:.3f} MHz): max relative error {err:.3e}"


def test_more_frequencies_than_slots_in_one_request_fails_cleanly(built_lib):
    raw = synth.noise_only([600e6], 384, seed=3)
    vin = dev(np.repeat(raw, 9, axis=0))
    out = torch.empty(1024, 16 * 9, 1, dtype=torch.float32, device="cuda")
    with B.Plan(max_tables=8) as p:
        with pytest.raises(B.BfError) as e:
            p.submit(vin, [500e6 + 1e5 * k for k in range(9)], out, stream_id=1, flags=B.BF_END_OF_STREAM)
        assert e.value.code == B.BF_ENOMEM
        # the plan still works, and a request that fits after the failed one is correct
        got = p.run(vin[:8], [500e6 + 1e5 * k for k in range(8)]).cpu().numpy()
    ref = O.beamform(np.repeat(raw, 8, axis=0), [500e6 + 1e5 * k for k in range(8)])
    assert np.max(np.abs(got - ref) / ref) <= 1e-5

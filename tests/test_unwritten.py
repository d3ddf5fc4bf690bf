"""Every output element is written: output buffers filled with NaN before the run
hold only finite, positive intensities after it, for every N-S form, across
ragged multi-channel requests, requests small enough to run as split items,
and a stream cut into requests with carried samples."""
import numpy as np
import pytest

from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMS = [B.BF_FP32_FFT, B.BF_TC_DFT256, B.BF_TC_DFT256_X2, B.BF_TC_DFT256_X1, B.BF_TC_DFT512]


def poisoned(n_chan, nf):
    return torch.full((1024, 16 * n_chan, nf), float("nan"), dtype=torch.float32, device="cuda")


def run_into(p, raw, freqs, out, stream_id, flags):
    vin = torch.from_numpy(np.ascontiguousarray(raw)).cuda()
    torch.cuda.synchronize()
    _, t = p.submit(vin, freqs, out, stream_id=stream_id, flags=flags, n_samples=raw.shape[1])
    return p.poll(t)


def all_written(out):
    return bool(torch.isfinite(out).all()) and bool((out > 0).all())


@pytest.mark.parametrize("form", FORMS)
def test_every_output_element_is_written(built_lib, form):
    with B.Plan(form=form) as p:
        # ragged multi-channel request: 5 whole frames per channel, 100 samples dropped
        freqs = [430e6, 610e6, 777e6]
        raw = synth.noise_only(freqs, 384 * 5 + 100, seed=51)
        out = poisoned(3, 5)
        assert run_into(p, raw, freqs, out, 1, B.BF_END_OF_STREAM) == (B.BF_OK, 5)
        assert all_written(out)
        # one frame of one channel: 4 work items, run as split halves where the form splits
        raw1 = synth.noise_only([520e6], 384, seed=52)
        out1 = poisoned(1, 1)
        assert run_into(p, raw1, [520e6], out1, 2, B.BF_END_OF_STREAM) == (B.BF_OK, 1)
        assert all_written(out1)
        # a stream cut into two requests: 123 samples carried from the first into the second
        raw2 = synth.noise_only([690e6, 701e6], 384 * 4, seed=53)
        cut = 384 + 123
        outa, outb = poisoned(2, 1), poisoned(2, 3)
        assert run_into(p, raw2[:, :cut], [690e6, 701e6], outa, 3, 0) == (B.BF_OK, 1)
        assert run_into(p, raw2[:, cut:], [690e6, 701e6], outb, 3, B.BF_END_OF_STREAM) == (B.BF_OK, 3)
        assert all_written(outa) and all_written(outb)

"""Whole-frame parity at full size, in the launch configuration the benchmark
times (the 4-channel node slice in one request): every one of the 1024 beams x
64 sub-channels of frames 0, 37, 38, 126 and 127 against the FP64 oracle.

With 152 SMs one wave of work items is 38 frames (4 E-W beams each), so frames
37 / 38 straddle the first wave edge, and the last frames of each channel
fall in the final partial wave, whose items run as two halves on two CTAs
(the tail split).  Tolerance 1e-5 relative for the FP32 form and the 3-term
tensor-core form, 1e-3 for the 1-term form.
"""
import numpy as np
import pytest

import oracle.chime_fftbf as O
from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FRAMES = (0, 37, 38, 126, 127)


@pytest.fixture(scope="module")
def node_slice(built_lib):
    raw, freqs, _ = synth.config_node_slice(0)
    ref = {}
    for F in FRAMES:
        rows = raw[:, 384 * F:384 * (F + 1)]
        ref[F] = O.beamform(rows, list(freqs))[:, :, 0]          # [1024, 64]
    return raw, list(freqs), ref


@pytest.mark.parametrize("form,tol", [(B.BF_FP32_FFT, 1e-5), (B.BF_TC_DFT256, 1e-5), (B.BF_TC_DFT256_X1, 1e-3),
                                      (B.BF_TC_DFT512, 1e-3)])
def test_whole_frames_of_the_node_slice(node_slice, form, tol):
    raw, freqs, ref = node_slice
    vin = torch.from_numpy(raw).cuda()
    with B.Plan(form=form) as p:
        out = p.run(vin, freqs)
        torch.cuda.synchronize()
        assert out.shape == (1024, 64, 128)
        for F in FRAMES:
            got = out[:, :, F].cpu().numpy().astype(np.float64)
            err = np.abs(got - ref[F]) / ref[F]
            assert err.max() <= tol, f"frame {F}: max relative error {err.max():.3e} at {np.unravel_index(err.argmax(), err.shape)}"

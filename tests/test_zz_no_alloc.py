"""Allocation-free dedispersion (bf_dedisperse_static) against bf_dedisperse.

bf_dedisperse_static serves callers that cannot allocate device memory (its
delay table is a file-scope device array instead of plan memory grown with
cudaFree + cudaMalloc).  Collected last on purpose: it must hold both in a
fresh process (the first call performs the per-device set-up) and after every
other test.  Two calls
in a row with different channel sets and DMs check that the shared static
delay table carries nothing over from one call to the next.
"""
import ctypes

import numpy as np
import pytest

from paper_1702_04728_gb300 import binding as B
from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_static_table_matches_allocating_entry_point(built_lib):
    cases = [([410e6, 520e6, 650e6, 790e6], 12 * 384 + 40, 0.5),      # max delay 9 of 12 frames
             ([600e6, 605e6], 9 * 384, 20.0)]                       # max delay 4 of 9 frames
    with B.Plan() as p:
        outs = [(p.run(dev(synth.noise_only(f, n, seed=80 + i)), f), f, dm) for i, (f, n, dm) in enumerate(cases)]
        for out, freqs, dm in outs:                  # two calls in a row, different tables
            nf = out.shape[2]
            a = torch.full((1024 * nf,), -1.0, dtype=torch.float32, device="cuda")
            b = torch.full((1024 * nf,), -2.0, dtype=torch.float32, device="cuda")
            na = B.bf_dedisperse(p.handle, out, freqs, nf, dm, a)
            nb = B.bf_dedisperse_static(p.handle, out, freqs, nf, dm, b)
            assert na == nb and na > 0
            # the same kernel on the same delays: identical bits, and nothing past n_out written
            assert torch.equal(a[:1024 * na], b[:1024 * nb])
            assert torch.all(b[1024 * nb:] == -2.0)


def test_static_table_rejects_too_many_channels(built_lib):
    with B.Plan() as p:
        out = torch.zeros(1024, 16 * 4097, 1, dtype=torch.float32, device="cuda")
        series = torch.empty(1024, dtype=torch.float32, device="cuda")
        with pytest.raises(B.BfError) as e:
            B.bf_dedisperse_static(p.handle, out, [500e6] * 4097, 1, 10.0, series)
        assert e.value.code == B.BF_EINVAL
        # channel counts whose sub-channel count overflows an int are refused before the
        # frequency array (one entry here) is read
        one = (ctypes.c_double * 1)(500e6)
        n = ctypes.c_int64()
        for n_chan in (2 ** 31 - 1, 2 ** 28, 4097):
            rc = B.lib().bf_dedisperse_static(p.handle, out.data_ptr(), n_chan, one, 1, 10.0, series.data_ptr(),
                                              ctypes.byref(n))
            assert rc == B.BF_EINVAL

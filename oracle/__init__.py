"""FP64 reference implementation of the fan-beam path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.
"""
from .chime_fftbf import *  # noqa: F401,F403

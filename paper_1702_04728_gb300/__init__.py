"""GB300-native CHIME/FRB hybrid FFT beamformer (arXiv 1702.04728).

The compute path lives in the CUDA library ``libchimebf.so`` built from
``csrc/`` and is reached through the C ABI declared in ``include/chimebf.h``;
``binding`` is the thin ctypes layer over it.  ``synth`` generates seeded
synthetic voltages.
"""
__all__ = ["binding", "synth"]

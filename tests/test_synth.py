"""The seeded input generators: host and device counter-based noise agree bit
for bit, and the quantised noise has the variance of clip(round(N(0, 2.5^2)))."""
import numpy as np
import pytest

from paper_1702_04728_gb300 import synth

torch = pytest.importorskip("torch")


def test_hash_noise_host_equals_device_on_cpu():
    dev = synth.hash_noise_device(5, 3, 50, device="cpu", chunk=1 << 12).numpy()
    for ch in range(3):
        assert np.array_equal(synth.hash_noise_rows(5, ch, 50, 0, 50), dev[ch])
    assert np.array_equal(synth.hash_noise_rows(5, 2, 50, 17, 23), dev[2, 17:23])


def test_hash_noise_distribution():
    x = synth.hash_noise_rows(9, 0, 3000, 0, 3000)
    re = (x >> 4).astype(int) - 8
    im = (x & 15).astype(int) - 8
    v = synth.quantized_noise_variance()
    n = re.size
    for part in (re, im):
        assert part.min() >= -7 and part.max() <= 7
        assert abs(part.mean()) < 5 * np.sqrt(v / n)
        assert abs(part.var() / v - 1) < 0.005
    assert abs(np.corrcoef(re.ravel()[:200000], im.ravel()[:200000])[0, 1]) < 0.01


def test_encode_rejects_out_of_range():
    with pytest.raises(ValueError):
        synth.encode(np.array([8]), np.array([0]))


def test_burst_offsets_host_equals_device_on_cpu():
    rng = np.random.default_rng(1)
    off = (rng.integers(-127, 128, size=(3, 50)).astype(np.int8), rng.integers(-127, 128, size=(3, 50)).astype(np.int8))
    dev = synth.hash_noise_device(5, 3, 50, device="cpu", chunk=1 << 12, offsets=off).numpy()
    for ch in range(3):
        assert np.array_equal(synth.hash_noise_rows(5, ch, 50, 0, 50, offsets=off), dev[ch])
    zero = (np.zeros((3, 50), np.int8), np.zeros((3, 50), np.int8))
    assert np.array_equal(synth.hash_noise_device(5, 3, 50, device="cpu", chunk=1 << 12, offsets=zero).numpy(),
                          synth.hash_noise_device(5, 3, 50, device="cpu", chunk=1 << 12).numpy())
    # row BURST_R of the table is the plain noise threshold set
    assert synth.burst_thresholds()[synth.BURST_R].tolist() == synth.noise_thresholds()


def test_burst_offset_shifts_the_quantised_mean():
    """A constant offset b moves the mean of clip(round(N(0, 2.5^2) + b)) by b
    (to first order: the clip at +-7 is 2.8 sigma away)."""
    n = 200000
    b = 40                                                   # 40 / 256 count
    off = (np.full((1, n // 2048 + 1), b, np.int8), np.zeros((1, n // 2048 + 1), np.int8))
    x = synth.hash_noise_rows(3, 0, n // 2048 + 1, 0, n // 2048 + 1, offsets=off)
    re = (x >> 4).astype(float) - 8
    im = (x & 15).astype(float) - 8
    se = np.sqrt(synth.quantized_noise_variance() / re.size)
    assert abs(re.mean() - b / synth.BURST_Q) < 5 * se + 0.002
    assert abs(im.mean()) < 5 * se

"""The shared seeded input generator (no FFT arithmetic)."""
import numpy as np

from fftu_inputs import complex_uniform, complex_uniform_range, splitmix64


def test_splitmix64_known_words():
    # SplitMix64 with seed 0: the first outputs of the published generator
    # (state advanced by 0x9E3779B97F4A7C15 before mixing).
    got = splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_range_and_determinism():
    a = complex_uniform(7, (4, 8, 16))
    b = complex_uniform(7, (4, 8, 16))
    assert np.array_equal(a, b)
    assert np.all(np.abs(a.real) <= 1) and np.all(np.abs(a.imag) <= 1)
    assert abs(a.real.mean()) < 0.1 and abs(a.imag.mean()) < 0.1
    assert not np.array_equal(a, complex_uniform(8, (4, 8, 16)))


def test_subrange_matches_full_array():
    full = complex_uniform(9, (1000,))
    part = complex_uniform_range(9, 123, 456)
    assert np.array_equal(full[123:579], part)


def test_complex64_is_rounded_fp64_draw():
    d = complex_uniform(5, (257,))
    s = complex_uniform(5, (257,), dtype=np.complex64)
    assert s.dtype == np.complex64
    assert np.array_equal(s, d.astype(np.complex64))


def test_loguniform_range_and_determinism():
    from fftu_inputs import complex_loguniform
    x = complex_loguniform(5, (64, 64), dtype=np.complex128)
    y = complex_loguniform(5, (64, 64), dtype=np.complex128)
    assert np.array_equal(x, y)
    mag = np.abs(x)
    assert mag.min() >= 1e-3 * (1 - 1e-12) and mag.max() < 1e3
    # log-uniform: each decade holds about a sixth of the values
    hist = np.histogram(np.log10(mag), bins=6, range=(-3, 3))[0]
    assert hist.min() > 0.8 * x.size / 6
    z = complex_loguniform(5, (64, 64), dtype=np.complex64)
    assert z.dtype == np.complex64 and np.allclose(z, x.astype(np.complex64))

"""Pins for the FP64 oracle: checks against what the mathematics fixes.

The paper prints no numeric worked example, so the oracle is pinned by
hand-derived exact DFTs (tests/golden/dft_exact.txt), brute-force sums of
eq. dftd, closed forms (impulse, single mode, constant), identities (Parseval,
linearity, shift theorem, round trip) and numpy's FFT as an independent
library.  Each pin is chosen so that a dropped term, a wrong sign or index, or a
transposed operand fails at least one of them; ``test_pins_catch_planted_mistakes``
shows that on deliberately wrong arrays.
"""
import os

import numpy as np
import pytest

import oracle
from fftu_inputs import complex_uniform

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dft_exact.txt")
TOL64 = 1e-13


def _read_golden():
    cases, cur = [], {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "shape":
                cur = {"shape": tuple(int(v) for v in vals)}
            else:
                arr = np.array([float(v) for v in vals])
                cur[key] = (arr[0::2] + 1j * arr[1::2]).reshape(cur["shape"])
                if key == "y":
                    cases.append(cur)
    return cases


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


@pytest.mark.parametrize("case", _read_golden(), ids=lambda c: "x".join(map(str, c["shape"])))
def test_golden_exact(case):
    assert _maxrel(oracle.fftn(case["x"]), case["y"]) < 1e-15
    assert _maxrel(oracle.dft_bruteforce(case["x"]), case["y"]) < 1e-15
    # inverse of the golden output gives the golden input back (1/N included)
    assert _maxrel(oracle.fftn(case["y"], inverse=True), case["x"]) < 1e-15


@pytest.mark.parametrize("shape", [(8, 8, 8), (16,), (5,), (4, 8, 2), (2, 3, 4, 5),
                                   (2, 2, 2, 2, 4), (7, 9), (1, 8, 1)])
def test_fftn_matches_bruteforce(shape):
    x = complex_uniform(11, shape)
    y = oracle.fftn(x)
    yb = oracle.dft_bruteforce(x)
    assert oracle.rel_l2(y, yb) < TOL64
    yi = oracle.fftn(x, inverse=True)
    assert oracle.rel_l2(yi, oracle.dft_bruteforce(x, inverse=True)) < TOL64


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 10, 7), (64, 64), (2, 4, 8, 16, 2)])
def test_fftn_matches_numpy(shape):
    x = complex_uniform(12, shape)
    assert oracle.rel_l2(oracle.fftn(x), np.fft.fftn(x)) < TOL64
    assert oracle.rel_l2(oracle.fftn(x, inverse=True), np.fft.ifftn(x)) < TOL64


@pytest.mark.parametrize("shape", [(8, 8, 8), (4, 6, 10)])
def test_impulse_closed_form(shape):
    # X = delta at j0  ->  Y[k] = prod_l w_{n_l}^{j0_l k_l}
    j0 = tuple(min(3, n - 1) for n in shape)
    x = np.zeros(shape, dtype=np.complex128)
    x[j0] = 1.0
    k = np.indices(shape)
    phase = sum(((k[l] * j0[l]) % shape[l]) / shape[l] for l in range(len(shape)))
    expect = np.exp(-2j * np.pi * phase)
    for fn in (oracle.fftn, oracle.dft_bruteforce):
        assert _maxrel(fn(x), expect) < TOL64


@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 4)])
def test_single_mode_and_constant(shape):
    # X[j] = prod_l w_{n_l}^{-m_l j_l}  ->  Y = N * delta_{k = m}
    N = int(np.prod(shape))
    m = tuple(1 + l for l in range(len(shape)))
    j = np.indices(shape)
    phase = sum(((j[l] * m[l]) % shape[l]) / shape[l] for l in range(len(shape)))
    x = np.exp(2j * np.pi * phase)
    expect = np.zeros(shape, dtype=np.complex128)
    expect[m] = N
    assert np.max(np.abs(oracle.fftn(x) - expect)) < 1e-11 * N
    c = np.full(shape, 2.5 - 1j)
    e0 = np.zeros(shape, dtype=np.complex128)
    e0[(0,) * len(shape)] = N * (2.5 - 1j)
    assert np.max(np.abs(oracle.fftn(c) - e0)) < 1e-11 * N


def test_parseval_linearity_roundtrip_shift():
    shape = (16, 8, 32)
    N = int(np.prod(shape))
    x = complex_uniform(21, shape)
    z = complex_uniform(22, shape)
    X, Z = oracle.fftn(x), oracle.fftn(z)
    # Parseval: sum |Y|^2 = N sum |X|^2
    assert abs(np.sum(np.abs(X) ** 2) - N * np.sum(np.abs(x) ** 2)) < 1e-12 * N * np.sum(np.abs(x) ** 2)
    # linearity
    a, b = 0.75 - 0.5j, -1.25 + 2j
    assert oracle.rel_l2(oracle.fftn(a * x + b * z), a * X + b * Z) < TOL64
    # round trip
    assert oracle.rel_l2(oracle.fftn(X, inverse=True), x) < TOL64
    # shift theorem: x[j - c] -> X[k] w^{c k}
    c = (3, 5, 7)
    xs = np.roll(x, c, axis=(0, 1, 2))
    k = np.indices(shape)
    phase = sum(((k[l] * c[l]) % shape[l]) / shape[l] for l in range(3))
    assert oracle.rel_l2(oracle.fftn(xs), X * np.exp(-2j * np.pi * phase)) < TOL64


def test_dft_points_match_fftn():
    shape = (32, 16, 8)
    x = complex_uniform(31, shape)
    Y = oracle.fftn(x)
    rng = np.random.default_rng(0)
    ks = np.stack([rng.integers(0, n, 12) for n in shape], axis=1)
    ks[0] = 0
    ks[1] = [n - 1 for n in shape]
    got = oracle.dft_points(x, ks)
    assert _maxrel(got, Y[tuple(ks.T)]) < TOL64
    goti = oracle.dft_points(Y, ks, inverse=True)
    assert _maxrel(goti, x[tuple(ks.T)]) < TOL64


def test_pins_catch_planted_mistakes():
    """Plausible oracle mistakes, planted in copies of its output, fail the pins."""
    x = complex_uniform(41, (4, 8, 2))
    good = oracle.fftn(x)
    ref = oracle.dft_bruteforce(x)
    assert oracle.rel_l2(good, ref) < TOL64
    wrong = {
        "flipped sign": (oracle.fftn(x, inverse=True) * x.size, ref),
        "missing 1/N on inverse": (oracle.fftn(good, inverse=True) * x.size, x),
        "row-major read as another shape": (oracle.fftn(x.reshape(4, 2, 8)).reshape(4, 8, 2), ref),
        "one axis skipped": (oracle.fft_axis(oracle.fft_axis(x, 0), 1), ref),
        "index off by one": (np.roll(good, 1, axis=1), ref),
        "dropped term": (oracle.fftn(np.where(np.arange(x.size).reshape(x.shape) == 5, 0, x)), ref),
    }
    assert oracle.rel_l2(oracle.fftn(good, inverse=True), x) < TOL64
    for name, (arr, expect) in wrong.items():
        assert oracle.rel_l2(arr, expect) > 1e-3, name


def test_error_metrics():
    """rel_l2 and max_abs_rel on hand-checkable arrays."""
    import oracle
    ref = np.array([3 + 4j, 0, 0, 0])
    y = np.array([3 + 4j, 0.5, 0, 0])
    assert oracle.rel_l2(y, ref) == pytest.approx(0.1)
    assert oracle.max_abs_rel(y, ref) == pytest.approx(0.1)
    y = np.array([3 + 4j, 0.3, 0.4j, 0])
    assert oracle.rel_l2(y, ref) == pytest.approx(0.1)
    assert oracle.max_abs_rel(y, ref) == pytest.approx(0.08)

"""CPU model of the parallel d-dimensional four-step FFT (Algorithm 2.3, Sec. 2.2).

TEST INFRASTRUCTURE ONLY.  FP64, explicit virtual processors P(s), s in
[p_1] x ... x [p_d], each holding a local array indexed by k in [n/p]
(elementwise n_l / p_l).  The local FFTs use the oracle's own 1D FFT.

Distribution (Sec. 1.1): X^{(s)}[k] = X[s + k p] per axis (the cyclic map
phi(s, k) = s + k p).  The supersteps, in the paper's order and notation:

  Superstep 0   Y^{(s)} = (F_{n_1/p_1} x ... x F_{n_d/p_d})(X^{(s)})
                Z^{(s)}[k] = (prod_l w_{n_l}^{k_l s_l}) Y^{(s)}[k]
  Superstep 1   for every destination k in [p]:
                Put Z^{(s)}(k : p : n/p) in P(k) as W^{(k)}[s n/p^2 : (s+1) n/p^2 - 1]
                (the block is the d-dim box with corner s * n/p^2, elementwise)
  Superstep 2   for t in [n/p^2]:
                V^{(s)}(t : n/p^2 : n/p) = (F_{p_1} x ... x F_{p_d})(W^{(s)}(t : n/p^2 : n/p))

The output V is in the same cyclic distribution: V[s + r p] = V^{(s)}[r].
Theorem 2.1 states that V is the d-dim DFT of X.  The inverse uses conjugated
weights throughout and scales by 1/N at the end (Sec. 1.3).

Global view of the exchanged data: element W^{(s)}[r] sits at global index
s + r p, and W^{(s)}[t + s' n/p^2] = Z^{(s')}[s + t p], so the value
Z^{(s')}[m] lands at global index m + s' (n/p).  ``phase_a`` returns that global
array; it is what a single-memory implementation stores after its
redistribution step.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import fft_axis


def _check(shape, p):
    shape = tuple(int(v) for v in shape)
    p = tuple(int(v) for v in p)
    if len(shape) != len(p):
        raise ValueError("n and p must have the same length d")
    for n_l, p_l in zip(shape, p):
        if p_l < 1 or n_l % (p_l * p_l) != 0:
            raise ValueError(f"need p_l^2 | n_l, got n_l={n_l}, p_l={p_l}")
    return shape, p


def processors(p):
    """All processor indices s in [p_1] x ... x [p_d], row-major."""
    return list(itertools.product(*[range(v) for v in p]))


def distribute(X, p):
    """Cyclic distribution: local arrays X^{(s)}[k] = X[s + k p] (Sec. 1.1)."""
    X = np.asarray(X)
    _check(X.shape, p)
    return {s: X[tuple(slice(s_l, None, p_l) for s_l, p_l in zip(s, p))].copy()
            for s in processors(p)}


def collect(local, shape, p):
    """Inverse of ``distribute``: global array with X[s + r p] = X^{(s)}[r]."""
    out = np.empty(tuple(shape), dtype=np.complex128)
    for s, arr in local.items():
        out[tuple(slice(s_l, None, p_l) for s_l, p_l in zip(s, p))] = arr
    return out


def _local_dft(a, sign):
    """(F_{m_1} x ... x F_{m_d}) on a local array, unscaled, one axis at a time."""
    y = np.asarray(a, dtype=np.complex128)
    for ax in range(y.ndim):
        y = fft_axis(y, ax, sign)
    return y


def twiddle_factors(shape, p, s, sign):
    """prod_l w_{n_l}^{k_l s_l} over k in [n/p] (Alg. 2.3, Superstep 0 twiddle)."""
    fac = np.ones(tuple(n // q for n, q in zip(shape, p)), dtype=np.complex128)
    for l, (n_l, p_l, s_l) in enumerate(zip(shape, p, s)):
        k = np.arange(n_l // p_l, dtype=np.int64)
        e = (k * s_l) % n_l
        w = np.exp(sign * 2j * np.pi * e / n_l)
        view = [1] * len(shape)
        view[l] = -1
        fac = fac * w.reshape(view)
    return fac


def superstep0(local_x, shape, p, inverse=False):
    """Z^{(s)} for every s: local DFT of shape n/p, then the twiddle."""
    sign = 1 if inverse else -1
    return {s: _local_dft(xs, sign) * twiddle_factors(shape, p, s, sign)
            for s, xs in local_x.items()}


def superstep1(local_z, shape, p):
    """The single all-to-all: W^{(k)} built from the Put of every Z^{(s)}."""
    L = tuple(n // q for n, q in zip(shape, p))
    M = tuple(n // (q * q) for n, q in zip(shape, p))
    local_w = {k: np.empty(L, dtype=np.complex128) for k in processors(p)}
    for s, zs in local_z.items():
        for k in processors(p):
            packet = zs[tuple(slice(k_l, None, p_l) for k_l, p_l in zip(k, p))]
            block = tuple(slice(s_l * m_l, (s_l + 1) * m_l) for s_l, m_l in zip(s, M))
            local_w[k][block] = packet
    return local_w


def superstep2(local_w, shape, p, inverse=False):
    """V^{(s)}(t : n/p^2 : n/p) = (F_{p_1} x ... x F_{p_d})(W^{(s)}(t : n/p^2 : n/p)) for all t.

    The local index r = t + s' n/p^2 (per axis) is split into the pair (s', t);
    the length-p DFTs run over the s' axes for every t at once.
    With inverse, the weights are conjugated and the result is scaled by 1/N.
    """
    sign = 1 if inverse else -1
    d = len(shape)
    M = tuple(n // (q * q) for n, q in zip(shape, p))
    split = []
    for p_l, m_l in zip(p, M):
        split += [p_l, m_l]
    N = int(np.prod(shape))
    out = {}
    for s, ws in local_w.items():
        a = np.asarray(ws, dtype=np.complex128).reshape(split)
        for l in range(d):
            a = fft_axis(a, 2 * l, sign)
        a = a.reshape(ws.shape)
        out[s] = a / N if inverse else a
    return out


def run(X, p, inverse=False):
    """Algorithm 2.3 end to end on a global array; returns the global V."""
    X = np.asarray(X, dtype=np.complex128)
    shape, p = _check(X.shape, p)
    z = superstep0(distribute(X, p), shape, p, inverse)
    w = superstep1(z, shape, p)
    v = superstep2(w, shape, p, inverse)
    return collect(v, shape, p)


def phase_a(X, p, inverse=False):
    """Supersteps 0 and 1; returns the exchanged data W in the global view."""
    X = np.asarray(X, dtype=np.complex128)
    shape, p = _check(X.shape, p)
    return collect(superstep1(superstep0(distribute(X, p), shape, p, inverse), shape, p),
                   shape, p)


def phase_b(Wg, p, inverse=False):
    """Superstep 2 on the global view of W; returns the global V."""
    Wg = np.asarray(Wg, dtype=np.complex128)
    shape, p = _check(Wg.shape, p)
    return collect(superstep2(distribute(Wg, p), shape, p, inverse), shape, p)


def z_closed_form(X, p, s, inverse=False):
    """Z^{(s)}[k] = sum_j X^{(s)}[j] prod_l w_{n_l}^{k_l (j_l p_l + s_l)}, summed directly.

    The closed form of the Superstep 0 output stated in the proof of
    Theorem 2.1; O((N/p)^2), for small arrays.
    """
    X = np.asarray(X, dtype=np.complex128)
    shape, p = _check(X.shape, p)
    sign = 1 if inverse else -1
    xs = distribute(X, p)[tuple(s)]
    L = xs.shape
    out = np.zeros(L, dtype=np.complex128)
    jj = np.indices(L).reshape(len(L), -1)
    xv = xs.reshape(-1)
    for k in itertools.product(*[range(v) for v in L]):
        phase = np.zeros(jj.shape[1])
        for l in range(len(L)):
            e = (k[l] * (jj[l] * p[l] + s[l])) % shape[l]
            phase = phase + e / shape[l]
        out[k] = np.sum(xv * np.exp(sign * 2j * np.pi * phase))
    return out

"""CPU mirror of the register-resident generic phase B (phase_b_reg.cuh, phase_b.cu), no GPU.

Phase B applies F_{p_0} x ... x F_{p_{d-1}} to the values at m + s' (n/p) for every m (Superstep 2 of
Algorithm 2.3).  The kernel takes a tile of all P = prod p_l values for Mt consecutive m along the last axis
(tile index e = mt + Mt flat(s')), groups its axes from the last one down (two adjacent axes where
p_l p_{l-1} <= 16), and runs one stage per group: a thread's fiber is the group's values for fixed other tile
indices, the first stage loads it from global memory, the last one stores it back, shared memory in between.
This file restates the grouping (pb_groups), the fiber addressing and the global offsets in numpy, runs them
over a whole small array, and compares with phase B of the CPU model (oracle/cyclic_model.py); it also checks
that every stage touches every tile element exactly once.
"""
import math

import numpy as np
import pytest

from fftu_inputs import complex_uniform
from oracle import cyclic_model as cm


def lg(x):
    return int(math.log2(x))


def groups(p, Mt, L, stride):
    out, off, l = [], lg(Mt), len(p) - 1
    while l >= 0:
        if p[l] == 1:
            l -= 1
            continue
        pp = p[l] * p[l - 1] if (l > 0 and p[l - 1] > 1) else 0
        if 0 < pp <= 16:
            out.append(dict(off=off, lo=p[l], hi=p[l - 1], slo=L[l] * stride[l], shi=L[l - 1] * stride[l - 1]))
            off += lg(p[l]) + lg(p[l - 1])
            l -= 2
        else:
            out.append(dict(off=off, lo=p[l], hi=1, slo=L[l] * stride[l], shi=0))
            off += lg(p[l])
            l -= 1
    return out


def tile_offset(e, p, Mt, L, stride):
    """Global offset of tile element e from the tile base (phaseb_offset)."""
    d = len(p)
    mt, sf = e & (Mt - 1), e >> lg(Mt)
    g = mt * stride[d - 1]
    for l in range(d - 1, -1, -1):
        s = sf & (p[l] - 1)
        sf >>= lg(p[l])
        g += s * L[l] * stride[l]
    return g


def tile_base(t, p, Mt, L, stride):
    d = len(p)
    lg_td = lg(L[d - 1]) - lg(Mt)
    rem = t >> lg_td
    base = ((t & ((1 << lg_td) - 1)) << lg(Mt)) * stride[d - 1]
    for l in range(d - 2, -1, -1):
        base += (rem & (L[l] - 1)) * stride[l]
        rem >>= lg(L[l])
    return base


def dft(x, sign):
    return np.fft.fft(x) if sign < 0 else np.conj(np.fft.fft(np.conj(x)))


def run_mirror(W, p, Mt, sign, scale):
    shape = W.shape
    d = len(shape)
    L = [shape[l] // p[l] for l in range(d)]
    stride = [int(np.prod(shape[l + 1:])) for l in range(d)]
    P = int(np.prod(p))
    total = P * Mt
    flat = W.reshape(-1).copy()
    gs = groups(p, Mt, L, stride)
    tiles = int(np.prod(L[:-1])) * (L[-1] // Mt)
    for t in range(tiles):
        base = tile_base(t, p, Mt, L, stride)
        sm = np.full(total, np.nan + 0j)
        for gi, g in enumerate(gs):
            first, last = gi == 0, gi == len(gs) - 1
            PG, LG = g["lo"] * g["hi"], lg(g["lo"] * g["hi"])
            seen = np.zeros(total, np.int64)
            for phi in range(total >> LG):
                e0 = ((phi >> g["off"]) << (g["off"] + LG)) | (phi & ((1 << g["off"]) - 1))
                go = base + tile_offset(e0, p, Mt, L, stride)
                js = range(PG)
                gidx = [go + (j % g["lo"]) * g["slo"] + (j // g["lo"]) * g["shi"] for j in js]
                sidx = [e0 + (j << g["off"]) for j in js]
                for e in sidx:
                    seen[e] += 1
                v = flat[gidx] if first else sm[sidx]
                v = np.asarray(v).reshape(g["hi"], g["lo"])
                v = np.apply_along_axis(dft, 1, v, sign)
                v = np.apply_along_axis(dft, 0, v, sign).reshape(-1)
                if last:
                    flat[gidx] = v * scale
                else:
                    sm[sidx] = v
            assert np.all(seen == 1), (t, gi)
    return flat.reshape(shape)


@pytest.mark.parametrize("shape,p,Mt", [
    ((32, 32, 32), (4, 4, 4), 8),          # pair then single
    ((16, 16, 16, 16), (4, 4, 2, 2), 4),   # two pairs
    ((64, 16), (8, 4), 4),                 # 8 x 4 > 16: two single stages
    ((8, 16, 32), (1, 4, 4), 8),           # p = 1 axis skipped
    ((256,), (16,), 16),                   # one stage: load and store in the same stage
])
@pytest.mark.parametrize("inverse", [False, True])
def test_register_stages_equal_the_model(shape, p, Mt, inverse):
    W = complex_uniform(9090 + len(shape), shape, dtype=np.complex128)
    scale = 1.0 / W.size if inverse else 1.0
    got = run_mirror(W, p, Mt, 1 if inverse else -1, scale)
    want = cm.phase_b(W, p, inverse=inverse)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)

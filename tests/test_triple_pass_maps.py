"""CPU mirror of the three-axis phase-A pass (triple_pass.cu), no GPU.

For the last three axes with 8-point sub-FFTs and p_b p_c = 16 the kernel computes, per residue class
(s_a, s_b, s_c), Superstep 0 of Algorithm 2.3 on those axes (an 8 x 8 x 8 DFT), the twiddles of Sec. 2.2 and
the Put position (s_a 8 + k_a, s_b 8 + k_b, s_c 8 + k_c) of Superstep 1, one CTA per (outer position, s_a).
This file restates its fibers, swizzled shared layout and CTA decode in numpy and checks:

* the data carried through the three stages equals the 3D DFT of every class times the three twiddles
  (numpy's FFT as the DFT primitive), both directions;
* every shared access stays in the 8192-element buffer, each stage's stores fill it exactly once, and
  every warp access takes 2 wavefronts (1 per half-warp);
* the CTA decode reads every input element and writes every Put position of a small array exactly once,
  and a warp's stage-3 stores are whole rows of n_c consecutive elements.
"""
import math
from collections import defaultdict

import numpy as np
import pytest

from fftu_inputs import uniform_pm1

THREADS = 512


def lg(x):
    return int(math.log2(x))


def tsw(q):
    return ((q >> 1) & 7) | ((q & 1) << 3)


def elem(q, x, y, z):
    return q * 512 + ((x * 64 + y * 8 + z) ^ tsw(q))


def dft(x, sign):
    return np.fft.fft(x) if sign < 0 else np.conj(np.fft.fft(np.conj(x)))


def root(n, e, sign):
    return np.exp(sign * 2j * np.pi * (np.asarray(e) % n) / n)


def wavefronts(idx):
    banks = defaultdict(set)
    for a in idx:
        for k in range(2):
            w = 2 * a + k
            banks[w % 32].add(w)
    return max(len(s) for s in banks.values()) if banks else 0


def fiber1(f, pb, pc):
    sc, sb, mb, ma = f & (pc - 1), (f >> lg(pc)) & (pb - 1), (f >> 4) & 7, f >> 7
    return sb, sc, ma, mb


def fiber23(f, pb, pc):
    kc, sc, sb, top = f & 7, (f >> 3) & (pc - 1), (f >> (3 + lg(pc))) & (pb - 1), f >> 7
    return sb, sc, top, kc


SPLITS = [(4, 4), (2, 8), (8, 2)]


@pytest.mark.parametrize("pb,pc", SPLITS)
def test_shared_maps_bijective_and_conflict_free(pb, pc):
    pats = []
    for z in range(8):
        pats.append(("s1_store", [elem(sb * pc + sc, ma, mb, z) for sb, sc, ma, mb in
                                  (fiber1(f, pb, pc) for f in range(1024))]))
    for y in range(8):
        pats.append(("s2", [elem(sb * pc + sc, x, y, kc) for sb, sc, x, kc in
                            (fiber23(f, pb, pc) for f in range(1024))]))
    for x in range(8):
        pats.append(("s3_load", [elem(sb * pc + sc, x, kb, kc) for sb, sc, kb, kc in
                                 (fiber23(f, pb, pc) for f in range(1024))]))
    for name in ("s1_store", "s2"):
        idx = np.concatenate([np.asarray(i) for n, i in pats if n == name])
        assert len(np.unique(idx)) == len(idx) == 8192 and idx.min() >= 0 and idx.max() < 8192, name
    for name, idx in pats:
        for h in range(2):  # fibers f and f + 512 are the two halves of a thread's work
            for w0 in range(h * THREADS, (h + 1) * THREADS, 32):
                lanes = idx[w0:w0 + 32]
                assert wavefronts(lanes) == 2, (name, w0)
                assert wavefronts(lanes[:16]) == 1 and wavefronts(lanes[16:]) == 1, (name, w0)


def run_item(planes, sa, pa, pb, pc, sign):
    """planes: the 8 input planes m_a p_a + s_a (shape [8, nb, nc]); returns the 8 Put-ordered output planes."""
    nb, nc, na = 8 * pb, 8 * pc, 8 * pa
    sm = np.full(8192, np.nan + 0j)
    for f in range(1024):
        sb, sc, ma, mb = fiber1(f, pb, pc)
        v = dft(np.array([planes[ma, mb * pb + sb, mc * pc + sc] for mc in range(8)]), sign)
        v = v * root(nc, sc * np.arange(8), sign)
        for kc in range(8):
            sm[elem(sb * pc + sc, ma, mb, kc)] = v[kc]
    for f in range(1024):
        sb, sc, ma, kc = fiber23(f, pb, pc)
        q = sb * pc + sc
        v = dft(np.array([sm[elem(q, ma, mb, kc)] for mb in range(8)]), sign) * root(nb, sb * np.arange(8), sign)
        for kb in range(8):
            sm[elem(q, ma, kb, kc)] = v[kb]
    out = np.full((8, nb, nc), np.nan + 0j)
    for f in range(1024):
        sb, sc, kb, kc = fiber23(f, pb, pc)
        q = sb * pc + sc
        v = dft(np.array([sm[elem(q, ma, kb, kc)] for ma in range(8)]), sign) * root(na, sa * np.arange(8), sign)
        for ka in range(8):
            out[ka, sb * 8 + kb, sc * 8 + kc] = v[ka]
    return out


@pytest.mark.parametrize("pa,pb,pc", [(4, 4, 4), (2, 2, 8), (8, 8, 2)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_item_data_equals_3d_dft_with_twiddles(pa, pb, pc, sign):
    na, nb, nc = 8 * pa, 8 * pb, 8 * pc
    u = uniform_pm1(777 + pa + pb, np.arange(2 * na * nb * nc, dtype=np.uint64))
    x = (u[0::2] + 1j * u[1::2]).reshape(na, nb, nc)
    sa = pa - 1
    got = run_item(x[sa::pa], sa, pa, pb, pc, sign)
    k = np.arange(8)
    for sb in range(pb):
        for sc in range(pc):
            blk = x[sa::pa, sb::pb, sc::pc]
            z = blk
            for ax in range(3):
                z = np.apply_along_axis(dft, ax, z, sign)
            z = z * root(na, sa * k, sign)[:, None, None] * root(nb, sb * k, sign)[None, :, None] \
                * root(nc, sc * k, sign)[None, None, :]
            np.testing.assert_allclose(got[:, sb * 8:(sb + 1) * 8, sc * 8:(sc + 1) * 8], z, rtol=0, atol=1e-9)


def test_cta_decode_covers_input_and_put_positions():
    outer, pa, pb, pc = 3, 4, 4, 4
    na, nb, nc = 8 * pa, 8 * pb, 8 * pc
    plane = nb * nc
    N = outer * na * plane
    seen_in = np.zeros(N, np.int64)
    seen_out = np.zeros(N, np.int64)
    for blk in range(outer * pa):
        sa, o = blk & (pa - 1), blk >> lg(pa)
        base = o * na * plane
        for f in range(1024):
            sb, sc, ma, mb = fiber1(f, pb, pc)
            idx = base + (ma * pa + sa) * plane + (mb * pb + sb) * nc + sc + np.arange(8) * pc
            np.add.at(seen_in, idx, 1)
            sb, sc, kb, kc = fiber23(f, pb, pc)
            idx = base + (sa * 8 + np.arange(8)) * plane + (sb * 8 + kb) * nc + sc * 8 + kc
            np.add.at(seen_out, idx, 1)
    assert np.all(seen_in == 1) and np.all(seen_out == 1)


def test_stage3_warp_stores_are_rows():
    pb, pc = 4, 4
    for f0 in range(0, 1024, 32):
        cols, rows = set(), set()
        for f in range(f0, f0 + 32):
            sb, sc, kb, kc = fiber23(f, pb, pc)
            rows.add(sb * 8 + kb)
            cols.add(sc * 8 + kc)
        assert len(rows) == 1 and cols == set(range(8 * pc))

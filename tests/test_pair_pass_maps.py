"""CPU mirror of the two-axis phase-A pass (pair_pass.cu), no GPU.

For two adjacent axes a, b = a + 1 with equal sub-FFT lengths L (8 or 16) the kernel computes, per residue
class (s_a, s_b) of every plane, Superstep 0 of Algorithm 2.3 on those two axes (an L x L DFT), the twiddles
of Sec. 2.2 and the Put positions (s_a L + k_a, s_b L + k_b) of Superstep 1.  This file restates its
thread roles, swizzled exchange and CTA decode in numpy and checks, for the configurations the planner can
choose (p_a p_b >= 16, at most 1024 threads):

* the data carried through the maps equals the 2D DFT of every class times w_{n_a}^{k_a s_a} w_{n_b}^{k_b s_b}
  (numpy's FFT as the DFT primitive), both directions;
* every exchange access stays in the CTA's buffer, each stage's stores are a bijection onto the items'
  class blocks, and every warp access takes the minimum number of wavefronts (2 per 32 lanes of 8 bytes,
  1 per half-warp);
* the CTA decode covers every input element and every Put position of a small array exactly once, and
  stage-2 stores of a contiguous pair are runs of n_b elements.
"""
import math
from collections import defaultdict

import numpy as np
import pytest

from fftu_inputs import uniform_pm1


def lg(x):
    return int(math.log2(x))


def pair_sw(c, L):
    return c & 15 if L == 16 else (c & 7) | (((c ^ (c >> 3)) & 1) << 3)


def dft(x, sign):
    return np.fft.fft(x) if sign < 0 else np.conj(np.fft.fft(np.conj(x)))


def root(n, e, sign):
    return np.exp(sign * 2j * np.pi * (np.asarray(e) % n) / n)


def wavefronts(elem_idx):
    banks = defaultdict(set)
    for a in elem_idx:
        for k in range(2):
            w = 2 * a + k
            banks[w % 32].add(w)
    return max(len(s) for s in banks.values()) if banks else 0


class Mirror:
    def __init__(self, L, pa, pb, W, contig):
        self.L, self.pa, self.pb, self.W, self.contig = L, pa, pb, W, contig
        self.per_item = pa * pb * L
        self.threads = W * self.per_item
        self.pad = 0 if contig else 16 // W
        self.region = pa * pb * L * L + self.pad
        self.size = W * self.region

    def split(self, t):
        if self.contig:
            lr = lg(self.per_item)
            return t >> lr, t & ((1 << lr) - 1)
        return t % self.W, t // self.W

    def role1(self, t):
        it, r = self.split(t)
        sb = r & (self.pb - 1)
        sa = (r >> lg(self.pb)) & (self.pa - 1)
        ma = r >> (lg(self.pb) + lg(self.pa))
        return it, sa, sb, ma

    def role2(self, t):
        it, r = self.split(t)
        kb = r & (self.L - 1)
        sb = (r >> lg(self.L)) & (self.pb - 1)
        sa = r >> (lg(self.L) + lg(self.pb))
        return it, sa, sb, kb

    def elem(self, it, c, ma, kb):
        L = self.L
        return it * self.region + c * L * L + ((ma * L + kb) ^ pair_sw(c, L))

    def accesses(self):
        acc = []
        th = range(self.threads)
        for kb in range(self.L):
            acc.append(("store", [self.elem(it, sa * self.pb + sb, ma, kb)
                                  for it, sa, sb, ma in map(self.role1, th)]))
        for ma in range(self.L):
            acc.append(("load", [self.elem(it, sa * self.pb + sb, ma, kb)
                                 for it, sa, sb, kb in map(self.role2, th)]))
        return acc

    def run(self, planes, na, nb, sign):
        """planes: [W, na, nb] (the items' planes).  Returns the Put-ordered output planes."""
        L, pa, pb = self.L, self.pa, self.pb
        sm = np.full(self.size, np.nan + 0j)
        out = np.full(planes.shape, np.nan + 0j)
        for t in range(self.threads):
            it, sa, sb, ma = self.role1(t)
            v = dft(np.array([planes[it, ma * pa + sa, mb * pb + sb] for mb in range(L)]), sign)
            v = v * root(nb, sb * np.arange(L), sign)
            for kb in range(L):
                sm[self.elem(it, sa * pb + sb, ma, kb)] = v[kb]
        for t in range(self.threads):
            it, sa, sb, kb = self.role2(t)
            v = dft(np.array([sm[self.elem(it, sa * pb + sb, ma, kb)] for ma in range(L)]), sign)
            v = v * root(na, sa * np.arange(L), sign)
            for ka in range(L):
                out[it, sa * L + ka, sb * L + kb] = v[ka]
        return out


def configs():
    out = []
    for L in (8, 16):
        for pa in (2, 4, 8, 16):
            for pb in (2, 4, 8, 16):
                per = pa * pb * L
                if pa * pb < 16 or per > 1024:
                    continue
                out.append((L, pa, pb, max(1, 512 // per), True))
                W = min(16, 1024 // per)
                if W >= 4:
                    out.append((L, pa, pb, W, False))
    return out


@pytest.mark.parametrize("cfg", configs(), ids=lambda c: "L%d_p%dx%d_W%d_%s" % (c[0], c[1], c[2], c[3],
                                                                             "contig" if c[4] else "strided"))
def test_exchange_in_bounds_bijective_conflict_free(cfg):
    m = Mirror(*cfg)
    acc = m.accesses()
    stores = np.concatenate([np.asarray(i) for n, i in acc if n == "store"])
    assert len(np.unique(stores)) == len(stores) == m.W * m.pa * m.pb * m.L * m.L
    for name, idx in acc:
        idx = np.asarray(idx)
        assert idx.min() >= 0 and idx.max() < m.size, name
        for w0 in range(0, m.threads, 32):
            lanes = idx[w0:w0 + 32]
            assert wavefronts(lanes) == max(1, math.ceil(len(lanes) * 8 / 128)), (name, w0)
            for h in (lanes[:16], lanes[16:]):
                if len(h):
                    assert wavefronts(h) == 1, (name, w0)


@pytest.mark.parametrize("cfg", [(8, 4, 4, 4, True), (8, 4, 4, 8, False), (16, 4, 4, 2, True),
                                 (16, 4, 4, 4, False), (8, 8, 8, 1, True), (8, 2, 8, 4, True)],
                         ids=lambda c: "L%d_p%dx%d_W%d" % c[:4])
@pytest.mark.parametrize("sign", [-1, 1])
def test_pair_data_equals_2d_dft_with_twiddles(cfg, sign):
    m = Mirror(*cfg)
    L, pa, pb = m.L, m.pa, m.pb
    na, nb = L * pa, L * pb
    u = uniform_pm1(31 + L + pa + 3 * pb, np.arange(2 * m.W * na * nb, dtype=np.uint64))
    planes = (u[0::2] + 1j * u[1::2]).reshape(m.W, na, nb)
    got = m.run(planes, na, nb, sign)
    want = np.empty_like(planes)
    k = np.arange(L)
    for it in range(m.W):
        for sa in range(pa):
            for sb in range(pb):
                blk = planes[it, sa::pa, sb::pb]
                z = np.apply_along_axis(dft, 1, np.apply_along_axis(dft, 0, blk, sign), sign)
                z = z * root(na, sa * k, sign)[:, None] * root(nb, sb * k, sign)[None, :]
                want[it, sa * L:(sa + 1) * L, sb * L:(sb + 1) * L] = z
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10 * L * L)


@pytest.mark.parametrize("case", [
    dict(shape=(8, 32, 32), a=1, L=8, W=4),          # contiguous pair, 4 planes per CTA
    dict(shape=(32, 32, 16), a=0, L=8, W=8),         # strided pair, 8 inner positions per CTA
    dict(shape=(2, 64, 64, 4), a=1, L=16, W=4),      # strided pair in the middle of the array
])
def test_cta_decode_covers_input_and_put_positions(case):
    shape, a, L, W = case["shape"], case["a"], case["L"], case["W"]
    na, nb = shape[a], shape[a + 1]
    pa, pb = na // L, nb // L
    outer = int(np.prod(shape[:a]))
    inner = int(np.prod(shape[a + 2:]))
    N = outer * na * nb * inner
    contig = inner == 1
    per = pa * pb * L
    seen_in = np.zeros(N, np.int64)
    seen_out = np.zeros(N, np.int64)
    ctas = outer // W if contig else outer * (inner // W)
    for b in range(ctas):
        for t in range(W * per):
            if contig:
                it, r = t >> lg(per), t & (per - 1)
                base = (b * W + it) * na * nb
                s = 1
            else:
                it, r = t % W, t // W
                vg, o = b % (inner // W), b // (inner // W)
                base = o * na * nb * inner + vg * W + it
                s = inner
            sb, sa, ma = r & (pb - 1), (r >> lg(pb)) & (pa - 1), r >> (lg(pb) + lg(pa))
            idx_in = base + ((ma * pa + sa) * nb + sb + np.arange(L) * pb) * s
            kb, sb2, sa2 = r & (L - 1), (r >> lg(L)) & (pb - 1), r >> (lg(L) + lg(pb))
            idx_out = base + ((sa2 * L + np.arange(L)) * nb + sb2 * L + kb) * s
            assert idx_in.max() < N and idx_out.max() < N
            np.add.at(seen_in, idx_in, 1)
            np.add.at(seen_out, idx_out, 1)
    assert np.all(seen_in == 1) and np.all(seen_out == 1)


def test_contiguous_pair_stores_are_runs_of_a_row():
    """Stage-2 stores of one warp on a contiguous pair (fixed k_a): 32 consecutive elements of a row."""
    m = Mirror(8, 4, 4, 4, True)
    nb = m.L * m.pb
    for w0 in range(0, m.threads, 32):
        cols = sorted(sb * m.L + kb for it, sa, sb, kb in map(m.role2, range(w0, w0 + 32)))
        rows = {(it, sa) for it, sa, sb, kb in map(m.role2, range(w0, w0 + 32))}
        assert len(rows) == 1 and cols == list(range(nb))

"""CPU mirror of the register-resident phase-A line pass (line_pass.cu), no GPU.

The kernel computes mode 0 of the strided pass (Superstep 0 of Algorithm 2.3 on one axis, the axis'
twiddle of Sec. 2.2 and the Put position s len + k of Superstep 1) with len = 16 T split twice by the
radix split of Sec. 2.1.1 (eq. radix).  This file restates its thread roles and shared-memory maps in
numpy and checks, for every T and CTA width W the planner can choose:

* on the contiguous axis, where stages 2 and 3 take line-major roles, a warp's Put stores are runs of 16
  consecutive outputs of one line;
* the data carried through the maps for one CTA equals the length-len DFT of every line times
  w_{n_l}^{k c} (numpy's FFT as the DFT primitive), both directions;
* every shared-memory access stays inside the CTA's buffer and each exchange's store map is a
  bijection onto the lines' regions;
* every warp-wide shared access takes the minimum number of wavefronts (2 for 32 lanes of 8 bytes),
  counted per 4-byte bank over the whole warp and, separately, within each half-warp;
* the CTA decode covers every input element and every Put position of a small array exactly once.
"""
import math
from collections import defaultdict

import numpy as np
import pytest

from fftu_inputs import uniform_pm1


def pad_of(W):
    return 16 // W if W >= 2 else 0


def line_configs():
    out = []
    for T in (16, 32, 64, 128):
        for W in (1, 2, 4, 8, 16):
            if 32 <= T * W <= (1024 if T == 128 else 512):
                out.append((T, W))
    return out


def dft(x, sign):
    return np.fft.fft(x) if sign < 0 else np.conj(np.fft.fft(np.conj(x)))


def root(n, e, sign):
    return np.exp(sign * 2j * np.pi * (np.asarray(e) % n) / n)


def wavefronts(byte_addrs):
    banks = defaultdict(set)
    for a in byte_addrs:
        for k in range(2):  # 8-byte element: two 4-byte words
            word = a // 4 + k
            banks[word % 32].add(word)
    return max(len(s) for s in banks.values()) if banks else 0


class Mirror:
    """One CTA of W lines.  Stage 1: thread t takes line t % W and role q = t / W.  Stages 2 and 3: the same
    on a strided axis; on the contiguous axis line t / T and role t % T."""

    def __init__(self, T, W, contig=False):
        self.T, self.W, self.contig = T, W, contig
        self.LEN = 16 * T
        self.R3 = T // 16
        self.P = pad_of(W)
        self.size = W * (self.LEN + self.P)
        self.threads = T * W

    def region(self, w):
        return w * (self.LEN + self.P)

    def role2(self, t):
        return (t // self.T, t % self.T) if self.contig else (t % self.W, t // self.W)

    def ex1(self, k1, j):
        return k1 * self.T + (j ^ k1)

    def ex2(self, k1, j1, k2):
        return ((j1 * 16 + k2) << 4) + k1

    def accesses(self):
        """Per shared-memory instruction: the element index of every thread."""
        T, W, R3 = self.T, self.W, self.R3
        th = range(self.threads)
        acc = []
        for k1 in range(16):  # stage-1 store
            acc.append(("ex1_store", [self.region(t % W) + self.ex1(k1, t // W) for t in th]))
        r2 = [self.role2(t) for t in th]
        for j2 in range(16):  # stage-2 load
            acc.append(("ex1_load", [self.region(w) + self.ex1(q & 15, (q >> 4) + R3 * j2) for w, q in r2]))
        if R3 > 1:
            for k2 in range(16):  # stage-2 store
                acc.append(("ex2_store", [self.region(w) + self.ex2(q & 15, q >> 4, k2) for w, q in r2]))
            for i in range(16 // R3):  # stage-3 loads
                for jj in range(R3):
                    acc.append(("ex2_load", [self.region(w) + self.ex2(q & 15, jj, (q >> 4) + R3 * i)
                                             for w, q in r2]))
        return acc

    def run(self, x, c, nl, sign):
        """x: [W, LEN] lines; c: class of each line.  Returns [W, LEN] outputs in k order."""
        T, W, R3, LEN = self.T, self.W, self.R3, self.LEN
        sm = np.full(self.size, np.nan + 0j)
        out = np.full((W, LEN), np.nan + 0j)
        regs = {}
        for t in range(self.threads):
            w, j = t % W, t // W
            v = dft(np.array([x[w, j + T * r] for r in range(16)]), sign)
            v = v * root(LEN, j * np.arange(16), sign)
            for k1 in range(16):
                sm[self.region(w) + self.ex1(k1, j)] = v[k1]
        for t in range(self.threads):
            w, q = self.role2(t)
            k1, j1 = q & 15, q >> 4
            v = np.array([sm[self.region(w) + self.ex1(k1, j1 + R3 * j2)] for j2 in range(16)])
            regs[t] = dft(v, sign)
        if R3 == 1:
            for t in range(self.threads):
                w, q = self.role2(t)
                k1 = q & 15
                for k2 in range(16):
                    k = k1 + 16 * k2
                    out[w, k] = regs[t][k2] * root(nl, c[w] * k, sign)
            return out
        sm[:] = np.nan
        for t in range(self.threads):
            w, q = self.role2(t)
            k1, j1 = q & 15, q >> 4
            v = regs[t] * root(T, j1 * np.arange(16), sign)
            for k2 in range(16):
                sm[self.region(w) + self.ex2(k1, j1, k2)] = v[k2]
        for t in range(self.threads):
            w, q = self.role2(t)
            k1, h = q & 15, q >> 4
            for i in range(16 // R3):
                k2 = h + R3 * i
                y = dft(np.array([sm[self.region(w) + self.ex2(k1, jj, k2)] for jj in range(R3)]), sign)
                for k3 in range(R3):
                    k = k1 + 16 * k2 + 256 * k3
                    out[w, k] = y[k3] * root(nl, c[w] * k, sign)
        return out


@pytest.mark.parametrize("T,W", line_configs(), ids=lambda v: str(v))
@pytest.mark.parametrize("contig", [False, True], ids=["strided", "contiguous"])
def test_shared_maps_in_bounds_bijective_and_conflict_free(T, W, contig):
    m = Mirror(T, W, contig)
    acc = m.accesses()
    for name, idx in acc:
        idx = np.asarray(idx)
        assert idx.min() >= 0 and idx.max() < m.size, name
        if name.endswith("store"):
            assert len(np.unique(idx)) == m.threads, name  # one element per thread, all distinct
        for w0 in range(0, m.threads, 32):
            lanes = idx[w0:w0 + 32]
            assert wavefronts(8 * lanes) == max(1, math.ceil(len(lanes) * 8 / 128)), (name, w0)
            for h0 in (0, 16):  # half-warp model: 16 distinct 8-byte slots per half
                half = lanes[h0:h0 + 16]
                if len(half):
                    assert wavefronts(8 * half) == 1, (name, w0, h0)
    # each exchange's stores fill every line's region exactly once
    for name in ("ex1_store", "ex2_store"):
        parts = [np.asarray(i) for n, i in acc if n == name]
        if not parts:
            continue
        idx = np.concatenate(parts)
        assert len(idx) == m.W * m.LEN and len(np.unique(idx)) == m.W * m.LEN, name


@pytest.mark.parametrize("T,W", [(16, 16), (32, 8), (64, 4), (128, 2), (64, 1), (128, 4)], ids=lambda v: str(v))
@pytest.mark.parametrize("sign", [-1, 1])
@pytest.mark.parametrize("contig", [False, True], ids=["strided", "contiguous"])
def test_line_data_equals_dft_twiddle(T, W, sign, contig):
    m = Mirror(T, W, contig)
    G = 4
    nl = m.LEN * G
    u = uniform_pm1(1000 + T + W, np.arange(2 * W * m.LEN, dtype=np.uint64))
    x = (u[0::2] + 1j * u[1::2]).reshape(W, m.LEN)
    c = np.array([(w * 3 + 1) % G for w in range(W)])
    got = m.run(x, c, nl, sign)
    k = np.arange(m.LEN)
    want = np.stack([dft(x[w], sign) * root(nl, c[w] * k, sign) for w in range(W)])
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9 * m.LEN)


def decode_contig(b, w, G, Wc, Wo, nl, LEN):
    lg_wc = int(math.log2(Wc))
    lg_cgroups = int(math.log2(G)) - lg_wc
    cg, og = b & ((1 << lg_cgroups) - 1), b >> lg_cgroups
    o = og * Wo + (w >> lg_wc)
    c = (cg << lg_wc) + (w & (Wc - 1))
    return o * nl + c, o * nl + c * LEN, G, 1


def decode_strided(b, w, G, W, nl, inner, LEN):
    vgroups = inner // W
    vg, rest = b % vgroups, b // vgroups
    c, o = rest % G, rest // G
    v = vg * W + w
    return o * nl * inner + c * inner + v, o * nl * inner + c * LEN * inner + v, G * inner, inner


@pytest.mark.parametrize("case", [
    dict(shape=(16, 512), axis=1, G=2, Wc=2, Wo=8),     # contiguous, len 256, W = 16
    dict(shape=(2, 4096), axis=1, G=16, Wc=4, Wo=1),    # contiguous, len 256, W = 4 (long line)
    dict(shape=(512, 8), axis=0, G=2, W=8),             # strided, len 256
    dict(shape=(2, 1024, 4), axis=1, G=4, W=4),         # strided middle axis, len 256
])
def test_cta_decode_covers_input_and_put_positions(case):
    shape, axis, G = case["shape"], case["axis"], case["G"]
    nl = shape[axis]
    LEN = nl // G
    outer = int(np.prod(shape[:axis]))
    inner = int(np.prod(shape[axis + 1:]))
    N = outer * nl * inner
    seen_in = np.zeros(N, np.int64)
    seen_out = np.zeros(N, np.int64)
    if inner == 1:
        Wc, Wo = case["Wc"], case["Wo"]
        W = Wc * Wo
        ctas = (outer // Wo) * (G // Wc)
        dec = lambda b, w: decode_contig(b, w, G, Wc, Wo, nl, LEN)  # noqa: E731
    else:
        W = case["W"]
        ctas = outer * G * (inner // W)
        dec = lambda b, w: decode_strided(b, w, G, W, nl, inner, LEN)  # noqa: E731
    for b in range(ctas):
        for w in range(W):
            i0, o0, s_in, s_out = dec(b, w)
            idx_in = i0 + np.arange(LEN) * s_in
            idx_out = o0 + np.arange(LEN) * s_out
            assert idx_in.max() < N and idx_out.max() < N
            np.add.at(seen_in, idx_in, 1)
            np.add.at(seen_out, idx_out, 1)
    assert np.all(seen_in == 1) and np.all(seen_out == 1)


@pytest.mark.parametrize("T,W", line_configs(), ids=lambda v: str(v))
def test_contiguous_put_stores_are_runs(T, W):
    """Stage-3 (or, for T = 16, stage-2) stores of one warp on the contiguous axis: runs of at least 16
    consecutive k of one line."""
    m = Mirror(T, W, contig=True)
    for w0 in range(0, m.threads, 32):
        roles = [m.role2(t) for t in range(w0, min(w0 + 32, m.threads))]
        for k2 in range(16 if m.R3 == 1 else 1):
            by_line = defaultdict(list)
            for w, q in roles:
                by_line[w].append((q & 15) + 16 * (k2 if m.R3 == 1 else (q >> 4)))
            for ks in by_line.values():
                ks = sorted(ks)
                runs = sum(1 for i, k in enumerate(ks) if i == 0 or k != ks[i - 1] + 1)
                assert len(ks) % 16 == 0 and runs <= len(ks) // 16  # every run at least 16 long

"""CPU mirrors of the CUDA kernels' index arithmetic (no GPU).

compute-sanitizer is not available where the kernels run, so their address arithmetic is
checked here instead, by restating it in numpy and running it over every thread and task:

* the fused 3D phase A (phase_a3.cu), for every compile-time configuration, whose parameters
  are read from the `using ... = Cfg<...>` lines of the source itself: every shared-memory
  load and store stays inside its buffer, every store map is a bijection, every 16-byte pair
  access is 16-byte aligned, the bulk copies are 16-byte aligned, the scratch layout of a
  residue unit is a bijection, and the Put-position store of stage 2 (Superstep 1 of
  Algorithm 2.3) covers the unit's box of the output exactly once.  The mirror then carries
  data through those maps (small DFTs by numpy, twiddles from the maps' exponents) for one
  residue unit and compares with Superstep 0 of the CPU model of Algorithm 2.3 placed by the
  Put map m + s (n/p);
* the persistent ring's task decode: a bijection onto (unit, task, stage), and every task
  waits only on tasks that come earlier in the order, so the earliest unfinished task can
  always run;
* the 3D phase B (phase_b3.cu): loads and stores of all tiles cover the array exactly once and
  the data carried through the maps equals Superstep 2 of the model (Theorem 2.1's output map
  m + k (n/p)).
"""
import os
import re

import numpy as np
import pytest

from fftu_inputs import uniform_pm1
from oracle import cyclic_model as cm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2203_11795_gb300", "csrc")
SEED = 99


# ---- configurations, read from the kernel source ---------------------------------------------

class Cfg:
    NAMES = ("N2", "P2", "R1", "B", "A", "L0", "Q1", "W", "MINB", "NS", "PP", "GT", "NT")
    DEFAULTS = {"GT": False, "NT": 256}

    def __init__(self, name, args):
        self.name = name
        vals = dict(self.DEFAULTS)
        for k, v in zip(self.NAMES, args):
            vals[k] = {"true": True, "false": False}.get(v, None) if v in ("true", "false") else int(v)
        self.__dict__.update(vals)
        self.L2 = self.N2 // self.P2
        self.R2 = self.L2 // self.R1
        self.L1 = self.A * self.B
        self.Q2 = self.L0 // self.Q1
        self.NCH = self.N2 // self.W
        self.TILE1 = self.B * self.N2
        self.TILE2 = self.L0 * self.A * self.W
        self.TILE = max(self.TILE1, self.TILE2)
        self.UNIT = self.L0 * self.L1 * self.N2
        self.S1_TASKS = self.L0 * self.A
        self.S2_TASKS = self.B * self.NCH
        self.SW1 = min(16 // self.P2, self.R2)
        self.SW2 = min(16 // self.W, self.Q2)
        self.SWA = min(16 // self.W, self.A) - 1
        self.SIG = 16 // self.P2 if 16 // self.P2 > 1 else 2


def phase_a_configs():
    src = open(os.path.join(CSRC, "phase_a3.cu")).read()
    found = re.findall(r"using\s+(\w+)\s*=\s*Cfg<([^>]*)>;", src)
    assert found, "no phase-A configurations found in phase_a3.cu"
    return [Cfg(name, [a.strip() for a in args.split(",")]) for name, args in found]


CONFIGS = phase_a_configs()


def x2_index(K, b, k2, s2):
    """Stage-1 Put-order shared layout (x2_index in phase_a3.cu)."""
    sw = (s2 * K.SIG) & (K.L2 - 1) & 15
    return b * K.N2 + K.L2 * s2 + (k2 ^ sw)


def w(n, e, sign):
    """w_n^e = exp(sign 2 pi i e / n)."""
    return np.exp(sign * 2j * np.pi * (np.asarray(e) % n) / n)


def dft_last(v, sign):
    """Unscaled DFT over the last axis (exponent sign as given)."""
    r = v.shape[-1]
    return np.fft.fft(v, axis=-1) if sign < 0 else np.fft.ifft(v, axis=-1) * r


def assert_bijection(idx, size, what):
    idx = np.asarray(idx).ravel()
    assert idx.min() >= 0 and idx.max() < size, f"{what}: index out of [0, {size})"
    assert idx.size == size and np.bincount(idx, minlength=size).max() == 1, f"{what}: not a bijection"


def stage(src, load, store, dst_size, twiddle, sign, what):
    """Gather src[:, load] (load: items x R), DFT over R, times twiddle, scatter to dst[:, store]."""
    assert load.shape == store.shape
    assert_bijection(load, src.shape[1], what + " loads")
    assert_bijection(store, dst_size, what + " stores")
    vals = dft_last(src[:, load], sign) * twiddle
    dst = np.empty((src.shape[0], dst_size), dtype=np.complex128)
    dst[:, store] = vals
    return dst


def pair_axis(base, e):
    """Element e (0, 1) of the 16-byte pair whose first element is at base; base must be even."""
    assert np.all(np.asarray(base) % 2 == 0), "pair access not 16-byte aligned"
    return base + e


# ---- phase A: maps and a unit of data carried through them ----------------------------------

def emulate_unit(K, P0, P1, s0, s1, sign):
    """The ring kernel's work on residue unit (s0, s1): stage 1 over its L0 x A tasks, the scratch
    block, stage 2 over its B x NCH tasks.  Returns {global output index: value}."""
    n0, n1, N2 = P0 * K.L0, P1 * K.L1, K.N2
    HP2, HW = K.P2 // 2, K.W // 2
    # producer: B rows of N2 elements per stage-1 task, bulk copies of N2 * 8 bytes
    assert (N2 * 8) % 16 == 0 and (K.TILE2 * 8) % 16 == 0
    m0, a = np.meshgrid(np.arange(K.L0), np.arange(K.A), indexing="ij")
    m0, a = m0.ravel(), a.ravel()
    b = np.arange(K.B)
    row_off = ((s0 + P0 * m0)[:, None] * n1 + (s1 + P1 * (a[:, None] + K.A * b[None, :]))) * N2
    assert np.all(row_off % 2 == 0)
    g = row_off[:, :, None] + np.arange(N2)[None, None, :]            # tasks x B x N2 global indices
    buf = (uniform_pm1(SEED, 2 * g) + 1j * uniform_pm1(SEED, 2 * g + 1)).reshape(len(m0), K.TILE1)

    # S1a: items (b, q, sp, e) x r
    bb, q, sp, e = np.meshgrid(b, np.arange(K.R2), np.arange(HP2), [0, 1], indexing="ij")
    r = np.arange(K.R1)
    load = pair_axis((bb * N2 + 2 * sp + K.P2 * q)[..., None] + (N2 // K.R1) * r, e[..., None])
    u = np.arange(K.R1)
    store = pair_axis((((bb[..., None] * K.R1 + u) * K.R2 + (q[..., None] ^ (u % K.SW1))) * K.P2
                       + 2 * sp[..., None]), e[..., None])
    tw = w(N2, q[..., None] * u * K.P2, sign)
    x1 = stage(buf, load.reshape(-1, K.R1), store.reshape(-1, K.R1), K.TILE1, tw.reshape(-1, K.R1), sign, "S1a")

    # S1b: items (b, u, sp, e) x q
    bb, u, sp, e = np.meshgrid(b, np.arange(K.R1), np.arange(HP2), [0, 1], indexing="ij")
    q = np.arange(K.R2)
    load = pair_axis((((bb[..., None] * K.R1 + u[..., None]) * K.R2 + (q ^ (u[..., None] % K.SW1))) * K.P2
                      + 2 * sp[..., None]), e[..., None])
    v = np.arange(K.R2)
    k2 = u[..., None] + K.R1 * v
    s2 = 2 * sp[..., None] + e[..., None]
    store = x2_index(K, bb[..., None], k2, s2)
    tw = w(N2, k2 * s2, sign)
    x2 = stage(x1, load.reshape(-1, K.R2), store.reshape(-1, K.R2), K.TILE1, tw.reshape(-1, K.R2), sign, "S1b")

    # S1c: items (ip pair, e) x b; output to the unit's scratch (stage-1 tasks x their stores)
    ip, e = np.meshgrid(2 * np.arange(N2 // 2), [0, 1], indexing="ij")
    s2, k2 = ip // K.L2, ip % K.L2
    load = pair_axis(x2_index(K, b, k2[..., None], s2[..., None]), e[..., None])
    assert_bijection(load.ravel(), K.TILE1, "S1c loads")
    vals = dft_last(x2[:, load.reshape(-1, K.B)], sign)                 # tasks x items x c
    c = np.arange(K.B)
    vals = vals * w(n1, (a[:, None, None] * c * P1), sign)
    arow = m0 * K.A + (a ^ (m0 & K.SWA))
    ipe = (ip + e).reshape(-1)
    dst = ((ip // K.W).reshape(-1)[None, :, None] * K.TILE2 + arow[:, None, None] * K.W
           + (ipe % K.W)[None, :, None] + c[None, None, :] * K.NCH * K.TILE2)
    assert np.all(((ip // K.W) * K.TILE2 + (ip % K.W)) % 2 == 0)
    assert_bijection(dst, K.UNIT, "scratch layout of a residue unit")
    scratch = np.empty(K.UNIT, dtype=np.complex128)
    scratch[dst] = vals

    # stage 2: task lt = c * NCH + chunk lands the contiguous block scratch[lt * TILE2 : +TILE2]
    lt = np.arange(K.S2_TASKS)
    cc, chunk = lt // K.NCH, lt % K.NCH
    blk = scratch.reshape(K.S2_TASKS, K.TILE2)
    # S2a: items (m0, wp, e) x a
    mm, wp, e = np.meshgrid(np.arange(K.L0), np.arange(HW), [0, 1], indexing="ij")
    aa = np.arange(K.A)
    load = pair_axis((mm[..., None] * K.A + (aa ^ (mm[..., None] & K.SWA))) * K.W + 2 * wp[..., None],
                     e[..., None])
    ee = np.arange(K.A)
    store = pair_axis((ee * K.L0 + mm[..., None]) * K.W + 2 * wp[..., None], e[..., None])
    k1 = cc[:, None, None] + K.B * ee[None, None, :]
    tw = np.broadcast_to(w(n1, k1 * s1, sign), (K.S2_TASKS, load.reshape(-1, K.A).shape[0], K.A))
    y1 = stage(blk, load.reshape(-1, K.A), store.reshape(-1, K.A), K.TILE2, tw, sign, "S2a")
    # S2b: items (e, q, wp, pe) x r
    ee, q, wp, pe = np.meshgrid(np.arange(K.A), np.arange(K.Q2), np.arange(HW), [0, 1], indexing="ij")
    r = np.arange(K.Q1)
    load = pair_axis((ee[..., None] * K.L0 + q[..., None] + K.Q2 * r) * K.W + 2 * wp[..., None], pe[..., None])
    u = np.arange(K.Q1)
    store = pair_axis((((ee[..., None] * K.Q1 + u) * K.Q2 + (q[..., None] ^ (u % K.SW2))) * K.W
                       + 2 * wp[..., None]), pe[..., None])
    tw = w(n0, q[..., None] * u * P0, sign)
    y2 = stage(y1, load.reshape(-1, K.Q1), store.reshape(-1, K.Q1), K.TILE2, tw.reshape(-1, K.Q1), sign, "S2b")
    # S2c: items (e, u, wp, pe) x q; store at the Put position in the output
    ee, u, wp, pe = np.meshgrid(np.arange(K.A), np.arange(K.Q1), np.arange(HW), [0, 1], indexing="ij")
    q = np.arange(K.Q2)
    load = pair_axis((((ee[..., None] * K.Q1 + u[..., None]) * K.Q2 + (q ^ (u[..., None] % K.SW2))) * K.W
                      + 2 * wp[..., None]), pe[..., None])
    assert_bijection(load.ravel(), K.TILE2, "S2c loads")
    vals = dft_last(y2[:, load.reshape(-1, K.Q2)], sign)               # tasks x items x v
    vv = np.arange(K.Q2)
    k0 = u.reshape(-1)[:, None] + K.Q1 * vv                             # items x v
    vals = vals * w(n0, k0 * s0, sign)[None]
    base = ((cc[:, None] + K.B * ee.reshape(-1)[None, :] + K.L1 * s1) * N2 + chunk[:, None] * K.W
            + 2 * wp.reshape(-1)[None, :])
    assert np.all(base % 2 == 0)
    out = (base + pe.reshape(-1)[None, :])[..., None] + (k0 + K.L0 * s0)[None] * n1 * N2
    return out.ravel(), vals.ravel(), (n0, n1, N2)


# Both directions share every index map; the inverse (conjugated twiddles) runs on the smaller units.
PA_CASES = [(K, sgn) for K in CONFIGS for sgn in (-1, 1) if sgn < 0 or K.UNIT <= 1 << 22]


@pytest.mark.parametrize("K,sign", PA_CASES, ids=[k.name + ("_inv" if sg > 0 else "_fwd") for k, sg in PA_CASES])
def test_phase_a_maps_and_data(K, sign):
    P0, P1 = 2, 4            # n_0 = 2 L0, n_1 = 4 L1 (p_l^2 | n_l), unit (1, 3): no twiddle is trivially 1
    s0, s1 = 1, 3
    out, vals, (n0, n1, N2) = emulate_unit(K, P0, P1, s0, s1, sign)
    # the Put box of unit (s0, s1): rows k0 + L0 s0, k1 + L1 s1, all of axis 2, each exactly once
    i0, i1, i2 = out // (n1 * N2), (out // N2) % n1, out % N2
    assert np.all((i0 // K.L0 == s0) & (i1 // K.L1 == s1))
    local = ((i0 - K.L0 * s0) * K.L1 + (i1 - K.L1 * s1)) * N2 + i2
    assert_bijection(local, K.UNIT, "stage-2 Put stores of a unit")
    got = np.empty(K.UNIT, dtype=np.complex128)
    got[local] = vals
    # expected: Z^{(s0, s1, s2)} of Superstep 0, placed at m + s (n/p) along every axis
    p = (P0, P1, K.P2)
    L2 = K.L2
    j0, j1, j2 = np.meshgrid(np.arange(K.L0), np.arange(K.L1), np.arange(L2), indexing="ij")
    xs = {}
    for s2 in range(K.P2):
        gidx = ((s0 + P0 * j0) * n1 + (s1 + P1 * j1)) * N2 + (s2 + K.P2 * j2)
        xs[(s0, s1, s2)] = uniform_pm1(SEED, 2 * gidx) + 1j * uniform_pm1(SEED, 2 * gidx + 1)
    z = cm.superstep0(xs, (n0, n1, N2), p, inverse=sign > 0)
    want = np.concatenate([z[(s0, s1, s2)] for s2 in range(K.P2)], axis=2).reshape(-1)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 1e-12, (K.name, err)


# ---- the persistent ring's task order ----------------------------------------------------------

def decode_task(t, U, S1, S2, mode, lag):
    """decode_task in phase_a3.cu: task index -> (unit, local task, is stage 1)."""
    if mode == 0:
        return t // S1, t % S1, 1
    if mode == 1:
        return t // S2, t % S2, 0
    if t < lag * S1:
        return t // S1, t % S1, 1
    if t < lag * S1 + (U - lag) * (S1 + S2):
        rr = t - lag * S1
        j, o = rr // (S1 + S2) + lag, rr % (S1 + S2)
        return (j, o, 1) if o < S1 else (j - lag, o - S1, 0)
    rr = t - lag * S1 - (U - lag) * (S1 + S2)
    return U - lag + rr // S2, rr % S2, 0


@pytest.mark.parametrize("U,S1,S2,lag,ring", [(64, 512, 512, 1, 3), (64, 512, 512, 1, 2), (8, 4, 6, 2, 3),
                                              (256, 1024, 512, 1, 3), (3, 5, 7, 1, 2), (4, 4, 4, 3, 4)])
def test_ring_task_order(U, S1, S2, lag, ring):
    total = U * (S1 + S2)
    seen = set()
    first_s1, first_s2 = {}, {}
    last_s1, last_s2 = {}, {}
    for t in range(total):
        unit, loc, is_s1 = decode_task(t, U, S1, S2, 2, lag)
        assert 0 <= unit < U and 0 <= loc < (S1 if is_s1 else S2)
        seen.add((unit, loc, is_s1))
        if is_s1:
            first_s1.setdefault(unit, t)
            last_s1[unit] = t
        else:
            first_s2.setdefault(unit, t)
            last_s2[unit] = t
    assert len(seen) == total
    for unit in range(U):
        # stage 2 of a unit waits for all of its stage-1 tasks: they all come earlier
        assert last_s1[unit] < first_s2[unit]
        # stage 1 of unit u >= ring reuses the slot of unit u - ring: its stage-2 tasks come earlier
        if unit >= ring:
            assert last_s2[unit - ring] < first_s1[unit]
    for mode, S in ((0, S1), (1, S2)):
        got = {decode_task(t, U, S1, S2, mode, lag) for t in range(U * S)}
        assert len(got) == U * S


# ---- phase B (phase_b3.cu) -------------------------------------------------------------------

def phase_b3_kinds():
    """(P0, P1, P2, MT) of every instantiated 3D phase-B kernel, from the source's dispatch."""
    src = open(os.path.join(CSRC, "phase_b3.cu")).read()
    kinds = set()
    for args in re.findall(r"launch_t<C, DIR, (\d+), (\d+), (\d+), (\d+)>", src):
        kinds.add(tuple(int(a) for a in args))
    assert kinds
    return sorted(kinds)


def emulate_phase_b3(data, shape, kind, sign):
    P0, P1, P2, MT = kind
    HALF = MT // 2
    single = P0 >= 16 or P1 >= 16
    L0, L1, L2 = (n // q for n, q in zip(shape, (P0, P1, P2)))
    st0, st1 = shape[1] * shape[2], shape[2]
    tiles2 = L2 // MT
    tiles = L0 * L1 * tiles2
    RS = MT
    flat = data.reshape(-1)
    t = np.arange(tiles)
    m2t = (t % tiles2) * MT
    m1, m0 = (t // tiles2) % L1, (t // tiles2) // L1
    tbase = m0 * st0 + m1 * st1 + m2t                                  # base - 2 hp
    # step 1: thread (s0, s1, hp), pair element e, r along s2'
    s0, s1, hp, e = np.meshgrid(np.arange(P0), np.arange(P1), np.arange(HALF), [0, 1], indexing="ij")
    r = np.arange(P2)
    src_off = (pair_axis(2 * hp, e) + s0 * L0 * st0 + s1 * L1 * st1)[..., None] + r * L2
    sh = (((s0 * P1 + s1)[..., None] * P2 + r) * RS + pair_axis(2 * hp, e)[..., None])
    loads1 = tbase[:, None] + src_off.reshape(-1)[None, :]
    assert_bijection(loads1.ravel(), flat.size, "phase B loads")
    smem = np.empty((tiles, P0 * P1 * P2 * MT), dtype=np.complex128)
    assert_bijection(sh.ravel(), smem.shape[1], "phase B step-1 shared stores")
    smem[:, sh.reshape(-1, P2)] = dft_last(flat[loads1.reshape(tiles, -1, P2)], sign)
    # step 2: F_{P1} along s1' in place
    if single:
        s0, k2, el = np.meshgrid(np.arange(P0), np.arange(P2), np.arange(MT), indexing="ij")
        pos = ((s0[..., None] * P1 + np.arange(P1)) * P2 + k2[..., None]) * RS + el[..., None]
    else:
        s0, k2, h, e = np.meshgrid(np.arange(P0), np.arange(P2), np.arange(HALF), [0, 1], indexing="ij")
        pos = ((s0[..., None] * P1 + np.arange(P1)) * P2 + k2[..., None]) * RS + pair_axis(2 * h, e)[..., None]
    assert_bijection(pos.ravel(), smem.shape[1], "phase B step-2 shared accesses")
    smem[:, pos.reshape(-1, P1)] = dft_last(smem[:, pos.reshape(-1, P1)], sign)
    # step 3: F_{P0} along s0' and the store
    if single:
        k1, k2, el = np.meshgrid(np.arange(P1), np.arange(P2), np.arange(MT), indexing="ij")
        col = el
    else:
        k1, k2, h, e = np.meshgrid(np.arange(P1), np.arange(P2), np.arange(HALF), [0, 1], indexing="ij")
        col = pair_axis(2 * h, e)
    rr = np.arange(P0)
    pos = ((rr * P1 + k1[..., None]) * P2 + k2[..., None]) * RS + col[..., None]
    assert_bijection(pos.ravel(), smem.shape[1], "phase B step-3 shared loads")
    dst = (col + k1 * L1 * st1 + k2 * L2)[..., None] + rr * L0 * st0
    stores = tbase[:, None] + dst.reshape(-1)[None, :]
    assert_bijection(stores.ravel(), flat.size, "phase B stores")
    out = np.empty_like(flat)
    out[stores.reshape(tiles, -1, P0)] = dft_last(smem[:, pos.reshape(-1, P0)], sign)
    N = flat.size
    return (out / N if sign > 0 else out).reshape(shape)


def phase_b_shape(kind):
    P0, P1, P2, MT = kind
    # the smallest shape with p_l^2 | n_l whose last axis holds a whole number of tiles
    L = [max(P0, 2), max(P1, 2), max(P2, MT)]
    return tuple(q * l for q, l in zip((P0, P1, P2), L))


PB_CASES = [(k, sgn) for k in phase_b3_kinds() for sgn in (-1, 1)
            if sgn < 0 or int(np.prod(phase_b_shape(k))) <= 1 << 22]


@pytest.mark.parametrize("kind,sign", PB_CASES,
                         ids=["x".join(map(str, k)) + ("_inv" if sg > 0 else "_fwd") for k, sg in PB_CASES])
def test_phase_b3_maps_and_data(kind, sign):
    shape = phase_b_shape(kind)
    n = int(np.prod(shape))
    g = np.arange(n)
    wg = (uniform_pm1(SEED, 2 * g) + 1j * uniform_pm1(SEED, 2 * g + 1)).reshape(shape)
    got = emulate_phase_b3(wg, shape, kind, sign)
    want = cm.phase_b(wg, kind[:3], inverse=sign > 0)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12


# ---- the tensor-core radix-16 stage (umma16.cuh): operand layout and the real form of F_16 --------

def umma_off(m, k):
    """Byte offset of (row m, k) in a K = 32 operand tile of 16-bit values (umma_off in umma16.cuh)."""
    return (m & 7) * 16 + (m >> 3) * 512 + (k & 7) * 2 + (k >> 3) * 128


def canonical_element(tile, m, k, start, lbo=128, sbo=512):
    """Element (m, k) of an MMA operand read through a no-swizzle K-major descriptor at byte `start`
    (core matrices of 8 rows x 16 bytes, next along K at lbo, next 8 rows at sbo), k within one
    instruction's K = 16."""
    off = start + (m % 8) * 16 + (m // 8) * sbo + (k % 8) * 2 + (k // 8) * lbo
    return tile[off // 2]


def bf16_round(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("kind", ["bf16", "fp16"])
@pytest.mark.parametrize("sign", [-1, 1], ids=["fwd", "inv"])
def test_umma16_operands_compute_the_dft(kind, sign):
    """Rows written by umma_write_row and read back through the descriptors' layout, multiplied as
    the six MMAs do (x_hi G_hi + x_lo G_hi + x_hi G_lo, two K halves each), give the 16-point DFT
    of every row within the split's error; every offset stays inside its 8 KB / 2 KB tile."""
    rnd = bf16_round if kind == "bf16" else (lambda v: np.asarray(v, np.float32).astype(np.float16).astype(np.float32))
    rows = 128
    assert max(umma_off(m, k) for m in range(rows) for k in range(32)) + 2 <= rows * 32 * 2
    assert max(umma_off(n, k) for n in range(32) for k in range(32)) + 2 <= 32 * 32 * 2
    rng = np.random.default_rng(5)
    xc = (rng.uniform(-1, 1, (rows, 16)) + 1j * rng.uniform(-1, 1, (rows, 16))).astype(np.complex64)
    x = np.concatenate([xc.real, xc.imag], axis=1).astype(np.float32)        # rows x 32
    kk, r = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    F = np.exp(sign * 2j * np.pi * ((kk * r) % 16) / 16)                      # F[k][r]
    Gt = np.zeros((32, 32), dtype=np.float32)                                # row n of B = column n of G
    Gt[:16, :16], Gt[:16, 16:] = F.real, -F.imag                             # y_re = F_re x_re - F_im x_im
    Gt[16:, :16], Gt[16:, 16:] = F.imag, F.real                              # y_im = F_im x_re + F_re x_im

    def tiles(v, nrows):
        hi = rnd(v)
        lo = rnd(v - hi)
        out = []
        for part in (hi, lo):
            t = np.full(nrows * 32, np.nan, dtype=np.float32)
            for m in range(nrows):
                for k in range(32):
                    t[umma_off(m, k) // 2] = part[m, k]
            out.append(t)
        return out

    a_hi, a_lo = tiles(x, rows)
    g_hi, g_lo = tiles(Gt, 32)

    def operand(t, nrows, half):
        return np.array([[canonical_element(t, m, k, 256 * half) for k in range(16)] for m in range(nrows)])

    D = np.zeros((rows, 32), dtype=np.float64)
    for half in (0, 1):
        for A, B in ((a_hi, g_hi), (a_lo, g_hi), (a_hi, g_lo)):
            D += operand(A, rows, half).astype(np.float64) @ operand(B, 32, half).astype(np.float64).T
    y = D[:, :16] + 1j * D[:, 16:]
    ref = (xc.astype(np.complex128) @ F.T)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    u = 2.0 ** -8 if kind == "bf16" else 2.0 ** -11
    assert err <= 12 * u * u, err

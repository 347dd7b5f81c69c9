"""CPU mirror of the generic fused phase B's shared tile (generic_tiles.cuh, phaseb_dfts), no GPU.

A tile holds all P = prod p_l values of Superstep 2 of Algorithm 2.3 for Mt consecutive m along the last axis
(element e = mt + Mt * flat(s')).  Its DFT passes take the axes from the last one down, two adjacent axes per
pass where p_l p_{l-1} <= 16.  For complex64 whose first pass is a single axis over runs of Mt < 16 elements,
the tile slot of e is e ^ (((e >> log2(S R)) & (16/S - 1)) << log2(S)) (fftu_api.cu, make_phase_b_fused;
a two-axis first pass keeps the identity, which measured faster).  Checked here: the slot map is a bijection
that keeps the 16-byte pairs (2k, 2k + 1) together, and where it is on, every warp access of every pass and
of the paired loads and stores takes the minimum number of wavefronts.
"""
import math
from collections import defaultdict

import pytest


def wavefronts(idx):
    banks = defaultdict(set)
    for a in idx:
        for k in range(2):
            w = 2 * a + k
            banks[w % 32].add(w)
    return max(len(s) for s in banks.values())


def passes(p, Mt):
    d, S, out, l = len(p), Mt, [], len(p) - 1
    while l >= 0:
        pp = p[l] * p[l - 1] if (l > 0 and p[l] > 1 and p[l - 1] > 1) else 0
        if 0 < pp <= 16:
            out.append((S, pp))
            S *= pp
            l -= 2
        else:
            if p[l] > 1:
                out.append((S, p[l]))
            S *= p[l]
            l -= 1
    return out


def first_pass_paired(p):
    l = len(p) - 1
    while l >= 0:
        pp = p[l] * p[l - 1] if (l > 0 and p[l] > 1 and p[l - 1] > 1) else 0
        if 0 < pp <= 16:
            return True
        if p[l] > 1:
            return False
        l -= 1
    return False


def swizzle(p, Mt):
    ps = passes(p, Mt)
    if ps and not first_pass_paired(p) and ps[0][0] < 16 and ps[0][0] * ps[0][1] >= 16:
        S, R = ps[0]
        return int(math.log2(S * R)), 16 // S - 1, int(math.log2(S))
    return 0, 0, 0


def slot(e, sw):
    src, mask, dst = sw
    return e ^ (((e >> src) & mask) << dst)


def accesses(p, Mt, nt=256):
    total = math.prod(p) * Mt
    for S, R in passes(p, Mt):
        groups, lg_s = total // R, int(math.log2(S))
        for w0 in range(0, groups, 32):
            gs = range(w0, min(w0 + 32, groups))
            for r in range(R):
                yield 8, [((g >> lg_s) << lg_s) * R + (g & (S - 1)) + r * S for g in gs]
    for w0 in range(0, total // 2, 32):  # 16-byte pair loads and stores
        yield 16, [2 * t for t in range(w0, min(w0 + 32, total // 2))]


@pytest.mark.parametrize("p,Mt", [((8, 8, 8, 8), 8), ((8, 8, 8), 4), ((16, 16), 32), ((4, 4, 4, 4), 16),
                                  ((8, 8), 64), ((16, 16, 16), 8)])
def test_slot_map_bijective_pairs_and_minimum_wavefronts(p, Mt):
    sw = swizzle(p, Mt)
    total = math.prod(p) * Mt
    slots = [slot(e, sw) for e in range(total)]
    assert sorted(slots) == list(range(total))
    assert all(slot(e + 1, sw) == slot(e, sw) + 1 for e in range(0, total, 2))
    for width, idx in accesses(p, Mt):
        phys = [slot(e, sw) for e in idx]
        if width == 16:
            phys = [q for e in phys for q in (e, e + 1)]
        assert wavefronts(phys) == max(1, math.ceil(len(phys) * 8 / 128))


def test_swizzle_on_for_single_axis_first_pass_only():
    # 64^4 at p = 8^4: the first pass (one axis, runs of 8) had 4-way conflicts; the swizzle is on
    assert swizzle((8, 8, 8, 8), 8) == (6, 1, 3)
    plain = sum(wavefronts(i) for w, i in accesses((8, 8, 8, 8), 8) if w == 8)
    swz = sum(wavefronts([slot(e, (6, 1, 3)) for e in i]) for w, i in accesses((8, 8, 8, 8), 8) if w == 8)
    assert swz < plain
    # 32^5 at p = 4^5: the first pass takes two axes; the identity is kept (measured faster)
    assert swizzle((4, 4, 4, 4, 4), 8) == (0, 0, 0)

"""Stage-level pins for the CPU model of Algorithm 2.3 (Sec. 2.2).

The model is checked against the plain d-dim DFT (Theorem 2.1) and against the
intermediate closed forms of the theorem's proof: the Superstep 0 output Z, the
exchanged data W, and the output index map.  Special cases: p = 1 (Superstep 2
is the identity and every twiddle is 1), d = 1 (Algorithm 2.2), n_l = p_l^2.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import cyclic_model as cm
from fftu_inputs import complex_uniform

TOL = 1e-13

CASES = [
    ((8, 8, 8), (2, 2, 2)),
    ((64, 64, 64), (2, 2, 2)),
    ((16, 8, 32), (4, 2, 4)),
    ((64,), (8,)),
    ((16, 16), (4, 4)),
    ((4, 4, 4, 4, 16), (2, 2, 2, 2, 4)),
    ((32, 8), (1, 2)),
    ((8, 4, 16), (1, 1, 1)),
]


@pytest.mark.parametrize("shape,p", CASES, ids=lambda v: "x".join(map(str, v)))
@pytest.mark.parametrize("inverse", [False, True])
def test_model_computes_the_dft(shape, p, inverse):
    x = complex_uniform(101, shape)
    v = cm.run(x, p, inverse=inverse)
    assert oracle.rel_l2(v, oracle.fftn(x, inverse=inverse)) < TOL
    # the two halves compose to the whole
    assert oracle.rel_l2(cm.phase_b(cm.phase_a(x, p, inverse), p, inverse), v) < TOL


@pytest.mark.parametrize("shape,p", [((8, 8, 8), (2, 2, 2)), ((16, 4), (4, 2)), ((16,), (4,))])
def test_superstep0_closed_form(shape, p):
    # Z^{(s)}[k] = sum_j X^{(s)}[j] prod_l w_{n_l}^{k_l (j_l p_l + s_l)}
    x = complex_uniform(102, shape)
    z = cm.superstep0(cm.distribute(x, p), shape, p)
    for s in cm.processors(p):
        assert np.max(np.abs(z[s] - cm.z_closed_form(x, p, s))) < 1e-12


@pytest.mark.parametrize("shape,p", [((16, 8, 32), (4, 2, 4)), ((8, 8, 8), (2, 2, 2))])
def test_exchange_and_output_maps(shape, p):
    x = complex_uniform(103, shape)
    L = tuple(n // q for n, q in zip(shape, p))
    M = tuple(n // (q * q) for n, q in zip(shape, p))
    z = cm.superstep0(cm.distribute(x, p), shape, p)
    w = cm.superstep1(z, shape, p)
    v = cm.superstep2(w, shape, p)
    Y = oracle.fftn(x)
    for s in cm.processors(p):
        for t in itertools.product(*[range(m) for m in M]):
            for s2 in cm.processors(p):
                # W^{(s)}(t : n/p^2 : n/p)[s'] = Z^{(s')}[s + t p]
                r = tuple(t_l + a * m_l for t_l, a, m_l in zip(t, s2, M))
                src = tuple(a + t_l * q for a, t_l, q in zip(s, t, p))
                assert w[s][r] == z[s2][src]
            for k in cm.processors(p):
                # V^{(s)}[t + k n/p^2] = V[s + t p + k n/p]
                r = tuple(t_l + k_l * m_l for t_l, k_l, m_l in zip(t, k, M))
                g = tuple(a + t_l * q + k_l * ll for a, t_l, q, k_l, ll in zip(s, t, p, k, L))
                assert abs(v[s][r] - Y[g]) < 1e-11


def test_p_one_special_case():
    shape, p = (8, 4, 16), (1, 1, 1)
    x = complex_uniform(104, shape)
    w = cm.phase_a(x, p)
    assert oracle.rel_l2(w, oracle.fftn(x)) < TOL          # all twiddles are 1
    assert oracle.rel_l2(cm.phase_b(w, p), w) < 1e-15      # F_1 is the identity
    f = cm.twiddle_factors(shape, p, (0, 0, 0), -1)
    assert np.all(f == 1)


def test_put_layout_global_position():
    # Z^{(s')}[m] lands at global index m + s' (n/p) in the global view of W
    shape, p = (16, 32), (2, 4)
    L = tuple(n // q for n, q in zip(shape, p))
    x = complex_uniform(105, shape)
    z = cm.superstep0(cm.distribute(x, p), shape, p)
    wg = cm.phase_a(x, p)
    for s2 in cm.processors(p):
        block = tuple(slice(a * ll, (a + 1) * ll) for a, ll in zip(s2, L))
        assert np.array_equal(wg[block], z[s2])


def test_model_rejects_bad_p():
    with pytest.raises(ValueError):
        cm.run(np.zeros((8, 8)), (4, 2))   # 16 does not divide 8
    with pytest.raises(ValueError):
        cm.run(np.zeros((8, 8)), (2,))


def test_planted_model_mistakes_fail(monkeypatch):
    """Mistakes planted in the model (on the CPU) are caught by the DFT pin."""
    shape, p = (16, 8), (4, 2)
    x = complex_uniform(106, shape)
    ref = oracle.fftn(x)
    good = cm.twiddle_factors

    monkeypatch.setattr(cm, "twiddle_factors", lambda sh, pp, s, sign: good(sh, pp, s, -sign))
    assert oracle.rel_l2(cm.run(x, p), ref) > 1e-3           # twiddle sign flipped
    monkeypatch.setattr(cm, "twiddle_factors", lambda sh, pp, s, sign: np.ones(
        tuple(n // q for n, q in zip(sh, pp))))
    assert oracle.rel_l2(cm.run(x, p), ref) > 1e-3           # twiddle dropped
    monkeypatch.setattr(cm, "twiddle_factors", good)

    orig_put = cm.superstep1

    def bad_put(local_z, sh, pp):
        w = orig_put(local_z, sh, pp)
        s0 = cm.processors(pp)
        w[s0[0]], w[s0[1]] = w[s0[1]], w[s0[0]]              # packets to the wrong processor
        return w

    monkeypatch.setattr(cm, "superstep1", bad_put)
    assert oracle.rel_l2(cm.run(x, p), ref) > 1e-3


# Sec. 2.3 prints the largest processor counts the single-exchange method allows, p_max = prod_l p_l
# with p_l the largest power of two whose square divides n_l: 32^3 = 32,768 for 1024^3, 16^3 = 4096
# for 256^3 and 512^3, and 32,768 for the 2^24 x 64 array.
PRINTED_PMAX = [((1024, 1024, 1024), 32768), ((512, 512, 512), 4096), ((256, 256, 256), 4096),
                ((1 << 24, 64), 32768)]


def _largest_grid(shape):
    grid = []
    for n_l in shape:
        q = 1
        while n_l % ((2 * q) * (2 * q)) == 0:
            q *= 2
        grid.append(q)
    return tuple(grid)


@pytest.mark.parametrize("shape,pmax", PRINTED_PMAX, ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_printed_pmax(shape, pmax):
    """The model's condition p_l^2 | n_l admits exactly the grids of the printed p_max: the largest grid
    is accepted, doubling any axis of it is refused, and its product is the printed number."""
    grid = _largest_grid(shape)
    assert int(np.prod(grid)) == pmax
    cm._check(shape, grid)
    for l in range(len(shape)):
        bigger = list(grid)
        bigger[l] *= 2
        with pytest.raises(ValueError):
            cm._check(shape, tuple(bigger))


@pytest.mark.parametrize("shape,pmax", PRINTED_PMAX, ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_boundary_refuses_grids_beyond_printed_pmax(shape, pmax):
    """fftu_plan refuses (FFTU_ERR_DIVISIBILITY, before touching a device) every grid that doubles
    one axis of the largest admissible grid."""
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as f
    grid = _largest_grid(shape)
    for l in range(len(shape)):
        bigger = list(grid)
        bigger[l] *= 2
        with pytest.raises(f.FFTUError) as ei:
            f.fftu_plan(len(shape), list(shape), bigger, f.FFTU_C64, f.FFTU_FORWARD)
        assert ei.value.status == 2

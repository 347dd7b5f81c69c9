"""The serving loop (include/fftu_serve.h) on the GPU: every request of a mixed stream matches the
FP64 oracle, a request's result is bit-identical alone and in the mix, memory admission holds the
budget, and pageable, solo and graph-replayed requests all take their intended path."""
import math
import time

import numpy as np
import pytest

import oracle
from fftu_inputs import complex_uniform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fftu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as f
    return f


SHAPES = [(32, 32, 32), (64, 32, 16), (16, 16, 16, 16), (256, 128), (1024,), (64, 64, 64)]


def make_mix(count, seed, shapes=SHAPES, c128_share=0.25):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        shape = shapes[rng.integers(len(shapes))]
        dt = np.complex128 if rng.random() < c128_share else np.complex64
        inverse = bool(rng.integers(2))
        reqs.append((shape, dt, inverse, 500 + i))
    return reqs


def run_server(fftu, reqs, pinned=True, poll_timeout=60.0, passes=1, **cfg):
    """Submit every request (passes times, waiting for all completions after each pass); returns
    (outputs by tag, completions of the last pass, stats)."""
    import torch
    bufs = {}
    for shape, dt, inverse, seed in reqs:  # every buffer first, so that the submissions come in a burst
        x = torch.from_numpy(complex_uniform(seed, shape, dtype=dt))
        y = torch.empty_like(x)
        if pinned:
            x, y = x.pin_memory(), y.pin_memory()
        bufs[seed] = (x, y)
    s = fftu.fftu_server_create(**cfg)
    try:
        for _ in range(passes):
            for shape, dt, inverse, seed in reqs:
                x, y = bufs[seed]
                code = fftu.FFTU_C128 if dt == np.complex128 else fftu.FFTU_C64
                fftu.fftu_server_submit(s, shape, code, fftu.FFTU_INVERSE if inverse else fftu.FFTU_FORWARD,
                                        x.data_ptr(), y.data_ptr(), seed)
            fftu.fftu_server_drain(s, poll_timeout)
            done = fftu.fftu_server_poll(s, 4096)
        stats = fftu.fftu_server_stats_get(s)
    finally:
        fftu.fftu_server_destroy(s)
    return {tag: bufs[tag][1].numpy().copy() for tag in bufs}, done, stats


def check_against_oracle(reqs, outs, done):
    assert sorted(c["tag"] for c in done) == sorted(r[3] for r in reqs)
    assert all(c["status"] == 0 for c in done)
    for shape, dt, inverse, seed in reqs:
        x = complex_uniform(seed, shape, dtype=dt).astype(np.complex128)
        ref = oracle.fftn(x, inverse=inverse)
        tol = 1e-12 if dt == np.complex128 else 1e-5 * max(1.0, math.log2(x.size))
        assert oracle.rel_l2(outs[seed], ref) <= tol, (shape, dt, inverse)


def test_mixed_stream_matches_oracle(fftu):
    reqs = make_mix(60, seed=1)
    outs, done, stats = run_server(fftu, reqs, max_batch=16, max_inflight=1, passes=2)
    check_against_oracle(reqs, outs, done)
    assert stats["completed"] == 120 and stats["rejected"] == 0
    assert stats["batches"] < 120                                     # batched
    assert stats["graph_builds"] > 0 and stats["graph_replays"] > 0   # graphs built while idle, then replayed
    assert stats["graph_replays"] + stats["direct_launches"] == stats["batches"]
    for c in done:
        assert c["submit_s"] <= c["start_s"] <= c["done_s"]


def test_alone_equals_in_mix(fftu):
    probe = [((64, 32, 16), np.complex64, False, 9001), ((256, 128), np.complex128, True, 9002),
             ((64, 64, 64), np.complex64, True, 9003)]
    alone = {}
    for r in probe:
        outs, done, _ = run_server(fftu, [r])
        alone[r[3]] = outs[r[3]]
    mix = make_mix(80, seed=2) + probe
    rng = np.random.default_rng(3)
    order = list(rng.permutation(len(mix)))
    mixed, done, stats = run_server(fftu, [mix[i] for i in order], max_batch=32, max_inflight=1)
    assert all(c["status"] == 0 for c in done)
    assert any(c["batch_size"] > 1 for c in done if c["tag"] in alone)
    for tag, y in alone.items():
        assert np.array_equal(y, mixed[tag]), tag


def test_pageable_and_solo_paths(fftu):
    reqs = make_mix(12, seed=4, shapes=[(32, 32, 32), (128, 64)])
    outs, done, stats = run_server(fftu, reqs, pinned=False)
    check_against_oracle(reqs, outs, done)
    assert stats["graph_replays"] == 0 and stats["direct_launches"] == stats["batches"]
    # every request at or above large_elems runs alone through its own plan's kernels
    reqs = make_mix(10, seed=5, shapes=[(32, 32, 32), (16, 16)])
    outs, done, stats = run_server(fftu, reqs, large_elems=1024)
    check_against_oracle(reqs, outs, done)
    assert all(c["batch_size"] == 1 for c in done if c["tag"] in {r[3] for r in reqs if math.prod(r[0]) >= 1024})


def test_memory_admission(fftu):
    # a budget that holds one 64^3 complex64 batch of one at a time (plus its plan)
    N = 64 ** 3
    budget = 3 * N * 8 + (1 << 20)
    reqs = [((64, 64, 64), np.complex64, bool(i % 2), 700 + i) for i in range(6)]
    outs, done, stats = run_server(fftu, reqs, device_bytes=budget, max_batch=1)
    check_against_oracle(reqs, outs, done)
    assert stats["peak_bytes"] <= budget
    # a request that cannot fit even alone is refused, the others still run
    reqs = [((64, 64, 64), np.complex64, False, 800), ((256, 256, 256), np.complex64, False, 801)]
    outs, done, stats = run_server(fftu, reqs, device_bytes=budget)
    status = {c["tag"]: c["status"] for c in done}
    assert status[801] == 4 and status[800] == 0 and stats["rejected"] == 1
    check_against_oracle(reqs[:1], outs, [c for c in done if c["tag"] == 800])


def test_long_line_key_falls_back_to_solo(fftu):
    # a 1D line longer than one tile is not batchable; the server runs it alone
    reqs = [((32768,), np.complex64, False, 900), ((32768,), np.complex64, True, 901)]
    outs, done, stats = run_server(fftu, reqs)
    check_against_oracle(reqs, outs, done)


def test_warm_prebuilds_instances_and_graphs(fftu):
    """After fftu_server_warm, requests of the key replay graphs that already exist: no instance is
    created and no graph is built while they run, and every result still matches the oracle."""
    import torch
    shape, dt = (64, 32, 16), np.complex64
    x0 = torch.from_numpy(complex_uniform(1, shape, dtype=dt)).pin_memory()
    y0 = torch.empty_like(x0).pin_memory()
    s = fftu.fftu_server_create(max_batch=8, max_inflight=1)
    try:
        for inverse in (False, True):
            fftu.fftu_server_warm(s, shape, fftu.FFTU_C64, fftu.FFTU_INVERSE if inverse else fftu.FFTU_FORWARD,
                                  x0.data_ptr(), y0.data_ptr(), 8)
        warm = fftu.fftu_server_stats_get(s)
        # batch sizes 1, 2, 4, 8, one instance per batched stream (4 of the default 8), both directions
        assert warm["instances"] == 2 * 4 * 4 and warm["graph_builds"] == 2 * 4 * 4 and warm["completed"] == 0
        reqs = [(shape, dt, bool(i % 2), 1100 + i) for i in range(24)]
        bufs = {}
        for _, _, inverse, seed in reqs:
            x = torch.from_numpy(complex_uniform(seed, shape, dtype=dt)).pin_memory()
            bufs[seed] = (x, torch.empty_like(x).pin_memory())
        for _, _, inverse, seed in reqs:
            x, y = bufs[seed]
            fftu.fftu_server_submit(s, shape, fftu.FFTU_C64, fftu.FFTU_INVERSE if inverse else fftu.FFTU_FORWARD,
                                    x.data_ptr(), y.data_ptr(), seed)
        fftu.fftu_server_drain(s, 60.0)
        done = fftu.fftu_server_poll(s, 64)
        after = fftu.fftu_server_stats_get(s)
    finally:
        fftu.fftu_server_destroy(s)
    assert after["instance_creations"] == warm["instance_creations"]
    assert after["graph_builds"] == warm["graph_builds"] and after["graph_replays"] == after["batches"]
    check_against_oracle(reqs, {tag: bufs[tag][1].numpy() for tag in bufs}, done)
    with pytest.raises(fftu.FFTUError):  # max_k < 1
        s2 = fftu.fftu_server_create()
        try:
            fftu.fftu_server_warm(s2, shape, fftu.FFTU_C64, fftu.FFTU_FORWARD, x0.data_ptr(), y0.data_ptr(), 0)
        finally:
            fftu.fftu_server_destroy(s2)

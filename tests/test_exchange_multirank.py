"""The multi-GPU form of Algorithm 2.3 on CPU ranks (gloo): one rank per virtual processor s, each
holding only its local array X^{(s)}, and exactly one all-to-all between Superstep 0 and Superstep 2.

This checks the exchange design a multi-GPU build would use (the one-GPU library realises the same
redistribution as phase A's store pattern): rank s sends to rank k the packet Z^{(s)}(k : p : n/p)
of N/P^2 elements, and rank k places the packet from s as the box of W^{(k)} with corner s n/p^2
(Superstep 1).  The local supersteps come from the CPU model; the gathered output must be the d-dim
DFT of the whole array (Theorem 2.1), forward and inverse.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import oracle.cyclic_model as cm
from fftu_inputs import complex_uniform

SHAPE, P = (8, 4, 16), (2, 1, 2)  # four ranks, p_l^2 | n_l on every axis


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pack(z, p):
    """Packets for every destination k in rank order: Z^{(s)}(k : p : n/p), flattened."""
    return np.concatenate([z[tuple(slice(k_l, None, p_l) for k_l, p_l in zip(k, p))].reshape(-1)
                           for k in cm.processors(p)])


def _unpack(buf, shape, p):
    """W^{(k)} from the packets of every source s' in rank order (box with corner s' n/p^2)."""
    L = tuple(n // q for n, q in zip(shape, p))
    M = tuple(n // (q * q) for n, q in zip(shape, p))
    size = int(np.prod(M))
    w = np.empty(L, dtype=np.complex128)
    for i, s in enumerate(cm.processors(p)):
        w[tuple(slice(s_l * m_l, (s_l + 1) * m_l) for s_l, m_l in zip(s, M))] = \
            buf[i * size:(i + 1) * size].reshape(M)
    return w


def _rank(rank, world, port, inverse, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = cm.processors(P)[rank]
        X = complex_uniform(31, SHAPE, dtype=np.complex64).astype(np.complex128)
        xs = X[tuple(slice(s_l, None, p_l) for s_l, p_l in zip(s, P))].copy()  # this rank's data only
        z = cm.superstep0({s: xs}, SHAPE, P, inverse)[s]                      # Superstep 0, local
        send = torch.from_numpy(np.ascontiguousarray(_pack(z, P)))
        recv = torch.empty_like(send)
        dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send))  # Superstep 1: one exchange
        w = _unpack(recv.numpy(), SHAPE, P)
        v = cm.superstep2({s: w}, SHAPE, P, inverse)[s]                       # Superstep 2, local
        q.put((rank, s, v, send.numel()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("inverse", [False, True])
def test_one_all_to_all_between_local_supersteps(inverse):
    world = int(np.prod(P))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, inverse, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=180) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    N = int(np.prod(SHAPE))
    assert all(sent == N // world for _, _, _, sent in got)  # N/P elements leave every rank
    V = cm.collect({s: v for _, s, v, _ in got}, SHAPE, P)
    X = complex_uniform(31, SHAPE, dtype=np.complex64).astype(np.complex128)
    assert oracle.rel_l2(V, oracle.fftn(X, inverse=inverse)) < 1e-13


def test_pack_unpack_is_the_superstep1_put():
    """In one process: packing every Z^{(s)} and unpacking per destination equals the model's Put."""
    X = complex_uniform(32, SHAPE, dtype=np.complex64).astype(np.complex128)
    z = cm.superstep0(cm.distribute(X, P), SHAPE, P)
    procs = cm.processors(P)
    packs = {s: _pack(z[s], P) for s in procs}
    per = int(np.prod(SHAPE)) // len(procs) // len(procs)
    ref = cm.superstep1(z, SHAPE, P)
    for j, k in enumerate(procs):
        buf = np.concatenate([packs[s][j * per:(j + 1) * per] for s in procs])  # what rank k receives
        np.testing.assert_array_equal(_unpack(buf, SHAPE, P), ref[k])

"""Host logic of the x-slab block partition, on the CPU: the ghost layers'
flags, the exchange plan, and the exchange between ranks over gloo (world
size 2, one block per rank) with a stand-in for the pack and unpack calls."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2001_11806_gb300 import blocks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_block_flags():
    g = np.zeros((2, 3, 6), np.uint8)
    g[..., 2] = 1
    g[..., 5] = 4
    b = blocks.block_flags(g, 0, 3, periodic_x=True)
    assert b.shape == (2, 3, 5)
    assert np.all(b[..., 0] == 4)  # wraps to x = 5 (outlet): its own flag
    assert np.all(b[..., 1:4] == g[..., 0:3])
    assert np.all(b[..., 4] == blocks.GHOST)  # x = 3 is fluid: a ghost
    b = blocks.block_flags(g, 3, 6, periodic_x=False)
    assert np.all(b[..., 0] == 1)  # x = 2: a wall
    assert np.all(b[..., 4] == 1)  # outside a non-periodic axis
    b = blocks.block_flags(g, 0, 3, periodic_x=False)
    assert np.all(b[..., 0] == 1)


@pytest.mark.parametrize("n,periodic", [(1, True), (2, True), (2, False), (3, True), (4, False)])
def test_exchange_plan(n, periodic):
    plan = blocks.exchange_plan(n, periodic)
    faces = n if periodic else n - 1
    assert len(plan) == 2 * faces
    for s, f, r, rf in plan:
        assert rf != f
        assert r == ((s + 1) % n if f == blocks.XHIGH else (s - 1) % n)
        assert (r, rf, s, f) in plan
    assert len({(s, f) for s, f, _, _ in plan}) == len(plan)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, periodic, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = {}

    def pack(face):
        return torch.full((4,), float(10 * rank + face))

    def unpack(face, t):
        got[face] = float(t[0])

    blocks.exchange_ranks(pack, unpack, rank, world, periodic, dist)
    q.put((rank, got))
    dist.destroy_process_group()


@pytest.mark.parametrize("periodic", [True, False])
def test_exchange_between_two_ranks_over_gloo(periodic):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(world))
    # rank 0's XHIGH face receives what rank 1 sent across its XLOW face, and back
    assert res[0][blocks.XHIGH] == 10 * 1 + blocks.XLOW
    assert res[1][blocks.XLOW] == 10 * 0 + blocks.XHIGH
    if periodic:
        assert res[0][blocks.XLOW] == 10 * 1 + blocks.XHIGH
        assert res[1][blocks.XHIGH] == 10 * 0 + blocks.XLOW
    else:
        assert blocks.XLOW not in res[0] and blocks.XHIGH not in res[1]


def test_single_periodic_rank_exchanges_with_itself():
    got = {}
    blocks.exchange_ranks(lambda f: torch.full((2,), float(f)), lambda f, t: got.__setitem__(f, float(t[0])), 0, 1,
                          True, None)
    assert got == {blocks.XHIGH: float(blocks.XLOW), blocks.XLOW: float(blocks.XHIGH)}

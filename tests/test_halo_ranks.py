"""The halo exchange between ranks on CPU: world_size 2 and 3 gloo ranks,
each with its local mesh from the library's partition.  Every rank fills its
send buffers with codes of its own face-node traces (global element, node,
variable); after the exchange each received row must hold the codes of the
neighbour's matching traces, which the test derives from the global mesh."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _face_node(n, l, a, b):
    N = n - 1
    return [n * (a + n * b), N + n * (a + n * b), a + n * n * b, a + n * (N + n * b), a + n * b,
            a + n * (b + n * N)][l]


def _codes(elem, l, n, rows):
    """[rows][n2] codes of element elem's traces on its face l."""
    out = np.zeros((rows, n * n))
    for ab in range(n * n):
        p = _face_node(n, l, ab % n, ab // n)
        for v in range(rows):
            out[v, ab] = (elem * n ** 3 + p) * 10 + v
    return out


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    from paper_2606_18927_gb300 import dg, halo, inputs as I
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        N = 2
        n = N + 1
        spec = I.BoxSpec(N, 4, 3, 3, periodic=(True, False, True))
        x, w = dg.lgl_nodes(N)
        X = I.node_coordinates(spec, x)
        nbr = I.connectivity(spec)
        part = dg.partition_sfc(N, X, world)
        l2g, nbl, _, _, hl = dg.partition_local(nbr, part, rank)
        nh = len(hl)
        sendU = torch.zeros((nh, 5, n * n), dtype=torch.float64)
        sendG = torch.zeros((nh, 4, n * n), dtype=torch.float64)
        for h, (peer, e, l, m) in enumerate(hl):
            sendU[h] = torch.from_numpy(_codes(l2g[e], l, n, 5))
            sendG[h] = torch.from_numpy(_codes(l2g[e], l, n, 4))
        recvU = torch.full_like(sendU, -1.0)
        recvG = torch.full_like(sendG, -1.0)
        halo.exchange(sendU, recvU, hl)
        halo.exchange(sendG, recvG, hl)
        bad = 0
        for h, (peer, e, l, m) in enumerate(hl):
            gn = nbr[l2g[e], l]
            bad += int(not np.array_equal(recvU[h].numpy(), _codes(gn, l ^ 1, n, 5)))
            bad += int(not np.array_equal(recvG[h].numpy(), _codes(gn, l ^ 1, n, 4)))
            bad += int(part[gn] != peer)
        q.put((rank, nh, bad))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_between_gloo_ranks(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(nh > 0 for _, nh, _ in out)
    assert all(bad == 0 for _, _, bad in out), out

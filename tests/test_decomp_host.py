"""Host logic of the block decomposition (paper_2608_09615_b300.decomp) on the CPU: the
exchange plans fill every ghost element of every sub-domain with the right neighbour's
data (checked against the periodic window of the global grid), the BR1 face-gradient plan
delivers the owners' face blocks to exactly the ghost faces that owned elements read, and
two gloo ranks (127.0.0.1) running the same plans over torch.distributed messages agree
with the single-process result; the FP64 all-reduce of the diagnostics sums the ranks."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

from paper_2608_09615_b300.decomp import (Partition, allreduce_diagnostics, depth_for, dist_deliver,
                                          run_plan)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

NV, NPT = 2, 3          # two variables, three "points" per element: enough to see any mix-up


def _global_state(ne, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (NV, ne[2], ne[1], ne[0], NPT))


def _flat(A):
    """[v][z][y][x][pt] -> [v][element][pt] (element index x fastest)."""
    return A.reshape(A.shape[0], -1, A.shape[-1])


def _cpu_pack(A):
    def pack(m):
        return _flat(A)[:, m.send, :].copy()
    return pack


def _cpu_unpack(A):
    def unpack(m, buf):
        F = _flat(A)
        F[:, m.recv, :] = buf
    return unpack


def _local_exchange(part, boxes):
    """All ranks in one process: axis by axis, every rank's messages packed, then delivered
    to the peer's matching ghost indices."""
    plans = [part.state_plan(r) for r in range(part.size)]
    for a in range(3):
        outbox = {}
        for r in range(part.size):
            for m in plans[r]:
                if m.axis == a:
                    outbox[(m.peer, a, 1 - m.side)] = _flat(boxes[r])[:, m.send, :].copy()
        for r in range(part.size):
            for m in plans[r]:
                if m.axis == a:
                    _flat(boxes[r])[:, m.recv, :] = outbox[(r, a, m.side)]


PARTS = [((6, 5, 4), (2, 2, 2), 1), ((6, 5, 4), (3, 1, 2), 1), ((8, 6, 4), (2, 3, 1), 2),
         ((5, 4, 6), (1, 1, 3), 2), ((4, 4, 4), (4, 1, 1), 1), ((9, 7, 5), (3, 2, 2), 1)]


@pytest.mark.parametrize("ne,parts,depth", PARTS)
def test_state_exchange_fills_every_ghost(ne, parts, depth):
    part = Partition(ne, parts, depth)
    U = _global_state(ne)
    ref = part.scatter(U)
    boxes = []
    for r in range(part.size):
        B = np.full_like(ref[r], np.nan)
        (lo, hi) = part.owned_local(r)
        sl = (slice(None), slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        B[sl] = ref[r][sl]                       # only the owned block is known before
        boxes.append(B)
    _local_exchange(part, boxes)
    for r in range(part.size):
        assert np.array_equal(boxes[r], ref[r]), "rank %d" % r
    # the owned blocks tile the grid exactly once
    assert np.array_equal(part.gather_owned(boxes, U), U)


def test_partition_geometry():
    part = Partition((10, 7, 4), (3, 2, 1), 2)
    assert part.size == 6
    assert [part.owned(r)[0][0] for r in range(3)] == [0, 3, 6]
    assert part.local_shape(0) == (3 + 4, 3 + 4, 4)            # z not split: no ghosts
    assert part.neighbour(0, 0, 0) == 2 and part.neighbour(2, 0, 1) == 0
    assert part.box_origin(0) == (-2, -2, 0)
    assert depth_for("compact", False) == 1 and depth_for("br1", True) == 1 and depth_for("br1", False) == 2
    with pytest.raises(ValueError):
        Partition((4, 4, 4), (3, 1, 1), 2)                      # blocks of 1 cannot feed 2 layers
    with pytest.raises(ValueError):
        Partition((4, 4, 4), (5, 1, 1), 1)


@pytest.mark.parametrize("ne,parts", [((6, 5, 4), (2, 2, 2)), ((6, 4, 5), (3, 1, 2)), ((4, 6, 4), (1, 3, 1))])
def test_face_gradient_plan_reaches_exactly_the_faces_owned_elements_read(ne, parts):
    # Synthetic face blocks: the value of (global element g, face f) is 10 g + f on its owner.
    part = Partition(ne, parts, 1)
    G = 4
    boxes = []
    for r in range(part.size):
        shp = part.local_shape(r)
        o = part.box_origin(r)
        T = np.full((int(np.prod(shp)), 6, G), np.nan)
        (lo, hi) = part.owned_local(r)
        for z, y, x in itertools.product(range(lo[2], hi[2]), range(lo[1], hi[1]), range(lo[0], hi[0])):
            gx, gy, gz = ((x + o[0]) % ne[0], (y + o[1]) % ne[1], (z + o[2]) % ne[2])
            g = gx + ne[0] * (gy + ne[1] * gz)
            T[x + shp[0] * (y + shp[1] * z)] = (10.0 * g + np.arange(6))[:, None]
        boxes.append(T)
    plans = [part.grad_plan(r) for r in range(part.size)]
    for a in range(3):
        outbox = {}
        for r in range(part.size):
            for m in plans[r]:
                if m.axis == a:
                    outbox[(m.peer, a, 1 - m.side)] = boxes[r][m.send, m.send_faces].copy()
        for r in range(part.size):
            for m in plans[r]:
                if m.axis == a:
                    boxes[r][m.recv, m.recv_faces] = outbox[(r, a, m.side)]
    # every face of a face-neighbour ghost that an owned element shares holds the owner's value
    for r in range(part.size):
        shp = part.local_shape(r)
        o = part.box_origin(r)
        (lo, hi) = part.owned_local(r)
        for z, y, x in itertools.product(range(lo[2], hi[2]), range(lo[1], hi[1]), range(lo[0], hi[0])):
            c = [x, y, z]
            for d in range(3):
                for side in (0, 1):
                    nb = list(c)
                    nb[d] += 1 if side else -1
                    if lo[d] <= nb[d] < hi[d] or part.halo(d) == 0:
                        continue                          # owned, or periodic inside the box
                    gx, gy, gz = ((nb[0] + o[0]) % ne[0], (nb[1] + o[1]) % ne[1], (nb[2] + o[2]) % ne[2])
                    g = gx + ne[0] * (gy + ne[1] * gz)
                    f = 2 * d + (1 - side)                # the neighbour's face towards us
                    le = nb[0] + shp[0] * (nb[1] + shp[1] * nb[2])
                    assert np.all(boxes[r][le, f] == 10.0 * g + f), (r, c, d, side)


def test_run_plan_with_a_local_deliver_matches_the_reference():
    ne, parts = (6, 4, 4), (2, 2, 1)
    part = Partition(ne, parts, 1)
    U = _global_state(ne, seed=3)
    ref = part.scatter(U)
    boxes = [np.zeros_like(b) for b in ref]
    for r in range(part.size):
        (lo, hi) = part.owned_local(r)
        sl = (slice(None), slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        boxes[r][sl] = ref[r][sl]
    plans = [part.state_plan(r) for r in range(part.size)]
    # one deliver per axis over all ranks: emulate the transport by a shared mailbox
    for a in range(3):
        mail = {}
        for r in range(part.size):
            for m in plans[r]:
                if m.axis == a:
                    mail[(m.peer, a, 1 - m.side)] = _cpu_pack(boxes[r])(m)
        for r in range(part.size):
            run_plan([m for m in plans[r] if m.axis == a], lambda m: None, _cpu_unpack(boxes[r]),
                     lambda msgs, bufs, r=r: [mail[(r, m.axis, m.side)] for m in msgs])
    for r in range(part.size):
        assert np.array_equal(boxes[r], ref[r])


# ---------------------------------------------------------------------- two gloo ranks
def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2608_09615_b300.decomp import Partition as P, allreduce_diagnostics as ar, dist_deliver as dd, \
        run_plan as rp
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ne, parts = (6, 4, 5), (2, 1, 1)
    part = P(ne, parts, 2)
    rng = np.random.default_rng(0)
    U = rng.uniform(-1, 1, (NV, ne[2], ne[1], ne[0], NPT))
    ref = part.extend(rank, U)
    box = np.zeros_like(ref)
    (lo, hi) = part.owned_local(rank)
    sl = (slice(None), slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
    box[sl] = ref[sl]
    T = torch.from_numpy(np.ascontiguousarray(box))

    def pack(m):
        return T.reshape(NV, -1, NPT)[:, torch.from_numpy(m.send).long(), :].contiguous()

    def unpack(m, buf):
        T.reshape(NV, -1, NPT)[:, torch.from_numpy(m.recv).long(), :] = buf

    rp(part.state_plan(rank), pack, unpack, dd(dist, rank))
    ok = bool(np.array_equal(T.numpy(), ref))
    d = {"ke": 1.0 + rank, "ke_rho": 2.0, "enstrophy": 0.5 * rank, "mass": 3.0, "energy": 4.0, "l2sq": 0.0,
         "volume": 10.0, "mom": [rank, -rank, 0.25], "nonfinite": rank == 1, "t": 0.5}
    s = ar(d, dist)
    out[rank] = (ok, s["ke"], s["volume"], s["mom"], s["nonfinite"])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_exchange_halos():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        ok, ke, vol, mom, nonfinite = out[r]
        assert ok, "rank %d ghosts differ from the periodic window" % r
        assert ke == 3.0 and vol == 20.0 and mom == [1.0, -1.0, 0.5] and nonfinite == 1
    del torch


def test_allreduce_is_importable_without_a_group():
    assert callable(allreduce_diagnostics) and callable(dist_deliver)

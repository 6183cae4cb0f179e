"""The 1-D row partition and the sparse-x all-gather on 2 and 3 gloo ranks (CPU).

Each rank owns a row block with about half the nonzeros and the matching part
of x; after the all-gather every rank computes its block of y (here with the
oracle standing in for the device kernel) and the parts reassemble into the
full oracle product. A distributed BFS step checks the frontier union."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import gen
import oracle
from paper_2006_16767_gb300 import dist as pdist


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def sparse_input(n, bounds, world):
    """300 listed nonzeros; with three ranks all of them fall in rank 0's
    rows, so the other ranks contribute empty lists to the all-gather."""
    idx, val = gen.sparse_x(n, 300, seed=23)
    if world == 3:
        keep = idx < bounds[1]
        idx, val = idx[keep], val[keep]
    return idx, val


def worker(rank, world, port, q):
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        rp, c = gen.rmat(12, 8, seed=21)
        n = 1 << 12
        v = gen.uniform(len(c), -1, 1, seed=22)
        bounds = pdist.row_partition(rp, world)
        r0, r1 = bounds[rank], bounds[rank + 1]
        lrp, lc, lv = pdist.local_rows(rp, c, v, r0, r1)
        # x: listed nonzeros, each rank holds the ones in its own row range
        idx, val = sparse_input(n, bounds, world)
        mine = (idx >= r0) & (idx < r1)

        def local_product(gi, gv):
            y, _, _ = oracle.spmspv_rowmajor(n, lrp, lc, lv, gi.numpy(), gv.numpy())
            return torch.from_numpy(y)

        y_local = pdist.partitioned_spmspv(local_product, torch.from_numpy(idx[mine]),
                                           torch.from_numpy(val[mine]))
        parts = [None] * world
        dist.all_gather_object(parts, (r0, r1, y_local.numpy()))
        # a BFS step: the next frontier is the union of the ranks' parts
        level, L = oracle.bfs(n, rp, c, int(np.flatnonzero(np.diff(rp) > 0)[0]))
        f = np.flatnonzero(level == 1).astype(np.int32)
        fm = f[(f >= r0) & (f < r1)]
        gi, _ = pdist.allgather_list(torch.from_numpy(fm), None)
        xb = np.zeros(n, np.uint8)
        xb[gi.numpy()] = 1
        yb = oracle.bool_pull(lrp, lc, xb)
        nxt_local = (np.flatnonzero(yb) + r0).astype(np.int32)
        fr = [None] * world
        dist.all_gather_object(fr, nxt_local)
        # the same exchange with the lengths kept in device tensors: the packed
        # buffer's first `total` entries equal the host-side concatenation
        cap = pdist.list_capacity(bounds)
        xi, xv = torch.from_numpy(idx[mine]), torch.from_numpy(val[mine])
        bi, bv, tot = pdist.allgather_list_device(xi, xv, torch.tensor([xi.numel()], dtype=torch.int64), cap)
        hi, hv = pdist.allgather_list(xi, xv)
        k = int(tot.item())
        same = k == hi.numel() and torch.equal(bi[:k], hi) and torch.equal(bv[:k], hv)
        ei, ev, etot = pdist.allgather_list_device(xi[:0], None, torch.zeros(1, dtype=torch.int64), cap)
        same = same and int(etot.item()) == 0 and ev is None
        if rank == 0:
            q.put(("ok", bounds, parts, fr, len(c), same))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # report to the parent instead of hanging it
        q.put(("err", repr(e)))


def test_row_partition_balances_nonzeros():
    rp, c = gen.rmat(14, 16, seed=3)
    for world in (1, 2, 3, 4, 8):
        b = pdist.row_partition(rp, world)
        assert b[0] == 0 and b[-1] == len(rp) - 1 and all(b[i] <= b[i + 1] for i in range(world))
        loads = [rp[b[i + 1]] - rp[b[i]] for i in range(world)]
        assert sum(loads) == rp[-1]
        assert max(loads) - min(loads) <= 2 * np.diff(rp).max() + 1
    assert pdist.owner_of([0, 5, 9], np.array([0, 4, 5, 8])).tolist() == [0, 0, 1, 1]


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reassemble_the_product(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
    assert res[0] == "ok", res
    _, bounds, parts, fr, nnz, same = res
    assert same, "device-count exchange differs from the host-count one"
    rp, c = gen.rmat(12, 8, seed=21)
    n = 1 << 12
    v = gen.uniform(len(c), -1, 1, seed=22)
    idx, val = sparse_input(n, bounds, world)
    if world == 3:
        assert 0 < len(idx) < 300
    y_ref, s, _ = oracle.spmspv_rowmajor(n, rp, c, v, idx, val)
    y = np.zeros(n)
    for (r0, r1, yl) in parts:
        y[r0:r1] = yl
    assert np.array_equal(y, y_ref)
    level, L = oracle.bfs(n, rp, c, int(np.flatnonzero(np.diff(rp) > 0)[0]))
    reached = np.flatnonzero(level == 2)
    union = np.concatenate(fr)
    visited = np.flatnonzero((level >= 0) & (level <= 1))
    assert np.array_equal(np.setdiff1d(union, visited), reached)

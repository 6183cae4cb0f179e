"""1-D row partition of y = A x across ranks (one process per GPU).

A is split into contiguous row blocks with about equal nonzero counts; rank
r keeps rows [r0, r1) in CSR (and builds its own handle, CSC included, on its
GPU). For a square A whose x and y share the row partition -- BFS frontiers,
PageRank vectors -- every rank holds the listed nonzeros of x in its own
range, all ranks exchange them with one all-gather of variable-length lists,
and each rank multiplies its row block by the gathered x, producing its own
part of y. No reduction is needed: y stays partitioned, and the next
frontier of a BFS is the union of the ranks' parts.

The exchange runs through torch.distributed (NCCL between GPUs, gloo on CPU
ranks in tests). The local product is a callable, so the same driver serves
the library's device kernels and host-side checks. allgather_list reads the
list lengths on the host; allgather_list_device keeps them on the device
(padded exchange, packing by a scatter), so a device-side loop of products
is not stalled by the exchange.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def row_partition(rowptr, world: int):
    """Row bounds [b_0 = 0, ..., b_world = m] splitting the nonzeros evenly
    (each bound is the first row whose start reaches r * nnz / world)."""
    rowptr = np.asarray(rowptr, np.int64)
    m = len(rowptr) - 1
    nnz = int(rowptr[-1])
    bounds = [0]
    for r in range(1, world):
        target = (nnz * r) // world
        bounds.append(int(np.searchsorted(rowptr[:m], target, "left")))
    bounds.append(m)
    for r in range(1, world + 1):
        bounds[r] = max(bounds[r], bounds[r - 1])
    return bounds


def local_rows(rowptr, col, val, r0: int, r1: int):
    """CSR of rows [r0, r1) (column ids unchanged)."""
    rowptr = np.asarray(rowptr, np.int64)
    lo, hi = int(rowptr[r0]), int(rowptr[r1])
    rp = (rowptr[r0:r1 + 1] - lo).astype(np.int32)
    return rp, np.asarray(col[lo:hi]), (None if val is None else np.asarray(val[lo:hi]))


def owner_of(bounds, j: np.ndarray):
    """Rank owning each index j under the row bounds."""
    return np.searchsorted(np.asarray(bounds[1:], np.int64), j, "right")


def allgather_list(idx: torch.Tensor, val: torch.Tensor | None, group=None):
    """All-gather variable-length (idx, val) lists; returns the concatenation
    in rank order (so locally ascending lists stay globally ascending)."""
    world = dist.get_world_size(group)
    n = torch.tensor([idx.numel()], dtype=torch.int64, device=idx.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(max(sizes), 1)
    pad_i = torch.zeros(cap, dtype=idx.dtype, device=idx.device)
    pad_i[: idx.numel()] = idx
    gi = [torch.empty_like(pad_i) for _ in range(world)]
    dist.all_gather(gi, pad_i, group=group)
    out_i = torch.cat([g[:s] for g, s in zip(gi, sizes)])
    if val is None:
        return out_i, None
    pad_v = torch.zeros(cap, dtype=val.dtype, device=val.device)
    pad_v[: val.numel()] = val
    gv = [torch.empty_like(pad_v) for _ in range(world)]
    dist.all_gather(gv, pad_v, group=group)
    return out_i, torch.cat([g[:s] for g, s in zip(gv, sizes)])


def list_capacity(bounds):
    """Entries a rank's part of x can hold at most: its row-block length
    (x shares the row partition, and listed ids are distinct)."""
    return max(1, max(bounds[r + 1] - bounds[r] for r in range(len(bounds) - 1)))


def allgather_list_device(idx: torch.Tensor, val: torch.Tensor | None, count: torch.Tensor, cap: int,
                          group=None):
    """All-gather of variable-length lists without a host synchronisation:
    every rank sends its list padded to `cap` entries and its length as a
    one-element int64 tensor `count` (on the lists' device); the gathered
    segments are packed in rank order by a scatter whose target positions
    come from the counts' prefix sums, all on the device. Returns
    (idx_buffer, val_buffer or None, total) where the first `total` entries
    (a one-element device tensor, the form the library's list count takes)
    hold the concatenation. No operation reads a count on the host, so the
    exchange can sit between device-side products without stalling them."""
    world = dist.get_world_size(group)
    dev = idx.device
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(counts, count.reshape(1).to(torch.int64), group=group)
    counts = torch.cat(counts)
    offs = torch.cumsum(counts, 0) - counts
    pos = torch.arange(cap, dtype=torch.int64, device=dev)
    # target of entry i of rank r: offs[r] + i when i < counts[r], else the
    # dump slot world * cap (one past the packed region's largest extent)
    tgt = torch.where(pos[None, :] < counts[:, None], offs[:, None] + pos[None, :],
                      torch.full((1, 1), world * cap, dtype=torch.int64, device=dev)).reshape(-1)

    def gather_pack(t):
        pad = torch.zeros(cap, dtype=t.dtype, device=dev)
        pad[: t.numel()] = t
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        out = torch.zeros(world * cap + 1, dtype=t.dtype, device=dev)
        out.scatter_(0, tgt, torch.cat(parts))
        return out

    out_i = gather_pack(idx)
    out_v = None if val is None else gather_pack(val)
    return out_i, out_v, counts.sum().reshape(1)


def partitioned_spmspv(local_product, x_idx_local, x_val_local, group=None):
    """One distributed product: gather x's listed nonzeros from every rank,
    then run this rank's row block. local_product(idx, val) returns this
    rank's part of y."""
    idx, val = allgather_list(x_idx_local, x_val_local, group)
    return local_product(idx, val)

"""Sharded skyline across processes (torch.distributed), host-side logic.

The skyline of a point set split over R ranks is the skyline of the union of
the ranks' local skylines: any point dominated inside its own shard is
dominated globally, and any dominator of a point has a skyline dominator
(transitivity of Definition 1). So each rank reduces its shard locally, the
ranks exchange only their local skylines (all-gather of points and global row
ids), and every rank reduces the union the same way.

`local_skyline` is the function that computes one skyline (on a GPU rank:
`paper_2107_09993_b300.skyline`); this module does no skyline arithmetic of
its own. The benchmark runs independent replicas instead (one point set per
GPU); this path serves callers whose single point set is spread over ranks.
"""
from __future__ import annotations

import numpy as np


def _all_gather_rows(group, rows: np.ndarray, width: int, dtype):
    """All-gather a variable number of rows from every rank (numpy in/out)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    n = torch.tensor([rows.shape[0]], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(max(sizes), 1)
    buf = torch.zeros((cap, width), dtype=dtype)
    if rows.shape[0]:
        buf[:rows.shape[0]] = torch.from_numpy(np.ascontiguousarray(rows))
    outs = [torch.zeros((cap, width), dtype=dtype) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    return np.concatenate([o[:s].numpy() for o, s in zip(outs, sizes)], axis=0)


def skyline_sharded(points: np.ndarray, row_offset: int, local_skyline, group=None) -> np.ndarray:
    """Global skyline of the union of all ranks' `points` (float32 [n_r, d],
    this rank holding global rows row_offset .. row_offset + n_r - 1).
    Returns the ascending global row ids, identical on every rank."""
    import torch

    P = np.ascontiguousarray(points, dtype=np.float32)
    d = P.shape[1]
    loc = np.asarray(local_skyline(P), dtype=np.int64)
    cand = P[loc]
    ids = loc + int(row_offset)
    allP = _all_gather_rows(group, cand, d, torch.float32)
    allI = _all_gather_rows(group, ids.reshape(-1, 1), 1, torch.int64).ravel()
    keep = np.asarray(local_skyline(allP), dtype=np.int64)
    return np.sort(allI[keep])

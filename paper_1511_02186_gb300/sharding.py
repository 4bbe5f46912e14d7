"""Query sharding over ranks: one process per GPU, each interpolating a contiguous range of the
queries against its own replica of the dataset.

Every interpolated point is computed independently of the others (Sec. 3.1.1: one thread per
interpolated point, no communication between them), so m queries split into contiguous ranges
with the dataset replicated on every device need no exchange while they are computed. Each rank
creates its dataset copy from the host arrays into its own device memory (no peer loads, no
multicast), runs the library's single-GPU call on its range, and, when the caller wants all
results in one place, the per-rank slices are gathered back in the caller's order (the one
collective, after the compute).

``query_ranges`` is pure host logic; ``shard_interpolate`` takes the per-rank compute as a
function, so that the partition and gather can be exercised on CPU ranks with any compute.
"""
from __future__ import annotations

import numpy as np


def query_ranges(m: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [begin, end) ranges of m queries for `world` ranks: every query in exactly one
    range, in rank order, sizes differing by at most one (the first m % world ranks take one
    more)."""
    if m < 0 or world < 1:
        raise ValueError("m >= 0 and world >= 1 required")
    per, extra = divmod(m, world)
    out, b = [], 0
    for r in range(world):
        e = b + per + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


def shard_interpolate(compute, qx, qy, rank: int, world: int, gather: bool = True):
    """Runs `compute(qx_slice, qy_slice) -> dict of per-query arrays` (first axis = query) on
    this rank's contiguous range of the queries. Without `gather`, returns (begin, end, dict) of
    the rank's own slice. With `gather` and world > 1, every rank receives the full arrays in
    the caller's order through torch.distributed.all_gather (ranges padded to the longest;
    CPU tensors under gloo, CUDA tensors under NCCL) and gets (0, m, dict)."""
    m = len(qx)
    b, e = query_ranges(m, world)[rank]
    part = compute(qx[b:e], qy[b:e])
    if not gather or world == 1:
        return b, e, part
    import torch
    import torch.distributed as dist
    longest = max(hi - lo for lo, hi in query_ranges(m, world))
    full = {}
    for key in sorted(part):
        v = part[key]
        t = v if isinstance(v, torch.Tensor) else torch.as_tensor(np.ascontiguousarray(v))
        pad = torch.zeros((longest,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        pad[: t.shape[0]] = t
        bufs = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(bufs, pad)
        pieces = [bufs[r][: hi - lo] for r, (lo, hi) in enumerate(query_ranges(m, world))]
        cat = torch.cat(pieces, dim=0)
        full[key] = cat if isinstance(v, torch.Tensor) else cat.numpy()
    return 0, m, full


def interpolate_on_rank(ctx, ds, qx, qy, params, rank: int, world: int, gather: bool = False,
                        stream=None):
    """The library's AIDW (ctx.interpolate, this rank's GPU) on this rank's range of the
    queries; returns (begin, end, {"z": ...}), or the gathered full result with `gather`."""
    def compute(a, b):
        out, _, _ = ctx.interpolate(ds, a, b, params, stream=stream)
        return {"z": out}

    return shard_interpolate(compute, qx, qy, rank, world, gather=gather)

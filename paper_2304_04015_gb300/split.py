"""One single-source query split across ranks by target range.

Section 5.5 of the paper gives every target u to the machine with index
floor(u M / n) (M machines), which then holds every walk pair of u and
emits u's score.  Here a rank is one GPU: rank r computes the targets
[ceil(r n / N), ceil((r + 1) n / N)) (exactly the u with floor(u N / n) = r)
from its own full copy of the graph, through ``srk_single_source`` with that
target range.  The source side of the query (walks, shuffle, hit table) is
keyed by (seed, s) alone, so every rank recomputes it identically and nothing
is exchanged before the walks; the only collective is one all-gather of the
per-rank score slices at the end.

Only argument marshalling and the gather live here; every step of the query
runs in the library's kernels.
"""
from __future__ import annotations

from typing import Optional, Tuple

__all__ = ["owner_range", "owner_of", "gather_slices", "split_query"]


def owner_of(u: int, n: int, world: int) -> int:
    """The rank that owns target u: floor(u N / n) (Section 5.5)."""
    return (u * world) // n


def owner_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """[begin, end) of the targets whose owner is ``rank``: begin =
    ceil(rank n / N), so that owner_of(u) = rank exactly for u in it."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside [0, %d)" % (rank, world))
    return (rank * n + world - 1) // world, ((rank + 1) * n + world - 1) // world


def gather_slices(local, n: int, rank: int, world: int, group=None):
    """All-gather of the ranks' slices into one length-n vector.

    ``local`` holds this rank's slice (owner_range(n, rank, world) entries,
    any dtype, on the device the process group communicates from: CUDA for
    NCCL, CPU for gloo).  One ``all_gather`` of equal-size padded buffers; the
    result is the concatenation in rank order."""
    import torch
    import torch.distributed as dist
    b, e = owner_range(n, rank, world)
    if local.numel() != e - b:
        raise ValueError("slice of rank %d has %d entries, expected %d"
                         % (rank, local.numel(), e - b))
    if world == 1:
        return local.clone()
    width = max(owner_range(n, r, world)[1] - owner_range(n, r, world)[0] for r in range(world))
    pad = torch.zeros(width, dtype=local.dtype, device=local.device)
    pad[:e - b] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    out = []
    for r in range(world):
        rb, re = owner_range(n, r, world)
        out.append(parts[r][:re - rb])
    return torch.cat(out)


def split_query(g, s: int, c: float, eps: float, seed: int, rank: int, world: int,
                group=None, stream=None, counts: bool = False, **opts):
    """One query over all ranks: this rank walks its owned targets, then the
    slices are all-gathered.  Returns the full FP64 score vector (and the
    uint32 meet counts when ``counts``) on every rank, on the graph's device.
    ``opts`` are passed to ``srk_single_source`` (z_override, L_override, p,
    q, warmup_rule, literal_shuffle, stats)."""
    import torch
    from . import srk_graph_info, srk_single_source
    n, _ = srk_graph_info(g)
    b, e = owner_range(n, rank, world)
    dev = torch.device("cuda", torch.cuda.current_device())
    scores = torch.empty(n, dtype=torch.float64, device=dev)
    cnt: Optional[torch.Tensor] = torch.empty(n, dtype=torch.int32, device=dev) if counts else None
    srk_single_source(g, s, c, eps, seed, scores, cnt, target_range=(b, e), stream=stream,
                      **opts)
    full = gather_slices(scores[b:e], n, rank, world, group)
    if counts:
        return full, gather_slices(cnt[b:e], n, rank, world, group)
    return full

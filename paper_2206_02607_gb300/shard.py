"""Host-side sharding of independent latent-step instances over ranks.

Instances are independent (each has its own q, coefficient and sample set), so
a multi-GPU run needs no data-path collective: every rank steps a contiguous
range of instances.  The ranges are balanced by work, the number of integration
samples sum |M_i|, which is what the step's cost is proportional to.
"""
from __future__ import annotations

import numpy as np

__all__ = ["partition_by_work", "shard_of"]


def partition_by_work(sizes, world: int):
    """Split instances 0..n-1 into `world` contiguous ranges [lo, hi) whose total
    sizes are as equal as a prefix split allows (cut at the cumulative-work
    quantiles).  Every instance lands in exactly one range; ranges may be empty
    when world > n."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    n = sizes.size
    cum = np.concatenate([[0], np.cumsum(sizes)])
    total = cum[-1]
    cuts = [0]
    for k in range(1, world):
        target = total * k / world
        cut = int(np.searchsorted(cum, target, side="left"))
        cuts.append(min(max(cut, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def shard_of(s_off, rank: int, world: int):
    """(lo, hi, local offsets) of this rank's instances for a ragged batch given by
    its sample offsets s_off [n+1]."""
    s_off = np.asarray(s_off, dtype=np.int64)
    lo, hi = partition_by_work(np.diff(s_off), world)[rank]
    local = (s_off[lo:hi + 1] - s_off[lo]).astype(np.int32)
    return lo, hi, local

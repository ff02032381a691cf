"""Scatter/gather of one trace over ranks (Sec. II.C).

The paper runs ncount/N histories on each of N MPI ranks (or GPUs) and then
merges the detectors on the master rank. Here a history depends only on
(seed, experiment id, index), so the scatter is a split of the index range
and the gather is one sum-reduce of the FP64 detector (per pixel sum of
weights, sum of squared weights, histories, and the transmitted weight).

Plumbing only: the histories run in the library's kernels; this module
computes index ranges and hands the detector arrays to torch.distributed
(NCCL on GPUs, gloo on CPUs), the collective that performs the exchange.
"""
from __future__ import annotations

DETECTOR_KEYS = ("sum_w", "sum_w2", "count", "trans")


def rank_range(rank: int, world: int, n: int):
    """Share of rank `rank` when a fixed total of n histories is split over
    `world` ranks (strong scaling): contiguous, disjoint, covering [0, n);
    the first n % world ranks take one history more. Returns (first, count)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    base, extra = divmod(n, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def weak_range(rank: int, n_per_rank: int):
    """Share of rank `rank` when every rank traces n_per_rank histories of
    its own (weak scaling): [rank n, (rank + 1) n)."""
    if rank < 0 or n_per_rank < 0:
        raise ValueError("need rank >= 0 and n_per_rank >= 0")
    return rank * n_per_rank, n_per_rank


def experiment_partition(costs, world: int):
    """Split a batch of experiments over `world` ranks with no exchange:
    every experiment's detector stays on the rank that traces it (its
    histories are keyed by its own experiment id). Longest-processing-time
    assignment: experiments in decreasing cost (histories x per-history
    cost) go to the least-loaded rank, ties to the lowest rank, which keeps
    the largest load within 4/3 of the optimum. Returns one ascending list
    of experiment indices per rank."""
    if world < 1:
        raise ValueError("need world >= 1")
    costs = [float(c) for c in costs]
    if any(not c >= 0.0 for c in costs):
        raise ValueError("costs must be >= 0")
    order = sorted(range(len(costs)), key=lambda e: (-costs[e], e))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for e in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(e)
        load[r] += costs[e]
    return [sorted(p) for p in parts]


class _CudaArray:
    """__cuda_array_interface__ of a library-owned device array, so that
    torch can view it without a copy."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def detector_views(exp, n_pixels):
    """Zero-copy torch views of an experiment's device detector: sum_w,
    sum_w2 (float64 [n_pixels]), count (the uint64 counts read as int64;
    counts stay below 2^63) and trans (float64 [1]). The views alias the
    library's arrays and are valid until the experiment is destroyed."""
    import torch
    from . import sas_detector_device
    sw, sw2, cnt, tr = sas_detector_device(exp)
    dev = torch.device("cuda", torch.cuda.current_device())
    return {"sum_w": torch.as_tensor(_CudaArray(sw, n_pixels, "<f8"), device=dev),
            "sum_w2": torch.as_tensor(_CudaArray(sw2, n_pixels, "<f8"), device=dev),
            "count": torch.as_tensor(_CudaArray(cnt, n_pixels, "<i8"), device=dev),
            "trans": torch.as_tensor(_CudaArray(tr, 1, "<f8"), device=dev)}


def merge_detector(det, dst=None, group=None):
    """The gather: sum every rank's detector arrays (a dict with the keys of
    DETECTOR_KEYS: float64 sums and int64 counts) in place, onto every rank
    (dst None: all-reduce) or onto rank dst only (reduce; the other ranks'
    arrays are left undefined by the collective). One collective per array,
    FP64 sums: the merged tallies equal those of one process tracing the
    union of the ranges up to the order of the FP64 additions."""
    import torch.distributed as dist
    for k in DETECTOR_KEYS:
        t = det[k]
        if dst is None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        else:
            dist.reduce(t, dst=dst, op=dist.ReduceOp.SUM, group=group)
    return det

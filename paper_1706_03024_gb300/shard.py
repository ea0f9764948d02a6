"""Sharding of the light tracer over ranks (one process per GPU).

Photon paths are independent and keyed by (seed, medium id, path id), so the work partitions by
path-id range with no exchange on the data path: rank r traces ids [r * n, (r + 1) * n) of the same
seed (weak scaling, n paths per rank). The only cross-rank step is the final reduction of what a
user reads: tallies and films are normalised per launched path, so the job's tally is the
path-weighted mean of the ranks' tallies, and a job's step time is the slowest rank's.

These helpers run on any torch.distributed backend: NCCL with CUDA tensors on GPUs, gloo with CPU
tensors in the multi-process tests.
"""
from __future__ import annotations

import numpy as np


def path_range(n_per_rank: int, rank: int) -> tuple[int, int]:
    """(first path id, count) of `rank` when every rank traces n_per_rank paths."""
    if n_per_rank < 0 or rank < 0:
        raise ValueError("n_per_rank and rank must be non-negative")
    return rank * n_per_rank, n_per_rank


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def reduce_scalar(x: float, op: str = "sum", device=None) -> float:
    """Sum or max of a scalar over all ranks (x itself without an initialised process group)."""
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX)
    return float(t.item())


def combine_tallies(local: dict, n_local: int, keys=("face", "absorbed", "emitted", "film"),
                    device=None) -> dict:
    """The job's normalised tallies from each rank's (normalised over its own n_local paths):
    sum_r n_r t_r / sum_r n_r, for every key present (numpy arrays, fp64). Counters are summed."""
    dist = _dist()
    out = {}
    n_tot = reduce_scalar(n_local, "sum", device)
    for k in keys:
        v = local.get(k)
        if v is None:
            out[k] = None
            continue
        a = np.asarray(v, dtype=np.float64) * float(n_local)
        if dist is not None and dist.get_world_size() > 1:
            import torch
            t = torch.from_numpy(np.ascontiguousarray(a)).to(device if device is not None else "cpu")
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            a = t.cpu().numpy()
        out[k] = a / n_tot if n_tot > 0 else a
    if "counters" in local:
        out["counters"] = {name: int(reduce_scalar(val, "sum", device))
                           for name, val in local["counters"].items()}
    return out

"""Merge Peaks across processes (Sec. 3.4): in the slab form of the path
each rank finds the strict 26-neighbour maxima of its own output planes;
the exchange is one all-gather of those candidate lists, after which every
rank runs the same Merge Peaks (ttm_merge_peaks: value descending, index
ascending, greedy exclusion) and holds the same list as Find Peaks on the
whole tomogram. Host logic only: it runs over any torch.distributed
backend (gloo on CPU, NCCL between GPUs)."""
import numpy as np

from . import ttm


def gather_merge_peaks(idx, val, shape, P: int, min_dist: float, group=None):
    """All-gather this rank's candidates (tomogram linear indices and
    values) and merge them; returns (indices, values) of the P best."""
    import torch.distributed as dist
    mine = (np.ascontiguousarray(idx, dtype=np.int64), np.ascontiguousarray(val, dtype=np.float32))
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, mine, group=group)
    all_idx = np.concatenate([p[0] for p in parts]) if parts else np.zeros(0, np.int64)
    all_val = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0, np.float32)
    return ttm.ttm_merge_peaks(all_idx, all_val, shape, P, min_dist)

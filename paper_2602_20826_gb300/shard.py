"""Sharding one batch of DAGs over several GPUs (one process per GPU).

DAGs are independent problems -- their schedules and bounds share nothing -- so a batch
splits across ranks with no exchange on the data path: each rank loads and schedules its
own share with its own GPU, and the only communication is gathering the per-DAG results
(bound, status, and for a search the winning candidate: 12-16 bytes per DAG) afterwards.

The share of work of a DAG is about proportional to its node count times the number of
candidate schedules evaluated on it, so the DAGs are balanced greedily by that cost:
longest first, each to the rank with the least work so far (LPT).
"""
from __future__ import annotations

import heapq

import numpy as np


def partition(costs, n_ranks: int):
    """Greedy LPT split of DAGs with the given costs over n_ranks: a list of n_ranks
    arrays of DAG ids (ascending within a rank). Ties go to the lower rank, so the split is
    deterministic and identical on every rank."""
    costs = np.asarray(costs, np.int64)
    order = np.lexsort((np.arange(len(costs)), -costs))  # descending cost, then id
    heap = [(0, r) for r in range(n_ranks)]
    parts = [[] for _ in range(n_ranks)]
    for d in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(d))
        heapq.heappush(heap, (load + int(costs[d]), r))
    return [np.asarray(sorted(p), np.int64) for p in parts]


def gather(parts, per_rank_values, n_dags: int, fill=-1):
    """Inverse of partition: per_rank_values[r][i] is the value of DAG parts[r][i]; returns
    one array over all n_dags DAGs in the original order."""
    first = next((np.asarray(v) for v in per_rank_values if len(v)), np.zeros(0, np.int64))
    out = np.full(n_dags, fill, dtype=first.dtype if first.size else np.int64)
    for ids, vals in zip(parts, per_rank_values):
        out[np.asarray(ids, np.int64)] = np.asarray(vals)
    return out


def gather_over_ranks(dist, parts, local_values, n_dags: int, fill=-1):
    """gather() across a torch.distributed process group (any backend): every rank passes
    its own values, rank 0 receives the whole batch's array (other ranks get None). Host
    objects only -- after the timed region, off the data path."""
    world = dist.get_world_size()
    got = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(np.asarray(local_values), got, dst=0)
    if dist.get_rank() != 0:
        return None
    return gather(parts, got, n_dags, fill)

"""Splitting one batch of tracking environments over several GPUs.

The environments of a batch are independent (Sec. III-A: each episode is its
own team of agents and targets), so a batch shards by contiguous env ranges
with no exchange on the data path.  Every random draw of the step is keyed by
the global id of the env, agent, target or filter it belongs to, so a shard
that knows where its first env, agent, target and filter sit in the whole
batch reproduces exactly the draws, and hence the states, that the unsplit
batch would produce for those envs.  Only the per-step summary metrics cross
ranks, as a sum.

Pure host code: it runs the same with or without a GPU.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np


def _counts(params) -> Tuple[np.ndarray, np.ndarray]:
    E = int(params.n_envs)
    a = params.agents_per_env
    t = params.targets_per_env
    a = np.full(E, params.max_agents, np.int64) if a is None else np.asarray(a, np.int64)
    t = np.full(E, params.max_targets, np.int64) if t is None else np.asarray(t, np.int64)
    if a.shape != (E,) or t.shape != (E,):
        raise ValueError("agents_per_env / targets_per_env must have n_envs entries")
    return a, t


def env_cost(params) -> np.ndarray:
    """Relative work of each env in one step: the particle filters dominate
    (A_e * T_e filters of P particles), the agents' policy rows and kinematics
    add a term per agent."""
    a, t = _counts(params)
    return a * t * int(params.n_particles) + a * 64


def shard_bounds(params, world_size: int) -> List[Tuple[int, int]]:
    """Contiguous env ranges [e0, e1), one per rank, balanced by
    :func:`env_cost`.  Uniform fleets split into equal counts (the first
    ``n_envs % world_size`` ranks take one env more)."""
    E = int(params.n_envs)
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    if E < world_size:
        raise ValueError(f"cannot split {E} envs over {world_size} ranks")
    cost = env_cost(params)
    if np.all(cost == cost[0]):
        q, r = divmod(E, world_size)
        sizes = [q + (1 if k < r else 0) for k in range(world_size)]
        edges = np.concatenate([[0], np.cumsum(sizes)])
    else:
        csum = np.concatenate([[0], np.cumsum(cost)])
        total = csum[-1]
        edges = [0]
        for k in range(1, world_size):
            cut = int(np.searchsorted(csum, total * k / world_size, side="left"))
            # keep at least one env per rank on both sides of the cut
            cut = max(cut, edges[-1] + 1)
            cut = min(cut, E - (world_size - k))
            edges.append(cut)
        edges.append(E)
    return [(int(edges[k]), int(edges[k + 1])) for k in range(world_size)]


def shard_params(params, rank: int, world_size: int):
    """The parameters of rank ``rank``'s shard: its env count, its slice of a
    ragged fleet and the global ids of its first env, agent, target and
    filter (added to any offsets ``params`` already carries)."""
    a, t = _counts(params)
    e0, e1 = shard_bounds(params, world_size)[rank]
    ragged = params.agents_per_env is not None or params.targets_per_env is not None
    kw = dict(
        n_envs=e1 - e0,
        id_env0=int(getattr(params, "id_env0", 0)) + e0,
        id_agent0=int(getattr(params, "id_agent0", 0)) + int(a[:e0].sum()),
        id_target0=int(getattr(params, "id_target0", 0)) + int(t[:e0].sum()),
        id_filter0=int(getattr(params, "id_filter0", 0)) + int((a[:e0] * t[:e0]).sum()),
    )
    if ragged:
        kw["agents_per_env"] = a[e0:e1].astype(np.int32)
        kw["targets_per_env"] = t[e0:e1].astype(np.int32)
    return dataclasses.replace(params, **kw)


def reduce_sums(values: Sequence[float], group=None) -> np.ndarray:
    """Element-wise sum of per-rank partial sums (float64) over the default
    process group; the identity when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist

    buf = torch.tensor(np.asarray(values, np.float64))
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        if dist.get_backend(group) == "nccl":
            buf = buf.cuda()
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf.cpu().numpy()

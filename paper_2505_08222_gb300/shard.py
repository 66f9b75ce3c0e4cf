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
import math
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


def _filters(params, a, t) -> np.ndarray:
    """Filters of each env: A_e T_e per-agent filters, or T_e shared ones."""
    return t.copy() if getattr(params, "shared_filter", 0) else a * t


def env_cost(params) -> np.ndarray:
    """Relative work of each env in one step: the particle filters dominate
    (A_e T_e filters of P particles, T_e when shared), the agents' policy
    rows and kinematics add a term per agent."""
    a, t = _counts(params)
    return _filters(params, a, t) * int(params.n_particles) + a * 64


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
    ragged fleet and the global ids of its first env, agent, target, filter
    and (agent, target) pair (added to any offsets ``params`` already
    carries)."""
    a, t = _counts(params)
    e0, e1 = shard_bounds(params, world_size)[rank]
    ragged = params.agents_per_env is not None or params.targets_per_env is not None
    kw = dict(
        n_envs=e1 - e0,
        id_env0=int(getattr(params, "id_env0", 0)) + e0,
        id_agent0=int(getattr(params, "id_agent0", 0)) + int(a[:e0].sum()),
        id_target0=int(getattr(params, "id_target0", 0)) + int(t[:e0].sum()),
        id_filter0=int(getattr(params, "id_filter0", 0)) + int(_filters(params, a[:e0], t[:e0]).sum()),
        id_pair0=int(getattr(params, "id_pair0", 0)) + int((a[:e0] * t[:e0]).sum()),
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


def lr_schedule(lr: float, step: int, steps: int, cosine: bool = True) -> float:
    """Learning rate of step ``step`` of ``steps``: cosine decay from ``lr``
    (held in FP32, as the training entry point receives it) to 0 at the last
    step, or constant."""
    lr32 = float(np.float32(lr))
    if not cosine:
        return lr32
    frac = step / (steps - 1) if steps > 1 else 0.0
    return lr32 * 0.5 * (1.0 + math.cos(math.pi * frac))


def rank_seed(seed: int, rank: int) -> int:
    """Batch-sampling seed of one rank: rank 0 keeps ``seed`` (a one-rank run
    draws what the single-device trainer draws), the others are spread by the
    64-bit golden-ratio increment."""
    return (int(seed) + 0x9E3779B97F4A7C15 * int(rank)) % (1 << 64)


def _weighted_mean_(buf, weight: float, weight_sum: float, group):
    """buf <- sum_r w_r buf_r / sum_r w_r over the ranks, in place (NCCL
    reduces on the device, gloo on the host)."""
    import torch.distributed as dist

    on_dev = dist.get_backend(group) == "nccl"
    work = buf if buf.is_cuda == on_dev else buf.to("cuda" if on_dev else "cpu")
    work.mul_(weight / weight_sum)
    dist.all_reduce(work, op=dist.ReduceOp.SUM, group=group)
    if work is not buf:
        buf.copy_(work)
    return buf


def dp_train(backend, X, Y, steps: int, batch: int, lr: float = 1e-3, cosine: bool = True, seed: int = 0,
             beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, huber: float = 0.0, group=None) -> dict:
    """Data-parallel training of the learned estimator: every rank holds its
    own recorded rows (X, Y) and an identical copy of the weights.  Each step
    a rank computes the loss gradient of its share of the global batch on its
    own device, the ranks' gradients are averaged weighted by their rows (the
    loss is a mean over rows, so this is the gradient of the union batch),
    and every rank applies the same Adam update, so the copies stay equal.

    ``batch`` is the global batch; rank r takes ``batch // W`` rows (the first
    ``batch % W`` ranks one more), drawn from its own rows by the
    counter-based stream under :func:`rank_seed`; ``batch=None`` uses every
    row of every rank each step (full-batch gradient descent).  With one rank
    this is the single-device trainer, step for step.

    ``backend`` provides ``est_loss_grad(X, Y, huber=, batch=, seed=,
    step=) -> (loss, grad)`` and ``est_adam_step(grad, lr, beta1, beta2,
    eps)`` (the environment handle does).  Returns the row-weighted mean
    loss of the first and last steps."""
    import torch.distributed as dist

    if steps < 1:
        raise ValueError("steps must be >= 1")
    dist_on = dist.is_available() and dist.is_initialized()
    rank = dist.get_rank(group) if dist_on else 0
    world = dist.get_world_size(group) if dist_on else 1
    n_local = int(X.shape[0])
    if batch is None:
        b_local = n_local
    else:
        q, r = divmod(int(batch), world)
        b_local = q + (1 if rank < r else 0)
        if b_local < 1:
            raise ValueError(f"global batch {batch} leaves rank {rank} of {world} no rows")
    b_total = b_local if world == 1 else int(reduce_sums([b_local], group)[0])
    s_rank = rank_seed(seed, rank)
    first = last = None
    for s in range(steps):
        loss, grad = backend.est_loss_grad(X, Y, huber=huber, batch=b_local, seed=s_rank, step=s)
        mean_loss = float(loss)
        if world > 1:
            _weighted_mean_(grad, b_local, b_total, group)
            mean_loss = float(reduce_sums([loss * b_local / b_total], group)[0])
        backend.est_adam_step(grad, lr_schedule(lr, s, steps, cosine), beta1, beta2, eps)
        if s == 0:
            first = mean_loss
        last = mean_loss
    return {"loss_first": first, "loss_last": last, "steps": steps, "world_size": world, "rows_per_step": b_local}

"""Env-sharded batches: two gloo ranks on the CPU, each running the FP64
oracle on its shard with global id offsets, reproduce the unsplit batch
exactly (per-filter errors and per-env rewards bit for bit), and the summed
metrics agree with the single-process sums."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from synth import preset
from paper_2505_08222_gb300 import shard

STEPS = 6
SEED = 17


def _params(kind):
    if kind == "uniform":
        return preset("fleet5", n_envs=5).replace(n_particles=64, d_model=0)
    if kind == "shared":  # one filter per (env, target), ragged counts
        return preset("ragged", n_envs=7, seed=4).replace(n_particles=32, d_model=0, shared_filter=1)
    return preset("ragged", n_envs=7, seed=3).replace(n_particles=32, d_model=0)


def _run(p, steps=STEPS):
    """Per-step per-filter error, per-env reward and crash flags of ``p``."""
    o = oracle.OracleEnv(p, SEED)
    o.reset(0)
    errs, rews = [], []
    for _ in range(steps):
        out = o.step(o.random_actions(o.step_count))
        errs.append(out["err"].copy())
        rews.append(out["reward"].copy())
    return np.stack(errs), np.stack(rews)


def _sums(err, rew):
    return [float((err ** 2).sum()), float(err.size), float(rew.sum())]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, kind, outdir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sp = shard.shard_params(_params(kind), rank, world)
        err, rew = _run(sp)
        tot = shard.reduce_sums(_sums(err, rew))
        np.savez(os.path.join(outdir, f"r{rank}.npz"), err=err, rew=rew, tot=tot)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["uniform", "ragged", "shared"])
def test_two_rank_shards_reproduce_whole_batch(kind):
    p = _params(kind)
    err_all, rew_all = _run(p)
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(2, _free_port(), kind, d), nprocs=2, join=True, start_method="spawn")
        parts = [np.load(os.path.join(d, f"r{k}.npz")) for k in range(2)]
    np.testing.assert_array_equal(np.concatenate([q["err"] for q in parts], axis=1), err_all)
    np.testing.assert_array_equal(np.concatenate([q["rew"] for q in parts], axis=1), rew_all)
    want = np.array(_sums(err_all, rew_all))
    for q in parts:  # every rank holds the reduced sums
        np.testing.assert_allclose(q["tot"], want, rtol=1e-12)


def test_shard_bounds_cover_and_balance():
    p = preset("ragged", n_envs=1000, seed=1)
    for world in (1, 2, 3, 8):
        b = shard.shard_bounds(p, world)
        assert b[0][0] == 0 and b[-1][1] == p.n_envs
        assert all(b[k][1] == b[k + 1][0] and b[k][1] > b[k][0] for k in range(world - 1))
        cost = shard.env_cost(p)
        loads = np.array([cost[e0:e1].sum() for e0, e1 in b])
        assert loads.max() <= loads.mean() + cost.max()
    u = preset("fleet5", n_envs=4099)
    assert [e1 - e0 for e0, e1 in shard.shard_bounds(u, 4)] == [1025, 1025, 1025, 1024]
    with pytest.raises(ValueError):
        shard.shard_bounds(preset("fleet5", n_envs=2), 3)


def test_shard_ids_are_prefix_sums():
    p = preset("ragged", n_envs=50, seed=2)
    a, t = p.counts()
    for rank in range(4):
        sp = shard.shard_params(p, rank, 4)
        e0 = sp.id_env0
        assert sp.id_agent0 == a[:e0].sum() and sp.id_target0 == t[:e0].sum()
        assert sp.id_filter0 == (a[:e0].astype(np.int64) * t[:e0]).sum()
        assert sp.id_pair0 == (a[:e0].astype(np.int64) * t[:e0]).sum()
        np.testing.assert_array_equal(sp.agents_per_env, a[e0:e0 + sp.n_envs])
        # shared filters: one per target (the cost, hence the bounds, change)
        ss = shard.shard_params(p.replace(shared_filter=1), rank, 4)
        s0 = ss.id_env0
        assert ss.id_filter0 == t[:s0].sum() and ss.id_pair0 == (a[:s0].astype(np.int64) * t[:s0]).sum()

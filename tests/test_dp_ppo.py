"""Data-parallel PPO gradients (the Trainer's ``dp_average``) on two gloo
ranks (CPU).  Each rank holds the FP64 oracle's gradient of the mean loss
over its own samples (unequal counts); after the row-weighted all-reduce both
hold the gradient of the mean loss over the union, which the oracle computes
in one process."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import synth

D, L, H, NACT, NS = 16, 2, 2, 5, 6
SPLIT, N = 5, 13  # rank 0 holds samples [0, 5), rank 1 [5, 13)


def _data():
    rng = np.random.default_rng(71)
    n_ent = rng.integers(0, NS + 1, N).astype(np.int32)
    tok = synth.random_tokens(N, NS, n_ent, seed=72).astype(np.float64)
    h = 0.5 * rng.standard_normal((N, D))
    act = rng.integers(0, NACT, N).astype(np.int32)
    logp_old = -np.log(NACT) + 0.3 * rng.standard_normal(N)
    adv = rng.standard_normal(N)
    ret = rng.standard_normal(N)
    return tok, n_ent, h, act, logp_old, adv, ret


def _grad(kind, lo, hi):
    tok, ne, h, act, lp, adv, ret = _data()
    no = NACT if kind == oracle.ACTOR else 1
    prm = synth.policy_params(synth.PolicyDims(D, L, H, no), seed=73 + kind)
    s = slice(lo, hi)
    _, g, _ = oracle.tfm_loss_grad(prm, D, L, H, no, kind, tok[s], ne[s], h[s], act[s], lp[s], adv[s], 0.2, 0.01,
                                   ret[s])
    return g


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import torch.distributed as dist

    from paper_2505_08222_gb300 import ppo

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = (0, SPLIT) if rank == 0 else (SPLIT, N)
        out = {}
        for kind in (oracle.ACTOR, oracle.CRITIC):
            g = torch.from_numpy(_grad(kind, lo, hi))
            total = ppo.dp_average(g, hi - lo)
            out[f"g{kind}"] = g.numpy()
            out["total"] = total
        np.savez(os.path.join(outdir, f"r{rank}.npz"), **out)
    finally:
        dist.destroy_process_group()


def test_two_ranks_average_to_the_union_gradient():
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(2, _free_port(), d), nprocs=2, join=True, start_method="spawn")
        r = [dict(np.load(os.path.join(d, f"r{k}.npz"))) for k in range(2)]
    for kind in (oracle.ACTOR, oracle.CRITIC):
        full = _grad(kind, 0, N)
        assert np.array_equal(r[0][f"g{kind}"], r[1][f"g{kind}"])
        np.testing.assert_allclose(r[0][f"g{kind}"], full, rtol=1e-10, atol=1e-14)
        # the two halves alone differ from the union: the average is not trivially one of them
        assert np.abs(_grad(kind, 0, SPLIT) - full).max() > 1e-6
    assert int(r[0]["total"]) == N and int(r[1]["total"]) == N


def test_one_process_is_a_no_op():
    from paper_2505_08222_gb300 import ppo

    g = torch.arange(5, dtype=torch.float64)
    assert ppo.dp_average(g, 7) == 7
    assert torch.equal(g, torch.arange(5, dtype=torch.float64))


def _empty_worker(rank, world, port, outdir):
    import torch.distributed as dist

    from paper_2505_08222_gb300 import ppo

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank 0's slice is empty (zeroed gradient, n_local = 0), rank 1 holds every sample
        g = torch.zeros(_grad(oracle.ACTOR, 0, N).size, dtype=torch.float64) if rank == 0 else torch.from_numpy(_grad(oracle.ACTOR, 0, N))
        total = ppo.dp_average(g, 0 if rank == 0 else N)
        # then a minibatch empty on both ranks: no average, the gradient is left alone
        h = torch.full((4,), float(rank + 1), dtype=torch.float64)
        none = ppo.dp_average(h, 0)
        np.savez(os.path.join(outdir, f"r{rank}.npz"), g=g.numpy(), total=total, h=h.numpy(), none=none)
    finally:
        dist.destroy_process_group()


def test_a_rank_with_an_empty_slice_still_joins_the_average():
    """Ragged shards can leave one rank's last minibatch empty; the trainer
    then zeroes that rank's gradient and calls dp_average with n_local = 0,
    so both ranks enter the same all-reduces and end with the other rank's
    gradient."""
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_empty_worker, args=(2, _free_port(), d), nprocs=2, join=True, start_method="spawn")
        r = [dict(np.load(os.path.join(d, f"r{k}.npz"))) for k in range(2)]
    full = _grad(oracle.ACTOR, 0, N)
    for k in range(2):
        np.testing.assert_allclose(r[k]["g"], full, rtol=1e-12, atol=1e-15)
        assert int(r[k]["total"]) == N
        assert int(r[k]["none"]) == 0
        assert np.all(r[k]["h"] == k + 1)

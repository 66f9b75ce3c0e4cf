"""Data-parallel training of the learned estimator on two gloo ranks (CPU).

The backend is the FP64 oracle (its loss gradient and Adam step), so the
check is of the host logic alone: with full batches the row-weighted average
of the ranks' gradients is the gradient of all rows, so two ranks holding
unequal halves of the rows follow the one-process run to rounding; with
sampled batches both ranks keep identical weights step after step."""
import math
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import synth
from paper_2505_08222_gb300 import shard

N_ROWS = 48
SPLIT = 22  # rank 0 holds rows [0, 22), rank 1 rows [22, 48)
STEPS = 3


class OracleEstimator:
    """The two calls data-parallel training makes, on the oracle's FP64
    network; batches are drawn with numpy keyed by (seed, step)."""

    def __init__(self, params):
        self.theta = np.asarray(params, np.float64).copy()
        self.m = np.zeros_like(self.theta)
        self.v = np.zeros_like(self.theta)
        self.t = 0

    def est_loss_grad(self, X, Y, huber=0.0, batch=None, seed=0, step=0):
        n = len(X)
        rows = np.arange(n) if batch in (None, n) else np.random.default_rng([seed, step]).integers(0, n, batch)
        loss, g = oracle.mlp_loss_grad(self.theta, X[rows], Y[rows], huber=huber)
        return loss, torch.from_numpy(g)

    def est_adam_step(self, grad, lr, beta1, beta2, eps):
        self.t += 1
        self.theta, self.m, self.v = oracle.adam(self.theta, self.m, self.v, grad.numpy(), self.t, lr=lr,
                                                 beta1=beta1, beta2=beta2, eps=eps)


def _data():
    X = synth.random_features(N_ROWS, seed=21).astype(np.float64)
    Y = np.random.default_rng(22).standard_normal((N_ROWS, 2)) * 0.4
    return X, Y


def _init():
    return synth.mlp_params(seed=23, bias_scale=0.1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, outdir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, Y = _data()
        lo, hi = (0, SPLIT) if rank == 0 else (SPLIT, N_ROWS)
        be = OracleEstimator(_init())
        batch = None if mode == "full" else 16
        st = shard.dp_train(be, X[lo:hi], Y[lo:hi], steps=STEPS, batch=batch, lr=1e-3, seed=5, huber=0.5)
        np.savez(os.path.join(outdir, f"r{rank}.npz"), theta=be.theta, first=st["loss_first"],
                 last=st["loss_last"], rows=st["rows_per_step"])
    finally:
        dist.destroy_process_group()


def _two_ranks(mode):
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(2, _free_port(), mode, d), nprocs=2, join=True, start_method="spawn")
        return [dict(np.load(os.path.join(d, f"r{r}.npz"))) for r in range(2)]


def test_two_ranks_full_batch_follow_single_process():
    r0, r1 = _two_ranks("full")
    X, Y = _data()
    be = OracleEstimator(_init())
    st = shard.dp_train(be, X, Y, steps=STEPS, batch=None, lr=1e-3, seed=5, huber=0.5)
    assert np.array_equal(r0["theta"], r1["theta"])
    np.testing.assert_allclose(r0["theta"], be.theta, rtol=1e-9, atol=1e-12)
    # the weights moved: the comparison is not of the initial weights
    assert np.abs(be.theta - _init()).max() > 0.5e-3
    assert float(r0["first"]) == pytest.approx(st["loss_first"], rel=1e-12)
    assert float(r1["last"]) == pytest.approx(st["loss_last"], rel=1e-12)
    assert int(r0["rows"]) == SPLIT and int(r1["rows"]) == N_ROWS - SPLIT


def test_two_ranks_sampled_batches_stay_identical():
    r0, r1 = _two_ranks("sampled")
    assert np.array_equal(r0["theta"], r1["theta"])
    assert int(r0["rows"]) == 8 and int(r1["rows"]) == 8
    assert float(r0["first"]) == float(r1["first"])


def test_single_process_is_a_plain_adam_loop():
    """Without a process group, dp_train is the loop est_loss_grad +
    est_adam_step with the cosine schedule and rank 0's seed."""
    X, Y = _data()
    a, b = OracleEstimator(_init()), OracleEstimator(_init())
    shard.dp_train(a, X, Y, steps=4, batch=10, lr=2e-3, seed=9, huber=0.0)
    for s in range(4):
        _, g = b.est_loss_grad(X, Y, batch=10, seed=9, step=s)
        b.est_adam_step(g, shard.lr_schedule(2e-3, s, 4), 0.9, 0.999, 1e-8)
    assert np.array_equal(a.theta, b.theta)


def test_lr_schedule_and_rank_seeds():
    lr32 = float(np.float32(1e-3))
    assert shard.lr_schedule(1e-3, 0, 5) == lr32
    assert shard.lr_schedule(1e-3, 4, 5) == pytest.approx(0.0, abs=1e-20)
    assert shard.lr_schedule(1e-3, 2, 5) == pytest.approx(lr32 * 0.5 * (1 + math.cos(math.pi / 2)), rel=1e-15)
    assert shard.lr_schedule(1e-3, 3, 5, cosine=False) == lr32
    assert shard.lr_schedule(1e-3, 0, 1) == lr32
    assert shard.rank_seed(7, 0) == 7
    seeds = {shard.rank_seed(7, r) for r in range(64)}
    assert len(seeds) == 64 and all(0 <= s < 2 ** 64 for s in seeds)
    with pytest.raises(ValueError):
        shard.dp_train(OracleEstimator(_init()), *_data(), steps=0, batch=4)

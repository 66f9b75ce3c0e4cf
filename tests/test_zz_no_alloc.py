"""tracker_update_noalloc: the allocation-free tracker update, for callers that
cannot allocate device memory (real-time threads that forbid allocator
calls, simulators that own every buffer and the GPU's memory budget, plug-ins
whose process gave all device memory to another framework's pool).  Called
through the C ABI and checked against env_step's own tracker output on two
calls in a row, and against the FP64 oracle's tracker from an injected state.

This file is collected last on purpose: the entry point shares one static
device array across calls, and it must work both in a fresh process and after
every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from synth import preset

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_08222_gb300 as ut  # noqa: E402
from paper_2505_08222_gb300 import _abi, make_config, shard  # noqa: E402
from gpu_util import oracle_state_f32, rel_close  # noqa: E402


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _call(cfg, seed, g, pos, parts, est, stream=None):
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream if stream is None else stream)
    return ut.lib.tracker_update_noalloc(ctypes.byref(cfg), ctypes.c_uint64(seed), g,
                                         _ptr(pos["ax"]), _ptr(pos["ay"]), _ptr(pos["tx"]), _ptr(pos["ty"]),
                                         _ptr(pos["tz"]), _ptr(parts["px"]), _ptr(parts["py"]), _ptr(parts["pvx"]),
                                         _ptr(parts["pvy"]), _ptr(est["estx"]), _ptr(est["esty"]), _ptr(est["err"]),
                                         st)


@pytest.mark.parametrize("P,rank", [(512, 0), (1000, 0), (512, 1)])
def test_noalloc_tracker_matches_env_step_twice(P, rank):
    """P = 512 takes the float4 particle path, P = 1000 the scalar one; rank 1
    of a two-way split carries nonzero global ids, which every random draw
    of the call adds to its local ids, as env_step does."""
    full = preset("fleet5", n_envs=96).replace(n_particles=P, d_model=0, comm_drop=0.2, target_depth_max=30.0)
    p = shard.shard_params(full, rank, 2)
    if rank:
        assert p.id_agent0 > 0 and p.id_filter0 > 0
    env = ut.Env(p)
    seed = 77
    env.reset(seed)
    cfg, keep = make_config(p)
    st = env.state()
    # the caller's own particle buffers start from the handle's reset state
    mine = {k: st[k].clone() for k in ("px", "py", "pvx", "pvy")}
    F = env.F
    est = {k: torch.empty(F, device="cuda") for k in ("estx", "esty", "err")}
    for call in range(2):
        g = env.state()["step"] + 1
        out = env.step()  # the existing entry point: move, ping, communicate, filter
        post = env.state()
        rc = _call(cfg, seed, g, post, mine, est)
        assert rc == 0, _abi.STATUS.get(rc)
        torch.cuda.synchronize()
        for k in ("px", "py", "pvx", "pvy"):
            a, b = mine[k].cpu().numpy(), post[k].cpu().numpy()
            floor = 100.0 if k in ("px", "py") else 1.0
            assert np.all(np.abs(a - b) <= 1e-5 * np.maximum(np.abs(b), floor)), (call, k)
        for k in ("estx", "esty", "err"):
            a, b = est[k].cpu().numpy(), out[k].cpu().numpy()
            assert np.all(np.abs(a - b) < 5e-3), (call, k)
    env.close()


@pytest.mark.parametrize("P,rank", [(512, 0), (1000, 1)])
def test_noalloc_tracker_matches_the_oracle(P, rank):
    """From an injected state: the oracle steps (move, ping, communicate,
    filter) in FP64; the entry point gets the oracle's moved positions and
    the same pre-step particles (FP32) at the same global step.  Estimates
    and errors agree within the filter step's tolerance (5 mm).  Resampled
    particles agree within 1e-5 relative except where a systematic-resampling
    threshold lies within the FP32 weights' rounding of a CDF step, so that
    the two sides pick neighbouring particles for that output: with
    P = 1000 thresholds per filter and weight errors ~1e-5 relative that
    happens in a few per cent of filters, to one or two of their outputs;
    more than 99.5 % of all resampled particles must agree."""
    full = preset("fleet5", n_envs=64).replace(n_particles=P, d_model=0, comm_drop=0.2, target_depth_max=30.0)
    p = shard.shard_params(full, rank, 2)
    seed = 5
    o = oracle.OracleEnv(p, seed)
    o.reset(0)
    rng = np.random.default_rng(3)
    for _ in range(2):  # a state some steps into the episode
        o.step(rng.integers(0, p.n_actions, o.NA).astype(np.int32))
    st32 = oracle_state_f32(o)
    o.set_arrays(**{k: v.astype(np.float64) if v.dtype == np.float32 else v for k, v in st32.items()})
    g = o.step_count + 1
    pre = {k: torch.from_numpy(st32[k].copy()).cuda() for k in ("px", "py", "pvx", "pvy")}
    ref = o.step(rng.integers(0, p.n_actions, o.NA).astype(np.int32), want=("meas_n",))
    pos = {k: torch.from_numpy(o.arr[k].astype(np.float32)).cuda() for k in ("ax", "ay", "tx", "ty", "tz")}
    est = {k: torch.empty(o.F, device="cuda") for k in ("estx", "esty", "err")}
    cfg, keep = make_config(p)
    for call in range(2):  # the same inputs twice: the shared scratch starts each call afresh
        parts = {k: v.clone() for k, v in pre.items()}
        rc = _call(cfg, seed, g, pos, parts, est)
        assert rc == 0, _abi.STATUS.get(rc)
        torch.cuda.synchronize()
        assert np.all(ref["meas_n"] > 0)  # every filter heard its target: each one resampled
        for k in ("estx", "esty"):
            assert np.all(np.abs(est[k].cpu().numpy() - o.arr[k]) < 5e-3), (call, k)
        assert np.all(np.abs(est["err"].cpu().numpy() - ref["err"]) < 5e-3), call
        same = np.ones(o.F * P, bool)
        for k in ("px", "py", "pvx", "pvy"):
            floor = 100.0 if k in ("px", "py") else 1.0
            same &= rel_close(parts[k].cpu().numpy(), o.arr[k], 1e-5, floor)
        print(f"P={P} rank {rank}: {same.mean():.5f} of resampled particles equal to the oracle's; "
              f"{same.reshape(o.F, P).all(1).mean():.3f} of filters entirely")
        assert same.mean() > 0.995, (call, same.mean())


def test_noalloc_rejects_sizes_beyond_its_static_limit():
    p = preset("large", n_envs=1024).replace(d_model=0)  # 65536 filters > 32768
    cfg, keep = make_config(p)
    dummy = torch.zeros(16, device="cuda")
    args = [_ptr(dummy)] * 12
    rc = ut.lib.tracker_update_noalloc(ctypes.byref(cfg), ctypes.c_uint64(1), 1, *args, None)
    assert rc == 1
    ragged = preset("ragged", n_envs=8).replace(d_model=0)
    cfg2, keep2 = make_config(ragged)
    assert ut.lib.tracker_update_noalloc(ctypes.byref(cfg2), ctypes.c_uint64(1), 1, *args, None) == 1

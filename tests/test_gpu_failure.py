"""Failure detection without a GPU fault.

* Bounded device waits: the test hook env_test_wait_timeout makes the
  tensor-core kernels (transformer agent, learned estimator) wait on a
  barrier that nothing signals, give up after a bounded number of polls and
  take the timed-out exit.  The next synchronising call reports
  UT_ERR_TIMEOUT; once the hook is off and the status word cleared, the same
  handle runs on and gives the same results as a fresh handle.
* Allocation failures: a caller allocator that returns NULL on its n-th call,
  for every n a handle's creation (and its policy / estimator buffers) goes
  through: the call returns UT_ERR_NOMEM and every buffer it had obtained is
  handed back (nothing leaks).
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from synth import preset

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_08222_gb300 as ut  # noqa: E402
from paper_2505_08222_gb300 import _abi, make_config  # noqa: E402

POLLS = 2000


def _policy_env(seed=3):
    p = preset("fleet5", n_envs=8).replace(n_particles=256)
    env = ut.Env(p)
    env.set_policy(synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, p.n_actions), seed=seed))
    return env, p


def _state(env):
    torch.cuda.synchronize()
    st = env.state()
    return {k: st[k].cpu().numpy().copy() for k in ("ax", "ay", "apsi", "px", "py", "estx")}


def test_policy_wait_that_runs_out_reports_timeout_and_the_handle_recovers():
    env, p = _policy_env()
    env.reset(5)
    env.step()
    assert env.metrics()["device_status"] == 0
    env.test_wait_timeout(POLLS)
    env.step()
    with pytest.raises(ut.UtError, match="UT_ERR_TIMEOUT"):
        env.metrics()
    # a graph rollout with the hook on reports it too
    with pytest.raises(ut.UtError, match="UT_ERR_TIMEOUT"):
        env.rollout(3)
    # hook off, status cleared: the same handle matches a fresh one bit for bit
    env.test_wait_timeout(0)
    env.metrics_reset()
    twin, _ = _policy_env()
    for e in (env, twin):
        e.reset(11)
        for _ in range(3):
            e.step()
    a, b = _state(env), _state(twin)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    assert env.metrics()["device_status"] == 0
    stats = env.rollout(4)
    assert stats["device_status"] == 0 and stats["steps"] == 4
    env.close()
    twin.close()


def test_estimator_wait_that_runs_out_reports_timeout_and_the_handle_recovers():
    p = preset("fleet5", n_envs=8).replace(n_particles=256, d_model=0)
    env = ut.Env(p, ring=True)
    env.est_set_weights(synth.mlp_params(seed=7, bias_scale=0.1))
    env.est_set_mode(2)
    env.reset(5)
    env.step()
    assert env.metrics()["device_status"] == 0
    env.test_wait_timeout(POLLS)
    before = env.state()["estx"].cpu().numpy().copy()
    env.step()
    with pytest.raises(ut.UtError, match="UT_ERR_TIMEOUT"):
        env.metrics()
    # the timed-out launch wrote no estimate
    np.testing.assert_array_equal(env.state()["estx"].cpu().numpy(), before)
    env.test_wait_timeout(0)
    env.metrics_reset()
    env.step()
    assert env.metrics()["device_status"] == 0
    assert not np.array_equal(env.state()["estx"].cpu().numpy(), before)
    env.close()


class _FailingAllocator:
    """Torch's caching allocator behind the ABI's allocator callback, with
    NULL on call number `fail_at` (1-based; 0 never fails) and a count of the
    blocks currently handed out."""

    def __init__(self, fail_at=0):
        self.fail_at, self.calls, self.live = fail_at, 0, set()
        dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
            self.live.add(int(ptr))
            return ptr

        def _free(ptr, stream, ctx):
            self.live.discard(int(ptr))
            torch.cuda.caching_allocator_delete(int(ptr))

        self._a = _abi.ALLOC_FN(_alloc)
        self._f = _abi.FREE_FN(_free)
        self.struct = _abi.Allocator(self._a, self._f, None)


def _create(cfg, alloc):
    h = ctypes.c_void_p()
    rc = ut.lib.env_create(ctypes.byref(cfg), ctypes.byref(alloc.struct), None, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("name,kw", [("fleet5", {"n_particles": 64}), ("ragged", {"n_particles": 32}),
                                     ("small", {"n_particles": 100})])
def test_env_create_fails_cleanly_at_every_allocation(name, kw):
    p = preset(name, n_envs=6).replace(**kw)
    cfg, keep = make_config(p, _abi.UT_FLAG_RING | _abi.UT_FLAG_DEBUG)
    ok = _FailingAllocator()
    rc, h = _create(cfg, ok)
    assert rc == 0
    n_calls = ok.calls
    assert n_calls > 20
    ut.lib.env_destroy(h)
    assert not ok.live
    for n in range(1, n_calls + 1):
        a = _FailingAllocator(fail_at=n)
        rc, h = _create(cfg, a)
        assert rc == 2 and not h.value, (n, rc)
        assert not a.live, (n, len(a.live))


def test_weight_buffers_fail_cleanly_and_can_be_set_later():
    """env_set_policy and est_set_weights with an allocator that fails on
    their first, second, ... allocation: UT_ERR_NOMEM, then (allocator
    healthy again) the same call succeeds and the handle works; everything is
    handed back at destroy."""
    p = preset("fleet5", n_envs=4).replace(n_particles=64)
    cfg, keep = make_config(p, _abi.UT_FLAG_RING)
    prm = synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, p.n_actions), seed=2)
    mlp = synth.mlp_params(seed=3, bias_scale=0.1)
    for k in range(1, 5):
        a = _FailingAllocator()
        rc, h = _create(cfg, a)
        assert rc == 0
        a.fail_at = a.calls + k
        pr = np.ascontiguousarray(prm, np.float32)
        rc = ut.lib.env_set_policy(h, pr.ctypes.data_as(ctypes.c_void_p), pr.size)
        assert rc == 2, (k, rc)
        a.fail_at = 0
        assert ut.lib.env_set_policy(h, pr.ctypes.data_as(ctypes.c_void_p), pr.size) == 0
        a.fail_at = a.calls + k
        ml = np.ascontiguousarray(mlp, np.float32)
        rc = ut.lib.est_set_weights(h, ml.ctypes.data_as(ctypes.c_void_p), ml.size)
        assert rc == 2, (k, rc)
        a.fail_at = 0
        assert ut.lib.est_set_weights(h, ml.ctypes.data_as(ctypes.c_void_p), ml.size) == 0
        assert ut.lib.env_reset(h, ctypes.c_uint64(1)) == 0
        assert ut.lib.est_set_mode(h, 2) == 0
        out = _abi.StepOut()
        assert ut.lib.env_step(h, None, ctypes.byref(out)) == 0
        s = _abi.RolloutStats()
        assert ut.lib.env_metrics(h, ctypes.byref(s)) == 0 and s.device_status == 0
        ut.lib.env_destroy(h)
        assert not a.live, (k, len(a.live))

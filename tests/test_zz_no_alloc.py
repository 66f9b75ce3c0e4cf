"""tracker_update_noalloc: the allocation-free tracker update, for callers that
cannot allocate device memory (code inside another component's graph capture,
real-time threads, simulators that own every buffer).  Called through the C
ABI and checked against env_step's own tracker output on two calls in a row.

This file is collected last on purpose: the entry point shares one static
device array across calls, and it must work both in a fresh process and after
every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

from synth import preset

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_08222_gb300 as ut  # noqa: E402
from paper_2505_08222_gb300 import _abi, make_config  # noqa: E402


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_tracker_matches_env_step_twice():
    p = preset("fleet5", n_envs=48).replace(n_particles=512, d_model=0, comm_drop=0.2, target_depth_max=30.0)
    env = ut.Env(p)
    seed = 77
    env.reset(seed)
    cfg, keep = make_config(p)
    st = env.state()
    # the caller's own particle buffers start from the handle's reset state
    mine = {k: st[k].clone() for k in ("px", "py", "pvx", "pvy")}
    F = env.F
    est = {k: torch.empty(F, device="cuda") for k in ("estx", "esty", "err")}
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        g = env.state()["step"] + 1
        out = env.step()  # the existing entry point: move, ping, communicate, filter
        post = env.state()
        rc = ut.lib.tracker_update_noalloc(ctypes.byref(cfg), ctypes.c_uint64(seed), g,
                                           _ptr(post["ax"]), _ptr(post["ay"]), _ptr(post["tx"]), _ptr(post["ty"]),
                                           _ptr(post["tz"]), _ptr(mine["px"]), _ptr(mine["py"]), _ptr(mine["pvx"]),
                                           _ptr(mine["pvy"]), _ptr(est["estx"]), _ptr(est["esty"]), _ptr(est["err"]),
                                           stream)
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

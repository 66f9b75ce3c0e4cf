"""Persistent rollout kernel (one CTA per environment for all T steps)
against the captured-graph rollout: the same state bit for bit after T steps
from the same reset, with the same filter launch shape, on the small
workload (one filter per env: particles resident in registers), on ragged
fleets (several filters per env: streamed through HBM each step), with any P
(scalar particle path) and with shared filters; device metrics agree to
summation order.  The autotuner records the rollout form it picked."""
import numpy as np
import pytest
import torch

import synth
from synth import preset

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_08222_gb300 as ut  # noqa: E402

KEYS = ("ax", "ay", "apsi", "tx", "ty", "tpsi", "px", "py", "pvx", "pvy", "lpx", "lpy", "lpage", "estx", "esty",
        "prev_estx", "prev_esty", "prev2_estx", "prev2_esty", "velx", "vely", "rudder")


def _snapshot(env):
    torch.cuda.synchronize()
    st = env.state()
    out = {k: st[k].cpu().numpy().copy() for k in KEYS if st.get(k) is not None}
    out["step"], out["t_ep"] = st["step"], st["t_ep"]
    return out


def _run(p, form, seed, T, reps=2, variant=None):
    env = ut.Env(p)
    if variant is not None:
        env.set_pf_variant(variant)
    env.reset(seed)
    env.set_rollout_form(form)
    assert env.rollout_form() == form
    stats = [env.rollout(T) for _ in range(reps)]
    snap = _snapshot(env)
    last = env.step()  # one more (graph-free) step from the rolled-out state: reward / done / obs follow
    extra = {k: last[k].cpu().numpy().copy() for k in ("reward", "done", "err")}
    v = env.pf_variant()
    env.close()
    return snap, stats, extra, v


@pytest.mark.parametrize("name,n_envs,kw", [
    ("small", 64, {}),                                              # P = 1000: float4 path, resident particles
    ("small", 16, {"n_particles": 1022}),                           # any P: scalar path, resident
    ("ragged", 40, {"n_particles": 100, "d_model": 0}),             # several filters per env, streamed
    ("ragged", 24, {"n_particles": 13, "d_model": 0, "comm_drop": 0.3}),
    ("ragged", 24, {"n_particles": 64, "d_model": 0, "shared_filter": 1}),
    ("fleet5", 8, {"n_particles": 512, "d_model": 0, "horizon": 7}),  # episode end inside the rollout
])
def test_persistent_rollout_equals_graph_rollout(name, n_envs, kw):
    p = preset(name, n_envs=n_envs).replace(**kw)
    T = 9
    g_snap, g_stats, g_extra, v = _run(p, 0, 5, T)
    p_snap, p_stats, p_extra, v2 = _run(p, 1, 5, T, variant=v)
    assert v == v2
    for k in g_snap:
        if k in ("step", "t_ep"):
            assert g_snap[k] == p_snap[k] == 2 * T, k
            continue
        np.testing.assert_array_equal(p_snap[k], g_snap[k], err_msg=k)
    for k in g_extra:
        np.testing.assert_array_equal(p_extra[k], g_extra[k], err_msg=k)
    for a, b in zip(g_stats, p_stats):
        for k in ("n_err", "crash_count", "agent_steps", "steps", "device_status"):
            assert a[k] == b[k], k
        assert b["sum_sq_err"] == pytest.approx(a["sum_sq_err"], rel=1e-12)
        assert b["reward_sum"] == pytest.approx(a["reward_sum"], rel=1e-12, abs=1e-9)
        assert b["kernel_launches"] == 2


def test_persistent_form_needs_random_actions_and_the_filter():
    p = preset("fleet5", n_envs=4).replace(n_particles=128)
    env = ut.Env(p, ring=True)
    env.reset(1)
    env.set_rollout_form(1)
    assert env.rollout_form() == 1
    env.set_policy(synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, p.n_actions), seed=1))
    assert env.rollout_form() == 0  # the policy acts: the graph runs
    with pytest.raises(ut.UtError, match="UT_ERR_UNSUPPORTED"):
        env.set_rollout_form(1)
    stats = env.rollout(3)
    assert stats["steps"] == 3 and stats["device_status"] == 0
    env.close()
    q = preset("fleet5", n_envs=4).replace(n_particles=128, d_model=0, pf_ess_num=8)
    e2 = ut.Env(q)
    with pytest.raises(ut.UtError, match="UT_ERR_UNSUPPORTED"):
        e2.set_rollout_form(1)
    e2.close()


def test_autotune_records_the_rollout_form():
    p = preset("small", n_envs=64)
    a = ut.Env(p)
    a.reset(0)
    a.autotune(3)
    form, v = a.rollout_form(), a.pf_variant()
    assert form in (0, 1)
    b = ut.Env(p)
    b.reset(0)
    b.autotune(3)  # the cached choice, no timing
    assert (b.rollout_form(), b.pf_variant()) == (form, v)
    a.close()
    b.close()

"""The shared-filter option (one filter per (env, target) fed every ping of
the target, the alternative of the filters-per-(agent, target) reading) in
the oracle, pinned by reductions to the per-agent filters and brute force.

* With one agent per env the two layouts are the same computation: the same
  filter ids, pair ids, measurement lists, tokens and rewards, bit for bit.
* The shared filter's measurement list is every agent of the env that heard
  the target, in agent order (brute force from the pings).
* With perfect communication every agent's own list holds the same pings
  as the shared list.
* Every agent's target token carries the shared estimate."""
import numpy as np
import pytest

import oracle
from synth import preset

STEPS = 5


def _pair(p, shared, **kw):
    return oracle.OracleEnv(p.replace(shared_filter=shared, **kw), 23)


def _run(o, steps=STEPS, want=("tokens", "meas", "meas_n", "range", "valid")):
    o.reset(0)
    outs = []
    for _ in range(steps):
        outs.append(o.step(o.random_actions(o.step_count), want=want))
    return outs


def test_one_agent_per_env_is_the_per_agent_filter():
    p = preset("fleet5", n_envs=3).replace(max_agents=1, max_targets=3, n_particles=64, d_model=0,
                                             comm_drop=0.3)
    a, b = _pair(p, 0), _pair(p, 1)
    assert a.F == b.F == 9
    ra, rb = _run(a), _run(b)
    for oa, ob in zip(ra, rb):
        for k in oa:
            np.testing.assert_array_equal(oa[k], ob[k], err_msg=k)
    for k in ("px", "py", "pvx", "pvy", "estx", "esty", "ax", "tx"):
        np.testing.assert_array_equal(a.arr[k], b.arr[k], err_msg=k)


def test_shared_lists_hold_every_ping_of_the_target():
    p = preset("fleet5", n_envs=4).replace(n_particles=32, d_model=0, det_radius=400.0, comm_drop=0.5)
    o = _pair(p, 1)
    assert o.F == 4 * p.max_targets and o.NPAIR == 4 * p.max_agents * p.max_targets
    o.reset(0)
    seen = 0
    for _ in range(4):
        out = o.step(o.random_actions(o.step_count), want=("meas", "meas_n", "range", "valid"))
        for e in range(p.n_envs):
            A, T = p.max_agents, p.max_targets
            for k in range(T):
                f = e * T + k
                want = [b for b in range(A) if out["valid"][e * A * T + b * T + k]]
                assert out["meas_n"][f] == len(want)
                for n, b in enumerate(want):
                    ia = e * A + b
                    np.testing.assert_array_equal(out["meas"][f, n, :2], [o.arr["ax"][ia], o.arr["ay"][ia]])
                    assert out["meas"][f, n, 3] == out["range"][e * A * T + b * T + k]
                seen += len(want)
    assert seen > 0


def test_perfect_comms_every_agent_holds_the_shared_list():
    p = preset("fleet5", n_envs=3).replace(n_particles=32, d_model=0, comm_radius=1e9, comm_drop=0.0)
    a, b = _pair(p, 0), _pair(p, 1)
    A, T = p.max_agents, p.max_targets
    a.reset(0)
    b.reset(0)
    for _ in range(3):
        act = a.random_actions(a.step_count)
        oa = a.step(act, want=("meas", "meas_n", "range"))
        ob = b.step(act, want=("meas", "meas_n", "range"))
        # same pings: the keys are the pairs in both layouts
        np.testing.assert_array_equal(oa["range"], ob["range"])
        for e in range(p.n_envs):
            for k in range(T):
                fs = e * T + k
                for ag in range(A):
                    fa = e * A * T + ag * T + k
                    assert oa["meas_n"][fa] == ob["meas_n"][fs]
                    n = ob["meas_n"][fs]
                    np.testing.assert_array_equal(oa["meas"][fa, :n], ob["meas"][fs, :n])


def test_tokens_carry_the_shared_estimate():
    p = preset("fleet5", n_envs=2).replace(n_particles=32, d_model=0)
    o = _pair(p, 1)
    out = _run(o, steps=2)[-1]
    A, T, S = p.max_agents, p.max_targets, p.feature_scale
    for e in range(p.n_envs):
        for ag in range(A):
            ia = e * A + ag
            for k in range(T):
                f = e * T + k
                tok = out["tokens"][ia, A + k]
                assert tok[0] == pytest.approx((o.arr["estx"][f] - o.arr["ax"][ia]) / S, abs=1e-15)
                assert tok[1] == pytest.approx((o.arr["esty"][f] - o.arr["ay"][ia]) / S, abs=1e-15)
                assert tok[5] == 1.0

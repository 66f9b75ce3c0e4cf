"""Pins of the oracle's environment stages against closed forms, printed
constants and brute force (Sec. III-A.2 / III-A.3 of the paper)."""
import math
import os

import numpy as np
import pytest

import oracle
from synth import preset

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()[:2]
            rows[k] = float(v)
    return rows


def _env(name="small", n_envs=4, seed=0, **kw):
    p = preset(name, n_envs=n_envs).replace(**kw)
    e = oracle.OracleEnv(p, seed)
    e.reset(0)
    return e


# ---------------------------------------------------------------- kinematics
def test_straight_line_closed_form():
    """Action 'no turn' with no heading noise: p_T = p_0 + v dt T (cos psi, sin psi)."""
    e = _env(heading_noise=0.0)
    x0, y0, psi0 = e.arr["ax"].copy(), e.arr["ay"].copy(), e.arr["apsi"].copy()
    T = 25
    for _ in range(T):
        e.step(np.ones(e.NA, np.int32))
    np.testing.assert_allclose(e.arr["ax"], x0 + 1.0 * 30.0 * T * np.cos(psi0), rtol=0, atol=1e-9)
    np.testing.assert_allclose(e.arr["ay"], y0 + 1.0 * 30.0 * T * np.sin(psi0), rtol=0, atol=1e-9)


def test_constant_turn_is_a_circle():
    """Constant turn delta: p_T = p_0 + v dt sum_{t=1..T} exp(i(psi0 + t delta))."""
    e = _env(heading_noise=0.0)
    z0 = e.arr["ax"] + 1j * e.arr["ay"]
    psi0 = e.arr["apsi"].copy()
    T, delta = 17, math.pi / 6
    for _ in range(T):
        e.step(np.full(e.NA, 2, np.int32))
    q = np.exp(1j * delta)
    zT = z0 + 30.0 * np.exp(1j * (psi0 + delta)) * (1 - q ** T) / (1 - q)
    np.testing.assert_allclose(e.arr["ax"], zT.real, atol=1e-9)
    np.testing.assert_allclose(e.arr["ay"], zT.imag, atol=1e-9)


def test_rudder_anchor_heading_change():
    """Actions Space paragraph: rudder +-0.24 rad <-> heading change +-1.45 rad."""
    gold = _golden("paper_constants.txt")
    e = _env("fleet5", n_envs=2, heading_noise=0.0)
    psi0 = e.arr["apsi"].copy()
    e.step(np.full(e.NA, 6, np.int32))  # gamma = +0.24
    d = np.angle(np.exp(1j * (e.arr["apsi"] - psi0)))
    np.testing.assert_allclose(d, gold["heading_change_max"], atol=1e-12)
    psi1 = e.arr["apsi"].copy()
    e.step(np.full(e.NA, 0, np.int32))  # gamma = -0.24
    d = np.angle(np.exp(1j * (e.arr["apsi"] - psi1)))
    np.testing.assert_allclose(d, -gold["heading_change_max"], atol=1e-12)


def test_rudder_adjacent_moves():
    """Actions Space paragraph, five rudder angles in [-0.24, 0.24] rad that
    change only to an adjacent angle (action_mode 2: down / keep / up): the
    rudder starts straight, moves one position per up / down action, stops at
    the ends, and the heading turns by 1.45 / 0.24 times the rudder angle
    reached (1.45 rad at the end stop)."""
    gold = _golden("paper_constants.txt")
    e = _env("fleet5", n_envs=2, heading_noise=0.0, action_mode=2, n_rudder=5, n_actions=3)
    assert np.all(e.arr["rudder"] == 2)
    seq = [2, 2, 2, 0, 1, 0, 0, 0, 0]
    want_k = [3, 4, 4, 3, 3, 2, 1, 0, 0]
    for a, k in zip(seq, want_k):
        psi0 = e.arr["apsi"].copy()
        e.step(np.full(e.NA, a, np.int32))
        assert np.all(e.arr["rudder"] == k)
        d = np.angle(np.exp(1j * (e.arr["apsi"] - psi0)))
        gamma = -0.24 + 0.12 * k
        np.testing.assert_allclose(d, gold["heading_change_max"] * gamma / 0.24, atol=1e-12)
    # random actions: never more than one position per step, always in range
    rng = np.random.default_rng(3)
    prev = e.arr["rudder"].copy()
    for _ in range(50):
        e.step(rng.integers(0, 3, e.NA).astype(np.int32))
        k = e.arr["rudder"]
        assert np.all(np.abs(k - prev) <= 1) and np.all((k >= 0) & (k <= 4))
        prev = k.copy()


def test_heading_noise_std():
    """Sec. III-A.3: Gaussian heading noise of std 0.02 rad."""
    e = _env("fleet5", n_envs=400, n_particles=4, heading_noise=0.02)
    psi0 = e.arr["apsi"].copy()
    e.step(np.full(e.NA, 3, np.int32))  # gamma = 0
    d = np.angle(np.exp(1j * (e.arr["apsi"] - psi0)))
    assert abs(d.std() - 0.02) < 0.0015 and abs(d.mean()) < 0.002


def test_targets_drift_free_is_straight():
    e = _env("fleet5", n_envs=3, n_particles=8, target_drift_sigma=0.0)
    x0, y0, psi, s = (e.arr[k].copy() for k in ("tx", "ty", "tpsi", "tspeed"))
    for _ in range(9):
        e.step(np.full(e.NA, 3, np.int32))
    np.testing.assert_allclose(e.arr["tx"], x0 + s * 30 * 9 * np.cos(psi), atol=1e-9)
    np.testing.assert_allclose(e.arr["ty"], y0 + s * 30 * 9 * np.sin(psi), atol=1e-9)
    assert np.all((s >= 0.5) & (s < 1.5))


def test_random_walk_target_speed():
    e = _env(n_envs=16)
    for _ in range(5):
        x0, y0 = e.arr["tx"].copy(), e.arr["ty"].copy()
        e.step(e.random_actions(e.step_count + 1))
        np.testing.assert_allclose(np.hypot(e.arr["tx"] - x0, e.arr["ty"] - y0), 0.3 * 30, atol=1e-9)


# --------------------------------------------------------------- spawn
def test_spawn_geometry():
    gold = _golden("paper_constants.txt")
    e = _env("fleet5", n_envs=64, n_particles=4)
    ok = []
    for env in range(64):
        a0, t0 = env * 5, env * 5
        xs = np.concatenate([e.arr["ax"][a0:a0 + 5], e.arr["tx"][t0:t0 + 5]])
        ys = np.concatenate([e.arr["ay"][a0:a0 + 5], e.arr["ty"][t0:t0 + 5]])
        # on the 2^-16 m lattice
        assert np.all(xs * 65536 == np.round(xs * 65536))
        d = np.hypot(xs[:, None] - xs[None], ys[:, None] - ys[None])[np.triu_indices(10, 1)]
        assert d.max() <= gold["spawn_max"] + 1e-9
        ok.append(d >= gold["spawn_min"])
    # 10 entities in a 100 m disk: most pairs satisfy the minimum separation
    assert np.mean(ok) > 0.9
    e1 = _env("fleet5", n_envs=64, n_particles=4, max_agents=2, max_targets=1)
    for env in range(64):
        xs = np.concatenate([e1.arr["ax"][2 * env:2 * env + 2], e1.arr["tx"][env:env + 1]])
        ys = np.concatenate([e1.arr["ay"][2 * env:2 * env + 2], e1.arr["ty"][env:env + 1]])
        d = np.hypot(xs[:, None] - xs[None], ys[:, None] - ys[None])[np.triu_indices(3, 1)]
        assert d.min() >= gold["spawn_min"] and d.max() <= gold["spawn_max"]


# --------------------------------------------------------------- pings / comms
def test_noise_free_ranges_equal_distance_and_detection_edge():
    e = _env("fleet5", n_envs=3, n_particles=8, range_sigma=0.0, target_depth_max=40.0)
    # put target 0 of env 0 at exactly det_radius - 1e-6 from agent 0 after the move
    o = e.step(np.full(e.NA, 3, np.int32), want=("range", "valid"))
    for env in range(3):
        for a in range(5):
            for k in range(5):
                f = env * 25 + a * 5 + k
                ia, it = env * 5 + a, env * 5 + k
                d = math.sqrt((e.arr["ax"][ia] - e.arr["tx"][it]) ** 2 + (e.arr["ay"][ia] - e.arr["ty"][it]) ** 2
                              + e.arr["tz"][it] ** 2)
                assert o["valid"][f] == 1
                assert o["range"][f] == pytest.approx(d, abs=1e-12)
    for delta, expect in ((-1e-6, 1), (1e-6, 0)):
        e2 = _env(n_envs=1, range_sigma=0.0, heading_noise=0.0, target_speed_min=0.0, target_speed_max=0.0)
        psi = e2.arr["apsi"][0]
        R = 1500.0
        # place the target so that after the agent's 30 m straight move it sits at R + delta
        nx, ny = e2.arr["ax"][0] + 30 * math.cos(psi), e2.arr["ay"][0] + 30 * math.sin(psi)
        e2.set_arrays(tx=[nx + R + delta], ty=[ny])
        o2 = e2.step(np.ones(1, np.int32), want=("valid", "range"))
        assert o2["valid"][0] == expect


def test_comms_brute_force():
    rng = np.random.default_rng(3)
    e = _env("fleet5", n_envs=6, n_particles=4, comm_radius=900.0, det_radius=1000.0, comm_drop=0.25)
    # scatter agents and targets so that some links and pings fail
    e.set_arrays(ax=rng.uniform(-1500, 1500, e.NA), ay=rng.uniform(-1500, 1500, e.NA),
                 tx=rng.uniform(-1500, 1500, e.NT), ty=rng.uniform(-1500, 1500, e.NT))
    o = e.step(np.full(e.NA, 3, np.int32), want=("recv", "valid", "range", "meas", "meas_n"))
    g = e.step_count
    assert 0 < o["valid"].sum() < e.F
    for env in range(6):
        for a in range(5):
            ia = env * 5 + a
            for b in range(5):
                ib = env * 5 + b
                if a == b:
                    expect = 1
                else:
                    u, _ = oracle.uniform_normal(0, ia, b, g, 10)
                    near = math.hypot(e.arr["ax"][ia] - e.arr["ax"][ib], e.arr["ay"][ia] - e.arr["ay"][ib]) <= 900.0
                    expect = int(near and not (u[0] < 0.25))
                assert o["recv"][ia * 5 + b] == expect
            for k in range(5):
                f = env * 25 + a * 5 + k
                rows = [(e.arr["ax"][env * 5 + b], e.arr["ay"][env * 5 + b], 0.0, o["range"][env * 25 + b * 5 + k])
                        for b in range(5) if o["recv"][ia * 5 + b] and o["valid"][env * 25 + b * 5 + k]]
                assert o["meas_n"][f] == len(rows)
                if rows:
                    np.testing.assert_array_equal(o["meas"][f, :len(rows)], np.array(rows))


# --------------------------------------------------------------- reward
def test_tracking_reward_eq1_printed_values():
    for line in open(os.path.join(GOLDEN, "reward_eq1.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        err, want = (float(v) for v in line.split())
        assert oracle.tracking_reward(err) == pytest.approx(want, rel=1e-12, abs=1e-300)


def test_reward_follow_normalisation_and_crash():
    e = _env("fleet5", n_envs=1, n_particles=4, target_speed_min=0.0, target_speed_max=0.0,
             heading_noise=0.0)
    # agents move 30 m along their heading; put targets relative to the new positions
    psi = e.arr["apsi"]
    nx, ny = e.arr["ax"] + 30 * np.cos(psi), e.arr["ay"] + 30 * np.sin(psi)
    spread = np.arange(5) * 1000.0
    e.set_arrays(ax=e.arr["ax"] + spread, tx=nx + spread + np.array([10, 99, 101, 500, 20.0]), ty=ny)
    o = e.step(np.full(5, 3, np.int32))
    # Eq. (2) with d_min = 100: targets 0, 1, 4 followed -> 3/5
    assert o["reward"][0] == pytest.approx(3 / 5)
    # crash: two agents closer than d_safe -> -1
    e.set_arrays(ax=np.array([0, 5, 2000, 4000, 6000.0]), ay=np.zeros(5), apsi=np.zeros(5))
    o = e.step(np.full(5, 3, np.int32))
    assert o["reward"][0] == -1.0 and o["crash"][0] == 1


# --------------------------------------------------------------- observation
def test_observation_tokens_structure():
    e = _env("fleet5", n_envs=2, n_particles=16)
    o = e.step(np.full(e.NA, 3, np.int32), want=("tokens",))
    tok = o["tokens"]
    assert tok.shape == (10, 10, 8)
    for ia in range(10):
        env = ia // 5
        np.testing.assert_array_equal(tok[ia, 0], [0, 0, 0, 1, 0, 0, 0, 0])
        assert np.all(tok[ia, 1:5, 4] == 1) and np.all(tok[ia, 5:10, 5] == 1)
        # targets: tracker estimate relative to the agent, depth / S
        a = ia % 5
        for k in range(5):
            f = env * 25 + a * 5 + k
            assert tok[ia, 5 + k, 0] == pytest.approx((e.arr["estx"][f] - e.arr["ax"][ia]) / 1000.0)
            assert tok[ia, 5 + k, 1] == pytest.approx((e.arr["esty"][f] - e.arr["ay"][ia]) / 1000.0)
        # teammates (all within comm range): current pose, not missing
        mates = [b for b in range(5) if b != a]
        for s, b in enumerate(mates):
            ib = env * 5 + b
            assert tok[ia, 1 + s, 0] == pytest.approx((e.arr["ax"][ib] - e.arr["ax"][ia]) / 1000.0)
            assert tok[ia, 1 + s, 6] == 0.0

"""GPU parity: the CUDA library against the FP64 oracle on the same seeded
inputs, through the C ABI.

Tolerances (float32 kernel arithmetic against float64):
  positions, headings, ranges, predicted particles: 1e-5 relative, the
  required bound for one step from an injected state; relative to
  max(|x|, 100 m) for coordinates (a coordinate is the difference of terms of
  the spawn scale, so near the origin float32 cancellation leaves an
  absolute error of that scale times 1e-7), max(|v|, 1 m/s) for velocities;
  resample indices: bit-exact given the kernel's own weights and the shared
  uniform (the oracle recomputes the map from them);
  normalised weights: 3e-3 relative to the largest weight (float32 log-domain
  weights carry an absolute error of ~|residual| * 1e-7 * range / sigma^2);
  estimate: 5e-3 m (weights' relative error times the particle spread);
  detection and communication bits: exact except within 1e-3 m of the
  radius, where float32 and float64 distances may round to different sides.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from synth import preset

from gpu_util import (angle_diff, bf16_to_f32, ess_trigger, gpu_state, inject, oracle_state_f32, rel_close,
                      resample_u64)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the parity tests need the GB300
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_08222_gb300 as ut  # noqa: E402


def _pair(params, seed=0, debug=True, ring=False):
    env = ut.Env(params, debug=debug, ring=ring)
    env.reset(seed)
    o = oracle.OracleEnv(params, seed)
    o.reset(0)
    return env, o


# ---------------------------------------------------------------- Philox
def test_philox_bit_exact():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, (4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [1, 2, 3, 4], [0xFFFFFFFF] * 4, [7, 0, 0, 11]]
    seed = 0x1234567890ABCDEF
    got = ut.philox(torch.from_numpy(ctr.view(np.int32)).cuda(), seed).cpu().numpy().view(np.uint32)
    want = oracle.philox_many(ctr, [seed & 0xFFFFFFFF, seed >> 32])
    np.testing.assert_array_equal(got, want)


# ---------------------------------------------------------------- resampling
@pytest.mark.parametrize("P", [1, 2, 3, 13, 64, 100, 1000, 1024, 2048, 4096])
def test_resample_indices_bit_exact(P):
    rng = np.random.default_rng(P)
    F = 48
    w = np.empty((F, P), np.float32)
    for f in range(F):
        kind = f % 6
        if kind == 0:
            v = rng.uniform(0, 1, P)
        elif kind == 1:
            v = np.exp(-rng.exponential(20.0, P))
        elif kind == 2:
            v = rng.integers(0, 65, P) / 64.0     # dyadic: exact in every order
        elif kind == 3:
            v = np.zeros(P)                       # one particle carries everything
        elif kind == 4:
            v = np.ones(P)
        else:
            v = np.where(rng.uniform(0, 1, P) < 0.01, rng.uniform(0, 1, P), 0.0)
        v[rng.integers(0, P)] = 1.0
        w[f] = v.astype(np.float32)
    u64 = rng.integers(0, 2 ** 63, F, dtype=np.int64)
    # exact ties P Q_i = j W + U0: a zero offset on the uniform (kind 4) and
    # dyadic (kind 2) filters of the first rows
    u64[[2, 4, 8, 10]] = 0
    got = ut.pf_resample(torch.from_numpy(w).cuda(), torch.from_numpy(u64).cuda()).cpu().numpy()
    for f in range(F):
        want = oracle.systematic_resample(w[f].astype(np.float64), int(u64[f]) & (2 ** 64 - 1))
        np.testing.assert_array_equal(got[f], want)


# ---------------------------------------------------------------- reset
@pytest.mark.parametrize("name,n_envs,P,kw", [("small", 8, 1000, {}), ("fleet5", 6, 256, {}), ("ragged", 12, 100, {}),
                                             ("fleet5", 6, 256, {"shared_filter": 1})])
def test_reset_parity(name, n_envs, P, kw):
    p = preset(name, n_envs=n_envs).replace(n_particles=P, **kw)
    env, o = _pair(p, seed=7)
    g = gpu_state(env)
    # spawn lies on a 2^-16 m lattice: bit-exact
    for k in ("ax", "ay", "tx", "ty"):
        np.testing.assert_array_equal(g[k].astype(np.float64), o.arr[k])
    assert np.all(angle_diff(g["apsi"], o.arr["apsi"]) < 1e-5)
    assert np.all(rel_close(g["tspeed"], o.arr["tspeed"], 1e-6))
    for k in ("px", "py", "pvx", "pvy"):
        fl = 100.0 if k in ("px", "py") else 1.0
        assert np.all(rel_close(g[k], o.arr[k], 1e-5, fl)), (k, np.max(np.abs(g[k] - o.arr[k])))
    assert np.all(np.abs(g["estx"] - o.arr["estx"]) < 1e-3)
    np.testing.assert_array_equal(g["lpx"].astype(np.float64), o.arr["lpx"])
    assert g["step"] == 0 and g["t_ep"] == 0


# ---------------------------------------------------------------- one step from an injected state
def _compare_step(env, o, actions, check_tokens=True):
    p = o.p
    st = gpu_state(env)
    g_next = st["step"] + 1
    out = env.step(torch.from_numpy(actions).cuda())
    dbg = {k: (v.cpu().numpy() if v is not None else None) for k, v in env.debug().items()}
    gout = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    g = gpu_state(env)
    ref = o.step(actions, want=("range", "valid", "recv", "meas", "meas_n", "pred_px", "weight", "wmax", "idx",
                                "tokens"))
    # kinematics (and, for action_mode 2, the rudder positions, exactly)
    np.testing.assert_array_equal(g["rudder"], o.arr["rudder"])
    assert np.all(rel_close(g["ax"], o.arr["ax"], 1e-5, 100.0)) and np.all(rel_close(g["ay"], o.arr["ay"], 1e-5, 100.0))
    assert np.all(angle_diff(g["apsi"], o.arr["apsi"]) < 1e-5)
    assert np.all(rel_close(g["tx"], o.arr["tx"], 1e-5, 100.0)) and np.all(rel_close(g["ty"], o.arr["ty"], 1e-5, 100.0))
    # pings: detection exact away from the radius
    a_of_f = np.repeat(np.arange(o.NA), np.repeat(o.n_targets_env, o.n_agents_env))
    t_of_f = np.concatenate([o.target_off[e] + np.tile(np.arange(o.n_targets_env[e]), o.n_agents_env[e])
                             for e in range(p.n_envs)])
    dist = np.sqrt((o.arr["ax"][a_of_f] - o.arr["tx"][t_of_f]) ** 2 + (o.arr["ay"][a_of_f] - o.arr["ty"][t_of_f]) ** 2
                   + o.arr["tz"][t_of_f] ** 2)
    edge = np.abs(dist - p.det_radius) < 1e-3
    assert np.all((dbg["valid"] == ref["valid"]) | edge)
    both = (dbg["valid"] == 1) & (ref["valid"] == 1)
    assert np.all(rel_close(dbg["range"][both], ref["range"][both], 1e-5, 100.0))
    # measurement lists
    same_lists = dbg["meas_n"] == ref["meas_n"]
    assert np.mean(same_lists) > 0.999
    for f in np.nonzero(same_lists)[0][:2000]:
        n = ref["meas_n"][f]
        assert np.all(rel_close(dbg["meas"][f, :n][:, [0, 1, 3]], ref["meas"][f, :n][:, [0, 1, 3]], 1e-5, 100.0))
    # predicted particles
    for k in ("pred_px", "pred_py", "pred_pvx", "pred_pvy"):
        fl = 100.0 if k in ("pred_px", "pred_py") else 1.0
        assert np.all(rel_close(dbg[k], ref[k], 1e-5, fl)), (k, np.max(np.abs(dbg[k] - ref[k])))
    # weights (normalised), per filter, relative to the largest weight
    P = p.n_particles
    wg = dbg["weight"].reshape(-1, P)
    wo = ref["weight"].reshape(-1, P)
    sel = same_lists
    scale = wo.max(1, keepdims=True)
    assert np.all(np.abs(wg[sel] - wo[sel]) <= 3e-3 * scale[sel] + 1e-7)
    np.testing.assert_allclose(wg.sum(1), 1.0, atol=2e-5)
    # resample map: bit-exact against the definition applied to the kernel's own weights
    wmax = dbg["wmax"].reshape(-1, P)
    idx = dbg["idx"].reshape(-1, P)
    k_ess = int(getattr(p, "pf_ess_num", 0))
    for f in range(o.F):
        if dbg["meas_n"][f] > 0 and (k_ess == 0 or ess_trigger(wmax[f], k_ess, P)):
            want = oracle.systematic_resample(wmax[f].astype(np.float64), resample_u64(o.seed, f, g_next))
            np.testing.assert_array_equal(idx[f], want)
        else:
            np.testing.assert_array_equal(idx[f], np.arange(P))
    # carried log-weights (ESS form): 0 where the kernel resampled, else
    # log w - max log w, against the oracle's where both took the same decision
    if k_ess:
        trig_g = np.array([dbg["meas_n"][f] > 0 and ess_trigger(wmax[f], k_ess, P) for f in range(o.F)])
        wo_max = ref["wmax"].reshape(-1, P)
        trig_o = np.array([ref["meas_n"][f] > 0 and ess_trigger(wo_max[f], k_ess, P) for f in range(o.F)])
        pw_g, pw_o = g["pw"].reshape(-1, P), o.arr["pw"].reshape(-1, P)
        assert np.all(pw_g[trig_g] == 0.0)
        same = (trig_g == trig_o) & sel
        assert np.mean(trig_g == trig_o) > 0.99
        keep = same & ~trig_g
        assert np.all(np.abs(pw_g[keep] - pw_o[keep]) <= 2e-3 + 1e-4 * np.abs(pw_o[keep]))
    # gather: new particles are the predicted ones at the resample indices
    for k, pk in (("px", "pred_px"), ("py", "pred_py"), ("pvx", "pred_pvx"), ("pvy", "pred_pvy")):
        np.testing.assert_array_equal(g[k].reshape(-1, P), np.take_along_axis(dbg[pk].reshape(-1, P), idx, 1))
    # estimate and error
    ok = sel
    assert np.all(np.abs(g["estx"][ok] - o.arr["estx"][ok]) < 5e-3)
    assert np.all(np.abs(g["esty"][ok] - o.arr["esty"][ok]) < 5e-3)
    assert np.all(np.abs(gout["err"][ok] - ref["err"][ok]) < 5e-3)
    # observation tokens: bf16 of the same features
    if check_tokens:
        tok = bf16_to_f32(gout["obs"].view(np.uint16)).reshape(ref["tokens"].shape)
        assert np.all(np.abs(tok - ref["tokens"]) <= 2 ** -8 * np.abs(ref["tokens"]) + 1e-5)
    # reward
    if p.reward_type == 0:
        assert np.all(np.abs(gout["reward"] - ref["reward"]) < 2e-3)
    else:
        assert np.mean(np.abs(gout["reward"] - ref["reward"]) < 1e-6) > 0.99
    return ref


@pytest.mark.parametrize("name,n_envs,P,kw", [
    ("small", 16, 1000, {}),
    ("small", 4, 1, {}),
    ("small", 3, 4096, {}),
    ("fleet5", 8, 2048, {}),
    ("fleet5", 4, 13, {"comm_drop": 0.3, "comm_radius": 300.0, "target_depth_max": 50.0}),
    ("fleet5", 4, 512, {"det_radius": 60.0}),
    ("fleet5", 6, 256, {"action_mode": 2, "n_rudder": 5, "n_actions": 3}),
    ("fleet5", 6, 512, {"shared_filter": 1, "comm_drop": 0.3}),
    ("ragged", 24, 100, {}),
    ("ragged", 16, 100, {"shared_filter": 1}),
    ("fleet5", 6, 512, {"pf_ess_num": 8, "range_sigma": 30.0}),
    ("fleet5", 4, 2048, {"pf_ess_num": 4}),
    ("ragged", 12, 13, {"pf_ess_num": 8, "range_sigma": 20.0}),
    ("small", 3, 4096, {"pf_ess_num": 12, "range_sigma": 40.0}),
    ("fleet5", 4, 256, {"shared_filter": 1, "pf_ess_num": 8, "range_sigma": 25.0}),
    ("large", 2, 512, {}),
])
def test_step_parity_from_injected_state(name, n_envs, P, kw):
    """The oracle's own state (rounded to float32) is injected into both sides,
    then one step is compared; repeated from the oracle's next state."""
    p = preset(name, n_envs=n_envs).replace(n_particles=P, **kw)
    env, o = _pair(p, seed=3)
    for t in range(1, 4):
        o.step(o.random_actions(t))
    for t in range(2):
        inject(env, o, oracle_state_f32(o), step=o.step_count, t_ep=3 + t)
        act = np.random.default_rng(t).integers(0, p.n_actions, o.NA).astype(np.int32)
        _compare_step(env, o, act)


# ---------------------------------------------------------------- whole rollouts
@pytest.mark.parametrize("name,n_envs,T,P,kw", [("small", 1024, 200, 1000, {}), ("fleet5", 64, 100, 2048, {}),
                                              ("ragged", 96, 60, 1024, {}),
                                              ("fleet5", 256, 100, 1024, {"shared_filter": 1}),
                                              ("fleet5", 128, 100, 1024, {"pf_ess_num": 8})])
def test_rollout_rmse_matches_oracle(name, n_envs, T, P, kw):
    """Mean tracking RMSE of whole rollouts agrees within 2% (the required
    whole-rollout bound).  'Mean tracking RMSE' = mean over filters of each filter's RMSE
    over the rollout.  Both sides draw the same random numbers, but float32
    and float64 weights place a resampling threshold on different sides of a
    CDF step now and then, after which the two filters are different (equally
    valid) realisations; a single agent's range-only posterior is bimodal, so
    the statistic needs about a thousand environments to settle within 2%."""
    p = preset(name, n_envs=n_envs).replace(n_particles=P, d_model=0, **kw)
    env = ut.Env(p)
    env.reset(0)
    se_g = torch.zeros(env.F, dtype=torch.float64, device="cuda")
    for t in range(T):
        out = env.step()
        se_g += out["err"].double() ** 2
    stats = env.metrics()
    o = oracle.OracleEnv(p, 0)
    o.reset(0)
    se_o = np.zeros(o.F)
    rw = 0.0
    for t in range(1, T + 1):
        r = o.step(o.random_actions(t))
        se_o += r["err"] ** 2
        rw += float(r["reward"].sum())
    mean_rmse_g = float(torch.sqrt(se_g / T).mean())
    mean_rmse_o = float(np.sqrt(se_o / T).mean())
    assert stats["n_err"] == o.F * T and stats["steps"] == T and stats["agent_steps"] == T * o.NA
    assert abs(mean_rmse_g - mean_rmse_o) <= 0.02 * mean_rmse_o, (mean_rmse_g, mean_rmse_o)
    pooled_o = math.sqrt(se_o.sum() / (o.F * T))
    print(f"{name}: mean RMSE gpu {mean_rmse_g:.3f} oracle {mean_rmse_o:.3f}; pooled gpu {stats['rmse']:.3f} "
          f"oracle {pooled_o:.3f}; reward gpu {stats['reward_sum']:.1f} oracle {rw:.1f}")
    assert abs(stats["reward_sum"] - rw) <= 0.05 * abs(rw) + 1.0


def test_ess_k16_is_the_every_step_filter():
    """With k = 16 the trigger fires unless all quantised weights are equal,
    so the carried-weight filter runs the every-step filter's computation:
    the two handles' states agree bit for bit."""
    p = preset("fleet5", n_envs=16).replace(n_particles=512, d_model=0)
    a, b = ut.Env(p), ut.Env(p.replace(pf_ess_num=16))
    v = a.pf_variant()
    b.set_pf_variant(v)
    a.reset(4)
    b.reset(4)
    for _ in range(6):
        a.step()
        b.step()
    sa, sb = gpu_state(a), gpu_state(b)
    for k in ("px", "py", "pvx", "pvy", "estx", "esty"):
        np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)
    assert np.all(sb["pw"] == 0.0)


def test_rollout_graph_metrics():
    p = preset("fleet5", n_envs=32).replace(n_particles=128, d_model=0)
    env = ut.Env(p)
    env.reset(2)
    s = env.rollout(20)
    assert s["steps"] == 20 and s["agent_steps"] == 20 * 160 and s["n_err"] == 20 * 800
    assert s["kernel_launches"] == 20 * 4 and s["device_status"] == 0
    assert 0 < s["rmse"] < 1000 and math.isfinite(s["reward_sum"])


@pytest.mark.parametrize("kw", [{}, {"shared_filter": 1}, {"pf_ess_num": 8, "range_sigma": 30.0}])
def test_eager_steps_equal_graph_rollout(kw):
    p = preset("fleet5", n_envs=16).replace(n_particles=256, d_model=0, **kw)
    a = ut.Env(p)
    a.reset(5)
    for _ in range(10):
        a.step()
    b = ut.Env(p)
    b.reset(5)
    b.rollout(10)
    sa, sb = gpu_state(a), gpu_state(b)
    for k in ("ax", "px", "estx"):
        np.testing.assert_array_equal(sa[k], sb[k])
    assert sa["step"] == sb["step"] == 10


# ---------------------------------------------------------------- full size, sampled
def test_full_size_fleet5_sampled():
    """The 4096-env 5v5 workload with 2048 particles per filter, in the launch
    configuration the benchmark times.  Sampled environments are replayed by
    the oracle from the same seed (random draws are keyed by global ids, so a
    one-env oracle batch with the right id offsets reproduces them); every
    filter is checked by invariants on the device."""
    p = preset("fleet5").replace(d_model=0)
    P = p.n_particles
    env = ut.Env(p, debug=True)
    env.reset(11)
    env.step()
    torch.cuda.synchronize()
    dbg = env.debug()
    F = env.F
    idx = dbg["idx"].view(F, P)
    assert int(idx.min()) >= 0 and int(idx.max()) < P
    assert int(torch.diff(idx, dim=1).min()) >= 0
    wsum = dbg["weight"].view(F, P).double().sum(1)
    assert float((wsum - 1).abs().max()) < 3e-5
    st = env.state()
    for e in (0, 1, 777, 2048, 4095):
        o = oracle.OracleEnv(p.replace(n_envs=1), 11, id_base=(e, 5 * e, 5 * e, 25 * e))
        o.reset(0)
        ref = o.step(o.random_actions(1), want=("pred_px", "pred_py", "weight"))
        sa, sf = slice(5 * e, 5 * e + 5), slice(25 * e * P, 25 * (e + 1) * P)
        assert np.all(rel_close(st["ax"][sa].cpu().numpy(), o.arr["ax"], 1e-5, 100.0))
        assert np.all(rel_close(st["tx"][sa].cpu().numpy(), o.arr["tx"], 1e-5, 100.0))
        assert np.all(rel_close(dbg["pred_px"][sf].cpu().numpy(), ref["pred_px"], 1e-5, 100.0))
        assert np.all(rel_close(dbg["pred_py"][sf].cpu().numpy(), ref["pred_py"], 1e-5, 100.0))
        wg = dbg["weight"][sf].cpu().numpy().reshape(25, P)
        wo = ref["weight"].reshape(25, P)
        assert np.all(np.abs(wg - wo) <= 3e-3 * wo.max(1, keepdims=True) + 1e-7)
        wmax = dbg["wmax"][sf].cpu().numpy().reshape(25, P)
        for fl in range(25):
            want = oracle.systematic_resample(wmax[fl].astype(np.float64), resample_u64(11, 25 * e + fl, 1))
            np.testing.assert_array_equal(idx[25 * e + fl].cpu().numpy(), want)


def test_full_size_large_sampled():
    """The largest workload: 65536 envs x 8 agents x 8 targets with 512
    particles per filter, exactly 2^31 particles, so the last filters' particle
    offsets need 64-bit indexing.  The first, a middle and the last
    environment are replayed by the oracle (global-id offsets) and compared
    on the predicted particles, the weights and the exact resample map."""
    p = preset("large").replace(d_model=0)
    P, A, T = p.n_particles, p.max_agents, p.max_targets
    FA = A * T
    env = ut.Env(p, debug=True)
    assert env.F * P == 2 ** 31
    env.reset(13)
    env.step()
    torch.cuda.synchronize()
    dbg = env.debug()
    st = env.state()
    for e in (0, 33333, p.n_envs - 1):
        o = oracle.OracleEnv(p.replace(n_envs=1), 13, id_base=(e, A * e, T * e, FA * e))
        o.reset(0)
        ref = o.step(o.random_actions(1), want=("pred_px", "pred_py", "weight"))
        sa = slice(A * e, A * (e + 1))
        sf = slice(FA * e * P, FA * (e + 1) * P)
        assert np.all(rel_close(st["ax"][sa].cpu().numpy(), o.arr["ax"], 1e-5, 100.0))
        assert np.all(rel_close(dbg["pred_px"][sf].cpu().numpy(), ref["pred_px"], 1e-5, 100.0))
        assert np.all(rel_close(dbg["pred_py"][sf].cpu().numpy(), ref["pred_py"], 1e-5, 100.0))
        wg = dbg["weight"][sf].cpu().numpy().reshape(FA, P)
        wo = ref["weight"].reshape(FA, P)
        assert np.all(np.abs(wg - wo) <= 3e-3 * wo.max(1, keepdims=True) + 1e-7)
        wmax = dbg["wmax"][sf].cpu().numpy().reshape(FA, P)
        idx = dbg["idx"][sf].cpu().numpy().reshape(FA, P)
        for fl in range(FA):
            want = oracle.systematic_resample(wmax[fl].astype(np.float64), resample_u64(13, FA * e + fl, 1))
            np.testing.assert_array_equal(idx[fl], want)
    del env, dbg, st
    torch.cuda.empty_cache()

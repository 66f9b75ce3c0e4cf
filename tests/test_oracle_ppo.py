"""TransfMAPPO training parts of the oracle (MAPPO of Sec. II-B with the
transformer actor and critic of Sec. III-B.1 / Fig. 3), pinned by:

* central finite differences of the batch loss (actor: PPO clipped surrogate
  with entropy bonus; critic: squared value error) on a small network with
  ragged entity counts, every parameter tensor sampled;
* at ratio 1 (pi_old = pi) the PPO gradient is the policy gradient
  -mean(A grad log pi(a)), differentiated here from the forward logits alone;
* samples whose ratio left the clip range in the adverse direction carry no
  gradient; the favourable side keeps it;
* the entropy and the value loss recomputed from the forward outputs;
* the critic's value is invariant to the order of the entity tokens;
* GAE closed forms: lambda = 0 gives the one-step TD error, lambda = 1 and
  gamma = 1 the return to the episode end (bootstrapped at the batch end)
  minus the value, and the backward recursion of the estimator;
* the critic's state tokens against the state they are built from, and their
  velocities against the next step's displacement (no noise, no turn)."""
import numpy as np
import pytest

import oracle
import synth
from synth import preset

D, L, H, NACT = 16, 2, 2, 5


def _net(n_out, seed=3):
    dims = synth.PolicyDims(D, L, H, n_out)
    prm = synth.policy_params(dims, seed=seed).astype(np.float64)
    return prm


def _batch(n, seed=5, ns=6):
    rng = np.random.default_rng(seed)
    n_ent = rng.integers(0, ns + 1, n)
    n_ent[0] = ns
    tok = synth.random_tokens(n, ns, n_ent, seed + 1).astype(np.float64)
    h = 0.5 * rng.standard_normal((n, D))
    return tok, n_ent.astype(np.int32), h


def _logp(logits, act):
    m = logits.max(1, keepdims=True)
    ls = logits - m - np.log(np.exp(logits - m).sum(1, keepdims=True))
    return ls[np.arange(len(act)), act], ls


def _fd_check(f, prm, grad, n_probe=240, h=1e-6, seed=0):
    """Central differences on parameters drawn from every tensor."""
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([rng.integers(0, len(prm), n_probe), [0, len(prm) - 1]]))
    num = np.empty(len(idx))
    for k, i in enumerate(idx):
        p1, p2 = prm.copy(), prm.copy()
        p1[i] += h
        p2[i] -= h
        num[k] = (f(p1) - f(p2)) / (2 * h)
    scale = np.abs(grad).max()
    np.testing.assert_allclose(grad[idx], num, rtol=1e-5, atol=1e-7 * scale)
    # the probes saw non-zero gradient in most tensors
    assert (np.abs(num) > 1e-9 * scale).sum() > 0.5 * len(idx)


def _shape_offsets(n_out):
    out, o = {}, 0
    for name, shape, _ in synth.policy_shapes(synth.PolicyDims(D, L, H, n_out)):
        out[name] = (o, int(np.prod(shape)))
        o += int(np.prod(shape))
    return out


def test_actor_gradient_matches_finite_differences():
    prm = _net(NACT)
    tok, ne, h = _batch(6)
    logits, _ = oracle.tfm_forward(prm, D, L, H, NACT, tok, ne, h)
    rng = np.random.default_rng(9)
    act = rng.integers(0, NACT, 6).astype(np.int32)
    lp, _ = _logp(logits, act)
    # ratios 1.1, 0.9, 1.5, 0.6, 1.0, 1.3 against advantages of both signs:
    # unclipped, clipped adverse and clipped favourable samples
    logp_old = lp - np.log([1.1, 0.9, 1.5, 0.6, 1.0, 1.3])
    adv = np.array([0.7, -1.2, 0.4, 0.9, -0.3, -0.8])

    def f(p):
        return oracle.tfm_loss_grad(p, D, L, H, NACT, oracle.ACTOR, tok, ne, h, act, logp_old, adv, 0.2, 0.05,
                                    want_grad=False)[0]

    loss, g, st = oracle.tfm_loss_grad(prm, D, L, H, NACT, oracle.ACTOR, tok, ne, h, act, logp_old, adv, 0.2, 0.05)
    assert loss == pytest.approx(f(prm), rel=1e-14)
    _fd_check(f, prm, g)
    # every tensor receives gradient except the recurrent input (data)
    for name, (o, n) in _shape_offsets(NACT).items():
        assert np.abs(g[o:o + n]).max() > 0, name
    assert st[2] == pytest.approx(3 / 6)  # ratios 1.5, 0.6, 1.3 lie outside [0.8, 1.2]


def test_critic_gradient_matches_finite_differences():
    prm = _net(1, seed=4)
    tok, ne, h = _batch(5, seed=7, ns=7)
    ret = np.array([0.3, -0.5, 1.2, 0.0, 0.8])

    def f(p):
        return oracle.tfm_loss_grad(p, D, L, H, 1, oracle.CRITIC, tok, ne, h, returns=ret, want_grad=False)[0]

    loss, g, st = oracle.tfm_loss_grad(prm, D, L, H, 1, oracle.CRITIC, tok, ne, h, returns=ret)
    _fd_check(f, prm, g, seed=1)
    v, _ = oracle.tfm_forward(prm, D, L, H, 1, tok, ne, h)
    assert loss == pytest.approx(np.mean((v[:, 0] - ret) ** 2), rel=1e-13)
    assert st[1] == pytest.approx(v[:, 0].mean(), rel=1e-13)


def test_ratio_one_is_the_policy_gradient():
    prm = _net(NACT, seed=6)
    tok, ne, h = _batch(5, seed=11)
    act = np.array([0, 4, 2, 1, 3], np.int32)
    adv = np.array([1.0, -0.5, 0.25, 2.0, -1.5])
    logits, _ = oracle.tfm_forward(prm, D, L, H, NACT, tok, ne, h)
    lp, _ = _logp(logits, act)
    loss, g, st = oracle.tfm_loss_grad(prm, D, L, H, NACT, oracle.ACTOR, tok, ne, h, act, lp, adv, 0.2, 0.0)
    assert loss == pytest.approx(-adv.mean(), rel=1e-12)
    assert st[2] == 0.0 and st[3] == pytest.approx(0.0, abs=1e-14)

    def pg(p):  # -mean(A log pi(a)) from the forward logits only
        lg, _ = oracle.tfm_forward(p, D, L, H, NACT, tok, ne, h)
        return -np.mean(adv * _logp(lg, act)[0])

    _fd_check(pg, prm, g, seed=2)


def test_clipped_adverse_samples_carry_no_gradient():
    prm = _net(NACT, seed=8)
    tok, ne, h = _batch(4, seed=13)
    act = np.array([1, 2, 3, 0], np.int32)
    logits, _ = oracle.tfm_forward(prm, D, L, H, NACT, tok, ne, h)
    lp, _ = _logp(logits, act)
    # A > 0 with r = 1.5 and A < 0 with r = 0.6: the clipped term is the min
    adverse = oracle.tfm_loss_grad(prm, D, L, H, NACT, oracle.ACTOR, tok, ne, h, act,
                                   lp - np.log([1.5, 0.6, 1.5, 0.6]), np.array([1.0, -1.0, 2.0, -0.5]), 0.2, 0.0)
    assert np.all(adverse[1] == 0.0)
    assert adverse[0] == pytest.approx(-np.mean([1.2, -0.8, 2.4, -0.4]), rel=1e-14)
    # the favourable side (A > 0, r = 0.6) keeps the unclipped gradient
    fav = oracle.tfm_loss_grad(prm, D, L, H, NACT, oracle.ACTOR, tok, ne, h, act, lp - np.log(0.6),
                               np.ones(4), 0.2, 0.0)
    one = oracle.tfm_loss_grad(prm, D, L, H, NACT, oracle.ACTOR, tok, ne, h, act, lp, np.ones(4), 0.2, 0.0)
    np.testing.assert_allclose(fav[1], 0.6 * one[1], rtol=1e-12, atol=1e-15)


def test_entropy_bonus_from_the_logits():
    prm = _net(NACT, seed=10)
    tok, ne, h = _batch(6, seed=17)
    logits, _ = oracle.tfm_forward(prm, D, L, H, NACT, tok, ne, h)
    act = np.zeros(6, np.int32)
    lp, ls = _logp(logits, act)
    ent = -(np.exp(ls) * ls).sum(1)
    loss, _, st = oracle.tfm_loss_grad(prm, D, L, H, NACT, oracle.ACTOR, tok, ne, h, act, lp, np.zeros(6), 0.2, 0.3)
    assert st[1] == pytest.approx(ent.mean(), rel=1e-13)
    assert loss == pytest.approx(-0.3 * ent.mean(), rel=1e-13)


def test_forward_agrees_with_the_agent_forward():
    """The training forward and the agent's inference forward are separate
    oracle codes of the same network."""
    dims = synth.PolicyDims(D, L, H, NACT)
    prm = synth.policy_params(dims, seed=12)
    tok, ne, h = _batch(7, seed=19)
    a, ha = oracle.tfm_forward(prm, D, L, H, NACT, tok, ne, h)
    b, hb = oracle.policy_forward(prm, D, L, H, tok, ne, h, n_act=NACT)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ha, hb, rtol=1e-12, atol=1e-12)


def test_critic_value_is_invariant_to_entity_order():
    prm = _net(1, seed=14)
    tok, ne, h = _batch(4, seed=23, ns=8)
    ne[:] = 8
    v, hv = oracle.tfm_forward(prm, D, L, H, 1, tok, ne, h)
    perm = np.random.default_rng(1).permutation(8)
    v2, hv2 = oracle.tfm_forward(prm, D, L, H, 1, tok[:, perm], ne, h)
    np.testing.assert_allclose(v2, v, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(hv2, hv, rtol=1e-12, atol=1e-13)


def _rv(T, E, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((T, E)), rng.standard_normal((T + 1, E))


def test_gae_lambda_zero_is_the_td_error():
    T, E, gam = 7, 3, 0.9
    r, v = _rv(T, E, 1)
    done = np.zeros((T, E), np.int32)
    done[3, 1] = 1
    adv, ret = oracle.gae(r, v, done, gam, 0.0)
    td = r + gam * (1 - done) * v[1:] - v[:-1]
    np.testing.assert_allclose(adv, td, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(ret, td + v[:-1], rtol=1e-14, atol=1e-14)


def test_gae_lambda_one_is_return_minus_value():
    T, E = 6, 2
    r, v = _rv(T, E, 2)
    done = np.zeros((T, E), np.int32)
    done[2, 0] = 1  # env 0's episode ends after step 2
    adv, ret = oracle.gae(r, v, done, 1.0, 1.0)
    for t in range(T):
        # env 1: undiscounted return to the batch end, bootstrapped with V_T
        assert adv[t, 1] == pytest.approx(r[t:, 1].sum() + v[T, 1] - v[t, 1], rel=1e-13)
        end = 3 if t <= 2 else T
        boot = 0.0 if t <= 2 else v[T, 0]
        assert adv[t, 0] == pytest.approx(r[t:end, 0].sum() + boot - v[t, 0], rel=1e-13)


def test_gae_satisfies_the_backward_recursion():
    T, E, gam, lam = 9, 4, 0.97, 0.8
    r, v = _rv(T, E, 3)
    done = (np.random.default_rng(4).random((T, E)) < 0.2).astype(np.int32)
    adv, _ = oracle.gae(r, v, done, gam, lam)
    nd = 1 - done
    delta = r + gam * nd * v[1:] - v[:-1]
    np.testing.assert_allclose(adv[-1], delta[-1], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(adv[:-1], delta[:-1] + gam * lam * nd[:-1] * adv[1:], rtol=1e-12, atol=1e-13)


def test_state_tokens_describe_the_true_state():
    p = preset("fleet5", n_envs=3).replace(n_particles=16, d_model=0)
    o = oracle.OracleEnv(p, 3)
    o.reset(0)
    o.step(o.random_actions(1))
    tok, ne = oracle.state_tokens(o)
    A, T, S = p.max_agents, p.max_targets, p.feature_scale
    assert tok.shape == (3, A + T, 8) and np.all(ne == A + T)
    a = o.arr
    for e in range(3):
        for b in range(A):
            q, i = tok[e, b], e * A + b
            np.testing.assert_allclose(q[:3], [a["ax"][i] / S, a["ay"][i] / S, 0.0], rtol=1e-15)
            assert np.hypot(q[3], q[4]) == pytest.approx(p.agent_speed, rel=1e-14)
            assert q[5] ** 2 + q[6] ** 2 == pytest.approx(1.0, rel=1e-14) and q[7] == 1.0
            assert np.arctan2(q[6], q[5]) == pytest.approx(np.arctan2(np.sin(a["apsi"][i]), np.cos(a["apsi"][i])))
        for k in range(T):
            q, i = tok[e, A + k], e * T + k
            np.testing.assert_allclose(q[:3], [a["tx"][i] / S, a["ty"][i] / S, a["tz"][i] / S], rtol=1e-15)
            assert np.hypot(q[3], q[4]) == pytest.approx(a["tspeed"][i], rel=1e-14) and q[7] == 0.0


def test_state_token_velocities_are_the_next_displacement():
    """Without heading noise and target drift, and with every agent steering
    straight, each entity's next displacement divided by dt is the velocity
    its token reported."""
    p = preset("fleet5", n_envs=3).replace(n_particles=16, d_model=0, heading_noise=0.0, target_drift_sigma=0.0)
    o = oracle.OracleEnv(p, 4)
    o.reset(0)
    o.step(o.random_actions(1))
    tok0, _ = oracle.state_tokens(o)
    o.step(np.full(o.NA, 3, np.int32))  # the middle rudder angle: no turn
    tok1, _ = oracle.state_tokens(o)
    S, dt = p.feature_scale, p.dt
    vel = (tok1[:, :, :2] - tok0[:, :, :2]) * S / dt
    np.testing.assert_allclose(vel, tok0[:, :, 3:5], rtol=1e-9, atol=1e-9)
    assert np.abs(tok0[:, :, 3:5]).max() > 0.1

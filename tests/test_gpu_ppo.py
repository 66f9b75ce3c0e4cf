"""TransfMAPPO training path (Sec. II-B, Sec. III-B.1, Fig. 3) on the GPU
against the FP64 oracle: the transformer forward, the PPO actor and critic
loss gradients, Adam, GAE, the critic's state tokens and the rollout
recording.  The linear layers' GEMMs run on either path of the library:

* FP32 CUDA cores (tensor_cores=False): unit roundoff u = 6e-8; each output
  is a chain of dot products of length K <= 4d = 512, LayerNorms and erf/exp,
  so errors stay near sqrt(K) u per stage, a few 1e-6 after L blocks; the
  tests allow 1e-4 absolute + 1e-4 relative on outputs and, on gradients,
  2e-4 of each tensor's largest entry element-wise and 2e-4 relative in norm.
* BF16 tensor cores (tensor_cores=True, the default): every GEMM operand is
  rounded to BF16 (u = 2^-8) and accumulated in FP32, everything else is
  FP32.  A dot product of rounded operands moves by about u times the
  magnitude of its terms, and a forward value passes 4 L GEMMs and L
  LayerNorms (which rescale the errors with the rows), a gradient up to 12 L
  GEMMs.  Measured over these cases: 1.3e-2 on outputs, 2.3e-2 on the
  recurrent embedding, 1.3e-2 of a tensor's largest entry on gradients;
  BF16_TOL below keeps a factor of two to three above those.

PPO ratios are set away from the clip boundaries (0.5, 0.9, 1.0, 1.1, 1.5
with eps = 0.2) so that rounding cannot flip a clip decision."""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import preset

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_08222_gb300 as ut  # noqa: E402
from paper_2505_08222_gb300 import ppo  # noqa: E402

RATIOS = np.array([0.5, 0.9, 1.0, 1.1, 1.5])


def _bf16_dev(x):
    return torch.from_numpy(synth.bf16_bits(x).view(np.int16)).cuda()


def _inputs(n, NS, d, seed, bf16=True):
    rng = np.random.default_rng(seed)
    n_ent = rng.integers(0, NS + 1, n).astype(np.int32)
    n_ent[:2] = NS
    tok = synth.random_tokens(n, NS, n_ent, seed=seed + 1)
    if not bf16:
        tok = (tok + 0.01 * rng.standard_normal(tok.shape)).astype(np.float32)
    h = (0.5 * rng.standard_normal((n, d))).astype(np.float32)
    tok_dev = _bf16_dev(tok) if bf16 else torch.from_numpy(tok).cuda()
    return tok, n_ent, h, tok_dev, torch.from_numpy(n_ent).cuda(), torch.from_numpy(h).cuda()


# bounds of the BF16 tensor-core path: outputs (absolute + relative), gradients
# (fraction of each tensor's largest entry, element-wise and in norm)
BF16_TOL = {"out_atol": 4e-2, "out_rtol": 2e-2, "grad": 4e-2}
FP32_TOL = {"out_atol": 1e-4, "out_rtol": 1e-4, "grad": 2e-4}


def _tol(tc):
    return BF16_TOL if tc else FP32_TOL


def _close(got, ref, atol=1e-4, rtol=1e-4):
    err = np.abs(got - ref)
    assert np.all(err <= atol + rtol * np.abs(ref)), float(err.max())
    return float(err.max())


def _close_tc(got, ref, tc):
    t = _tol(tc)
    return _close(got, ref, t["out_atol"], t["out_rtol"])


def _grad_close(got, ref, shapes, tol=2e-4):
    o = 0
    worst = 0.0
    for name, shape, _ in shapes:
        n = int(np.prod(shape))
        g, r = got[o:o + n], ref[o:o + n]
        scale = np.abs(r).max()
        assert scale > 0, name
        e = np.abs(g - r).max() / scale
        rn = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert e <= tol and rn <= tol, (name, e, rn)
        worst = max(worst, e)
        o += n
    assert o == len(ref)
    return worst


CASES = {
    # name: (d, L, H, n_out, NS, bf16 tokens, n)
    "actor64": (64, 2, 4, 7, 10, True, 257),
    "critic64": (64, 2, 4, 1, 10, False, 200),
    "actor128": (128, 3, 8, 7, 16, True, 48),
    "small32": (32, 1, 4, 5, 6, True, 70),
}


@pytest.mark.parametrize("tc", [False, True])
@pytest.mark.parametrize("case", list(CASES))
def test_forward_matches_oracle(case, tc):
    d, L, H, no, NS, bf, n = CASES[case]
    prm = synth.policy_params(synth.PolicyDims(d, L, H, no), seed=31)
    net = ppo.Tfm(prm, d, L, H, no, NS, n + 5, bf, tensor_cores=tc)
    tok, ne, h, tok_d, ne_d, h_d = _inputs(n, NS, d, 3, bf)
    h_out = torch.empty_like(h_d)
    out = net.forward(tok_d, ne_d, h_d, h_out=h_out).cpu().numpy()
    ref, ref_h = oracle.tfm_forward(prm, d, L, H, no, tok, ne, h)
    e1 = _close_tc(out, ref, tc)
    e2 = _close_tc(h_out.cpu().numpy(), ref_h, tc)
    # rows selected through sel: a permutation with repeats
    sel = np.random.default_rng(4).integers(0, n, n + 5).astype(np.int32)
    out2 = net.forward(tok_d, ne_d, h_d, sel=torch.from_numpy(sel).cuda()).cpu().numpy()
    _close_tc(out2, ref[sel], tc)
    print(f"{case} tc={tc}: max |dout| {e1:.2e}, |dh| {e2:.2e}")


def _ppo_args(prm, d, L, H, no, tok, ne, h, seed):
    n = len(ne)
    logits, _ = oracle.tfm_forward(prm, d, L, H, no, tok, ne, h)
    rng = np.random.default_rng(seed)
    act = rng.integers(0, no, n).astype(np.int32)
    m = logits.max(1, keepdims=True)
    ls = logits - m - np.log(np.exp(logits - m).sum(1, keepdims=True))
    lp = ls[np.arange(n), act]
    logp_old = (lp - np.log(RATIOS[rng.integers(0, len(RATIOS), n)])).astype(np.float32)
    adv = rng.standard_normal(n).astype(np.float32)
    return act, logp_old, adv


@pytest.mark.parametrize("tc", [False, True])
@pytest.mark.parametrize("case", ["actor64", "actor128", "small32"])
def test_actor_gradient_matches_oracle(case, tc):
    d, L, H, no, NS, bf, n = CASES[case]
    prm = synth.policy_params(synth.PolicyDims(d, L, H, no), seed=37)
    net = ppo.Tfm(prm, d, L, H, no, NS, n, bf, tensor_cores=tc)
    tok, ne, h, tok_d, ne_d, h_d = _inputs(n, NS, d, 7, bf)
    act, logp_old, adv = _ppo_args(prm, d, L, H, no, tok, ne, h, 8)
    st = net.actor_grad(tok_d, ne_d, h_d, torch.from_numpy(act).cuda(), torch.from_numpy(logp_old).cuda(),
                        torch.from_numpy(adv).cuda(), clip_eps=0.2, ent_coef=0.01)
    loss, g, rst = oracle.tfm_loss_grad(prm, d, L, H, no, oracle.ACTOR, tok, ne, h, act, logp_old, adv, 0.2, 0.01)
    worst = _grad_close(net.grad.cpu().numpy(), g, synth.policy_shapes(synth.PolicyDims(d, L, H, no)),
                        tol=_tol(tc)["grad"])
    st_tol = (2e-2, 2e-3) if tc else (1e-4, 1e-5)
    np.testing.assert_allclose(st[:2], rst[:2], rtol=st_tol[0], atol=st_tol[1])
    assert st[2] == pytest.approx(rst[2], abs=1e-12)  # clipped fraction: the same decisions
    assert st[3] == pytest.approx(rst[3], abs=5e-3 if tc else 1e-4)
    print(f"{case} tc={tc}: worst per-tensor gradient error {worst:.2e}; loss {st[0]:.5f} vs {loss:.5f}")


ATTN_EDGES = {
    # the tensor-core attention kernels' edges (head width 16): 16 tokens
    # (no padded row), 2 tokens (14 padded rows), two samples (fewer items
    # than warps)
    "t16": (32, 1, 2, 5, 15, True, 37),
    "t2": (64, 1, 4, 7, 1, True, 45),
    "two_samples": (64, 2, 4, 7, 10, True, 2),
}


@pytest.mark.parametrize("case", list(ATTN_EDGES))
def test_tensor_core_attention_edges_match_oracle(case):
    """Forward outputs and the actor gradient on the tensor-core path (the
    attention on mma.sync) at token counts 16 and 2 and with two samples."""
    d, L, H, no, NS, bf, n = ATTN_EDGES[case]
    prm = synth.policy_params(synth.PolicyDims(d, L, H, no), seed=53)
    net = ppo.Tfm(prm, d, L, H, no, NS, n, bf, tensor_cores=True)
    tok, ne, h, tok_d, ne_d, h_d = _inputs(n, NS, d, 54, bf)
    h_out = torch.empty_like(h_d)
    out = net.forward(tok_d, ne_d, h_d, h_out=h_out).cpu().numpy()
    ref, ref_h = oracle.tfm_forward(prm, d, L, H, no, tok, ne, h)
    e1 = _close_tc(out, ref, True)
    _close_tc(h_out.cpu().numpy(), ref_h, True)
    act, logp_old, adv = _ppo_args(prm, d, L, H, no, tok, ne, h, 55)
    st = net.actor_grad(tok_d, ne_d, h_d, torch.from_numpy(act).cuda(), torch.from_numpy(logp_old).cuda(),
                        torch.from_numpy(adv).cuda(), clip_eps=0.2, ent_coef=0.01)
    loss, g, rst = oracle.tfm_loss_grad(prm, d, L, H, no, oracle.ACTOR, tok, ne, h, act, logp_old, adv, 0.2, 0.01)
    worst = _grad_close(net.grad.cpu().numpy(), g, synth.policy_shapes(synth.PolicyDims(d, L, H, no)),
                        tol=_tol(True)["grad"])
    np.testing.assert_allclose(st[:2], rst[:2], rtol=2e-2, atol=2e-3)
    print(f"{case}: max |dout| {e1:.2e}, worst per-tensor gradient error {worst:.2e}")


@pytest.mark.parametrize("tc", [False, True])
def test_value_gradient_matches_oracle(tc):
    d, L, H, no, NS, bf, n = CASES["critic64"]
    prm = synth.policy_params(synth.PolicyDims(d, L, H, 1), seed=41)
    net = ppo.Tfm(prm, d, L, H, 1, NS, n, bf, tensor_cores=tc)
    tok, ne, h, tok_d, ne_d, h_d = _inputs(n, NS, d, 9, bf)
    ret = np.random.default_rng(10).standard_normal(n).astype(np.float32)
    st = net.value_grad(tok_d, ne_d, h_d, torch.from_numpy(ret).cuda())
    loss, g, rst = oracle.tfm_loss_grad(prm, d, L, H, 1, oracle.CRITIC, tok, ne, h, returns=ret)
    worst = _grad_close(net.grad.cpu().numpy(), g, synth.policy_shapes(synth.PolicyDims(d, L, H, 1)),
                        tol=_tol(tc)["grad"])
    np.testing.assert_allclose(st[:2], rst[:2], rtol=2e-2 if tc else 1e-4, atol=2e-3 if tc else 1e-5)
    print(f"critic tc={tc}: worst per-tensor gradient error {worst:.2e}")


@pytest.mark.parametrize("tc", [False, True])
def test_gradient_is_deterministic_and_selection_is_a_gather(tc):
    d, L, H, no, NS, bf, n = CASES["actor64"]
    prm = synth.policy_params(synth.PolicyDims(d, L, H, no), seed=43)
    net = ppo.Tfm(prm, d, L, H, no, NS, n, bf, tensor_cores=tc)
    tok, ne, h, tok_d, ne_d, h_d = _inputs(n, NS, d, 11, bf)
    act, logp_old, adv = _ppo_args(prm, d, L, H, no, tok, ne, h, 12)
    a = [torch.from_numpy(x).cuda() for x in (act, logp_old, adv)]
    net.actor_grad(tok_d, ne_d, h_d, *a)
    g1 = net.grad.clone()
    net.actor_grad(tok_d, ne_d, h_d, *a)
    assert torch.equal(g1, net.grad)
    # the same samples in another order through sel: equal to rounding
    perm = torch.from_numpy(np.random.default_rng(13).permutation(n).astype(np.int32)).cuda()
    net.actor_grad(tok_d, ne_d, h_d, *a, sel=perm)
    _grad_close(net.grad.cpu().numpy(), g1.cpu().numpy().astype(np.float64),
                synth.policy_shapes(synth.PolicyDims(d, L, H, no)), tol=1e-5)


def test_adam_matches_oracle():
    d, L, H, no = 32, 1, 4, 5
    prm = synth.policy_params(synth.PolicyDims(d, L, H, no), seed=47)
    net = ppo.Tfm(prm, d, L, H, no, 6, 4, True)
    rng = np.random.default_rng(14)
    th, m, v = prm.astype(np.float64), np.zeros(len(prm)), np.zeros(len(prm))
    for t in range(1, 4):
        g = (rng.standard_normal(len(prm)) * 10.0 ** rng.uniform(-4, 0, len(prm))).astype(np.float32)
        net.adam_step(1e-3, 0.9, 0.999, 1e-8, grad=torch.from_numpy(g).cuda())
        th, m, v = oracle.adam(th, m, v, g, t, lr=1e-3)
    got = net.params().cpu().numpy()
    np.testing.assert_allclose(got, th, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("gamma,lam", [(0.99, 0.95), (1.0, 1.0), (0.9, 0.0)])
def test_gae_matches_oracle(gamma, lam):
    T, E, NA = 37, 300, 900
    rng = np.random.default_rng(15)
    r = rng.standard_normal((T, E)).astype(np.float32)
    v = rng.standard_normal((T + 1, E)).astype(np.float32)
    done = (rng.random((T, E)) < 0.05).astype(np.int32)
    agent_env = np.sort(rng.integers(0, E, NA)).astype(np.int32)
    adv, ret, adv_a = ppo.gae(*(torch.from_numpy(x).cuda() for x in (r, v, done)), gamma, lam,
                              torch.from_numpy(agent_env).cuda())
    ra, rr = oracle.gae(r, v, done, gamma, lam)
    _close(adv.cpu().numpy(), ra, atol=2e-5, rtol=1e-5)
    _close(ret.cpu().numpy(), rr, atol=2e-5, rtol=1e-5)
    assert np.array_equal(adv_a.cpu().numpy(), adv.cpu().numpy()[:, agent_env])


def _policy_env(n_envs=8, name="fleet5", **kw):
    p = preset(name, n_envs=n_envs).replace(n_particles=64, **kw)
    env = ut.Env(p)
    prm = synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, p.n_actions), seed=53)
    env.set_policy(prm)
    return env, p, prm


@pytest.mark.parametrize("name", ["fleet5", "ragged"])
def test_state_tokens_match_oracle(name):
    env, p, _ = _policy_env(n_envs=6, name=name, target_depth_max=30.0)
    env.reset(3)
    for _ in range(3):
        env.step()
    st = env.state()
    NS = env.NS
    tok = torch.zeros((env.E, NS, 8), device="cuda")
    ne = torch.zeros(env.E, dtype=torch.int32, device="cuda")
    assert ut.lib.env_state_tokens(env.h, tok.data_ptr(), ne.data_ptr()) == 0
    a_cnt, t_cnt = p.counts()
    ao = np.concatenate([[0], np.cumsum(a_cnt)])
    to = np.concatenate([[0], np.cumsum(t_cnt)])
    arrs = [st[k].double().cpu().numpy() for k in ("ax", "ay", "apsi", "tx", "ty", "tz", "tpsi", "tspeed")]
    ref, rne = oracle.state_tokens_arrays(ao, to, NS, p.feature_scale, p.agent_speed, *arrs)
    assert np.array_equal(ne.cpu().numpy(), rne) and np.array_equal(rne, a_cnt + t_cnt)
    _close(tok.cpu().numpy(), ref, atol=2e-6, rtol=2e-6)
    assert np.abs(ref[:, :, 2]).max() > 0  # targets at depth


@pytest.mark.parametrize("name", ["fleet5", "ragged"])
def test_snapshot_and_record(name):
    env, p, _ = _policy_env(n_envs=5, name=name)
    env.reset(4)
    env.step()
    NA, NS, d = env.NA, env.NS, p.d_model
    tok = torch.zeros((NA, NS, 8), dtype=torch.int16, device="cuda")
    ne = torch.zeros(NA, dtype=torch.int32, device="cuda")
    h = torch.zeros((NA, d), device="cuda")
    obs_before = env.state()["h"].clone()
    assert ut.lib.env_ppo_snapshot(env.h, tok.data_ptr(), ne.data_ptr(), h.data_ptr()) == 0
    out = env.step()
    obs_prev = tok.clone()
    act = torch.zeros(NA, dtype=torch.int32, device="cuda")
    logp = torch.zeros(NA, device="cuda")
    rew = torch.zeros(env.E, device="cuda")
    done = torch.ones(env.E, dtype=torch.int32, device="cuda")
    assert ut.lib.env_ppo_record(env.h, act.data_ptr(), logp.data_ptr(), rew.data_ptr(), done.data_ptr()) == 0
    torch.cuda.synchronize()
    assert torch.equal(act, out["actions"]) and torch.equal(rew, out["reward"]) and torch.equal(done, out["done"])
    z = out["logits"].double().cpu().numpy()
    m = z.max(1, keepdims=True)
    ls = z - m - np.log(np.exp(z - m).sum(1, keepdims=True))
    np.testing.assert_allclose(logp.cpu().numpy(), ls[np.arange(NA), act.cpu().numpy()], atol=2e-6, rtol=1e-6)
    a_cnt, t_cnt = p.counts()
    assert np.array_equal(ne.cpu().numpy(), np.repeat(a_cnt + t_cnt, a_cnt))
    # h: the BF16 recurrent embedding before the step, widened exactly
    hb = obs_before.view(torch.int16).cpu().numpy().astype(np.uint16).astype(np.uint32) << 16
    assert np.array_equal(h.cpu().numpy().view(np.uint32), hb)
    assert obs_prev.abs().sum() > 0


@pytest.mark.parametrize("tc", [False, True])
def test_full_minibatch_forward_sampled(tc):
    """The bench's actor minibatch (fleet5: 32 steps x 20480 agents / 4)
    through the training forward; 24 sampled samples against the oracle."""
    n, d, L, H, no, NS = 163840, 64, 2, 4, 7, 10
    prm = synth.policy_params(synth.PolicyDims(d, L, H, no), seed=59)
    net = ppo.Tfm(prm, d, L, H, no, NS, n, True, tensor_cores=tc)
    # 40 copies of a 4096-sample block, each copy with its own recurrent input
    tok0, ne0, _, _, _, _ = _inputs(4096, NS, d, 17, True)
    tok, ne = np.tile(tok0, (40, 1, 1)), np.tile(ne0, 40)
    h = (0.5 * np.random.default_rng(19).standard_normal((n, d))).astype(np.float32)
    tok_d, ne_d, h_d = _bf16_dev(tok), torch.from_numpy(ne).cuda(), torch.from_numpy(h).cuda()
    out = net.forward(tok_d, ne_d, h_d).cpu().numpy()
    idx = np.random.default_rng(18).choice(n, 24, replace=False)
    idx[0], idx[1] = 0, n - 1
    ref, _ = oracle.tfm_forward(prm, d, L, H, no, tok[idx], ne[idx], h[idx])
    _close_tc(out[idx], ref, tc)


def test_trainer_fits_the_value_and_moves_the_policy():
    env, p, prm = _policy_env(n_envs=32)
    crit = synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, 1), seed=61)
    tr = ppo.Trainer(env, prm, crit, ppo.PPOConfig(T=16, epochs=1, minibatches=1, lr_critic=1e-3))
    tr.collect(7)
    # one full-batch step per update: the statistics are those before the step
    first = tr.update(7)
    for _ in range(40):
        last = tr.update(7)  # the same batch: the critic fits its fixed returns
    for s in (first, last):
        assert all(np.isfinite(s["actor"])) and all(np.isfinite(s["critic"]))
    assert last["critic"][0] < 0.5 * first["critic"][0], (first["critic"], last["critic"])
    # log-probabilities of the BF16 agent (behaviour) and of the FP32 network agree closely
    assert abs(first["actor"][3]) < 0.02 and first["actor"][2] < 0.01
    # a whole iteration (collect + update) runs, and the env's agent runs the updated weights
    it = tr.iteration(8)
    assert all(np.isfinite(it["actor"])) and all(np.isfinite(it["critic"]))
    env.reset(7)
    o1 = env.step()["logits"].clone()
    env.set_policy(prm)
    env.reset(7)
    o0 = env.step()["logits"].clone()
    assert not torch.equal(o0, o1)


def test_trainer_on_a_ragged_fleet():
    """Agents and targets per env vary: per-agent entity counts, the agent
    -> env advantage map and ragged critic tokens all take part."""
    env, p, prm = _policy_env(n_envs=24, name="ragged")
    a_cnt, t_cnt = p.counts()
    assert len(set(a_cnt.tolist())) > 1 and len(set(t_cnt.tolist())) > 1
    crit = synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, 1), seed=67)
    tr = ppo.Trainer(env, prm, crit, ppo.PPOConfig(T=8, epochs=1, minibatches=2))
    st = tr.iteration(3)
    assert all(np.isfinite(st["actor"])) and all(np.isfinite(st["critic"]))
    T = tr.cfg.T
    assert np.array_equal(tr.ne[0].cpu().numpy(), np.repeat(a_cnt + t_cnt, a_cnt))
    assert np.array_equal(tr.cne[0].cpu().numpy(), a_cnt + t_cnt)
    # every agent carries its env's advantage
    adv_a, adv = tr.adv_a.cpu().numpy(), tr.adv.cpu().numpy()
    assert np.array_equal(adv_a, adv[:, np.repeat(np.arange(p.n_envs), a_cnt)])
    # the recorded GAE against the oracle's on the recorded rewards, values and episode ends
    ra, rr = oracle.gae(tr.rew.cpu().numpy(), tr.val.cpu().numpy(), tr.done.cpu().numpy(), tr.cfg.gamma,
                        tr.cfg.lam)
    _close(adv, ra, atol=2e-5, rtol=1e-5)
    assert adv.shape == (T, p.n_envs)


def test_graph_collection_equals_the_step_by_step_calls():
    env, p, prm = _policy_env(n_envs=16, name="ragged")
    crit = synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, 1), seed=71)
    tr = ppo.Trainer(env, prm, crit, ppo.PPOConfig(T=6, epochs=1, minibatches=1))
    names = ("tok", "ne", "h", "act", "logp", "rew", "done", "ctok", "cne", "ch", "val")
    tr.collect_eager(9)
    eager = {k: getattr(tr, k).clone() for k in names}
    for _ in range(2):  # the captured graph, then its replay
        for k in names:
            getattr(tr, k).fill_(-7)
        tr.collect(9)
        torch.cuda.synchronize()
        for k in names:
            assert torch.equal(getattr(tr, k), eager[k]), k


@pytest.mark.parametrize("tc", [False, True])
def test_actor_gradient_large_minibatch_matches_oracle(tc):
    """Gradient parity at 15,000 samples (165,000 token rows: 1,290 row tiles
    of the GEMMs, weight gradients split over many row ranges)."""
    d, L, H, no, NS, n = 64, 2, 4, 7, 10, 15000
    prm = synth.policy_params(synth.PolicyDims(d, L, H, no), seed=89)
    net = ppo.Tfm(prm, d, L, H, no, NS, n, True, tensor_cores=tc)
    tok, ne, h, tok_d, ne_d, h_d = _inputs(n, NS, d, 90, True)
    act, logp_old, adv = _ppo_args(prm, d, L, H, no, tok, ne, h, 91)
    st = net.actor_grad(tok_d, ne_d, h_d, torch.from_numpy(act).cuda(), torch.from_numpy(logp_old).cuda(),
                        torch.from_numpy(adv).cuda(), clip_eps=0.2, ent_coef=0.01)
    loss, g, rst = oracle.tfm_loss_grad(prm, d, L, H, no, oracle.ACTOR, tok, ne, h, act, logp_old, adv, 0.2, 0.01)
    worst = _grad_close(net.grad.cpu().numpy(), g, synth.policy_shapes(synth.PolicyDims(d, L, H, no)),
                        tol=_tol(tc)["grad"])
    np.testing.assert_allclose(st[:2], rst[:2], rtol=2e-2 if tc else 1e-4, atol=2e-3 if tc else 1e-5)
    print(f"large minibatch tc={tc}: worst per-tensor gradient error {worst:.2e}")

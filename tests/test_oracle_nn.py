"""Pins of the oracle's neural parts: the transformer agent against PyTorch's
own pre-LN encoder layer in float64 (a library routine), permutation
invariance over entity tokens (Sec. III-B.1), the estimator MLP's gradients
against central finite differences and autograd, Adam against its closed form
on a constant gradient and against torch.optim.Adam."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth


def _split(params, shapes):
    out, o = {}, 0
    for name, shape, _ in shapes:
        n = int(np.prod(shape))
        out[name] = params[o:o + n].reshape(shape)
        o += n
    assert o == len(params)
    return out


def _torch_policy(params, dims, tokens, n_ent, h):
    """Same network assembled from torch.nn.TransformerEncoderLayer(norm_first)."""
    d = dims.d
    W = {k: torch.tensor(v, dtype=torch.float64) for k, v in _split(params, synth.policy_shapes(dims)).items()}
    n, ns, _ = tokens.shape
    x = torch.zeros(n, 1 + ns, d, dtype=torch.float64)
    x[:, 0] = torch.tensor(h, dtype=torch.float64)
    x[:, 1:] = torch.tensor(tokens, dtype=torch.float64) @ W["W_emb"].T + W["b_emb"]
    pad = torch.arange(1 + ns)[None, :] > torch.tensor(n_ent)[:, None]
    for l in range(dims.n_layers):
        layer = torch.nn.TransformerEncoderLayer(d, dims.n_heads, 4 * d, dropout=0.0, activation="gelu",
                                                 layer_norm_eps=1e-5, batch_first=True, norm_first=True,
                                                 dtype=torch.float64)
        with torch.no_grad():
            layer.self_attn.in_proj_weight.copy_(W[f"Wqkv{l}"])
            layer.self_attn.in_proj_bias.copy_(W[f"bqkv{l}"])
            layer.self_attn.out_proj.weight.copy_(W[f"Wo{l}"])
            layer.self_attn.out_proj.bias.copy_(W[f"bo{l}"])
            layer.linear1.weight.copy_(W[f"W1{l}"])
            layer.linear1.bias.copy_(W[f"b1{l}"])
            layer.linear2.weight.copy_(W[f"W2{l}"])
            layer.linear2.bias.copy_(W[f"b2{l}"])
            layer.norm1.weight.copy_(W[f"ln1_g{l}"])
            layer.norm1.bias.copy_(W[f"ln1_b{l}"])
            layer.norm2.weight.copy_(W[f"ln2_g{l}"])
            layer.norm2.bias.copy_(W[f"ln2_b{l}"])
        layer.eval()
        with torch.no_grad():
            # the plain (non fast-path) math: training-mode flag off, no nested tensors
            x = layer._sa_block(layer.norm1(x), None, pad, False) + x
            x = x + layer._ff_block(layer.norm2(x))
    hr = x[:, 0]
    z = torch.nn.functional.layer_norm(hr, (d,), W["lnf_g"], W["lnf_b"], 1e-5)
    return (z @ W["Wh"].T + W["bh"]).numpy(), hr.numpy()


@pytest.mark.parametrize("d,L,H", [(64, 2, 4), (32, 1, 2), (128, 3, 8)])
def test_policy_matches_torch_encoder(d, L, H):
    dims = synth.PolicyDims(d, L, H)
    params = synth.policy_params(dims, seed=d + L)
    n, ns = 9, 16
    rng = np.random.default_rng(0)
    n_ent = rng.integers(1, ns + 1, n).astype(np.int32)
    tok = synth.random_tokens(n, ns, n_ent, seed=1)
    h = synth.round_bf16(rng.standard_normal((n, d)).astype(np.float32))
    logits, h_out = oracle.policy_forward(params, d, L, H, tok, n_ent, h)
    tl, th = _torch_policy(params, dims, tok, n_ent, h)
    np.testing.assert_allclose(logits, tl, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(h_out, th, rtol=1e-10, atol=1e-10)


def test_policy_entity_permutation_invariance():
    dims = synth.PolicyDims(64, 2, 4)
    params = synth.policy_params(dims)
    n, ns = 6, 10
    n_ent = np.full(n, 10, np.int32)
    tok = synth.random_tokens(n, ns, n_ent, seed=3)
    h = synth.round_bf16(np.random.default_rng(4).standard_normal((n, 64)).astype(np.float32))
    base, hb = oracle.policy_forward(params, 64, 2, 4, tok, n_ent, h)
    perm = np.random.default_rng(5).permutation(ns)
    pl, ph = oracle.policy_forward(params, 64, 2, 4, tok[:, perm], n_ent, h)
    np.testing.assert_allclose(pl, base, atol=1e-12)
    np.testing.assert_allclose(ph, hb, atol=1e-12)


def test_policy_single_token_reduces_to_value_path():
    """With no entities the attention over one token returns its value row:
    x1 = h + Wo (Wv LN1(h) + bv) + bo, then the FFN residual."""
    dims = synth.PolicyDims(32, 1, 2)
    params = synth.policy_params(dims, seed=7)
    W = _split(params.astype(np.float64), synth.policy_shapes(dims))
    h = np.random.default_rng(8).standard_normal((1, 32))

    def ln(x, g, b):
        return (x - x.mean()) / math.sqrt(x.var() + 1e-5) * g + b

    v = W["Wqkv0"][64:] @ ln(h[0], W["ln1_g0"], W["ln1_b0"]) + W["bqkv0"][64:]
    x = h[0] + W["Wo0"] @ v + W["bo0"]
    z = W["W10"] @ ln(x, W["ln2_g0"], W["ln2_b0"]) + W["b10"]
    z = np.array([0.5 * t * (1 + math.erf(t / math.sqrt(2))) for t in z])
    x = x + W["W20"] @ z + W["b20"]
    logits = W["Wh"] @ ln(x, W["lnf_g"], W["lnf_b"]) + W["bh"]
    tok = np.zeros((1, 4, 8), np.float32)
    lo, ho = oracle.policy_forward(params, 32, 1, 2, tok, np.zeros(1, np.int32), h)
    np.testing.assert_allclose(ho[0], x, atol=1e-12)
    np.testing.assert_allclose(lo[0], logits, atol=1e-12)


def test_gumbel_max_distribution():
    """Gumbel-max sampling draws action j with probability softmax(logits)_j."""
    logits = np.array([[0.3, -1.0, 2.0, 0.0, 0.5, -0.2, 1.1]])
    p = np.exp(logits[0]) / np.exp(logits[0]).sum()
    counts = np.zeros(7)
    for g in range(20000):
        a, _ = oracle.gumbel_actions(11, g, logits)
        counts[a[0]] += 1
    np.testing.assert_allclose(counts / counts.sum(), p, atol=0.012)


# ----------------------------------------------------------------- estimator
def _torch_mlp(params, X):
    W = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True)
         for k, v in _split(params.astype(np.float64), synth.mlp_shapes()).items()}
    x = torch.tensor(X, dtype=torch.float64)
    for l in range(1, 4):
        x = torch.nn.functional.gelu(x @ W[f"W{l}"].T + W[f"b{l}"])
    return x @ W["W4"].T + W["b4"], W


def test_mlp_forward_and_grad_match_autograd():
    params = synth.mlp_params(seed=1, bias_scale=0.1)
    X = synth.random_features(37, seed=2)
    Y = np.random.default_rng(3).standard_normal((37, 2)) * 0.3
    out = oracle.mlp_forward(params, X)
    loss, grad = oracle.mlp_loss_grad(params, X, Y)
    to, W = _torch_mlp(params, X)
    tl = ((to - torch.tensor(Y)) ** 2).sum() / (2 * 37)
    tl.backward()
    np.testing.assert_allclose(out, to.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert loss == pytest.approx(tl.item(), rel=1e-12)
    tg = np.concatenate([W[name].grad.numpy().ravel() for name, _, _ in synth.mlp_shapes()])
    np.testing.assert_allclose(grad, tg, rtol=1e-9, atol=1e-13)


def test_mlp_grad_central_differences():
    params = synth.mlp_params(seed=5, bias_scale=0.1).astype(np.float64)
    X = synth.random_features(5, seed=6)
    Y = np.random.default_rng(7).standard_normal((5, 2)) * 0.3
    _, grad = oracle.mlp_loss_grad(params, X, Y)
    rng = np.random.default_rng(8)
    n = oracle.mlp_param_count()
    idx = np.concatenate([rng.integers(0, n, 40), [n - 1, n - 3, 0, 24576, 24576 + 256 + 5]])
    h = 1e-5
    for i in idx:
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        fd = (oracle.mlp_loss_grad(p1, X, Y)[0] - oracle.mlp_loss_grad(p2, X, Y)[0]) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_mlp_huber_matches_torch_huber_loss():
    """The Huber loss of the training step against torch's huber_loss
    (summed over outputs, averaged over rows) and autograd; the threshold is
    chosen so that residuals fall on both sides of it."""
    params = synth.mlp_params(seed=11, bias_scale=0.1)
    X = synth.random_features(41, seed=12)
    Y = np.random.default_rng(13).standard_normal((41, 2)) * 0.5
    delta = 0.3
    loss, grad = oracle.mlp_loss_grad(params, X, Y, huber=delta)
    to, W = _torch_mlp(params, X)
    e = np.abs(to.detach().numpy() - Y)
    assert np.mean(e > delta) > 0.2 and np.mean(e < delta) > 0.2
    tl = torch.nn.functional.huber_loss(to, torch.tensor(Y), reduction="sum", delta=delta) / 41
    tl.backward()
    assert loss == pytest.approx(tl.item(), rel=1e-12)
    tg = np.concatenate([W[name].grad.numpy().ravel() for name, _, _ in synth.mlp_shapes()])
    np.testing.assert_allclose(grad, tg, rtol=1e-9, atol=1e-13)


def test_mlp_huber_constant_network_closed_form():
    """All weights zero and output bias c: every row outputs c, so
    L = mean_r sum_c rho(c - y) and dL/db4 = mean_r clip(c - y, -delta, delta)
    with every other gradient zero (GELU(0) = 0); delta = 0 is the squared error."""
    n = oracle.mlp_param_count()
    params = np.zeros(n)
    c = np.array([0.4, -1.1])
    params[-2:] = c
    X = synth.random_features(9, seed=1)
    Y = np.random.default_rng(2).standard_normal((9, 2))
    for delta in (0.0, 0.5, 100.0):
        loss, grad = oracle.mlp_loss_grad(params, X, Y, huber=delta)
        e = c - Y
        if delta == 0.0:
            rho, d = 0.5 * e * e, e
        else:
            rho = np.where(np.abs(e) <= delta, 0.5 * e * e, delta * (np.abs(e) - 0.5 * delta))
            d = np.clip(e, -delta, delta)
        assert loss == pytest.approx(rho.sum() / 9, rel=1e-13)
        np.testing.assert_allclose(grad[-2:], d.mean(axis=0), rtol=1e-13, atol=1e-15)
        assert np.all(grad[:-2] == 0.0)
    # a threshold above every residual leaves the squared error unchanged
    assert oracle.mlp_loss_grad(params, X, Y, huber=100.0)[0] == pytest.approx(
        oracle.mlp_loss_grad(params, X, Y)[0], rel=1e-15)


def test_adam_closed_form_constant_gradient():
    """With a constant gradient g, bias-corrected moments are exactly g and
    g^2, so every step moves theta by -lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 51):
        th, m, v = oracle.adam(th, m, v, g, t, lr=1e-2)
    np.testing.assert_allclose(th, -50 * 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-10, atol=1e-15)


def test_adam_matches_torch():
    rng = np.random.default_rng(0)
    theta = rng.standard_normal(50)
    p = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    m, v = np.zeros(50), np.zeros(50)
    for t in range(1, 21):
        g = rng.standard_normal(50)
        theta, m, v = oracle.adam(theta, m, v, g, t, lr=3e-3)
        p.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(theta, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def _learned_env(**kw):
    from synth import preset
    p = preset("fleet5", n_envs=3).replace(n_particles=64, d_model=0, **kw)
    o = oracle.OracleEnv(p, 5)
    o.reset(0)
    for t in range(1, 4):
        o.step(o.random_actions(t))
    return o


def _const_net(c0, c1):
    prm = np.zeros(oracle.mlp_param_count())
    prm[-2:] = (c0, c1)  # b4: the network outputs (c0, c1) for every input
    return prm


def test_learned_step_update_rule_closed_forms():
    """The learned tracker's update with a constant-output network
    (all weights zero, output bias (c0, c1)): with a fresh ping the estimate
    moves by L clamp(c, +-3); without one it is held (mode 1), moved all the
    same (mode 2) or coasts by the smoothed motion (mode 3)."""
    L = 100.0
    for mode in (1, 2, 3):
        o = _learned_env(det_radius=130.0)
        e0x, e0y = o.arr["estx"].copy(), o.arr["esty"].copy()
        p0x, p0y = o.arr["prev_estx"].copy(), o.arr["prev_esty"].copy()
        v0x = o.arr["velx"].copy()
        o.step(o.random_actions(4), mlp=_const_net(0.5, -4.0), mode=mode)
        feat, _ = o.est_features(o.step_count)
        fresh = (feat[:, 3] == 0) & (feat[:, 4] == 1)
        assert 0 < fresh.sum() < o.F
        np.testing.assert_allclose(o.arr["prev_estx"], e0x)
        np.testing.assert_allclose(o.arr["velx"], 0.85 * v0x + 0.15 * (e0x - p0x), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(o.arr["estx"][fresh], e0x[fresh] + 0.5 * L, rtol=1e-12)
        np.testing.assert_allclose(o.arr["esty"][fresh], e0y[fresh] - 3.0 * L, rtol=1e-12)
        st = ~fresh
        if mode == 1:
            np.testing.assert_array_equal(o.arr["estx"][st], e0x[st])
        elif mode == 2:
            np.testing.assert_allclose(o.arr["estx"][st], e0x[st] + 0.5 * L, rtol=1e-12)
        else:
            vx = o.arr["velx"][st]
            np.testing.assert_allclose(o.arr["estx"][st], e0x[st] + np.clip(vx, -3 * L, 3 * L), rtol=1e-12)


def test_learned_step_zero_network_holds_estimates():
    """A network that outputs zero leaves every estimate where it was; the
    reported error is then the distance from it to the (moved) target."""
    o = _learned_env()
    e0x, e0y = o.arr["estx"].copy(), o.arr["esty"].copy()
    out = o.step(o.random_actions(4), mlp=np.zeros(oracle.mlp_param_count()), mode=2)
    np.testing.assert_array_equal(o.arr["estx"], e0x)
    np.testing.assert_array_equal(o.arr["esty"], e0y)
    f = np.arange(o.F)
    tgt = (f // 25) * 5 + f % 5  # 5 x 5 fleets: filter (env, agent, target) -> target index
    np.testing.assert_allclose(out["err"], np.hypot(e0x - o.arr["tx"][tgt], e0y - o.arr["ty"][tgt]), rtol=1e-12)

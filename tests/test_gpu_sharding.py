"""Env-sharded batches on the GPU: handles built for consecutive env ranges of
one batch (global id offsets from ``shard.shard_params``) reproduce, bit for
bit, the state of the unsplit batch stepped by a single handle.  Agents act
through the transformer policy (Gumbel-max draws keyed by global agent id),
and the same filter launch variant runs on every handle."""
import numpy as np
import pytest
import torch

import synth
from synth import preset

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_08222_gb300 as ut  # noqa: E402
from paper_2505_08222_gb300 import shard  # noqa: E402

KEYS = ("ax", "ay", "apsi", "tx", "ty", "tz", "px", "py", "pvx", "pvy", "estx", "esty")


def _make(p, learned, variant=None):
    env = ut.Env(p, ring=learned)
    if variant is not None:
        env.set_pf_variant(variant)
    if p.d_model:
        env.set_policy(synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads), seed=5))
    if learned:
        env.est_set_weights(synth.mlp_params(seed=9, bias_scale=0.05))
    return env


def _roll(env, steps, learned):
    env.reset(23)
    rew = []
    for t in range(steps):
        if learned and t == 3:
            env.est_set_mode(True)
        rew.append(env.step()["reward"].clone())
    torch.cuda.synchronize()
    st = env.state()
    return {k: st[k].clone() for k in KEYS}, torch.stack(rew)


@pytest.mark.parametrize("kind,world,learned,kw", [("fleet5", 3, False, {}), ("ragged", 2, False, {}),
                                                  ("fleet5", 2, True, {}), ("ragged", 3, False, {"shared_filter": 1})])
def test_shards_reproduce_whole_batch(kind, world, learned, kw):
    p = preset(kind, n_envs=37, seed=4).replace(n_particles=256, **kw)
    env = _make(p, learned)
    v = env.pf_variant()
    whole, rew = _roll(env, 8, learned)
    parts = [_roll(_make(shard.shard_params(p, r, world), learned, v), 8, learned) for r in range(world)]
    for k in KEYS:
        got = torch.cat([s[k] for s, _ in parts])
        assert torch.equal(got, whole[k]), k
    assert torch.equal(torch.cat([r for _, r in parts], dim=1), rew)

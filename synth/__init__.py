"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds configuration presets, ragged fleet sizes and random
network weights.  It contains none of the method's arithmetic: it only draws
inputs (numpy's seeded generator) and states constants.  Both the FP64 oracle
(``oracle/``) and the CUDA library (``paper_2505_08222_gb300``) consume what it
produces; neither imports the other.

Presets restate the five workloads of the tracking benchmark:

* ``small``     64 envs x 1 agent x 1 target, 1000 particles, random heading
                actions in {-30, 0, +30} deg, target random walk at 0.3 m/s;
* ``fleet5``    4096 envs x 5 agents x 5 targets, 2048 particles, targets at
                U[0.5, 1.5] m/s with N(0, 10 deg) heading drift, transformer
                policy d=64, 2 layers, 4 heads, 7 rudder actions;
* ``ragged``    16384 envs, agents and targets U{1..8} per env, 1024 particles,
                128-step rollout;
* ``learned``   the fleet5 workload with the learned estimator;
* ``large``     65536 envs x 8 x 8, 512 particles, policy d=128, 3 layers, 8 heads.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# Tracking-error scale of features and observation tokens (metres).
FEATURE_SCALE = 1000.0


@dataclass
class EnvParams:
    """Every constant of the environment step (Sec. III-A.2 / III-A.3 of the
    paper plus the readings the paper leaves open)."""

    n_envs: int = 64
    max_agents: int = 1
    max_targets: int = 1
    n_particles: int = 1000
    horizon: int = 200
    agents_per_env: Optional[np.ndarray] = None   # int32 [n_envs], None = max_agents
    targets_per_env: Optional[np.ndarray] = None  # int32 [n_envs], None = max_targets
    dt: float = 30.0
    agent_speed: float = 1.0
    heading_noise: float = 0.0
    action_mode: int = 0            # 0: {-turn, 0, +turn}; 1: rudder angles; 2: rudder, adjacent moves
    n_rudder: int = 5               # action_mode 2: rudder positions
    n_actions: int = 3
    turn_angle: float = math.pi / 6
    rudder_max: float = 0.24
    rudder_gain: float = 1.45 / 0.24
    target_model: int = 0           # 0: heading redrawn each step; 1: drift
    target_speed_min: float = 0.3
    target_speed_max: float = 0.3
    target_drift_sigma: float = math.radians(10.0)
    target_depth_max: float = 0.0
    range_sigma: float = 1.0
    det_radius: float = 1500.0
    comm_radius: float = 1500.0
    comm_drop: float = 0.0
    pf_accel_sigma: float = 0.1
    pf_vcap: float = 1.2 * 0.3
    reward_type: int = 0            # 0: tracking Eq. 1; 1: follow Eq. 2
    eps_min: float = 10.0
    eps_max: float = 50.0
    follow_dmin: float = 50.0
    d_safe: float = 10.0
    spawn_min: float = 50.0
    spawn_radius: float = 100.0
    spawn_tries: int = 64
    feature_scale: float = FEATURE_SCALE
    est_scale: float = 100.0
    # global ids of the first env / agent / target / filter (sharded batches)
    id_env0: int = 0
    id_agent0: int = 0
    id_target0: int = 0
    id_filter0: int = 0
    # transformer agent; d_model == 0 means no policy (random actions)
    d_model: int = 0
    n_layers: int = 0
    n_heads: int = 0
    # 1: one filter per (env, target) fed every ping of the target (C1's
    # alternative); 0: one filter per (env, agent, target)
    shared_filter: int = 0
    id_pair0: int = 0  # global id of the first (agent, target) pair (sharded, shared filters)
    # resampling trigger: 0 every step with a measurement; k in 1..16: when ESS < k/16 P
    pf_ess_num: int = 0

    def counts(self):
        a = (np.full(self.n_envs, self.max_agents, np.int32) if self.agents_per_env is None
             else np.asarray(self.agents_per_env, np.int32))
        t = (np.full(self.n_envs, self.max_targets, np.int32) if self.targets_per_env is None
             else np.asarray(self.targets_per_env, np.int32))
        return a, t

    def replace(self, **kw) -> "EnvParams":
        return dataclasses.replace(self, **kw)


def preset(name: str, n_envs: Optional[int] = None, seed: int = 0) -> EnvParams:
    """The benchmark workloads; ``n_envs`` shrinks a preset for tests."""
    if name == "small":
        p = EnvParams()
    elif name in ("fleet5", "learned"):
        p = EnvParams(n_envs=4096, max_agents=5, max_targets=5, n_particles=2048, horizon=500,
                      heading_noise=0.02, action_mode=1, n_actions=7, target_model=1,
                      target_speed_min=0.5, target_speed_max=1.5, pf_vcap=1.2 * 1.5,
                      reward_type=1, follow_dmin=100.0, d_model=64, n_layers=2, n_heads=4)
    elif name == "ragged":
        p = EnvParams(n_envs=16384, max_agents=8, max_targets=8, n_particles=1024, horizon=128,
                      heading_noise=0.02, action_mode=1, n_actions=7, target_model=1,
                      target_speed_min=0.5, target_speed_max=1.5, pf_vcap=1.2 * 1.5,
                      reward_type=1, follow_dmin=100.0, d_model=64, n_layers=2, n_heads=4)
    elif name == "large":
        p = EnvParams(n_envs=65536, max_agents=8, max_targets=8, n_particles=512, horizon=256,
                      heading_noise=0.02, action_mode=1, n_actions=7, target_model=1,
                      target_speed_min=0.5, target_speed_max=1.5, pf_vcap=1.2 * 1.5,
                      reward_type=1, follow_dmin=100.0, d_model=128, n_layers=3, n_heads=8)
    else:
        raise ValueError(f"unknown preset {name!r}")
    if n_envs is not None:
        p = p.replace(n_envs=n_envs)
    if name == "ragged":
        rng = np.random.default_rng(seed)
        p = p.replace(agents_per_env=rng.integers(1, 9, p.n_envs).astype(np.int32),
                      targets_per_env=rng.integers(1, 9, p.n_envs).astype(np.int32))
    return p


# --------------------------------------------------------------------------
# BF16-representable random weights
# --------------------------------------------------------------------------
def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 value (ties to even); returns
    float32 holding BF16-representable values."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Upper 16 bits of BF16-representable float32 values."""
    return (np.ascontiguousarray(x, np.float32).view(np.uint32) >> 16).astype(np.uint16)


@dataclass
class PolicyDims:
    d: int
    n_layers: int
    n_heads: int
    n_act: int = 7
    n_in: int = 8


def policy_shapes(p: PolicyDims):
    """(name, shape, kind) of the transformer agent's parameters in canonical
    order; kind is 'w' (matrix, fan-in scaled), 'g' (LayerNorm gain) or 'b'."""
    d, f = p.d, 4 * p.d
    out = [("W_emb", (d, p.n_in), "w"), ("b_emb", (d,), "b")]
    for l in range(p.n_layers):
        out += [(f"ln1_g{l}", (d,), "g"), (f"ln1_b{l}", (d,), "b"),
                (f"Wqkv{l}", (3 * d, d), "w"), (f"bqkv{l}", (3 * d,), "b"),
                (f"Wo{l}", (d, d), "w"), (f"bo{l}", (d,), "b"),
                (f"ln2_g{l}", (d,), "g"), (f"ln2_b{l}", (d,), "b"),
                (f"W1{l}", (f, d), "w"), (f"b1{l}", (f,), "b"),
                (f"W2{l}", (d, f), "w"), (f"b2{l}", (d,), "b")]
    out += [("lnf_g", (d,), "g"), ("lnf_b", (d,), "b"),
            ("Wh", (p.n_act, d), "w"), ("bh", (p.n_act,), "b")]
    return out


def mlp_shapes():
    out = []
    for l, (i, o) in enumerate([(96, 256), (256, 256), (256, 256), (256, 2)]):
        out += [(f"W{l + 1}", (o, i), "w"), (f"b{l + 1}", (o,), "b")]
    return out


def random_params(shapes, seed: int, bias_scale: float = 0.1) -> np.ndarray:
    """Random init: matrices N(0, 1/fan_in), LayerNorm gains 1 + bias_scale N,
    biases bias_scale N; every value rounded to BF16.  Flat float32 array."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, shape, kind in shapes:
        if kind == "w":
            v = rng.standard_normal(shape) / math.sqrt(shape[-1])
        elif kind == "g":
            v = 1.0 + bias_scale * rng.standard_normal(shape)
        else:
            v = bias_scale * rng.standard_normal(shape)
        parts.append(round_bf16(v.astype(np.float32)).ravel())
    return np.concatenate(parts).astype(np.float32)


def policy_params(dims: PolicyDims, seed: int = 1234) -> np.ndarray:
    return random_params(policy_shapes(dims), seed)


def mlp_params(seed: int = 4321, bias_scale: float = 0.0) -> np.ndarray:
    return random_params(mlp_shapes(), seed, bias_scale)


def random_tokens(n_agents: int, n_slots: int, n_ent: np.ndarray, seed: int) -> np.ndarray:
    """Observation-like BF16 tokens [n_agents, n_slots, 8]: offsets of order
    0.3, one-hot kinds, flags; slots beyond n_ent are zero padding."""
    rng = np.random.default_rng(seed)
    tok = np.zeros((n_agents, n_slots, 8), np.float32)
    for a in range(n_agents):
        for s in range(int(n_ent[a])):
            tok[a, s, :3] = 0.3 * rng.standard_normal(3)
            tok[a, s, 3 + rng.integers(0, 3)] = 1.0
            tok[a, s, 6] = float(rng.integers(0, 2))
            tok[a, s, 7] = rng.integers(0, 17) / 16.0
    return round_bf16(tok)


def random_features(n_rows: int, seed: int) -> np.ndarray:
    """Estimator-like BF16 feature rows [n_rows, 96] (80 used, 16 zero)."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n_rows, 96), np.float32)
    x[:, :80] = 0.5 * rng.standard_normal((n_rows, 80))
    x[:, 4:80:5] = 1.0
    return round_bf16(x)

"""TransfMAPPO training on the device (Sec. II-B, Sec. III-B.1, Fig. 3).

Argument marshalling over the library's training calls (``include/utrack.h``):
``Tfm`` wraps one FP32 transformer (the actor, or the critic with one
output), ``gae`` the advantage estimator, and ``Trainer`` drives one PPO
iteration — collect T steps of every env with the transformer agent acting,
the critic's values from the true state, GAE, then epochs of minibatch
updates of both networks and the copy of the actor's weights into the env's
agent.  Every arithmetic step runs in the library's kernels; minibatch
orders are seeded permutations passed in as row indices.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _abi, lib, shard

_vp = ctypes.c_void_p


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else _vp(t.data_ptr())


class TfmError(RuntimeError):
    pass


class Tfm:
    """One transformer (actor: n_out = number of actions; critic: n_out = 1)
    with FP32 master weights, Adam moments and activation buffers for
    ``max_batch`` samples."""

    def __init__(self, params: np.ndarray, d_model: int, n_layers: int, n_heads: int, n_out: int, n_slots: int,
                 max_batch: int, tokens_bf16: bool, stream: Optional[int] = None, tensor_cores: bool = True):
        c = _abi.TfmConfig(_abi.UT_ABI_VERSION, d_model, n_layers, n_heads, n_out, n_slots, int(tokens_bf16), 0,
                           max_batch)
        self.cfg = c
        self.n_params = int(lib.tfm_param_count(ctypes.byref(c)))
        if self.n_params < 0:
            raise TfmError("tfm: unsupported configuration")
        prm = np.ascontiguousarray(params, np.float32)
        if prm.size != self.n_params:
            raise TfmError(f"tfm: {prm.size} parameters given, {self.n_params} expected")
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        h = _vp()
        self._check(lib.tfm_create(ctypes.byref(c), prm.ctypes.data_as(_vp), prm.size, _vp(self.stream),
                                   ctypes.byref(h)), "tfm_create", handle=False)
        self.h = h
        self.d, self.n_out, self.n_slots = d_model, n_out, n_slots
        self.grad = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        self.set_gemm_path(tensor_cores)

    def set_gemm_path(self, tensor_cores: bool):
        """True: the linear layers' GEMMs on the tensor cores (BF16 operands,
        FP32 accumulation); False: FP32 on the CUDA cores."""
        self._check(lib.tfm_set_gemm_path(self.h, 1 if tensor_cores else 0), "tfm_set_gemm_path")
        self.tensor_cores = bool(tensor_cores)

    def _check(self, rc, what, handle=True):
        if rc != 0:
            msg = ""
            if handle and getattr(self, "h", None):
                raw = lib.tfm_last_error(self.h)
                msg = raw.decode() if raw else ""
            raise TfmError(f"{what}: {_abi.STATUS.get(rc, rc)} {msg}".strip())

    def close(self):
        if getattr(self, "h", None):
            lib.tfm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> torch.Tensor:
        """Zero-copy view of the master weights."""
        p = _vp()
        self._check(lib.tfm_params(self.h, ctypes.byref(p)), "tfm_params")
        from . import device_view
        return device_view(p.value, (self.n_params,))

    def forward(self, tokens, n_ent, h, sel=None, h_out=None, out=None):
        n = len(sel) if sel is not None else tokens.shape[0]
        if out is None:
            out = torch.empty((n, self.n_out), dtype=torch.float32, device="cuda")
        self._check(lib.tfm_forward(self.h, _ptr(tokens), _ptr(n_ent), _ptr(h), _ptr(sel), n, _ptr(out),
                                    _ptr(h_out)), "tfm_forward")
        return out

    def actor_grad(self, tokens, n_ent, h, actions, logp_old, adv, sel=None, clip_eps=0.2, ent_coef=0.0,
                   stats=True):
        n = len(sel) if sel is not None else tokens.shape[0]
        st = (ctypes.c_double * 4)() if stats else None
        self._check(lib.tfm_ppo_actor_grad(self.h, _ptr(tokens), _ptr(n_ent), _ptr(h), _ptr(sel), n, _ptr(actions),
                                           _ptr(logp_old), _ptr(adv), clip_eps, ent_coef, _ptr(self.grad), st),
                    "tfm_ppo_actor_grad")
        return list(st) if stats else None

    def value_grad(self, tokens, n_ent, h, returns, sel=None, stats=True):
        n = len(sel) if sel is not None else tokens.shape[0]
        st = (ctypes.c_double * 4)() if stats else None
        self._check(lib.tfm_value_grad(self.h, _ptr(tokens), _ptr(n_ent), _ptr(h), _ptr(sel), n, _ptr(returns),
                                       _ptr(self.grad), st), "tfm_value_grad")
        return list(st) if stats else None

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, grad=None):
        self._check(lib.tfm_adam_step(self.h, _ptr(self.grad if grad is None else grad), lr, beta1, beta2, eps),
                    "tfm_adam_step")

    def sync_policy(self, env):
        self._check(lib.tfm_sync_policy(self.h, env.h), "tfm_sync_policy")
        env._policy_ready = True


def gae(reward, value, done, gamma, lam, agent_env=None, stream=None):
    """adv, ret [T, E] (and the per-agent advantages [T, NA] when agent_env
    [NA] gives each agent's env) from reward, done [T, E], value [T+1, E]."""
    T, E = reward.shape
    adv = torch.empty_like(reward)
    ret = torch.empty_like(reward)
    adv_a = None
    NA = 0
    if agent_env is not None:
        NA = agent_env.numel()
        adv_a = torch.empty((T, NA), dtype=torch.float32, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = lib.ppo_gae(_ptr(reward), _ptr(value), _ptr(done), T, E, gamma, lam, _ptr(adv), _ptr(ret), _ptr(agent_env),
                     NA, _ptr(adv_a), _vp(s))
    if rc != 0:
        raise TfmError(f"ppo_gae: {_abi.STATUS.get(rc, rc)}")
    return adv, ret, adv_a


def dp_average(grad: torch.Tensor, n_local: int, group=None) -> int:
    """Data parallelism: every rank holds a gradient of the mean loss over
    its own n_local samples; afterwards each holds the gradient of the mean
    over all ranks' samples (the row-weighted average), so identical Adam
    steps keep the ranks' weights equal.  A rank with no samples passes
    n_local = 0 (its gradient then carries no weight) and must still call,
    so that every rank enters the same collectives.  Returns the total sample
    count (0: no rank had samples, the gradient is left as it is).  No-op
    without an initialised process group of more than one rank."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return n_local
    total = int(shard.reduce_sums([n_local], group)[0])
    if total == 0:  # every rank's slice was empty: nothing to average, no step
        return 0
    shard._weighted_mean_(grad, n_local, total, group)
    return total


@dataclass
class PPOConfig:
    T: int = 64                 # steps collected per iteration
    epochs: int = 4
    minibatches: int = 4
    lr_actor: float = 3e-4
    lr_critic: float = 1e-3
    clip_eps: float = 0.2
    ent_coef: float = 0.01
    gamma: float = 0.99
    lam: float = 0.95
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8


class Trainer:
    """TransfMAPPO on one env batch: the env's transformer agent is the actor
    (its weights copied from the FP32 master after every update), the critic
    reads the true state of each env and keeps its own recurrent embedding
    (zero at reset, carried across the steps of the episode like the
    agents').

    Data parallelism is explicit: given ``group`` (a process group of
    several ranks, one env shard per rank, see ``shard.shard_params``), each
    rank collects its own batch and every minibatch gradient is averaged
    across the group's ranks by sample count before the Adam step
    (``dp_average``).  With ``group=None`` the trainer is one process, even
    when torch.distributed is initialised (e.g. one rank of a job that
    trains alone)."""

    def __init__(self, env, actor_params: np.ndarray, critic_params: np.ndarray, cfg: PPOConfig = PPOConfig(),
                 group=None):
        p = env.params
        self.env, self.cfg, self.group = env, cfg, group
        self.NA, self.E, self.NS, self.d = env.NA, env.E, env.NS, p.d_model
        T = cfg.T
        self.mb_actor = -(-T * self.NA // cfg.minibatches)
        self.mb_critic = -(-T * self.E // cfg.minibatches)
        st = env._stream
        self.actor = Tfm(actor_params, p.d_model, p.n_layers, p.n_heads, p.n_actions, self.NS, self.mb_actor, True,
                         stream=st)
        self.critic = Tfm(critic_params, p.d_model, p.n_layers, p.n_heads, 1, self.NS,
                          max(self.mb_critic, self.E), False, stream=st)
        dev = dict(device="cuda")
        NA, E, NS, d = self.NA, self.E, self.NS, self.d
        self.tok = torch.zeros((T, NA, NS, 8), dtype=torch.int16, **dev)
        self.ne = torch.zeros((T, NA), dtype=torch.int32, **dev)
        self.h = torch.zeros((T, NA, d), dtype=torch.float32, **dev)
        self.act = torch.zeros((T, NA), dtype=torch.int32, **dev)
        self.logp = torch.zeros((T, NA), dtype=torch.float32, **dev)
        self.rew = torch.zeros((T, E), dtype=torch.float32, **dev)
        self.done = torch.zeros((T, E), dtype=torch.int32, **dev)
        self.ctok = torch.zeros((T + 1, E, NS, 8), dtype=torch.float32, **dev)
        self.cne = torch.zeros((T + 1, E), dtype=torch.int32, **dev)
        self.ch = torch.zeros((T + 2, E, d), dtype=torch.float32, **dev)
        self.val = torch.zeros((T + 1, E), dtype=torch.float32, **dev)
        a_cnt, _ = p.counts()
        self.agent_env = torch.from_numpy(np.repeat(np.arange(E, dtype=np.int32), a_cnt)).cuda()
        self.actor.sync_policy(env)

    def _env_call(self, rc, what):
        if rc != 0:
            raw = lib.env_last_error(self.env.h)
            raise TfmError(f"{what}: {_abi.STATUS.get(rc, rc)} {raw.decode() if raw else ''}")

    def collect(self, seed: int):
        """T steps from env_reset(seed) as one CUDA graph (env_ppo_collect):
        actor inputs, actions, behaviour log-probabilities, rewards, episode
        ends, critic tokens and values (T + 1 of them: the last bootstraps)."""
        self.env.reset(seed)
        self.ch[0].zero_()
        b = self._buffers()
        self._env_call(lib.env_ppo_collect(self.env.h, self.critic.h, self.cfg.T, ctypes.byref(b)), "env_ppo_collect")

    def _buffers(self):
        if getattr(self, "_bufs", None) is None:
            self._bufs = _abi.PpoBuffers(*[t.data_ptr() for t in (self.tok, self.ne, self.h, self.act, self.logp,
                                                                   self.rew, self.done, self.ctok, self.cne, self.ch,
                                                                   self.val)])
        return self._bufs

    def collect_eager(self, seed: int):
        """The same collection as separate calls, step by step."""
        env, T = self.env, self.cfg.T
        env.reset(seed)
        self.ch[0].zero_()
        for t in range(T + 1):
            self._env_call(lib.env_state_tokens(env.h, _ptr(self.ctok[t]), _ptr(self.cne[t])), "env_state_tokens")
            self.critic.forward(self.ctok[t], self.cne[t], self.ch[t], h_out=self.ch[t + 1],
                                out=self.val[t].view(self.E, 1))
            if t == T:
                break
            self._env_call(lib.env_ppo_snapshot(env.h, _ptr(self.tok[t]), _ptr(self.ne[t]), _ptr(self.h[t])),
                           "env_ppo_snapshot")
            env.step()
            self._env_call(lib.env_ppo_record(env.h, _ptr(self.act[t]), _ptr(self.logp[t]), _ptr(self.rew[t]),
                                              _ptr(self.done[t])), "env_ppo_record")

    def update(self, seed: int):
        """GAE, then epochs x minibatches of actor and critic Adam steps;
        returns the last minibatch's statistics."""
        c, T = self.cfg, self.cfg.T
        self.adv, self.ret, self.adv_a = gae(self.rew, self.val, self.done, c.gamma, c.lam, self.agent_env,
                                             stream=self.env._stream)
        NA, E = self.NA, self.E
        tok = self.tok.view(T * NA, self.NS, 8)
        ne, h = self.ne.view(T * NA), self.h.view(T * NA, self.d)
        act, logp, adv = self.act.view(T * NA), self.logp.view(T * NA), self.adv_a.view(T * NA)
        ctok = self.ctok[:T].reshape(T * E, self.NS, 8)
        cne, ch, ret = self.cne[:T].reshape(T * E), self.ch[:T].reshape(T * E, self.d), self.ret.view(T * E)
        import torch.distributed as dist

        dp = self.group is not None
        rank = dist.get_rank(self.group) if dp else 0
        g = torch.Generator(device="cuda")
        g.manual_seed(shard.rank_seed(seed, rank) & 0x7FFFFFFFFFFFFFFF)
        sa = sc = None
        for ep in range(c.epochs):
            pa = torch.randperm(T * NA, generator=g, device="cuda").to(torch.int32)
            pc = torch.randperm(T * E, generator=g, device="cuda").to(torch.int32)
            for k in range(c.minibatches):
                last = ep == c.epochs - 1 and k == c.minibatches - 1
                # with a process group every rank takes part in every
                # all-reduce, its slice empty or not (ragged shards can leave
                # one rank's last slice empty while another's is not)
                sel = pa[k * self.mb_actor:(k + 1) * self.mb_actor]
                if sel.numel():
                    sa = self.actor.actor_grad(tok, ne, h, act, logp, adv, sel=sel, clip_eps=c.clip_eps,
                                               ent_coef=c.ent_coef, stats=last)
                elif dp:
                    self.actor.grad.zero_()
                n = dp_average(self.actor.grad, sel.numel(), self.group) if dp else sel.numel()
                if n:
                    self.actor.adam_step(c.lr_actor, c.beta1, c.beta2, c.eps)
                sel = pc[k * self.mb_critic:(k + 1) * self.mb_critic]
                if sel.numel():
                    sc = self.critic.value_grad(ctok, cne, ch, ret, sel=sel, stats=last)
                elif dp:
                    self.critic.grad.zero_()
                n = dp_average(self.critic.grad, sel.numel(), self.group) if dp else sel.numel()
                if n:
                    self.critic.adam_step(c.lr_critic, c.beta1, c.beta2, c.eps)
        self.actor.sync_policy(self.env)
        return {"actor": sa, "critic": sc}

    def iteration(self, seed: int):
        self.collect(seed)
        return self.update(seed)


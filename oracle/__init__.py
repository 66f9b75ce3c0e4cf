"""FP64 CPU oracle of the tracking-environment step — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library in
``paper_2505_08222_gb300``) never calls it and shares no code with it.

The arithmetic lives in ``utrack_oracle.c`` (environment, particle filter,
reward, observations) and ``utrack_oracle_nn.c`` (transformer agent,
estimator MLP, Adam) and ``utrack_oracle_ppo.c`` (TransfMAPPO: the
actor's and critic's loss gradients, GAE, the critic's state tokens),
compiled with gcc into ``_build/liboracle.so``.  This
module only marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# UTRACK_ORACLE_DIR points the oracle at another copy of its C sources (the
# planted-mistake tests build mutated copies there); unset, this directory.
_SRC_DIR = os.environ.get("UTRACK_ORACLE_DIR") or _HERE
_SRC = [os.path.join(_SRC_DIR, "utrack_oracle.c"), os.path.join(_SRC_DIR, "utrack_oracle_nn.c"),
        os.path.join(_SRC_DIR, "utrack_oracle_ppo.c")]
_LIB_PATH = os.path.join(_SRC_DIR, "_build", "liboracle.so")
_lib = None

N_SLOTS_FEATURES = 8
RING = 16
FEAT = 96


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction so that x86 and
    Arm hosts produce identical doubles)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp] + _SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB_PATH)
        _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_up = ctypes.POINTER(ctypes.c_uint32)


class OcConfig(ctypes.Structure):
    _fields_ = [
        ("n_envs", ctypes.c_int32), ("max_agents", ctypes.c_int32), ("max_targets", ctypes.c_int32),
        ("n_particles", ctypes.c_int32),
        ("agent_off", _ip), ("target_off", _ip), ("filter_off", _ip),
        ("dt", ctypes.c_double), ("agent_speed", ctypes.c_double), ("heading_noise", ctypes.c_double),
        ("action_mode", ctypes.c_int32), ("n_rudder", ctypes.c_int32), ("n_actions", ctypes.c_int32),
        ("turn_angle", ctypes.c_double), ("rudder_max", ctypes.c_double), ("rudder_gain", ctypes.c_double),
        ("target_model", ctypes.c_int32),
        ("target_speed_min", ctypes.c_double), ("target_speed_max", ctypes.c_double),
        ("target_drift_sigma", ctypes.c_double), ("target_depth_max", ctypes.c_double),
        ("range_sigma", ctypes.c_double), ("det_radius", ctypes.c_double), ("comm_radius", ctypes.c_double),
        ("comm_drop", ctypes.c_double),
        ("pf_accel_sigma", ctypes.c_double), ("pf_vcap", ctypes.c_double),
        ("reward_type", ctypes.c_int32),
        ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double), ("follow_dmin", ctypes.c_double),
        ("d_safe", ctypes.c_double),
        ("spawn_min", ctypes.c_double), ("spawn_radius", ctypes.c_double), ("spawn_tries", ctypes.c_int32),
        ("feature_scale", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("env0", ctypes.c_int32), ("agent0", ctypes.c_int32), ("target0", ctypes.c_int32),
        ("filter0", ctypes.c_int32), ("est_scale", ctypes.c_double),
        ("shared_filter", ctypes.c_int32), ("pair0", ctypes.c_int32), ("pair_off", _ip),
        ("pf_ess_num", ctypes.c_int32),
    ]


class OcState(ctypes.Structure):
    _fields_ = [(n, _dp) for n in ("ax", "ay", "apsi", "tx", "ty", "tz", "tpsi", "tspeed",
                                   "px", "py", "pvx", "pvy", "lpx", "lpy")] + [
        ("lpage", _ip), ("estx", _dp), ("esty", _dp), ("prev_estx", _dp), ("prev_esty", _dp),
        ("prev2_estx", _dp), ("prev2_esty", _dp), ("velx", _dp), ("vely", _dp), ("rudder", _ip), ("ring", _dp),
        ("ring_head", _ip),
        ("ring_count", _ip), ("step", ctypes.c_uint32), ("t_ep", ctypes.c_int32), ("pw", _dp)]


_OUT_FIELDS = [("range", _dp), ("valid", _ip), ("recv", _ip), ("meas", _dp), ("meas_n", _ip),
               ("pred_px", _dp), ("pred_py", _dp), ("pred_pvx", _dp), ("pred_pvy", _dp),
               ("weight", _dp), ("wmax", _dp), ("idx", _ip), ("err", _dp), ("tokens", _dp),
               ("reward", _dp), ("crash", _ip)]


class OcStepOut(ctypes.Structure):
    _fields_ = _OUT_FIELDS


class OcPolicyDims(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("n_layers", ctypes.c_int32), ("n_heads", ctypes.c_int32),
                ("n_act", ctypes.c_int32), ("n_in", ctypes.c_int32)]


def _declare(L):
    v = None
    L.oc_philox4x32_10.argtypes = [_up, _up, _up]
    L.oc_uniform_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, _dp, _dp]
    L.oc_reset.argtypes = [ctypes.POINTER(OcConfig), ctypes.POINTER(OcState), ctypes.c_uint32]
    L.oc_random_actions.argtypes = [ctypes.POINTER(OcConfig), ctypes.c_uint32, ctypes.c_int32, _ip]
    L.oc_gumbel_actions.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, _dp, _ip, _dp]
    L.oc_step.argtypes = [ctypes.POINTER(OcConfig), ctypes.POINTER(OcState), _ip, ctypes.POINTER(OcStepOut)]
    L.oc_ls_update.argtypes = [ctypes.POINTER(OcConfig), ctypes.POINTER(OcState), _dp]
    L.oc_step_learned.argtypes = [ctypes.POINTER(OcConfig), ctypes.POINTER(OcState), _ip, _dp, ctypes.c_int32,
                                  ctypes.POINTER(OcStepOut)]
    L.oc_systematic_resample.argtypes = [ctypes.c_int32, _dp, ctypes.c_uint64, _ip]
    L.oc_tracking_reward.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.oc_tracking_reward.restype = ctypes.c_double
    L.oc_obs.argtypes = [ctypes.POINTER(OcConfig), ctypes.POINTER(OcState), _dp]
    L.oc_est_features.argtypes = [ctypes.POINTER(OcConfig), ctypes.POINTER(OcState), ctypes.c_uint32, _dp, _dp]
    L.oc_policy_param_count.argtypes = [ctypes.POINTER(OcPolicyDims)]
    L.oc_policy_param_count.restype = ctypes.c_int64
    L.oc_policy_forward.argtypes = [ctypes.POINTER(OcPolicyDims), _dp, ctypes.c_int32, ctypes.c_int32, _dp,
                                    _ip, _dp, _dp, _dp]
    L.oc_mlp_param_count.restype = ctypes.c_int64
    L.oc_mlp_forward.argtypes = [ctypes.c_int32, _dp, _dp, _dp, _dp]
    L.oc_mlp_loss_grad.argtypes = [ctypes.c_int32, _dp, _dp, _dp, _dp, ctypes.c_double]
    L.oc_mlp_loss_grad.restype = ctypes.c_double
    L.oc_adam.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int32, ctypes.c_double,
                          ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.oc_tfm_param_count.argtypes = [ctypes.POINTER(OcPolicyDims)]
    L.oc_tfm_param_count.restype = ctypes.c_int64
    L.oc_tfm_forward.argtypes = [ctypes.POINTER(OcPolicyDims), _dp, ctypes.c_int32, ctypes.c_int32, _dp, _ip,
                                 _dp, _dp, _dp]
    L.oc_tfm_loss_grad.argtypes = [ctypes.POINTER(OcPolicyDims), _dp, ctypes.c_int32, ctypes.c_int32, _dp, _ip,
                                   _dp, ctypes.c_int32, _ip, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp,
                                   _dp, _dp]
    L.oc_tfm_loss_grad.restype = ctypes.c_double
    L.oc_gae.argtypes = [ctypes.c_int32, ctypes.c_int32, _dp, _dp, _ip, ctypes.c_double, ctypes.c_double,
                         _dp, _dp]
    L.oc_state_tokens.argtypes = [ctypes.c_int32, _ip, _ip, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                  _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _ip]
    return v


def _p(a: Optional[np.ndarray], t=_dp):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, np.int32)


# --------------------------------------------------------------------------
# Random numbers
# --------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oc_philox4x32_10(_p(c, _up), _p(k, _up), _p(out, _up))
    return out


def philox_many(ctrs: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of each counter row ([n, 4] uint32)."""
    L = lib()
    k = np.ascontiguousarray(key, np.uint32)
    ctrs = np.ascontiguousarray(ctrs, np.uint32)
    out = np.zeros_like(ctrs)
    for i in range(ctrs.shape[0]):
        L.oc_philox4x32_10(_p(ctrs[i], _up), _p(k, _up), _p(out[i], _up))
    return out


def uniform_normal(seed, id0, id1, step, tag):
    u = np.zeros(4)
    n = np.zeros(4)
    lib().oc_uniform_normal(seed, id0, id1, step, tag, _p(u), _p(n))
    return u, n


# --------------------------------------------------------------------------
# Environment
# --------------------------------------------------------------------------
class OracleEnv:
    """Batched environment state in float64 plus the stage functions."""

    def __init__(self, params, seed: int, id_base=None):
        self.p = params
        a, t = params.counts()
        self.n_agents_env, self.n_targets_env = a, t
        self.agent_off = _i32(np.concatenate([[0], np.cumsum(a)]))
        self.target_off = _i32(np.concatenate([[0], np.cumsum(t)]))
        shared = int(getattr(params, "shared_filter", 0))
        self.filter_off = _i32(np.concatenate([[0], np.cumsum(t if shared else a * t)]))
        self.pair_off = _i32(np.concatenate([[0], np.cumsum(a * t)]))
        self.NA = int(self.agent_off[-1])
        self.NT = int(self.target_off[-1])
        self.F = int(self.filter_off[-1])
        self.NPAIR = int(self.pair_off[-1])
        P = params.n_particles
        self.cfg = OcConfig()
        c = self.cfg
        c.n_envs, c.max_agents, c.max_targets, c.n_particles = (params.n_envs, params.max_agents,
                                                                params.max_targets, P)
        c.agent_off, c.target_off, c.filter_off = (_p(self.agent_off, _ip), _p(self.target_off, _ip),
                                                   _p(self.filter_off, _ip))
        c.pair_off = _p(self.pair_off, _ip)
        c.shared_filter = shared
        for name in ("dt", "agent_speed", "heading_noise", "action_mode", "n_rudder", "n_actions", "turn_angle",
                     "rudder_max", "rudder_gain", "target_model", "target_speed_min", "target_speed_max",
                     "target_drift_sigma", "target_depth_max", "range_sigma", "det_radius", "comm_radius",
                     "comm_drop", "pf_accel_sigma", "pf_vcap", "reward_type", "eps_min", "eps_max",
                     "follow_dmin", "d_safe", "spawn_min", "spawn_radius", "spawn_tries", "feature_scale",
                     "est_scale"):
            setattr(c, name, getattr(params, name))
        c.seed = seed
        if id_base is None:  # global ids of a shard of a larger batch, else 0
            id_base = tuple(getattr(params, k, 0)
                            for k in ("id_env0", "id_agent0", "id_target0", "id_filter0", "id_pair0"))
        id_base = tuple(id_base) + (0,) * (5 - len(id_base))
        c.env0, c.agent0, c.target0, c.filter0, c.pair0 = (int(v) for v in id_base)
        self.seed = seed
        AM = params.max_agents
        self.arr = {
            "ax": np.zeros(self.NA), "ay": np.zeros(self.NA), "apsi": np.zeros(self.NA),
            "tx": np.zeros(self.NT), "ty": np.zeros(self.NT), "tz": np.zeros(self.NT),
            "tpsi": np.zeros(self.NT), "tspeed": np.zeros(self.NT),
            "px": np.zeros(self.F * P), "py": np.zeros(self.F * P),
            "pvx": np.zeros(self.F * P), "pvy": np.zeros(self.F * P),
            "lpx": np.zeros(self.NA * AM), "lpy": np.zeros(self.NA * AM),
            "lpage": np.zeros(self.NA * AM, np.int32),
            "estx": np.zeros(self.F), "esty": np.zeros(self.F),
            "prev_estx": np.zeros(self.F), "prev_esty": np.zeros(self.F),
            "prev2_estx": np.zeros(self.F), "prev2_esty": np.zeros(self.F),
            "velx": np.zeros(self.F), "vely": np.zeros(self.F), "rudder": np.zeros(self.NA, np.int32),
            "ring": np.zeros(self.F * RING * 4), "ring_head": np.zeros(self.F, np.int32),
            "ring_count": np.zeros(self.F, np.int32),
        }
        c.pf_ess_num = int(getattr(params, "pf_ess_num", 0))
        if c.pf_ess_num > 0:  # carried particle log-weights
            self.arr["pw"] = np.zeros(self.F * P)
        self.st = OcState()
        self._bind()

    def _bind(self):
        for k, v in self.arr.items():
            setattr(self.st, k, _p(v, _ip if v.dtype == np.int32 else _dp))

    @property
    def step_count(self) -> int:
        return int(self.st.step)

    def set_arrays(self, **kw):
        for k, v in kw.items():
            dst = self.arr[k]
            dst[...] = np.asarray(v, dst.dtype).reshape(dst.shape)

    def set_counters(self, step: int, t_ep: int = 0):
        self.st.step = step
        self.st.t_ep = t_ep

    def reset(self, g: int = 0):
        lib().oc_reset(ctypes.byref(self.cfg), ctypes.byref(self.st), g)

    def random_actions(self, g: int) -> np.ndarray:
        act = np.zeros(self.NA, np.int32)
        lib().oc_random_actions(ctypes.byref(self.cfg), g, self.NA, _p(act, _ip))
        return act

    def step(self, actions: np.ndarray, want=(), mlp=None, mode: int = 2) -> dict:
        """One step.  ``want`` names the intermediates to return.  With ``mlp``
        (estimator parameters, canonical order) the learned tracker replaces
        the particle filter (``mode`` 1 hold / 2 network / 3 coast on steps
        without a fresh ping); ``mode=4`` selects the least-squares tracker."""
        P, AM = self.p.n_particles, self.p.max_agents
        NS = self.p.max_agents + self.p.max_targets
        shapes = {"range": (self.NPAIR, np.float64), "valid": (self.NPAIR, np.int32),
                  "recv": (self.NA * AM, np.int32), "meas": (self.F * AM * 4, np.float64),
                  "meas_n": (self.F, np.int32), "pred_px": (self.F * P, np.float64),
                  "pred_py": (self.F * P, np.float64), "pred_pvx": (self.F * P, np.float64),
                  "pred_pvy": (self.F * P, np.float64), "weight": (self.F * P, np.float64),
                  "wmax": (self.F * P, np.float64), "idx": (self.F * P, np.int32),
                  "err": (self.F, np.float64), "tokens": (self.NA * NS * 8, np.float64),
                  "reward": (self.p.n_envs, np.float64), "crash": (self.p.n_envs, np.int32)}
        want = set(want) | {"err", "reward", "crash"}
        if "pred_px" in want:
            want |= {"pred_py", "pred_pvx", "pred_pvy"}
        out = {k: np.zeros(n, dt) for k, (n, dt) in shapes.items() if k in want}
        so = OcStepOut()
        for k, v in out.items():
            setattr(so, k, _p(v, _ip if v.dtype == np.int32 else _dp))
        act = _i32(actions)
        if mode == 4:  # least-squares tracker
            lib().oc_step_learned(ctypes.byref(self.cfg), ctypes.byref(self.st), _p(act, _ip), None, 4,
                                  ctypes.byref(so))
        elif mlp is None:
            lib().oc_step(ctypes.byref(self.cfg), ctypes.byref(self.st), _p(act, _ip), ctypes.byref(so))
        else:
            prm = _f64(mlp)
            lib().oc_step_learned(ctypes.byref(self.cfg), ctypes.byref(self.st), _p(act, _ip), _p(prm), int(mode),
                                  ctypes.byref(so))
        if "tokens" in out:
            out["tokens"] = out["tokens"].reshape(self.NA, NS, 8)
        if "meas" in out:
            out["meas"] = out["meas"].reshape(self.F, AM, 4)
        return out

    def ls_update(self) -> np.ndarray:
        """The least-squares tracker's update on the current rings alone
        (history advanced, estimates replaced); returns the errors [F]."""
        err = np.zeros(self.F)
        lib().oc_ls_update(ctypes.byref(self.cfg), ctypes.byref(self.st), _p(err))
        return err

    def obs(self) -> np.ndarray:
        """Observation tokens of the current state [NA, A_max + T_max, 8]."""
        NS = self.p.max_agents + self.p.max_targets
        tok = np.zeros(self.NA * NS * 8)
        lib().oc_obs(ctypes.byref(self.cfg), ctypes.byref(self.st), _p(tok))
        return tok.reshape(self.NA, NS, 8)

    def est_features(self, g: Optional[int] = None):
        feat = np.zeros((self.F, FEAT))
        label = np.zeros((self.F, 2))
        lib().oc_est_features(ctypes.byref(self.cfg), ctypes.byref(self.st),
                              self.step_count if g is None else g, _p(feat), _p(label))
        return feat, label

    def n_entities(self) -> np.ndarray:
        """Entity tokens per agent (A_e + T_e), [NA]."""
        return np.repeat(self.n_agents_env + self.n_targets_env, self.n_agents_env).astype(np.int32)


def systematic_resample(wmax: np.ndarray, u64: int) -> np.ndarray:
    w = _f64(wmax)
    idx = np.zeros(len(w), np.int32)
    lib().oc_systematic_resample(len(w), _p(w), ctypes.c_uint64(u64), _p(idx, _ip))
    return idx


def tracking_reward(err: float, eps_min: float = 10.0, eps_max: float = 50.0) -> float:
    return lib().oc_tracking_reward(err, eps_min, eps_max)


def gumbel_actions(seed: int, g: int, logits: np.ndarray, agent0: int = 0):
    lg = _f64(logits)
    n, k = lg.shape
    act = np.zeros(n, np.int32)
    gum = np.zeros((n, k))
    lib().oc_gumbel_actions(ctypes.c_uint64(seed), g, agent0, n, k, _p(lg), _p(act, _ip), _p(gum))
    return act, gum


# --------------------------------------------------------------------------
# Neural parts
# --------------------------------------------------------------------------
def policy_param_count(d, n_layers, n_heads, n_act=7, n_in=8) -> int:
    dims = OcPolicyDims(d, n_layers, n_heads, n_act, n_in)
    return int(lib().oc_policy_param_count(ctypes.byref(dims)))


def policy_forward(params, d, n_layers, n_heads, tokens, n_ent, h_in, n_act=7):
    """logits [n, n_act], h_out [n, d]."""
    dims = OcPolicyDims(d, n_layers, n_heads, n_act, 8)
    prm = _f64(params)
    tok = _f64(tokens)
    n, ns, _ = tok.shape
    ne = _i32(n_ent)
    h = _f64(h_in)
    logits = np.zeros((n, n_act))
    h_out = np.zeros((n, d))
    lib().oc_policy_forward(ctypes.byref(dims), _p(prm), n, ns, _p(tok), _p(ne, _ip), _p(h),
                            _p(logits), _p(h_out))
    return logits, h_out


def mlp_param_count() -> int:
    return int(lib().oc_mlp_param_count())


def mlp_forward(params, X, want_pre=False):
    prm = _f64(params)
    x = _f64(X)
    B = x.shape[0]
    out = np.zeros((B, 2))
    pre = np.zeros((3, B, 256)) if want_pre else None
    lib().oc_mlp_forward(B, _p(prm), _p(x), _p(out), _p(pre))
    return (out, pre) if want_pre else out


def mlp_loss_grad(params, X, Y, huber=0.0):
    """Mean over rows of the summed per-output loss (squared error / 2, or
    the Huber loss with threshold ``huber`` > 0) and its gradient."""
    prm = _f64(params)
    x = _f64(X)
    y = _f64(Y)
    g = np.zeros_like(prm)
    loss = lib().oc_mlp_loss_grad(x.shape[0], _p(prm), _p(x), _p(y), _p(g), float(huber))
    return loss, g


def adam(theta, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    th, mm, vv, gg = _f64(theta).copy(), _f64(m).copy(), _f64(v).copy(), _f64(grad)
    lib().oc_adam(len(th), _p(th), _p(mm), _p(vv), _p(gg), t, lr, beta1, beta2, eps)
    return th, mm, vv


# --------------------------------------------------------------------------
# TransfMAPPO training (actor and critic losses, GAE, critic tokens)
# --------------------------------------------------------------------------
ACTOR, CRITIC = 0, 1


def tfm_param_count(d, n_layers, n_heads, n_out, n_in=8) -> int:
    return int(lib().oc_tfm_param_count(ctypes.byref(OcPolicyDims(d, n_layers, n_heads, n_out, n_in))))


def tfm_forward(params, d, n_layers, n_heads, n_out, tokens, n_ent, h_in):
    """out [n, n_out], h_out [n, d] of the transformer (actor or critic)."""
    if n_layers > 8:
        raise ValueError("at most 8 blocks")
    dims = OcPolicyDims(d, n_layers, n_heads, n_out, 8)
    prm, tok, ne, h = _f64(params), _f64(tokens), _i32(n_ent), _f64(h_in)
    n, ns, _ = tok.shape
    out = np.zeros((n, n_out))
    h_out = np.zeros((n, d))
    lib().oc_tfm_forward(ctypes.byref(dims), _p(prm), n, ns, _p(tok), _p(ne, _ip), _p(h), _p(out), _p(h_out))
    return out, h_out


def tfm_loss_grad(params, d, n_layers, n_heads, n_out, kind, tokens, n_ent, h_in, actions=None, logp_old=None,
                  adv=None, clip_eps=0.2, ent_coef=0.0, returns=None, want_grad=True):
    """Mean loss, its gradient (or None) and the mean stats [loss, entropy
    (actor) / V (critic), clipped fraction, approximate KL]."""
    if n_layers > 8 or n_out > 64:
        raise ValueError("at most 8 blocks and 64 outputs")
    dims = OcPolicyDims(d, n_layers, n_heads, n_out, 8)
    prm, tok, ne, h = _f64(params), _f64(tokens), _i32(n_ent), _f64(h_in)
    n, ns, _ = tok.shape
    act = None if actions is None else _i32(actions)
    lo = None if logp_old is None else _f64(logp_old)
    ad = None if adv is None else _f64(adv)
    rt = None if returns is None else _f64(returns)
    g = np.zeros_like(prm) if want_grad else None
    st = np.zeros(4)
    loss = lib().oc_tfm_loss_grad(ctypes.byref(dims), _p(prm), n, ns, _p(tok), _p(ne, _ip), _p(h), int(kind),
                                  _p(act, _ip), _p(lo), _p(ad), float(clip_eps), float(ent_coef), _p(rt), _p(g),
                                  _p(st))
    return loss, g, st


def gae(reward, value, done, gamma, lam):
    """adv, ret [T, E] from reward, done [T, E] and value [T + 1, E]."""
    r, v, dn = _f64(reward), _f64(value), _i32(done)
    T, E = r.shape
    assert v.shape == (T + 1, E) and dn.shape == (T, E)
    adv, ret = np.zeros((T, E)), np.zeros((T, E))
    lib().oc_gae(T, E, _p(r), _p(v), _p(dn, _ip), float(gamma), float(lam), _p(adv), _p(ret))
    return adv, ret


def state_tokens_arrays(agent_off, target_off, n_slots, S, agent_speed, ax, ay, apsi, tx, ty, tz, tpsi, tspeed):
    """Critic tokens [E, n_slots, 8] and n_ent [E] from state arrays."""
    ao, to = _i32(agent_off), _i32(target_off)
    E = len(ao) - 1
    arrs = [_f64(a) for a in (ax, ay, apsi, tx, ty, tz, tpsi, tspeed)]
    tok = np.zeros((E, n_slots, 8))
    ne = np.zeros(E, np.int32)
    lib().oc_state_tokens(E, _p(ao, _ip), _p(to, _ip), n_slots, float(S), float(agent_speed),
                          *[_p(a) for a in arrs], _p(tok), _p(ne, _ip))
    return tok, ne


def state_tokens(env: "OracleEnv", n_slots=None):
    """Critic tokens [E, n_slots, 8] and n_ent [E] from the env's true state."""
    c = env.cfg
    a = env.arr
    return state_tokens_arrays(env.agent_off, env.target_off, n_slots or (c.max_agents + c.max_targets),
                               c.feature_scale, c.agent_speed, a["ax"], a["ay"], a["apsi"], a["tx"], a["ty"],
                               a["tz"], a["tpsi"], a["tspeed"])

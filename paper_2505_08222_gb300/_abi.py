"""ctypes mirror of include/utrack.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# UTRACK_CHECKED=1 loads the index-checked build (build(checked=True))
CHECKED = os.environ.get("UTRACK_CHECKED", "") == "1"
LIB_PATH = os.path.join(HERE, "_build_checked" if CHECKED else "_build", "libutrack.so")

UT_ABI_VERSION = 8
UT_FLAG_DEBUG = 1
UT_FLAG_RING = 2

STATUS = {0: "UT_OK", 1: "UT_ERR_INVALID", 2: "UT_ERR_NOMEM", 3: "UT_ERR_CUDA", 4: "UT_ERR_TIMEOUT",
          5: "UT_ERR_STATE", 6: "UT_ERR_UNSUPPORTED"}

_i32p = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp, _vp)),
                ("free", ctypes.CFUNCTYPE(None, _vp, _vp, _vp)),
                ("ctx", _vp)]


ALLOC_FN = ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp, _vp)
FREE_FN = ctypes.CFUNCTYPE(None, _vp, _vp, _vp)

CONFIG_FIELDS = [
    ("abi_version", ctypes.c_uint32), ("flags", ctypes.c_uint32),
    ("n_envs", ctypes.c_int32), ("max_agents", ctypes.c_int32), ("max_targets", ctypes.c_int32),
    ("n_particles", ctypes.c_int32), ("horizon", ctypes.c_int32),
    ("agents_per_env_host", _i32p), ("targets_per_env_host", _i32p),
    ("dt", ctypes.c_float), ("agent_speed", ctypes.c_float), ("heading_noise", ctypes.c_float),
    ("action_mode", ctypes.c_int32), ("n_rudder", ctypes.c_int32), ("n_actions", ctypes.c_int32),
    ("turn_angle", ctypes.c_float), ("rudder_max", ctypes.c_float), ("rudder_gain", ctypes.c_float),
    ("target_model", ctypes.c_int32),
    ("target_speed_min", ctypes.c_float), ("target_speed_max", ctypes.c_float),
    ("target_drift_sigma", ctypes.c_float), ("target_depth_max", ctypes.c_float),
    ("range_sigma", ctypes.c_float), ("det_radius", ctypes.c_float), ("comm_radius", ctypes.c_float),
    ("comm_drop", ctypes.c_float), ("pf_accel_sigma", ctypes.c_float), ("pf_vcap", ctypes.c_float),
    ("reward_type", ctypes.c_int32), ("eps_min", ctypes.c_float), ("eps_max", ctypes.c_float),
    ("follow_dmin", ctypes.c_float), ("d_safe", ctypes.c_float),
    ("spawn_min", ctypes.c_float), ("spawn_radius", ctypes.c_float), ("spawn_tries", ctypes.c_int32),
    ("feature_scale", ctypes.c_float), ("est_scale", ctypes.c_float),
    ("id_env0", ctypes.c_uint32), ("id_agent0", ctypes.c_uint32), ("id_target0", ctypes.c_uint32),
    ("id_filter0", ctypes.c_uint32),
    ("d_model", ctypes.c_int32), ("n_layers", ctypes.c_int32), ("n_heads", ctypes.c_int32),
    ("shared_filter", ctypes.c_int32), ("id_pair0", ctypes.c_uint32), ("pf_ess_num", ctypes.c_int32),
]


class Config(ctypes.Structure):
    _fields_ = CONFIG_FIELDS


class StepOut(ctypes.Structure):
    _fields_ = [("reward", _vp), ("done", _vp), ("obs", _vp), ("estx", _vp), ("esty", _vp), ("err", _vp),
                ("actions", _vp), ("logits", _vp)]


STATE_PTRS = ["ax", "ay", "apsi", "tx", "ty", "tz", "tpsi", "tspeed", "px", "py", "pvx", "pvy",
              "lpx", "lpy", "lpage", "estx", "esty", "prev_estx", "prev_esty", "prev2_estx", "prev2_esty",
              "rudder", "velx", "vely", "ring", "ring_head", "ring_count", "h", "pw"]


class StateView(ctypes.Structure):
    _fields_ = [(n, _vp) for n in STATE_PTRS] + [
        ("step", ctypes.c_uint32), ("t_ep", ctypes.c_int32),
        ("n_agents", ctypes.c_int64), ("n_targets", ctypes.c_int64), ("n_filters", ctypes.c_int64)]


DEBUG_PTRS = ["range", "valid", "recv", "meas", "meas_n", "pred_px", "pred_py", "pred_pvx", "pred_pvy",
              "weight", "wmax", "idx"]


class DebugView(ctypes.Structure):
    _fields_ = [(n, _vp) for n in DEBUG_PTRS]


class EstTrainConfig(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("cosine", ctypes.c_int32), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("seed", ctypes.c_uint64), ("huber_delta", ctypes.c_float)]


class EstTrainStats(ctypes.Structure):
    _fields_ = [("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double), ("ms", ctypes.c_double),
                ("rows_seen", ctypes.c_int64)]


class TfmConfig(ctypes.Structure):
    _fields_ = [("abi_version", ctypes.c_uint32), ("d_model", ctypes.c_int32), ("n_layers", ctypes.c_int32),
                ("n_heads", ctypes.c_int32), ("n_out", ctypes.c_int32), ("n_slots", ctypes.c_int32),
                ("tokens_bf16", ctypes.c_int32), ("reserved", ctypes.c_int32), ("max_batch", ctypes.c_int64)]


class PpoBuffers(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("tokens", "n_ent", "h", "actions", "logp", "reward", "done", "ctokens",
                                              "cn_ent", "ch", "value")]


class RolloutStats(ctypes.Structure):
    _fields_ = [("sum_sq_err", ctypes.c_double), ("n_err", ctypes.c_int64), ("rmse", ctypes.c_double),
                ("reward_sum", ctypes.c_double), ("crash_count", ctypes.c_int64),
                ("agent_steps", ctypes.c_int64), ("steps", ctypes.c_int64), ("device_status", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64)]


# name -> (restype, argtypes); every function include/utrack.h declares
SIGNATURES = {
    "env_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Allocator), _vp, ctypes.POINTER(_vp)]),
    "env_destroy": (None, [_vp]),
    "env_last_error": (ctypes.c_char_p, [_vp]),
    "env_reset": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "env_step": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(StepOut)]),
    "rollout": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(RolloutStats)]),
    "env_get_state": (ctypes.c_int, [_vp, ctypes.POINTER(StateView)]),
    "env_set_state": (ctypes.c_int, [_vp, ctypes.POINTER(StateView)]),
    "env_debug": (ctypes.c_int, [_vp, ctypes.POINTER(DebugView)]),
    "env_metrics": (ctypes.c_int, [_vp, ctypes.POINTER(RolloutStats)]),
    "env_metrics_reset": (ctypes.c_int, [_vp]),
    "env_test_wait_timeout": (ctypes.c_int, [_vp, ctypes.c_uint32]),
    "env_set_rollout_form": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "env_get_rollout_form": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "rollout_prepare": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "env_profile": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "env_stage_time": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "pf_variant_count": (ctypes.c_int32, []),
    "pf_variant_usable": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32]),
    "pf_variant_label": (ctypes.c_char_p, [ctypes.c_int32]),
    "env_set_pf_variant": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "env_get_pf_variant": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "env_autotune": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "env_set_policy": (ctypes.c_int, [_vp, _vp, ctypes.c_int64]),
    "policy_forward": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                      _vp]),
    "est_set_weights": (ctypes.c_int, [_vp, _vp, ctypes.c_int64]),
    "est_get_weights": (ctypes.c_int, [_vp, _vp, ctypes.c_int64]),
    "est_set_mode": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "est_forward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64]),
    "est_record": (ctypes.c_int, [_vp, _vp, _vp]),
    "est_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_float, _vp, ctypes.POINTER(ctypes.c_double)]),
    "est_adam_step": (ctypes.c_int, [_vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "est_train": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.POINTER(EstTrainConfig),
                                 ctypes.POINTER(EstTrainStats)]),
    "est_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "est_load": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "ut_philox": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp, ctypes.c_int64, _vp]),
    "tc_gemm_bf16": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp]),
    "tracker_update_noalloc": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_uint64, ctypes.c_uint32] + [_vp] * 13),
    "pf_resample": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32, _vp, _vp]),
    "tfm_param_count": (ctypes.c_int64, [ctypes.POINTER(TfmConfig)]),
    "tfm_create": (ctypes.c_int, [ctypes.POINTER(TfmConfig), _vp, ctypes.c_int64, _vp, ctypes.POINTER(_vp)]),
    "tfm_destroy": (None, [_vp]),
    "tfm_last_error": (ctypes.c_char_p, [_vp]),
    "tfm_params": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "tfm_set_gemm_path": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "tfm_forward": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp]),
    "tfm_ppo_actor_grad": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_float,
                                          ctypes.c_float, _vp, ctypes.POINTER(ctypes.c_double)]),
    "tfm_value_grad": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp,
                                      ctypes.POINTER(ctypes.c_double)]),
    "tfm_adam_step": (ctypes.c_int, [_vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "tfm_sync_policy": (ctypes.c_int, [_vp, _vp]),
    "ppo_gae": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_float, _vp,
                               _vp, _vp, ctypes.c_int64, _vp, _vp]),
    "env_state_tokens": (ctypes.c_int, [_vp, _vp, _vp]),
    "env_ppo_snapshot": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "env_ppo_record": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "env_ppo_collect": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.POINTER(PpoBuffers)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libutrack.so; raises if it has not been built (there is no
    fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2505_08222_gb300.build.build() "
                          "(the library has no CPU or Python fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib

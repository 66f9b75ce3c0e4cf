"""Helpers for the GPU parity tests: run the CUDA library and the FP64 oracle
on the same seeded inputs and injected states."""
import math

import numpy as np
import torch

import oracle

STATE_KEYS_F = ["ax", "ay", "apsi", "tx", "ty", "tz", "tpsi", "tspeed", "px", "py", "pvx", "pvy", "lpx", "lpy",
                "estx", "esty"]
STATE_KEYS_I = ["lpage", "rudder"]


def gpu_state(env) -> dict:
    torch.cuda.synchronize()
    st = env.state()
    out = {}
    for k in STATE_KEYS_F + STATE_KEYS_I + ["ring", "ring_head", "ring_count", "pw"]:
        v = st.get(k)
        if v is not None:
            out[k] = v.detach().cpu().numpy().copy()
    out["step"], out["t_ep"] = st["step"], st["t_ep"]
    return out


def oracle_state_f32(o: oracle.OracleEnv) -> dict:
    """The oracle's state rounded to float32 (what a GPU handle can hold)."""
    out = {k: o.arr[k].astype(np.float32) for k in STATE_KEYS_F}
    if "pw" in o.arr:  # carried log-weights (resampling triggered by the effective sample size)
        out["pw"] = o.arr["pw"].astype(np.float32)
    out["lpage"] = o.arr["lpage"].copy()
    out["rudder"] = o.arr["rudder"].copy()
    return out


def inject(env, o: oracle.OracleEnv, st: dict, step: int, t_ep: int = 0):
    """Same float32 state into the GPU handle and the oracle."""
    tens = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in st.items()}
    env.set_state(step, t_ep, **tens)
    o.set_arrays(**{k: v.astype(np.float64) if v.dtype == np.float32 else v for k, v in st.items()})
    o.set_counters(step, t_ep)


def rel_close(a, b, rel, floor=1.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) <= rel * np.maximum(np.abs(b), floor)


def angle_diff(a, b):
    return np.abs(np.angle(np.exp(1j * (np.asarray(a, np.float64) - np.asarray(b, np.float64)))))


def ess_trigger(wmax, k: int, P: int) -> bool:
    """The filter's resampling trigger on its own max-normalised weights:
    16 (sum r)^2 < k P sum r^2 with r = floor(w 2^38) >> 23."""
    r = np.floor(np.asarray(wmax, np.float64) * 2.0 ** 38).astype(np.int64) >> 23
    s1, s2 = int(r.sum()), int((r * r).sum())
    return 16 * s1 * s1 < k * P * s2


def resample_u64(seed: int, filt_global: int, g: int) -> int:
    r = oracle.philox([filt_global, 0, g, 12], [seed & 0xFFFFFFFF, seed >> 32])
    return int(r[0]) | (int(r[1]) << 32)


def bf16_to_f32(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint16).astype(np.uint32) << 16).view(np.float32)

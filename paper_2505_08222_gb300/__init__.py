"""GB300-native batched underwater-tracking environment (arXiv 2505.08222).

A thin Python binding over the C ABI of ``_build/libutrack.so`` (declared in
``include/utrack.h``).  Every step of the environment runs in the library's
CUDA kernels; this module only marshals arguments.  PyTorch provides device
memory (its caching allocator is handed to the library as the allocator) and
streams, and wraps the library's borrowed device buffers as tensors.

There is no CPU or Python fallback: importing the binding without the built
library raises ImportError.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _abi

__all__ = ["Env", "UtError", "philox", "pf_resample", "lib"]

lib = _abi.load()
# checked build (UTRACK_CHECKED=1): handles closed with a failed index check
CHECK_FAILURES: list = []


class UtError(RuntimeError):
    pass


def _check(rc: int, handle=None, what: str = ""):
    if rc != 0:
        msg = ""
        if handle:
            raw = lib.env_last_error(handle)
            msg = raw.decode() if raw else ""
        raise UtError(f"{what}: {_abi.STATUS.get(rc, rc)} {msg}".strip())


class _DevArray:
    """Exposes a borrowed device pointer through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


_TYPESTR = {torch.float32: "<f4", torch.int32: "<i4", torch.int16: "<i2", torch.uint8: "|u1",
            torch.float64: "<f8", torch.int64: "<i8"}


def device_view(ptr: int, shape, dtype=torch.float32) -> Optional[torch.Tensor]:
    """Zero-copy tensor over a borrowed device buffer of the library."""
    if not ptr:
        return None
    n = int(np.prod(shape)) if len(shape) else 1
    if n == 0:
        return torch.empty(shape, dtype=dtype, device="cuda")
    return torch.as_tensor(_DevArray(ptr, shape, _TYPESTR[dtype]), device="cuda")


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class _TorchAllocator:
    """Routes the library's allocations through PyTorch's caching allocator."""

    def __init__(self):
        dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
            except Exception:
                return None

        def _free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self._a = _abi.ALLOC_FN(_alloc)
        self._f = _abi.FREE_FN(_free)
        self.struct = _abi.Allocator(self._a, self._f, None)


def make_config(params, flags: int = 0):
    """ut_config from an object carrying the EnvParams fields."""
    cfg = _abi.Config()
    cfg.abi_version = _abi.UT_ABI_VERSION
    cfg.flags = flags
    keep = []
    for name, _ in _abi.CONFIG_FIELDS:
        if name in ("abi_version", "flags"):
            continue
        if name in ("agents_per_env_host", "targets_per_env_host"):
            src = getattr(params, name.replace("_host", ""), None)
            if src is None:
                setattr(cfg, name, None)
            else:
                arr = np.ascontiguousarray(src, np.int32)
                keep.append(arr)
                setattr(cfg, name, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
            continue
        setattr(cfg, name, getattr(params, name))
    return cfg, keep


class Env:
    """One batch of independent tracking environments on the current GPU."""

    def __init__(self, params, debug: bool = False, ring: bool = False, stream=None,
                 use_torch_allocator: bool = True):
        self.params = params
        flags = (_abi.UT_FLAG_DEBUG if debug else 0) | (_abi.UT_FLAG_RING if ring else 0)
        self._cfg, self._keep = make_config(params, flags)
        self._stream = _stream_ptr(stream)
        self._alloc = _TorchAllocator() if use_torch_allocator else None
        h = ctypes.c_void_p()
        rc = lib.env_create(ctypes.byref(self._cfg),
                            ctypes.byref(self._alloc.struct) if self._alloc else None,
                            ctypes.c_void_p(self._stream), ctypes.byref(h))
        _check(rc, None, "env_create")
        self.h = h
        st = self._state_view()
        self.NA, self.NT, self.F = st.n_agents, st.n_targets, st.n_filters
        a_cnt, t_cnt = params.counts()
        self.NPAIR = int((a_cnt.astype(np.int64) * t_cnt).sum())  # (agent, target) pairs
        self.P = params.n_particles
        self.AM = params.max_agents
        self.NS = params.max_agents + params.max_targets
        self.E = params.n_envs

    # ------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "h", None):
            if _abi.CHECKED:  # checked build: record a failed index check before the handle goes
                s = _abi.RolloutStats()
                lib.env_metrics(self.h, ctypes.byref(s))
                if s.device_status == 3:
                    CHECK_FAILURES.append(lib.env_last_error(self.h).decode())
            lib.env_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, seed: int):
        _check(lib.env_reset(self.h, ctypes.c_uint64(seed)), self.h, "env_reset")

    def step(self, actions: Optional[torch.Tensor] = None) -> dict:
        ptr = None
        if actions is not None:
            assert actions.is_cuda and actions.dtype == torch.int32 and actions.is_contiguous()
            assert actions.numel() == self.NA
            ptr = ctypes.c_void_p(actions.data_ptr())
        out = _abi.StepOut()
        _check(lib.env_step(self.h, ptr, ctypes.byref(out)), self.h, "env_step")
        return self._step_views(out)

    def _step_views(self, out) -> dict:
        return {
            "reward": device_view(out.reward, (self.E,)),
            "done": device_view(out.done, (self.E,), torch.int32),
            "obs": device_view(out.obs, (self.NA, self.NS, 8), torch.int16),
            "estx": device_view(out.estx, (self.F,)),
            "esty": device_view(out.esty, (self.F,)),
            "err": device_view(out.err, (self.F,)),
            "actions": device_view(out.actions, (self.NA,), torch.int32),
            "logits": device_view(out.logits, (self.NA, self.params.n_actions)),
        }

    def rollout(self, T: int) -> dict:
        s = _abi.RolloutStats()
        _check(lib.rollout(self.h, T, ctypes.byref(s)), self.h, "rollout")
        return {k: getattr(s, k) for k, _ in _abi.RolloutStats._fields_}

    @property
    def policy_ready(self) -> bool:
        return getattr(self, "_policy_ready", False)

    def set_policy(self, params: np.ndarray):
        """Canonical float32 parameter blob of the transformer agent."""
        prm = np.ascontiguousarray(params, np.float32)
        _check(lib.env_set_policy(self.h, prm.ctypes.data_as(ctypes.c_void_p), prm.size), self.h, "env_set_policy")
        self._policy_ready = True

    def policy_forward(self, tokens: torch.Tensor, n_ent: torch.Tensor, h: torch.Tensor, step: int = 1,
                       sample: bool = False):
        """Forward of the agent on caller tensors: tokens [n, S, 8] bf16,
        n_ent [n] int32, h [n, d] bf16 (updated in place).  Returns logits
        (and actions if sample)."""
        assert tokens.dtype == torch.bfloat16 and h.dtype == torch.bfloat16 and n_ent.dtype == torch.int32
        tokens = tokens.contiguous()
        n, S, _ = tokens.shape
        logits = torch.empty((n, self.params.n_actions), dtype=torch.float32, device="cuda")
        act = torch.empty(n, dtype=torch.int32, device="cuda") if sample else None
        _check(lib.policy_forward(self.h, ctypes.c_void_p(tokens.data_ptr()), ctypes.c_void_p(n_ent.data_ptr()),
                                  ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(logits.data_ptr()),
                                  ctypes.c_void_p(act.data_ptr()) if act is not None else None, n, S, step,
                                  ctypes.c_void_p(_stream_ptr(None))), self.h, "policy_forward")
        return (logits, act) if sample else logits

    # ------------------------------------------------------------ estimator
    def est_set_weights(self, params: np.ndarray):
        prm = np.ascontiguousarray(params, np.float32)
        _check(lib.est_set_weights(self.h, prm.ctypes.data_as(ctypes.c_void_p), prm.size), self.h, "est_set_weights")

    def est_get_weights(self) -> np.ndarray:
        out = np.zeros(156930, np.float32)
        _check(lib.est_get_weights(self.h, out.ctypes.data_as(ctypes.c_void_p), out.size), self.h, "est_get_weights")
        return out

    def est_set_mode(self, mode):
        """0 / False: particle filter; 1 / True: learned estimator, estimate held
        on steps without a fresh ping; 2: network on every step; 3: coast at the
        estimate's smoothed motion on steps without a fresh ping; 4: least-squares
        trilateration over the ring's pings (no network)."""
        _check(lib.est_set_mode(self.h, int(mode)), self.h, "est_set_mode")

    def est_forward(self, X: torch.Tensor) -> torch.Tensor:
        assert X.is_cuda and X.dtype == torch.float32 and X.shape[-1] == 96
        X = X.contiguous()
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
        _check(lib.est_forward(self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(out.data_ptr()), X.shape[0]),
               self.h, "est_forward")
        return out

    def est_record(self, feat: torch.Tensor, label: torch.Tensor):
        """Writes the current features [F, 96] and labels [F, 2] into the given tensors."""
        assert feat.is_contiguous() and label.is_contiguous()
        _check(lib.est_record(self.h, ctypes.c_void_p(feat.data_ptr()), ctypes.c_void_p(label.data_ptr())), self.h,
               "est_record")

    def est_loss_grad(self, X: torch.Tensor, Y: torch.Tensor, huber: float = 0.0, batch: Optional[int] = None,
                      seed: int = 0, step: int = 0):
        """Loss and gradient [156930] (device) of one batch: all rows of X, Y
        in order (``batch`` None or len(X)), else ``batch`` rows drawn as
        :meth:`est_train`'s step ``step`` under ``seed``."""
        for t, c in ((X, 96), (Y, 2)):
            assert t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.shape[1] == c and t.is_contiguous()
        assert X.shape[0] == Y.shape[0]
        n = X.shape[0]
        grad = torch.empty(156930, dtype=torch.float32, device="cuda")
        loss = ctypes.c_double()
        _check(lib.est_loss_grad(self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), n,
                                 n if batch is None else int(batch), seed, step, huber,
                                 ctypes.c_void_p(grad.data_ptr()), ctypes.byref(loss)), self.h, "est_loss_grad")
        return loss.value, grad

    def est_adam_step(self, grad: torch.Tensor, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                      eps: float = 1e-8):
        """One Adam update of the master weights with ``grad`` [156930] (device)."""
        assert grad.is_cuda and grad.dtype == torch.float32 and grad.numel() == 156930 and grad.is_contiguous()
        _check(lib.est_adam_step(self.h, ctypes.c_void_p(grad.data_ptr()), lr, beta1, beta2, eps), self.h,
               "est_adam_step")

    def est_train(self, X: torch.Tensor, Y: torch.Tensor, steps: int, batch: int, lr: float = 1e-3,
                  cosine: bool = True, seed: int = 0, beta1=0.9, beta2=0.999, eps=1e-8, huber: float = 0.0) -> dict:
        cfg = _abi.EstTrainConfig(steps, batch, lr, 1 if cosine else 0, beta1, beta2, eps, seed, huber)
        st = _abi.EstTrainStats()
        _check(lib.est_train(self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), X.shape[0],
                             ctypes.byref(cfg), ctypes.byref(st)), self.h, "est_train")
        return {k: getattr(st, k) for k, _ in _abi.EstTrainStats._fields_}

    def est_save(self, path: str):
        _check(lib.est_save(self.h, path.encode()), self.h, "est_save")

    def est_load(self, path: str):
        _check(lib.est_load(self.h, path.encode()), self.h, "est_load")

    def set_rollout_form(self, form: int):
        """0: captured CUDA graph of T steps; 1: persistent kernel (random
        actions and the particle filter only; UtError otherwise)."""
        _check(lib.env_set_rollout_form(self.h, int(form)), self.h, "env_set_rollout_form")

    def rollout_form(self) -> int:
        v = ctypes.c_int32()
        _check(lib.env_get_rollout_form(self.h, ctypes.byref(v)), self.h, "env_get_rollout_form")
        return v.value

    def rollout_prepare(self, T: int):
        _check(lib.rollout_prepare(self.h, T), self.h, "rollout_prepare")

    def profile(self, enable: bool = True):
        _check(lib.env_profile(self.h, 1 if enable else 0), self.h, "env_profile")

    def stage_time(self):
        """(total ms, launches) of the tracker stage since the last read."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(lib.env_stage_time(self.h, ctypes.byref(ms), ctypes.byref(n)), self.h, "env_stage_time")
        return ms.value, n.value

    def pf_variants(self):
        """Usable particle-filter launch variants for this handle's P."""
        return [v for v in range(lib.pf_variant_count()) if lib.pf_variant_usable(v, self.P)]

    def set_pf_variant(self, v: int):
        _check(lib.env_set_pf_variant(self.h, v), self.h, "env_set_pf_variant")

    def pf_variant(self) -> int:
        v = ctypes.c_int32()
        _check(lib.env_get_pf_variant(self.h, ctypes.byref(v)), self.h, "env_get_pf_variant")
        return v.value

    def autotune(self, reps: int = 5) -> str:
        """Times every usable filter variant, keeps the fastest (advances the env)."""
        v = ctypes.c_int32()
        _check(lib.env_autotune(self.h, reps, ctypes.byref(v)), self.h, "env_autotune")
        return lib.pf_variant_label(v.value).decode()

    def pf_variant_name(self) -> str:
        return lib.pf_variant_label(self.pf_variant()).decode()

    def metrics(self) -> dict:
        s = _abi.RolloutStats()
        _check(lib.env_metrics(self.h, ctypes.byref(s)), self.h, "env_metrics")
        return {k: getattr(s, k) for k, _ in _abi.RolloutStats._fields_}

    def metrics_reset(self):
        """Clears the device metrics and the device status word."""
        _check(lib.env_metrics_reset(self.h), self.h, "env_metrics_reset")

    def test_wait_timeout(self, polls: int):
        """Failure-detection test hook: > 0 makes the tensor-core kernels'
        first wait run out after ``polls`` polls (status word -> timeout);
        0 switches it off."""
        _check(lib.env_test_wait_timeout(self.h, int(polls)), self.h, "env_test_wait_timeout")

    # ------------------------------------------------------------ state
    def _state_view(self):
        v = _abi.StateView()
        _check(lib.env_get_state(self.h, ctypes.byref(v)), self.h, "env_get_state")
        return v

    def state(self) -> dict:
        """Borrowed device views of every state buffer plus the counters."""
        v = self._state_view()
        NA, NT, FP, F, AM = self.NA, self.NT, self.F * self.P, self.F, self.AM
        shapes = {"ax": (NA,), "ay": (NA,), "apsi": (NA,), "tx": (NT,), "ty": (NT,), "tz": (NT,),
                  "tpsi": (NT,), "tspeed": (NT,), "px": (FP,), "py": (FP,), "pvx": (FP,), "pvy": (FP,),
                  "lpx": (NA * AM,), "lpy": (NA * AM,), "lpage": (NA * AM,), "estx": (F,), "esty": (F,),
                  "prev_estx": (F,), "prev_esty": (F,), "prev2_estx": (F,), "prev2_esty": (F,),
                  "rudder": (NA,), "velx": (F,), "vely": (F,),
                  "ring": (F, 16, 4), "ring_head": (F,), "ring_count": (F,), "pw": (FP,)}
        out = {}
        for k, shp in shapes.items():
            dt = torch.int32 if k in ("lpage", "ring_head", "ring_count", "rudder") else torch.float32
            out[k] = device_view(getattr(v, k), shp, dt)
        d = getattr(self.params, "d_model", 0)
        out["h"] = device_view(v.h, (NA, d), torch.int16) if d else None
        out["step"] = v.step
        out["t_ep"] = v.t_ep
        return out

    def set_state(self, step: int, t_ep: int = 0, **tensors):
        """Copies the given device tensors (float32 / int32, contiguous) in."""
        v = _abi.StateView()
        keep = []
        for k, t in tensors.items():
            if t is None:
                continue
            t = t.contiguous()
            keep.append(t)
            setattr(v, k, t.data_ptr())
        v.step = step
        v.t_ep = t_ep
        _check(lib.env_set_state(self.h, ctypes.byref(v)), self.h, "env_set_state")
        torch.cuda.synchronize()

    def debug(self) -> dict:
        v = _abi.DebugView()
        _check(lib.env_debug(self.h, ctypes.byref(v)), self.h, "env_debug")
        F, FP, NA, AM, NP = self.F, self.F * self.P, self.NA, self.AM, self.NPAIR
        return {
            "range": device_view(v.range, (NP,)), "valid": device_view(v.valid, (NP,), torch.int32),
            "recv": device_view(v.recv, (NA * AM,), torch.int32), "meas": device_view(v.meas, (F, AM, 4)),
            "meas_n": device_view(v.meas_n, (F,), torch.int32),
            "pred_px": device_view(v.pred_px, (FP,)), "pred_py": device_view(v.pred_py, (FP,)),
            "pred_pvx": device_view(v.pred_pvx, (FP,)), "pred_pvy": device_view(v.pred_pvy, (FP,)),
            "weight": device_view(v.weight, (FP,)), "wmax": device_view(v.wmax, (FP,)),
            "idx": device_view(v.idx, (FP,), torch.int32),
        }


# ---------------------------------------------------------------- stand-alone ops
def philox(ctr: torch.Tensor, seed: int) -> torch.Tensor:
    """Philox4x32-10 of counters ctr [n, 4] (int32 bit patterns on the GPU)."""
    assert ctr.is_cuda and ctr.dtype == torch.int32 and ctr.shape[-1] == 4
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    _check(lib.ut_philox(ctypes.c_void_p(ctr.data_ptr()), ctypes.c_uint64(seed), ctypes.c_void_p(out.data_ptr()),
                         ctr.shape[0], ctypes.c_void_p(_stream_ptr(None))), None, "ut_philox")
    return out


def tc_gemm(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """A [M, K] bf16 @ B [N, K]^T bf16 -> [M, N] fp32 on the tensor cores."""
    assert A.is_cuda and A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib.tc_gemm_bf16(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                            ctypes.c_void_p(C.data_ptr()), M, N, K, ctypes.c_void_p(status.data_ptr()),
                            ctypes.c_void_p(_stream_ptr(None))), None, "tc_gemm_bf16")
    if int(status.item()) != 0:
        raise UtError("tc_gemm_bf16: tensor-core wait timed out")
    return C


def pf_resample(wmax: torch.Tensor, u64: torch.Tensor) -> torch.Tensor:
    """Systematic resample map of wmax [n_filters, P] (float32) with offsets
    u64 [n_filters] (int64 bit patterns)."""
    assert wmax.is_cuda and wmax.dtype == torch.float32 and u64.dtype == torch.int64
    wmax = wmax.contiguous()
    u64 = u64.contiguous()
    F, P = wmax.shape
    idx = torch.empty((F, P), dtype=torch.int32, device=wmax.device)
    _check(lib.pf_resample(ctypes.c_void_p(wmax.data_ptr()), ctypes.c_void_p(u64.data_ptr()), F, P,
                           ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(_stream_ptr(None))), None, "pf_resample")
    return idx

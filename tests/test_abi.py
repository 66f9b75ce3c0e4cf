"""The C-ABI library loads and exports every entry point include/*.h declares;
host-side validation rejects bad configurations (no GPU needed: validation
happens before any CUDA call)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = re.sub(r"typedef\s+struct\s+\w*\s*\{.*?\}\s*\w+\s*;", "", text, flags=re.S)
        text = re.sub(r"typedef\s+enum\s*\{.*?\}\s*\w+\s*;", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\([^;{}]*\)\s*;", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("env_create", "env_reset", "env_step", "rollout", "env_get_state", "env_set_state",
                     "env_destroy", "env_last_error", "pf_resample", "ut_philox"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    path = lib._name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_covers_every_declared_symbol():
    from paper_2505_08222_gb300 import _abi
    assert _declared_functions() <= set(_abi.SIGNATURES)


def _cfg(**kw):
    from paper_2505_08222_gb300 import make_config
    from synth import preset
    p = preset("fleet5", n_envs=4)
    cfg, keep = make_config(p.replace(**kw))
    return cfg, keep


@pytest.mark.parametrize("kw", [
    {"n_envs": 0}, {"max_agents": 9}, {"max_targets": 0}, {"n_particles": 0}, {"n_particles": 4097},
    {"range_sigma": 0.0}, {"n_heads": 3}, {"n_actions": 9}, {"reward_type": 2}, {"spawn_tries": 65},
    {"action_mode": 3}, {"shared_filter": 2}, {"shared_filter": -1}, {"pf_ess_num": 17}, {"pf_ess_num": -1},
    {"action_mode": 2, "n_actions": 7}, {"action_mode": 2, "n_actions": 3, "n_rudder": 1},
    {"action_mode": 2, "n_actions": 3, "n_rudder": 9},
])
def test_create_rejects_invalid_config(lib, kw):
    from paper_2505_08222_gb300 import _abi
    import paper_2505_08222_gb300 as ut
    cfg, keep = _cfg(**kw)
    h = ctypes.c_void_p()
    rc = ut.lib.env_create(ctypes.byref(cfg), None, None, ctypes.byref(h))
    assert rc == 1 and not h.value


def test_create_rejects_bad_ragged_counts_and_abi(lib):
    import numpy as np
    import paper_2505_08222_gb300 as ut
    cfg, keep = _cfg(agents_per_env=np.array([1, 2, 9, 1], np.int32))
    h = ctypes.c_void_p()
    assert ut.lib.env_create(ctypes.byref(cfg), None, None, ctypes.byref(h)) == 1
    cfg, keep = _cfg()
    cfg.abi_version = 99
    assert ut.lib.env_create(ctypes.byref(cfg), None, None, ctypes.byref(h)) == 1


def test_noalloc_rejects_layouts_it_does_not_run(lib):
    """The allocation-free tracker runs per-agent filters resampled every
    step on uniform fleets; other configurations are refused before any
    device work (so this runs without a GPU)."""
    import paper_2505_08222_gb300 as ut
    dummy = [ctypes.c_void_p(16)] * 12
    for kw in ({"shared_filter": 1}, {"pf_ess_num": 8}, {"n_envs": 0}):
        cfg, keep = _cfg(**kw)
        assert ut.lib.tracker_update_noalloc(ctypes.byref(cfg), ctypes.c_uint64(1), 1, *dummy, None) == 1
    cfg, keep = _cfg()
    assert ut.lib.tracker_update_noalloc(ctypes.byref(cfg), ctypes.c_uint64(1), 0, *dummy, None) == 1


def test_noalloc_rejects_unaligned_particle_arrays(lib):
    """With P % 4 == 0 the filter reads and writes particles as float4: a
    particle array that does not start on a 16-byte boundary (a view at an
    odd float offset) is refused on the host, before any device work."""
    import paper_2505_08222_gb300 as ut
    cfg, keep = _cfg(n_particles=512)
    for bad in range(4):  # px, py, pvx, pvy in turn 4 bytes off the boundary
        args = [ctypes.c_void_p(4096)] * 12
        args[5 + bad] = ctypes.c_void_p(4096 + 4)
        assert ut.lib.tracker_update_noalloc(ctypes.byref(cfg), ctypes.c_uint64(1), 1, *args, None) == 1


def test_standalone_ops_validate_arguments(lib):
    import paper_2505_08222_gb300 as ut
    assert ut.lib.pf_resample(None, None, -1, 16, None, None) == 1
    assert ut.lib.pf_resample(None, None, 4, 0, None, None) == 1
    assert ut.lib.ut_philox(None, 0, None, -3, None) == 1


def test_estimator_entry_points_reject_null_handles(lib):
    import paper_2505_08222_gb300 as ut
    assert ut.lib.est_set_mode(None, 1) == 1
    assert ut.lib.est_set_mode(None, 4) == 1


def test_tfm_param_count_validates_the_configuration(lib):
    from paper_2505_08222_gb300 import _abi
    import oracle

    f = lib.tfm_param_count
    f.restype = ctypes.c_int64
    f.argtypes = [ctypes.POINTER(_abi.TfmConfig)]

    def cfg(**kw):
        base = dict(abi_version=_abi.UT_ABI_VERSION, d_model=64, n_layers=2, n_heads=4, n_out=7, n_slots=10,
                    tokens_bf16=1, reserved=0, max_batch=1024)
        base.update(kw)
        return _abi.TfmConfig(**base)

    for d, L, H, no in ((64, 2, 4, 7), (128, 3, 8, 7), (32, 1, 4, 1), (96, 2, 3, 5)):
        assert f(ctypes.byref(cfg(d_model=d, n_layers=L, n_heads=H, n_out=no))) == oracle.tfm_param_count(d, L, H, no)
    for bad in (dict(d_model=48), dict(d_model=256), dict(n_heads=1), dict(n_heads=16), dict(n_heads=5), dict(n_layers=0),
                dict(n_layers=9), dict(n_out=0), dict(n_out=17), dict(n_slots=0), dict(n_slots=17),
                dict(tokens_bf16=2), dict(max_batch=0), dict(max_batch=(1 << 22) + 1), dict(abi_version=1)):
        assert f(ctypes.byref(cfg(**bad))) == -1, bad


def test_training_calls_reject_bad_arguments_before_any_cuda_call(lib):
    from paper_2505_08222_gb300 import _abi

    for name, (res, args) in _abi.SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    one = ctypes.c_void_p(16)
    assert lib.tfm_create(None, None, 0, None, ctypes.byref(ctypes.c_void_p())) == 1
    c = _abi.TfmConfig(_abi.UT_ABI_VERSION, 64, 2, 4, 7, 10, 1, 0, 8)
    assert lib.tfm_create(ctypes.byref(c), one, 5, None, ctypes.byref(ctypes.c_void_p())) == 1  # count mismatch
    # GAE: bad sizes, discount outside [0, 1], agent map without output
    assert lib.ppo_gae(one, one, one, 0, 4, 0.99, 0.95, one, one, None, 0, None, None) == 1
    assert lib.ppo_gae(one, one, one, 4, 4, 1.5, 0.95, one, one, None, 0, None, None) == 1
    assert lib.ppo_gae(one, one, one, 4, 4, 0.99, -0.1, one, one, None, 0, None, None) == 1
    assert lib.ppo_gae(one, one, one, 4, 4, 0.99, 0.95, one, one, one, 8, None, None) == 1
    assert lib.tfm_forward(None, one, one, one, None, 1, one, None) == 1
    assert lib.tfm_sync_policy(None, None) == 1
    assert lib.env_ppo_record(None, None, None, None, None) == 1
    bufs = _abi.PpoBuffers()
    assert lib.env_ppo_collect(None, None, 4, ctypes.byref(bufs)) == 1
    assert lib.env_ppo_collect(one, one, 0, ctypes.byref(bufs)) == 1  # T < 1
    assert lib.env_ppo_collect(one, one, 4, None) == 1
    assert lib.env_ppo_collect(one, one, 4, ctypes.byref(bufs)) == 1  # null buffers

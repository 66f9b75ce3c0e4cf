"""Resampling triggered by the effective sample size (the ESS option of the
filter, reading C23) in the oracle, pinned by reductions and brute force.

* k = 16: the trigger is 16 (sum r)^2 < 16 P sum r^2, which by Cauchy-Schwarz
  holds unless all quantised weights are equal, so the filter resamples at
  every step with a measurement, as the default filter does: the two
  trajectories are the same, bit for bit.
* Without resampling the weights carry over: with a deterministic predict
  (no acceleration noise) the weights after two steps are the normalised
  product of the two steps' range likelihoods (brute force in numpy).
* The trigger is the integer rule applied to the step's own max-normalised
  weights; when it fires, the resample map is the systematic map of those
  weights, else the identity."""
import numpy as np
import pytest

import oracle
from synth import preset


def _trigger(wmax, k, P):
    r = np.floor(np.asarray(wmax, np.float64) * 2.0 ** 38).astype(np.int64) >> 23
    s1, s2 = int(r.sum()), int((r * r).sum())
    return 16 * s1 * s1 < k * P * s2


@pytest.mark.parametrize("shared", [0, 1])
def test_k16_is_the_every_step_filter(shared):
    p = preset("fleet5", n_envs=3).replace(n_particles=64, d_model=0, comm_drop=0.2, det_radius=300.0,
                                           shared_filter=shared)
    a = oracle.OracleEnv(p, 31)
    b = oracle.OracleEnv(p.replace(pf_ess_num=16), 31)
    a.reset(0)
    b.reset(0)
    for t in range(1, 8):
        act = a.random_actions(t)
        ra, rb = a.step(act, want=("idx",)), b.step(act, want=("idx",))
        np.testing.assert_array_equal(ra["idx"], rb["idx"])
        np.testing.assert_array_equal(ra["err"], rb["err"])
    for k in ("px", "py", "pvx", "pvy", "estx", "esty"):
        np.testing.assert_array_equal(a.arr[k], b.arr[k], err_msg=k)
    assert np.all(b.arr["pw"] == 0.0)


def test_carried_weights_are_the_product_of_likelihoods():
    """Broad likelihood (sigma_r = 200 m), a low trigger (k = 1, ESS < P/16)
    and a deterministic predict (sigma_a = 0); the filters whose trigger did
    not fire at either step are compared."""
    sig = 200.0
    p = preset("fleet5", n_envs=2).replace(n_particles=48, d_model=0, pf_accel_sigma=0.0, range_sigma=sig,
                                           pf_ess_num=1)
    o = oracle.OracleEnv(p, 5)
    o.reset(0)
    P, AM = p.n_particles, p.max_agents
    want = ("meas", "meas_n", "pred_px", "weight", "wmax", "idx")
    loglik = np.zeros((o.F, P))
    kept = np.ones(o.F, bool)
    for t in range(1, 3):
        out = o.step(o.random_actions(t), want=want)
        x = out["pred_px"].reshape(o.F, P)
        y = out["pred_py"].reshape(o.F, P)
        for f in range(o.F):
            e = int(np.searchsorted(o.filter_off, f, side="right") - 1)
            k = (f - o.filter_off[e]) % o.n_targets_env[e]
            tz = o.arr["tz"][o.target_off[e] + k]
            for m in range(out["meas_n"][f]):
                qx, qy, qz, r = out["meas"][f, m]
                d = np.sqrt((x[f] - qx) ** 2 + (y[f] - qy) ** 2 + (tz - qz) ** 2)
                loglik[f] += -(r - d) ** 2 / (2 * sig * sig)
            if out["meas_n"][f] > 0 and _trigger(out["wmax"].reshape(o.F, P)[f], 1, P):
                kept[f] = False
    w = np.exp(loglik - loglik.max(1, keepdims=True))
    w /= w.sum(1, keepdims=True)
    got = out["weight"].reshape(o.F, P)
    np.testing.assert_allclose(got[kept], w[kept], rtol=1e-9, atol=1e-15)
    # the carried log-weights are log w - max log w: the summed log-likelihoods
    # shifted to a maximum of exactly 0
    pw = o.arr["pw"].reshape(o.F, P)
    np.testing.assert_allclose(pw[kept], (loglik - loglik.max(1, keepdims=True))[kept], rtol=1e-9, atol=1e-9)
    assert np.all(pw[kept].max(1) == 0.0)
    # the compared filters carried weights through two steps with measurements
    assert kept.sum() >= 10 and (out["meas_n"][kept] > 0).sum() >= 10


def test_trigger_is_the_integer_rule_on_the_weights():
    p = preset("fleet5", n_envs=4).replace(n_particles=128, d_model=0, pf_ess_num=8, det_radius=400.0,
                                           range_sigma=50.0)
    o = oracle.OracleEnv(p, 11)
    o.reset(0)
    P = p.n_particles
    fired = idle = 0
    for t in range(1, 7):
        g = o.step_count + 1
        out = o.step(o.random_actions(t), want=("wmax", "idx", "meas_n"))
        wmax = out["wmax"].reshape(o.F, P)
        idx = out["idx"].reshape(o.F, P)
        for f in range(o.F):
            trig = out["meas_n"][f] > 0 and _trigger(wmax[f], 8, P)
            if trig:
                r = oracle.philox([f, 0, g, 12], [11, 0])
                u64 = int(r[0]) | (int(r[1]) << 32)
                np.testing.assert_array_equal(idx[f], oracle.systematic_resample(wmax[f], u64))
                fired += 1
            else:
                np.testing.assert_array_equal(idx[f], np.arange(P))
                idle += 1
    assert fired > 0 and idle > 0

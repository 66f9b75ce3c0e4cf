"""Pins of the oracle's particle filter (Sec. II-A; one tracker per agent per
target, Sec. III-A.2) against closed forms, brute-force Bayes, exact-rational
systematic resampling and textbook least-squares trilateration."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle
from synth import preset


def _env(n_envs=2, seed=0, **kw):
    p = preset("fleet5", n_envs=n_envs).replace(**kw)
    e = oracle.OracleEnv(p, seed)
    e.reset(0)
    return e


def test_predict_closed_form_without_noise_or_measurements():
    """sigma_a = 0 and nothing heard: p_T = p_0 + T dt v, velocities unchanged."""
    e = _env(n_envs=2, n_particles=64, pf_accel_sigma=0.0, det_radius=0.0)
    rng = np.random.default_rng(1)
    vx = rng.uniform(-1, 1, e.F * 64)
    vy = rng.uniform(-1, 1, e.F * 64)
    e.set_arrays(pvx=vx, pvy=vy)
    px0, py0 = e.arr["px"].copy(), e.arr["py"].copy()
    for _ in range(7):
        o = e.step(np.full(e.NA, 3, np.int32), want=("idx",))
        assert np.all(o["idx"].reshape(e.F, 64) == np.arange(64))
    np.testing.assert_allclose(e.arr["px"], px0 + 7 * 30 * vx, atol=1e-9)
    np.testing.assert_allclose(e.arr["py"], py0 + 7 * 30 * vy, atol=1e-9)


def test_velocity_cap():
    """Speeds above v_cap (far above, and just above) are cut to v_cap with
    the direction kept; speeds below it are left unchanged."""
    e = _env(n_envs=1, n_particles=8, pf_accel_sigma=0.0, det_radius=0.0)
    cap = 1.2 * 1.5
    speed = np.array([5.0, 1.05 * cap, 1.5 * cap, 0.95 * cap, 0.5 * cap, 0.0, 2.5 * cap, 0.999 * cap])
    ang = np.linspace(0.3, 5.9, 8)
    vx = np.tile(speed * np.cos(ang), e.F)
    vy = np.tile(speed * np.sin(ang), e.F)
    e.set_arrays(pvx=vx, pvy=vy)
    e.step(np.full(e.NA, 3, np.int32))
    got = np.hypot(e.arr["pvx"], e.arr["pvy"])
    want = np.tile(np.minimum(speed, cap), e.F)
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-15)
    moving = np.tile(speed > 0, e.F)
    np.testing.assert_allclose(np.arctan2(e.arr["pvy"], e.arr["pvx"])[moving],
                               np.arctan2(vy, vx)[moving], rtol=1e-13, atol=1e-13)


def test_weights_brute_force_bayes_p4():
    """Posterior of 4 particles = normalised product of Gaussian range pdfs."""
    e = _env(n_envs=1, n_particles=4, pf_accel_sigma=0.0, range_sigma=3.0, target_depth_max=30.0)
    rng = np.random.default_rng(5)
    e.set_arrays(px=e.arr["px"] + rng.normal(0, 5, e.F * 4), pvx=np.zeros(e.F * 4), pvy=np.zeros(e.F * 4))
    o = e.step(np.full(e.NA, 3, np.int32), want=("pred_px", "weight", "meas", "meas_n"))
    for f in range(e.F):
        k = f % 5
        n = o["meas_n"][f]
        assert n > 0
        post = np.ones(4)
        for m in o["meas"][f, :n]:
            dist = np.sqrt((o["pred_px"][f * 4:f * 4 + 4] - m[0]) ** 2 + (o["pred_py"][f * 4:f * 4 + 4] - m[1]) ** 2
                           + (e.arr["tz"][k] - m[2]) ** 2)
            post *= stats.norm.pdf(m[3], loc=dist, scale=3.0)
        w = o["weight"][f * 4:f * 4 + 4]
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        if post.sum() > 1e-250:
            np.testing.assert_allclose(w, post / post.sum(), rtol=1e-9, atol=1e-15)


def test_single_measurement_argmax_is_nearest_to_range_circle():
    e = _env(n_envs=1, n_particles=256, max_agents=1, max_targets=1, pf_accel_sigma=0.0)
    rng = np.random.default_rng(2)
    e.set_arrays(px=e.arr["tx"][0] + rng.uniform(-300, 300, 256), py=e.arr["ty"][0] + rng.uniform(-300, 300, 256),
                 pvx=np.zeros(256), pvy=np.zeros(256))
    o = e.step(np.zeros(1, np.int32), want=("pred_px", "weight", "meas", "meas_n"))
    assert o["meas_n"][0] == 1
    qx, qy, _, r = o["meas"][0, 0]
    gap = np.abs(np.hypot(o["pred_px"] - qx, o["pred_py"] - qy) - r)
    assert np.argmax(o["weight"]) == np.argmin(gap)


def _brute_resample(wmax, u64):
    """Systematic resampling by its definition in exact rationals: weights
    quantised to q_i = floor(w_i 2^38), C_i = Q_i / W, u0 = floor(u64 W / 2^64) / W,
    u_j = (j + u0) / P, idx_j = min{i : C_i > u_j}."""
    P = len(wmax)
    q = [int(math.floor(Fraction(w) * 2 ** 38)) for w in wmax]
    Q = np.cumsum(q).tolist()
    W = Q[-1]
    u0 = Fraction((u64 * W) >> 64, W)
    out = []
    for j in range(P):
        u = (j + u0) / P
        out.append(next(i for i in range(P) if Fraction(Q[i], W) > u))
    return np.array(out)


@pytest.mark.parametrize("P", [1, 2, 3, 5, 8, 13, 16])
def test_resample_brute_force_small(P):
    rng = np.random.default_rng(P)
    for trial in range(40):
        if trial % 3 == 0:   # dyadic weights: exact in any summation order
            w = rng.integers(0, 9, P) / 8.0
        elif trial % 3 == 1:  # heavy-tailed
            w = np.exp(-rng.exponential(8.0, P))
        else:
            w = rng.uniform(0, 1, P)
        w[rng.integers(0, P)] = 1.0  # max-normalised
        u64 = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        np.testing.assert_array_equal(oracle.systematic_resample(w, u64), _brute_resample(w, u64))
    # exact ties P Q_i = j W + U0 (offset 0): uniform weights give the identity
    # map only under the strict rule C_i > u_j; dyadic weights tie often
    np.testing.assert_array_equal(oracle.systematic_resample(np.ones(P), 0), np.arange(P))
    for _ in range(10):
        w = rng.integers(1, 5, P) / 4.0
        w[0] = 1.0
        np.testing.assert_array_equal(oracle.systematic_resample(w, 0), _brute_resample(w, 0))


def _exact_resample_real(wmax, u64):
    """Systematic resampling (Sec. II-A) on the unquantised FP64 weights in
    exact rationals: C_i = S_i / S with S_i the partial sums of the weights,
    offset u0 = u64 / 2^64, u_j = (j + u0) / P, idx_j = min{i : C_i > u_j}
    (clamped to P - 1).  Returns the map and the CDF."""
    P = len(wmax)
    S, acc = [], Fraction(0)
    for w in wmax:
        acc += Fraction(float(w))
        S.append(acc)
    C = [x / acc for x in S]
    u0 = Fraction(u64, 2 ** 64)
    out, i = [], 0
    for j in range(P):
        u = (j + u0) / P
        while i < P - 1 and not C[i] > u:
            i += 1
        out.append(i)
    return np.array(out), C


@pytest.mark.parametrize("P", [1, 2, 3, 7, 16, 100, 1000])
def test_quantised_map_is_systematic_resampling_on_the_real_weights(P):
    """The oracle resamples on weights quantised to q_i = floor(w_i 2^38)
    (reading C5).  On the real (unquantised) weights, systematic resampling
    gives the same map except where a threshold u_j lies within
    (P + 2) 2^-38 of a CDF step: flooring moves each partial sum Q_i / W
    from S_i / S by less than P 2^-38 (every w <= 1 with max w = 1, so
    W >= 2^38), and the offset U0 / W lies within 1/W of u64 / 2^64.
    Weights below 2^-38 of the maximum (dropped by the quantisation) are the
    only other departure, and they fall under the same bound."""
    rng = np.random.default_rng(100 + P)
    delta = Fraction(P + 2, 2 ** 38)
    n_diff = 0
    for trial in range(30 if P < 1000 else 6):
        kind = trial % 3
        if kind == 0:
            w = rng.uniform(0, 1, P)
        elif kind == 1:
            w = np.exp(-rng.exponential(8.0, P))
        else:  # some weights below 2^-38 of the maximum
            w = np.exp(-rng.exponential(20.0, P))
            w[rng.integers(0, P, max(1, P // 4))] = rng.uniform(0, 2.0 ** -39, max(1, P // 4))
        w[rng.integers(0, P)] = 1.0
        u64 = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        got = oracle.systematic_resample(w, u64)
        want, C = _exact_resample_real(w, u64)
        for j in np.nonzero(got != want)[0]:
            u = (int(j) + Fraction(u64, 2 ** 64)) / P
            gap = min(abs(c - u) for c in C)
            assert gap <= delta, (P, trial, int(j), float(gap))
            n_diff += 1
    assert n_diff <= 2, n_diff  # a coincidence within 2^-30 is rare on random draws


def test_quantised_map_departs_only_within_the_bound_near_a_step():
    """A threshold placed inside a dropped weight's interval, or within a
    few 2^-38 of a CDF step, is where the two maps may differ; one placed
    well away from every step gives the same index."""
    P = 4
    tiny = 2.0 ** -40  # below 2^-38: quantised to 0
    w = np.array([1.0, tiny, 1.0, 1.0])
    S = np.cumsum([Fraction(float(x)) for x in w])
    C = [x / S[-1] for x in S]
    # u_1 = (1 + u0) / P inside (C_0, C_1]: the real map picks particle 1,
    # the quantised one (q_1 = 0) cannot
    u0 = (C[0] + C[1]) / 2 * P - 1
    assert 0 < u0 < 1
    u64 = int(u0 * 2 ** 64)
    got = oracle.systematic_resample(w, u64)
    want, _ = _exact_resample_real(w, u64)
    assert want[1] == 1 and got[1] == 2
    gap = min(abs(c - (1 + Fraction(u64, 2 ** 64)) / P) for c in C)
    assert gap <= Fraction(P + 2, 2 ** 38)
    # thresholds (j + 1/2) / P, far from every step (1/3, 1/3 + 2^-40, 2/3, 1): identical maps
    u64 = 2 ** 63
    np.testing.assert_array_equal(oracle.systematic_resample(w, u64), _exact_resample_real(w, u64)[0])


def test_resample_structure():
    rng = np.random.default_rng(9)
    P = 1000
    # uniform weights give the identity map
    np.testing.assert_array_equal(oracle.systematic_resample(np.ones(P), int(rng.integers(0, 2 ** 63))),
                                  np.arange(P))
    for _ in range(20):
        w = np.exp(-rng.exponential(2.0, P))
        w /= w.max()
        idx = oracle.systematic_resample(w, int(rng.integers(0, 2 ** 63)))
        assert np.all(np.diff(idx) >= 0)
        counts = np.bincount(idx, minlength=P)
        q = np.floor(w * 2 ** 38)
        expect = P * q / q.sum()
        assert np.all(counts >= np.floor(expect) - 1e-9) and np.all(counts <= np.ceil(expect) + 1e-9)


def _ls_trilateration(q, r):
    """Textbook linearised least squares: subtract the first circle equation."""
    A = 2 * (q[1:] - q[0])
    b = (r[0] ** 2 - r[1:] ** 2) + (q[1:] ** 2).sum(1) - (q[0] ** 2).sum()
    return np.linalg.lstsq(A, b, rcond=None)[0]


def test_static_target_trilateration_convergence():
    """Static target, three non-collinear agents circling, small range noise:
    the filter estimate converges to the truth and to the LS fix."""
    e = _env(n_envs=1, n_particles=2000, max_agents=3, max_targets=1, target_speed_min=0.0,
             target_speed_max=0.0, range_sigma=0.2, pf_accel_sigma=0.02, pf_vcap=0.05, heading_noise=0.0,
             target_drift_sigma=0.0)
    pooled = [[] for _ in range(3)]
    for t in range(40):
        o = e.step(np.array([6, 0, 5], np.int32), want=("meas", "meas_n"))
        for a in range(3):
            pooled[a].extend(o["meas"][a, :o["meas_n"][a]])
    truth = np.array([e.arr["tx"][0], e.arr["ty"][0]])
    for a in range(3):
        est = np.array([e.arr["estx"][a], e.arr["esty"][a]])
        assert np.linalg.norm(est - truth) < 1.0
        m = np.array(pooled[a])  # static target: every step's pings constrain the same point
        ls = _ls_trilateration(m[:, :2], m[:, 3])
        assert np.linalg.norm(ls - truth) < 1.0
        assert np.linalg.norm(est - ls) < 1.5


def test_estimate_motion_features_closed_form():
    """Identical particles, no noise, nothing heard: the estimate moves by
    u = dt v every step, so after n updates the last-motion feature is u / L
    and the smoothed motion is the geometric sum u (1 - 0.85^(n-1)) / L
    (reading C18: v <- 0.85 v + 0.15 (e1 - e2), v = 0 at reset)."""
    P = 16
    e = _env(n_envs=1, n_particles=P, pf_accel_sigma=0.0, det_radius=0.0, target_depth_max=0.0)
    F = e.F
    vx0, vy0 = 0.7, -0.4
    X, Y = np.linspace(-50, 50, F), np.linspace(20, 80, F)
    e.set_arrays(px=np.repeat(X, P), py=np.repeat(Y, P), pvx=np.full(F * P, vx0), pvy=np.full(F * P, vy0),
                 estx=X, esty=Y, prev_estx=X, prev_esty=Y, prev2_estx=X, prev2_esty=Y)
    L = e.p.est_scale
    for n in range(1, 9):
        e.step(np.full(e.NA, 3, np.int32))
        feat, _ = e.est_features(e.step_count)
        if n >= 2:
            np.testing.assert_allclose(feat[:, 80], 30 * vx0 / L, rtol=1e-9)
            np.testing.assert_allclose(feat[:, 81], 30 * vy0 / L, rtol=1e-9)
        np.testing.assert_allclose(feat[:, 82], 30 * vx0 * (1 - 0.85 ** (n - 1)) / L, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(feat[:, 83], 30 * vy0 * (1 - 0.85 ** (n - 1)) / L, rtol=1e-9, atol=1e-12)


def test_estimator_features_translation_invariant():
    """Features live in the estimate's local frame: shifting every position
    (estimates, ping senders, targets) by one vector leaves them unchanged;
    a ping whose range equals the 3-D distance from the estimate has zero
    innovation."""
    e = _env(n_envs=3, n_particles=32, comm_drop=0.0)
    for t in range(1, 5):
        e.step(np.random.default_rng(t).integers(0, 7, e.NA).astype(np.int32))
    f0, _ = e.est_features(e.step_count)
    shift = np.array([123.25, -77.5])
    ring = e.arr["ring"].reshape(e.F, 16, 4).copy()
    ring[:, :, 0] += shift[0]
    ring[:, :, 1] += shift[1]
    e.set_arrays(ring=ring.reshape(-1), **{k: e.arr[k] + shift[i % 2] for i, k in
                                           enumerate(["estx", "esty", "prev_estx", "prev_esty",
                                                      "prev2_estx", "prev2_esty", "tx", "ty"])})
    f1, _ = e.est_features(e.step_count)
    np.testing.assert_allclose(f1, f0, atol=1e-9)
    # zero innovation for a range equal to the distance from e1
    ring = e.arr["ring"].reshape(e.F, 16, 4).copy()
    head = e.arr["ring_head"]
    newest = (head - 1) % 16
    rows = np.arange(e.F)
    e1x, e1y = e.arr["prev_estx"], e.arr["prev_esty"]
    depth = np.array([e.arr["tz"][e.target_off[f // 25] + (f % 25) % 5] for f in range(e.F)])
    ring[rows, newest, 2] = np.sqrt((ring[rows, newest, 0] - e1x) ** 2 + (ring[rows, newest, 1] - e1y) ** 2
                                    + depth ** 2)
    e.set_arrays(ring=ring.reshape(-1))
    f2, _ = e.est_features(e.step_count)
    has = e.arr["ring_count"] > 0
    np.testing.assert_allclose(f2[has, 2], 0.0, atol=1e-12)

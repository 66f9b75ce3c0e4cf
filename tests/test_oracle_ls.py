"""Pins of the oracle's least-squares trilateration tracker (Sec. II-A;
Sec. III-A.2 names LS next to the particle filter; reading C21): exact
recovery of a static target from noise-free ranges, invariance to the
origin and to the order of the pings, and the hold rule for too few pings
or collinear senders."""
import numpy as np

import oracle
from synth import preset


def _env(depth=0.0):
    p = preset("fleet5", n_envs=2).replace(n_particles=16, d_model=0, target_depth_max=depth)
    o = oracle.OracleEnv(p, 3)
    o.reset(0)
    return o


def _set_rings(o, q, r, counts, head=None):
    ring = np.zeros((o.F, 16, 4))
    ring[:, :, 0] = q[..., 0]
    ring[:, :, 1] = q[..., 1]
    ring[:, :, 2] = r
    ring[:, :, 3] = 1.0
    o.set_arrays(ring=ring.reshape(-1), ring_count=counts,
                 ring_head=counts % 16 if head is None else head)


def _target_of_filter(o):
    f = np.arange(o.F)
    return (f // 25) * 5 + f % 5


def test_exact_static_target_from_noise_free_ranges():
    rng = np.random.default_rng(0)
    o = _env()
    tz = rng.uniform(0, 60, o.NT)
    o.set_arrays(tz=tz)
    tgt = _target_of_filter(o)
    x = np.stack([o.arr["tx"][tgt], o.arr["ty"][tgt]], 1)
    q = x[:, None, :] + rng.uniform(-800, 800, (o.F, 16, 2))
    r = np.sqrt(((q - x[:, None, :]) ** 2).sum(-1) + tz[tgt][:, None] ** 2)
    counts = rng.integers(3, 17, o.F).astype(np.int32)
    _set_rings(o, q, r, counts)
    o.set_arrays(estx=x[:, 0] + rng.normal(0, 300, o.F), esty=x[:, 1] + rng.normal(0, 300, o.F))
    err = o.ls_update()
    np.testing.assert_allclose(o.arr["estx"], x[:, 0], atol=1e-6)
    np.testing.assert_allclose(o.arr["esty"], x[:, 1], atol=1e-6)
    np.testing.assert_allclose(err, 0.0, atol=1e-6)


def test_origin_and_order_invariance():
    rng = np.random.default_rng(1)
    o = _env()
    q = rng.uniform(-1000, 1000, (o.F, 16, 2))
    r = rng.uniform(100, 900, (o.F, 16))
    counts = np.full(o.F, 16, np.int32)
    _set_rings(o, q, r, counts)
    e0 = rng.uniform(-200, 200, (o.F, 2))
    o.set_arrays(estx=e0[:, 0], esty=e0[:, 1])
    o.ls_update()
    ref = np.stack([o.arr["estx"], o.arr["esty"]], 1).copy()
    # another previous estimate (the local origin) and reversed ping order
    o2 = _env()
    _set_rings(o2, q[:, ::-1], r[:, ::-1], counts, head=np.full(o2.F, 7, np.int32))
    o2.set_arrays(estx=e0[:, 0] + 555.0, esty=e0[:, 1] - 321.0)
    o2.ls_update()
    np.testing.assert_allclose(np.stack([o2.arr["estx"], o2.arr["esty"]], 1), ref, atol=1e-6)


def test_hold_with_too_few_pings_or_collinear_senders():
    rng = np.random.default_rng(2)
    o = _env()
    q = rng.uniform(-500, 500, (o.F, 16, 2))
    q[1::2, :, 1] = 2.0 * q[1::2, :, 0] + 7.0  # odd filters: all senders on one line
    r = rng.uniform(100, 600, (o.F, 16))
    counts = np.where(np.arange(o.F) % 4 == 0, 2, 16).astype(np.int32)  # every 4th: two pings only
    _set_rings(o, q, r, counts)
    e0 = rng.uniform(-100, 100, (o.F, 2))
    o.set_arrays(estx=e0[:, 0], esty=e0[:, 1])
    o.ls_update()
    held = (np.arange(o.F) % 2 == 1) | (np.arange(o.F) % 4 == 0)
    np.testing.assert_array_equal(o.arr["estx"][held], e0[held, 0])
    assert np.all(o.arr["estx"][~held] != e0[~held, 0])
    np.testing.assert_array_equal(o.arr["prev_estx"], e0[:, 0])

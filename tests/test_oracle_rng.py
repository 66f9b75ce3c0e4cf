"""Pins of the oracle's Philox4x32-10 generator and its uniform / normal maps.

The published definition (Salmon et al., SC'11) is a 10-round bijection of the
128-bit counter for a fixed key.  These tests do not retype the forward
round: they invert it (the inverse uses the modular inverses of the
multipliers) and check statistics that any mistake in the mixing breaks.
"""
import numpy as np
import pytest
from scipy import stats

import oracle

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def _inverse_philox(out, key):
    """Undo the 10 rounds: lo0 = M0*c0 (mod 2^32) gives c0 via the inverse of
    M0, the recomputed high half unmasks c3, likewise c2 and c1."""
    inv0, inv1 = pow(M0, -1, 1 << 32), pow(M1, -1, 1 << 32)
    keys = [((key[0] + r * W0) & MASK, (key[1] + r * W1) & MASK) for r in range(10)]
    n0, n1, n2, n3 = (int(v) for v in out)
    for k0, k1 in reversed(keys):
        c0 = (n3 * inv0) & MASK
        c2 = (n1 * inv1) & MASK
        hi0 = (M0 * c0) >> 32
        hi1 = (M1 * c2) >> 32
        c3 = n2 ^ hi0 ^ k1
        c1 = n0 ^ hi1 ^ k0
        n0, n1, n2, n3 = c0, c1, c2, c3
    return [n0, n1, n2, n3]


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 2, 3, 4], [5, 6]),
    ([MASK, MASK, MASK, MASK], [MASK, MASK]),
    ([123456789, 0, 77, 11], [0xDEADBEEF, 42]),
])
def test_philox_is_invertible_round_function(ctr, key):
    out = oracle.philox(ctr, key)
    assert _inverse_philox(out, key) == ctr


def test_philox_avalanche():
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(200):
        ctr = rng.integers(0, 1 << 32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 1 << 32, 2, dtype=np.uint64).astype(np.uint32)
        a = oracle.philox(ctr, key)
        bit = rng.integers(0, 128)
        c2 = ctr.copy()
        c2[bit // 32] ^= np.uint32(1 << (bit % 32))
        b = oracle.philox(c2, key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    # a single input bit flips about half of the 128 output bits
    assert 60 < np.mean(flips) < 68


def test_uniform_and_normal_statistics():
    n = 20000
    us, ns = [], []
    for i in range(n // 4):
        u, z = oracle.uniform_normal(7, i, 3, 11, 9)
        us.extend(u)
        ns.extend(z)
    us, ns = np.array(us), np.array(ns)
    assert us.min() >= 0.0 and us.max() < 1.0
    # 24-bit grid: every uniform is k / 2^24
    assert np.all(np.floor(us * 2**24) == us * 2**24)
    assert stats.kstest(us, "uniform").pvalue > 1e-3
    assert abs(ns.mean()) < 0.03 and abs(ns.var() - 1.0) < 0.04
    assert stats.kstest(ns, "norm").pvalue > 1e-3
    # neighbouring counters are uncorrelated
    assert abs(np.corrcoef(us[:-4], us[4:])[0, 1]) < 0.03


def test_streams_differ_by_tag_step_and_seed():
    base = oracle.philox([5, 0, 9, 7], [1, 0])
    assert not np.array_equal(base, oracle.philox([5, 0, 9, 8], [1, 0]))
    assert not np.array_equal(base, oracle.philox([5, 0, 10, 7], [1, 0]))
    assert not np.array_equal(base, oracle.philox([5, 0, 9, 7], [2, 0]))

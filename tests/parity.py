"""Element-wise parity checks shared by the GPU tests and their CPU self-tests.

Every GPU result is compared with the FP64 oracle element by element.  For a
gradient the bound of an element is a fraction of the largest entry of its
tensor: BF16 operand rounding (unit roundoff u = 2^-8) perturbs each product
in proportion to the magnitudes of the operands, so errors scale with the
tensor's magnitude, not with each element's own value (an entry near zero
carries the same absolute error as a large one).
"""
from __future__ import annotations

import numpy as np

# Element-wise bound of the learned estimator's gradients (FP32 accumulation,
# BF16 tensor-core operands), as a fraction of each tensor's largest entry.
# BF16 rounds to nearest with unit roundoff u = 2^-8; the longest chain of
# roundings (dW1: two hidden activations, three backward dz images and the
# BF16 features of the first layer's weight gradient) perturbs each product
# by a few u in relative terms, and the errors of a sum over K = 256 terms or
# a batch of rows partly cancel.  A numpy error model of exactly those
# roundings (tests/test_parity_checks.py) lands at 4e-4 of the largest entry
# per tensor on the test's batch; the bound leaves a factor ~7 for the
# kernels' other differences (the GELU evaluations, summation orders).
EST_GRAD_FRAC = 3e-3


def tensor_slices(shapes):
    """(name, slice) of each tensor in a flat canonical parameter blob."""
    out, off = [], 0
    for name, shape, _ in shapes:
        n = int(np.prod(shape))
        out.append((name, slice(off, off + n), tuple(shape)))
        off += n
    return out


def elementwise_worst(got, ref, shapes, frac):
    """Worst ratio |got - ref| / (frac * max|ref|) over each tensor's elements
    (a ratio above 1 fails)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    worst = {}
    for name, sl, _ in tensor_slices(shapes):
        scale = frac * float(np.max(np.abs(ref[sl])))
        if scale == 0.0:
            worst[name] = 0.0 if np.all(got[sl] == 0.0) else np.inf
            continue
        worst[name] = float(np.max(np.abs(got[sl] - ref[sl])) / scale)
    return worst


def check_elementwise(got, ref, shapes, frac):
    """Assert |got - ref| <= frac * max|ref| for every element of every
    tensor; returns the worst ratio per tensor."""
    worst = elementwise_worst(got, ref, shapes, frac)
    bad = {k: v for k, v in worst.items() if not v <= 1.0}
    assert not bad, f"element-wise parity failed (ratio to bound): {bad}"
    return worst

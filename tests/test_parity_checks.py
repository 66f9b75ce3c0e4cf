"""CPU self-tests of the element-wise parity checks the GPU tests use.

1. The bound on the estimator's gradients holds for a BF16 error model of
   the GPU path: a numpy emulation of the tensor-core training pass (FP32
   accumulation, every tensor-core operand rounded to BF16 where the kernels
   round it) stays inside it against the FP64 oracle.
2. The same check rejects planted mistakes of the kind a wrong kernel makes:
   one row of a weight gradient lost, a transposed weight gradient, a sign
   error in one row.  The mistakes are made on the host, in a copy of the
   oracle's gradient with the model's BF16 errors added.
"""
import numpy as np
import pytest
from scipy.special import erf

import oracle
import synth
from parity import EST_GRAD_FRAC, check_elementwise, elementwise_worst, tensor_slices


def _gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def _gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def _bf(x):
    return synth.round_bf16(np.asarray(x, np.float32))


def bf16_model_grad(params, X, Y):
    """Gradient of the mean squared-error loss as the GPU path rounds it:
    FP32 arithmetic, hidden activations and backward dz images rounded to
    BF16 (the tensor-core operands), the first layer's features kept to
    FP32 accuracy (its forward multiplies BF16 high and low parts) but
    rounded to BF16 in its weight gradient, the output layer in FP32."""
    f = np.float32
    sl = {n: s for n, s, _ in tensor_slices(synth.mlp_shapes())}
    shp = {n: sh for n, _, sh in tensor_slices(synth.mlp_shapes())}
    W = {n: params[sl[n]].astype(f).reshape(shp[n]) for n in sl}
    X = X.astype(f)
    z1 = X @ W["W1"].T + W["b1"]
    a1 = _bf(_gelu(z1))
    z2 = a1 @ W["W2"].T + W["b2"]
    a2 = _bf(_gelu(z2))
    z3 = a2 @ W["W3"].T + W["b3"]
    a3 = _gelu(z3).astype(f)
    out = a3 @ W["W4"].T + W["b4"]
    B = X.shape[0]
    dout = ((out - Y) / f(B)).astype(f)
    g = np.zeros(params.size, np.float64)
    g[sl["W4"]] = (dout.T @ a3).ravel()
    g[sl["b4"]] = dout.sum(0)
    dz3 = (dout @ W["W4"]) * _gelu_grad(z3).astype(f)
    g[sl["b3"]] = dz3.sum(0)
    dz3b = _bf(dz3)
    dz2 = (dz3b @ W["W3"]) * _gelu_grad(z2).astype(f)
    g[sl["b2"]] = dz2.sum(0)
    dz2b = _bf(dz2)
    dz1 = (dz2b @ W["W2"]) * _gelu_grad(z1).astype(f)
    g[sl["b1"]] = dz1.sum(0)
    dz1b = _bf(dz1)
    g[sl["W3"]] = (dz3b.T @ a2).ravel()
    g[sl["W2"]] = (dz2b.T @ a1).ravel()
    g[sl["W1"]] = (dz1b.T @ _bf(X)).ravel()
    return g


def _case(seed=5, n=700):
    params = synth.mlp_params(seed=seed, bias_scale=0.1)
    rng = np.random.default_rng(seed + 1)
    X = np.zeros((n, 96), np.float32)
    cnt = rng.integers(1, 17, n)
    for s in range(16):
        on = s < cnt
        X[on, 5 * s:5 * s + 2] = rng.uniform(-0.3, 0.3, (on.sum(), 2))
        X[on, 5 * s + 2] = rng.uniform(0.02, 0.6, on.sum())
        X[on, 5 * s + 3] = (s // 5) / 16.0
        X[on, 5 * s + 4] = 1.0
    Y = (rng.standard_normal((n, 2)) * 0.2).astype(np.float32)
    _, ref = oracle.mlp_loss_grad(params, X, Y)
    return params, X, Y, ref


def test_bf16_error_model_stays_inside_the_gradient_bound():
    params, X, Y, ref = _case()
    got = bf16_model_grad(params, X, Y)
    worst = check_elementwise(got, ref, synth.mlp_shapes(), EST_GRAD_FRAC)
    print("BF16 model, worst ratio to the bound per tensor:", {k: round(v, 3) for k, v in worst.items()})
    # the model is not trivially exact, and the bound leaves it a margin
    assert 0.02 < max(worst.values()) < 0.5


@pytest.mark.parametrize("name", ["W1", "W2", "W3", "W4"])
def test_a_lost_row_of_a_weight_gradient_is_rejected(name):
    """Zero each row of the weight gradient in turn (a dropped row of an
    operand image or a skipped output tile): nearly every such copy fails."""
    params, X, Y, ref = _case()
    base = bf16_model_grad(params, X, Y)
    sl = {n: (s, sh) for n, s, sh in tensor_slices(synth.mlp_shapes())}[name]
    s, shape = sl
    rows = shape[0]
    caught = 0
    for r in range(rows):
        bad = base.copy()
        view = bad[s].reshape(shape)
        view[r] = 0.0
        worst = elementwise_worst(bad, ref, synth.mlp_shapes(), EST_GRAD_FRAC)
        caught += worst[name] > 1.0
    assert caught >= 0.9 * rows, (name, caught, rows)


def test_transposed_and_sign_errors_are_rejected():
    params, X, Y, ref = _case()
    base = bf16_model_grad(params, X, Y)
    slices = {n: (s, sh) for n, s, sh in tensor_slices(synth.mlp_shapes())}
    for name in ("W2", "W3"):
        s, shape = slices[name]
        bad = base.copy()
        bad[s] = base[s].reshape(shape).T.ravel()
        with pytest.raises(AssertionError):
            check_elementwise(bad, ref, synth.mlp_shapes(), EST_GRAD_FRAC)
    s, shape = slices["W1"]
    bad = base.copy()
    view = bad[s].reshape(shape)
    r = int(np.argmax(np.abs(view).max(1)))
    view[r] = -view[r]
    with pytest.raises(AssertionError):
        check_elementwise(bad, ref, synth.mlp_shapes(), EST_GRAD_FRAC)
    # a bias gradient from the wrong layer
    bad = base.copy()
    bad[slices["b2"][0]] = base[slices["b3"][0]]
    with pytest.raises(AssertionError):
        check_elementwise(bad, ref, synth.mlp_shapes(), EST_GRAD_FRAC)

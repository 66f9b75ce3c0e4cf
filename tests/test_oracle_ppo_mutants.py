"""The TransfMAPPO oracle's pins catch plausible mistakes: copies of
``oracle/utrack_oracle_ppo.c`` with one planted mistake each (a dropped term,
a wrong sign or factor, a swapped operand, a lost clip branch or episode-end
mask) are compiled on the CPU, and every copy must fail one of the checks
the pins use: central finite differences of the batch loss with every
parameter tensor probed, the closed forms of GAE, and agreement of the
training forward with the separately written agent forward.  The unmodified
source passes the same checks (the control case)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import synth

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "utrack_oracle_ppo.c")
D, L, H, NACT, NS = 16, 2, 2, 5, 6

MUTANTS = {
    "gelu_grad_drops_gaussian_term": ("+ x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);", ";"),
    "layernorm_bwd_drops_projection": ("- m1 - xh[i] * m2);", "- m1);"),
    "attention_dK_uses_K_for_Q": ("dQKV[u * 3 * d + d + hh * dh + j] += ds * QKV[t * 3 * d + hh * dh + j];",
                                  "dQKV[u * 3 * d + d + hh * dh + j] += ds * QKV[t * 3 * d + d + hh * dh + j];"),
    "attention_dV_transposed_P": ("+= Pt[u] * dO[t * d + hh * dh + j];", "+= P[((int64_t)hh * n + u) * n + t] * dO[t * d + hh * dh + j];"),
    "entropy_gradient_sign": ("+ ent_coef * pj * (lp + Hn);", "- ent_coef * pj * (lp + Hn);"),
    "clip_branch_lost": ("const double gl = s1 <= s2 ? -adv * r : 0.0;", "const double gl = -adv * r;"),
    "value_gradient_factor": ("dout[0] = 2.0 * e;", "dout[0] = e;"),
    "embedding_bias_gradient_lost": ("for (int j = 0; j < d; ++j) g->b_emb[j] += dX[t * d + j];", ""),
    "ffn_weight_gradient_transposed": ("outer_add(f, d, dZ, y, g->W1[l]);", "outer_add(f, d, dZ, y, g->W2[l]);"),
    "residual_gradient_lost": ("memcpy(dM, dX, sizeof(double) * n * d);", "memset(dM, 0, sizeof(double) * n * d);"),
    "gae_bootstrap_ignores_done": ("gamma * nd * value[(int64_t)(u + 1) * E + e]", "gamma * value[(int64_t)(u + 1) * E + e]"),
    "gae_drops_lambda": ("w *= gamma * lam;", "w *= gamma;"),
    "attention_scale_lost": ("s[u] = acc / sqrt((double)dh);", "s[u] = acc;"),
}


def _build(text, d):
    src = os.path.join(d, "m.c")
    so = os.path.join(d, "m.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-o", so, src, "-lm"],
                   check=True)
    lib = ctypes.CDLL(so)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    dims = ctypes.POINTER(oracle.OcPolicyDims)
    lib.oc_tfm_forward.argtypes = [dims, dp, ctypes.c_int32, ctypes.c_int32, dp, ip, dp, dp, dp]
    lib.oc_tfm_loss_grad.argtypes = [dims, dp, ctypes.c_int32, ctypes.c_int32, dp, ip, dp, ctypes.c_int32, ip, dp,
                                     dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
    lib.oc_tfm_loss_grad.restype = ctypes.c_double
    lib.oc_gae.argtypes = [ctypes.c_int32, ctypes.c_int32, dp, dp, ip, ctypes.c_double, ctypes.c_double, dp, dp]
    return lib


def _p(a, t=ctypes.c_double):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(t))


def _batch():
    rng = np.random.default_rng(81)
    n = 5
    ne = rng.integers(1, NS + 1, n).astype(np.int32)
    ne[0] = NS
    tok = np.ascontiguousarray(synth.random_tokens(n, NS, ne, seed=82), np.float64)
    h = 0.5 * rng.standard_normal((n, D))
    act = rng.integers(0, NACT, n).astype(np.int32)
    adv = rng.standard_normal(n)
    ret = rng.standard_normal(n)
    return tok, ne, h, act, adv, ret


def _loss(lib, prm, kind, no, logp_old, grad=None):
    tok, ne, h, act, adv, ret = _batch()
    dims = oracle.OcPolicyDims(D, L, H, no, 8)
    return lib.oc_tfm_loss_grad(ctypes.byref(dims), _p(prm), len(ne), NS, _p(tok), _p(ne, ctypes.c_int32), _p(h),
                                kind, _p(act, ctypes.c_int32), _p(logp_old), _p(adv), 0.2, 0.05, _p(ret), _p(grad),
                                None)


def _forward(lib, prm, no):
    tok, ne, h, *_ = _batch()
    dims = oracle.OcPolicyDims(D, L, H, no, 8)
    out = np.zeros((len(ne), no))
    lib.oc_tfm_forward(ctypes.byref(dims), _p(prm), len(ne), NS, _p(tok), _p(ne, ctypes.c_int32), _p(h), _p(out),
                       None)
    return out


def _gradient_ok(lib, kind):
    """Analytic gradient of the mutant against its own central differences,
    four entries of every parameter tensor probed."""
    no = NACT if kind == oracle.ACTOR else 1
    prm = synth.policy_params(synth.PolicyDims(D, L, H, no), seed=83).astype(np.float64)
    logp_old = None
    if kind == oracle.ACTOR:
        out = _forward(lib, prm, no)
        _, _, _, act, _, _ = _batch()
        m = out.max(1, keepdims=True)
        lp = (out - m - np.log(np.exp(out - m).sum(1, keepdims=True)))[np.arange(len(act)), act]
        logp_old = lp - np.log([1.1, 0.9, 1.5, 0.6, 1.0])  # unclipped, clipped both ways
    g = np.zeros_like(prm)
    _loss(lib, prm, kind, no, logp_old, g)
    o = 0
    idx = []
    for _, shape, _ in synth.policy_shapes(synth.PolicyDims(D, L, H, no)):
        n = int(np.prod(shape))
        idx += list(o + np.linspace(0, n - 1, min(4, n)).astype(int))
        o += n
    for i in idx:
        e = 1e-6
        p1, p2 = prm.copy(), prm.copy()
        p1[i] += e
        p2[i] -= e
        num = (_loss(lib, p1, kind, no, logp_old) - _loss(lib, p2, kind, no, logp_old)) / (2 * e)
        if abs(num - g[i]) > 1e-6 * max(1.0, abs(num)) + 1e-9:
            return False
    return True


def _gae_ok(lib):
    T, E = 6, 3
    rng = np.random.default_rng(84)
    r, v = rng.standard_normal((T, E)), rng.standard_normal((T + 1, E))
    done = np.zeros((T, E), np.int32)
    done[2, 1] = 1
    for gam, lam in ((0.9, 0.0), (1.0, 1.0)):
        adv, ret = np.zeros((T, E)), np.zeros((T, E))
        lib.oc_gae(T, E, _p(r), _p(v), _p(done, ctypes.c_int32), gam, lam, _p(adv), _p(ret))
        if lam == 0.0:
            want = r + gam * (1 - done) * v[1:] - v[:-1]
        else:
            want = np.zeros((T, E))
            for e in range(E):
                for t in range(T):
                    acc = 0.0
                    for u in range(t, T):
                        acc += r[u, e]
                        if done[u, e]:
                            break
                    else:
                        acc += v[T, e]
                    want[t, e] = acc - v[t, e]
        if not np.allclose(adv, want, rtol=1e-12, atol=1e-12):
            return False
    return True


def _forward_ok(lib):
    prm = synth.policy_params(synth.PolicyDims(D, L, H, NACT), seed=85).astype(np.float64)
    tok, ne, h, *_ = _batch()
    ref, _ = oracle.policy_forward(prm, D, L, H, tok, ne, h, n_act=NACT)
    return np.allclose(_forward(lib, prm, NACT), ref, rtol=1e-12, atol=1e-12)


def _all_pins(lib):
    return {"actor_grad": _gradient_ok(lib, oracle.ACTOR), "critic_grad": _gradient_ok(lib, oracle.CRITIC),
            "gae": _gae_ok(lib), "forward": _forward_ok(lib)}


@pytest.fixture(scope="module")
def workdir():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tempfile.mkdtemp()
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_unmodified_oracle_passes_every_pin(workdir):
    res = _all_pins(_build(open(SRC).read(), os.path.join(workdir)))
    assert all(res.values()), res


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(name, workdir):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site of {name} not unique in the source"
    d = os.path.join(workdir, name)
    os.makedirs(d, exist_ok=True)
    res = _all_pins(_build(text.replace(old, new), d))
    assert not all(res.values()), f"{name} passed every pin: {res}"

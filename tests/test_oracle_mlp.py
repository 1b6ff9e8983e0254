"""Pins of the MLP oracle: exact FP64 gradients against central finite
differences, the bfloat16 rounding against bit-level facts, and planted
mistakes in a copy of the backward pass."""
import inspect
import sys
import types

import numpy as np
import pytest

from oracle import mlp


def _tiny(seed=0, d_in=7, w=5, d_out=3, B=4):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(rng, d_in, w, d_out, out_gain=1.0)
    p = p + 0.1 * rng.normal(size=p.size)          # nonzero biases too
    x = rng.normal(size=(B, d_in))
    t = rng.normal(size=(B, d_out))
    return p, x, t, d_in, w, d_out


def _fd_grad(mod, p, x, t, d_in, w, d_out, h=1e-6):
    g = np.zeros_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = mod.loss_and_grads(p + e, x, t, d_in, w, d_out, bf16=False)
        lm, _ = mod.loss_and_grads(p - e, x, t, d_in, w, d_out, bf16=False)
        g[i] = (lp - lm) / (2 * h)
    return g


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradients_match_finite_differences(seed):
    p, x, t, d_in, w, d_out = _tiny(seed)
    _, g = mlp.loss_and_grads(p, x, t, d_in, w, d_out, bf16=False)
    np.testing.assert_allclose(g, _fd_grad(mlp, p, x, t, d_in, w, d_out), rtol=1e-6, atol=1e-9)


def test_bf16_rounding_bit_facts():
    # 1 + 2^-8 is exactly halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16_round(1.0 + 2 ** -8) == 1.0
    assert mlp.bf16_round(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    assert mlp.bf16_round(-(1.0 + 2 ** -7 + 2 ** -8)) == -(1.0 + 2 ** -6)   # tie, odd neighbour -> even
    v = np.random.default_rng(3).normal(size=1000)
    r = mlp.bf16_round(v)
    assert np.all(np.abs(r - v) <= 2 ** -8 * np.abs(v) * (1 + 1e-6))          # half an ulp (8-bit significand)
    assert np.all(mlp.bf16_round(r) == r)


def test_adam_first_step_moves_by_lr_times_sign():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    q, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(q, p - 0.01 * np.sign(g), rtol=1e-9)


MUTATIONS = {
    "tanh derivative sign": ("* (1.0 - h2 * h2)", "* (1.0 + h2 * h2)"),
    "transposed weight in backward": ("dh1 = (r(dh2) @ r(W2).T)", "dh1 = (r(dh2) @ r(W2))"),
    "missing factor 2 in dy": ("dy = 2.0 * e / (B * d_out)", "dy = e / (B * d_out)"),
    "bias grad from wrong layer": ("gb2 = dh2.sum(axis=0)", "gb2 = dh1.sum(axis=0)"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    src = inspect.getsource(mlp)
    assert old in src
    mod = types.ModuleType("mlp_mutant")
    sys.modules["mlp_mutant"] = mod
    try:
        exec(compile(src.replace(old, new), "mlp_mutant", "exec"), mod.__dict__)
    finally:
        del sys.modules["mlp_mutant"]
    p, x, t, d_in, w, d_out = _tiny(5, d_in=6, w=6, d_out=6)
    try:
        _, g = mod.loss_and_grads(p, x, t, d_in, w, d_out, bf16=False)
        ok = np.allclose(g, _fd_grad(mlp, p, x, t, d_in, w, d_out), rtol=1e-6, atol=1e-9)
    except Exception:
        ok = False
    assert not ok

"""Pins of the regressor oracle (Sec. V) and of the feature counts.

Each check ties the fp64 oracle to something other than itself: values of
the normal distribution, central finite differences of its own loss, torch's
fp64 autograd and AdamW, torch's bfloat16 rounding, textbook cases of the
bf16 format, a symplectic restatement of commutation and the closed-form
commuting probability of uniform strings.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_2401_06713_b300 import synth


def _theta(seed=3):
    return synth.mlp_init(seed).astype(np.float64)


def _data(B, seed=5):
    g = np.random.default_rng(seed)
    X = g.normal(0.0, 1.0, size=(B, mlp.N_IN))
    T = g.normal(0.0, 1.0, size=(B, mlp.N_OUT))
    return X, T


def test_param_count_and_layout():
    assert mlp.N_PARAMS == 64 * 5 + 64 + 64 * 64 + 64 + 2 * 64 + 2 == 4674
    th = np.arange(mlp.N_PARAMS, dtype=np.float64)
    p = mlp.unpack(th)
    assert p["W1"][1, 0] == 5 and p["b1"][0] == 320 and p["W2"][0, 1] == 385
    assert p["b3"][1] == mlp.N_PARAMS - 1
    np.testing.assert_array_equal(mlp.pack(p), th)


def test_gelu_normal_table_values():
    # Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208 (normal table)
    assert mlp.gelu(0.0) == 0.0
    assert mlp.gelu(1.0) == pytest.approx(0.8413447460685429, abs=1e-15)
    assert mlp.gelu(-1.0) == pytest.approx(-(1.0 - 0.8413447460685429), abs=1e-15)
    assert mlp.gelu(2.0) == pytest.approx(2.0 * 0.9772498680518208, abs=1e-14)
    assert mlp.gelu(40.0) == 40.0 and mlp.gelu(-40.0) == pytest.approx(0.0, abs=1e-300)
    for z in np.linspace(-6, 6, 49):
        h = 1e-6
        fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
        assert mlp.gelu_grad(z) == pytest.approx(fd, abs=1e-8)


def test_forward_matches_torch_fp64():
    th = _theta()
    X, _ = _data(7)
    p = {k: torch.tensor(v) for k, v in mlp.unpack(th).items()}
    x = torch.tensor(X)
    h = torch.nn.functional.gelu(torch.nn.functional.linear(x, p["W1"], p["b1"]), approximate="none")
    h = torch.nn.functional.gelu(torch.nn.functional.linear(h, p["W2"], p["b2"]), approximate="none")
    y = torch.nn.functional.linear(h, p["W3"], p["b3"]).numpy()
    np.testing.assert_allclose(mlp.forward(th, X), y, rtol=1e-12, atol=1e-12)


def test_backward_matches_finite_differences():
    th = _theta(11)
    X, T = _data(4, seed=12)
    w = (1.0, 0.5)
    g, L = mlp.backward(th, X, T, w)
    assert L == pytest.approx(mlp.loss(th, X, T, w), rel=1e-13)
    rng = np.random.default_rng(0)
    sizes = [int(np.prod(s)) for _, s in mlp.SHAPES]
    starts = np.cumsum([0] + sizes[:-1])
    # every block of the vector: 12 coordinates each, plus all of b3
    idx = sorted(set(int(i) for s, n in zip(starts, sizes) for i in s + rng.choice(n, min(n, 12), replace=False))
                 | {mlp.N_PARAMS - 1, mlp.N_PARAMS - 2})
    h = 1e-6
    for i in idx:
        tp = th.copy()
        tm = th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, X, T, w) - mlp.loss(tm, X, T, w)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_backward_matches_torch_autograd():
    th = _theta(21)
    X, T = _data(9, seed=22)
    w = (0.7, 1.3)
    g, L = mlp.backward(th, X, T, w)
    t = torch.tensor(th, requires_grad=True)
    p, at = {}, 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        p[name] = t[at:at + n].reshape(shape)
        at += n
    x = torch.tensor(X)
    h = torch.nn.functional.gelu(x @ p["W1"].T + p["b1"])
    h = torch.nn.functional.gelu(h @ p["W2"].T + p["b2"])
    y = h @ p["W3"].T + p["b3"]
    loss = ((y - torch.tensor(T)) ** 2 * torch.tensor(w, dtype=torch.float64)).sum() / (2 * len(X))
    loss.backward()
    np.testing.assert_allclose(g, t.grad.numpy(), rtol=1e-10, atol=1e-13)
    assert L == pytest.approx(float(loss.detach()), rel=1e-12)


def test_adamw_matches_torch():
    rng = np.random.default_rng(4)
    th = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    t = torch.tensor(th.copy(), requires_grad=True)
    opt = torch.optim.AdamW([t], lr=3e-3, betas=(0.9, 0.98), eps=1e-7, weight_decay=0.05)
    for step in range(1, 8):
        grad = rng.normal(size=50)
        th, m, v = mlp.adamw_step(th, grad, m, v, step, lr=3e-3, beta1=0.9, beta2=0.98, eps=1e-7,
                                  weight_decay=0.05)
        opt.zero_grad()
        t.grad = torch.tensor(grad)
        opt.step()
        # torch applies the decay as p *= 1 - lr wd before the Adam step;
        # the two forms differ by lr^2 wd terms
        np.testing.assert_allclose(th, t.detach().numpy(), rtol=0, atol=1e-6)


def test_adamw_first_step_is_sign_step():
    # with zero moments, step 1 moves every weight by lr * g / (|g| + eps)
    g = np.array([3.0, -0.25, 1e-3])
    th, _, _ = mlp.adamw_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1, eps=1e-12)
    np.testing.assert_allclose(th, -0.1 * np.sign(g), rtol=1e-9)


def test_bf16_rounding_textbook_cases_and_torch():
    cases = {1.0: 0x3F80, -2.0: 0xC000, 1.0 + 2 ** -8: 0x3F80, 1.0 + 3 * 2 ** -8: 0x3F82,
             1.0 + 2 ** -7: 0x3F81, 0.0: 0x0000, 65280.0: 0x477F}
    for x, bits in cases.items():
        assert int(mlp.to_bf16_bits(np.float32(x))) == bits, x
    r = np.random.default_rng(9).normal(size=10000).astype(np.float32)
    ties = (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32)
    allv = np.concatenate([r, ties, -ties])
    ref = torch.from_numpy(allv).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(mlp.to_bf16_bits(allv), ref)
    np.testing.assert_array_equal(mlp.bf16_bits_to_f64(np.array([0x3F80, 0xC000])), [1.0, -2.0])


def _symplectic_commute(a, b):
    xa, za = (a == 1) | (a == 2), (a == 2) | (a == 3)
    xb, zb = (b == 1) | (b == 2), (b == 2) | (b == 3)
    return (int(np.sum(xa & zb)) + int(np.sum(za & xb))) % 2 == 0


def test_feature_counts_brute_force():
    chars = synth.pauli_weighted(37, 13, 0.4, seed=8)
    seed, samples = 77, 500
    w, c = oracle.feature_counts(chars, seed, samples)
    assert w == int(np.count_nonzero(chars))
    n = len(chars)
    want = 0
    for p in range(samples):
        d0 = oracle.draw_u32(seed, 0, p, 3, 0)
        d1 = oracle.draw_u32(seed, 0, p, 3, 1)
        a = (d0 * n) >> 32
        b = (d1 * (n - 1)) >> 32
        b += b >= a
        assert a != b and 0 <= a < n and 0 <= b < n
        want += _symplectic_commute(chars[a], chars[b])
    assert c == want


def test_feature_pairs_are_distinct_strings():
    # two anticommuting strings: a sampler that could pick a string twice
    # would count commuting pairs
    chars = np.array([[1], [3]], dtype=np.uint8)
    assert oracle.feature_counts(chars, 5, 1000) == (2, 0)
    assert oracle.feature_counts(np.array([[2]], dtype=np.uint8), 5, 1000) == (1, 0)


def test_feature_density_closed_form():
    # i.i.d. uniform characters: a position anticommutes with probability
    # (3/4)^2 (2/3) = 3/8, so P(commute) = (1 + (1 - 3/4)^q) / 2
    q, n, s = 3, 4000, 40000
    chars = synth.pauli_uniform(n, q, seed=4)
    f = oracle.features(chars, seed=1, samples=s, budget_bytes=n * 1024.0)
    p = (1 + 0.25 ** q) / 2
    assert abs(f[3] - p) < 5 * math.sqrt(p * (1 - p) / s)
    assert abs(f[2] - 0.75) < 0.01
    # n = 4000, budget 1024 bytes per string: log2(ln 4000) - 3 and 10 / 4 - 3
    assert f[0] == pytest.approx(math.log2(8.294049640102028) - 3) and f[1] == q / 64
    assert f[4] == pytest.approx(-0.5)

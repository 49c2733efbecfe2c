"""fp64 oracle of the parameter regressor -- TEST INFRASTRUCTURE ONLY.

Sec. V of the paper predicts the palette fraction P' and the list factor
alpha from instance features with a regressor trained on grid-search labels
(Eq. ml is the objective the labels minimise).  The regressor here is a
5 -> 64 -> 64 -> 2 multilayer perceptron with the exact GELU

    h1 = gelu(W1 x + b1),  h2 = gelu(W2 h1 + b2),  y = W3 h2 + b3,
    gelu(z) = z * Phi(z) = z (1 + erf(z / sqrt 2)) / 2,

trained on the loss (1/B) sum_b sum_o w_o (y_bo - t_bo)^2 / 2 with AdamW
(Loshchilov & Hutter, "Decoupled Weight Decay Regularization", Algorithm 2:
Adam moments with bias correction, weight decay applied to the weights
directly, not through the gradient).

Everything here is plain numpy in float64, one sample at a time for the
forward and the backward, so each step can be checked by eye against the
chain rule.  Parameters are one flat vector in the order
W1[64][5] | b1[64] | W2[64][64] | b2[64] | W3[2][64] | b3[2] (row-major).
Only ``tests/`` may import this module.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_OUT = 5, 64, 2
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    """Split the flat parameter vector into named float64 arrays."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAMS,)
    out, at = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[at:at + size].reshape(shape)
        at += size
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def phi(z: float) -> float:
    """Standard normal density."""
    return math.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def Phi(z: float) -> float:
    """Standard normal distribution function, through erf."""
    return 0.5 * (1.0 + math.erf(z / math.sqrt(2.0)))


def gelu(z: float) -> float:
    return z * Phi(z)


def gelu_grad(z: float) -> float:
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return Phi(z) + z * phi(z)


def forward_one(p: dict, x: np.ndarray):
    """One sample: returns (y, cache) with the pre-activations for backward."""
    z1 = p["W1"] @ x + p["b1"]
    h1 = np.array([gelu(v) for v in z1])
    z2 = p["W2"] @ h1 + p["b2"]
    h2 = np.array([gelu(v) for v in z2])
    y = p["W3"] @ h2 + p["b3"]
    return y, (x, z1, h1, z2, h2)


def forward(theta: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Outputs [B][2] for inputs X [B][5]."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    return np.array([forward_one(p, x)[0] for x in X]).reshape(len(X), N_OUT)


def loss(theta: np.ndarray, X: np.ndarray, T: np.ndarray, w=(1.0, 1.0)) -> float:
    Y = forward(theta, X)
    D = Y - np.asarray(T, dtype=np.float64)
    return float(np.sum(np.asarray(w) * D * D) / (2.0 * len(X)))


def backward(theta: np.ndarray, X: np.ndarray, T: np.ndarray, w=(1.0, 1.0)):
    """(gradient of ``loss`` w.r.t. theta, loss), by the chain rule per sample."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    B = len(X)
    g = {name: np.zeros(shape) for name, shape in SHAPES}
    total = 0.0
    for b in range(B):
        y, (x, z1, h1, z2, h2) = forward_one(p, X[b])
        d = y - T[b]
        total += float(np.sum(w * d * d)) / (2.0 * B)
        dy = w * d / B                      # dL/dy
        g["W3"] += np.outer(dy, h2)
        g["b3"] += dy
        dh2 = p["W3"].T @ dy                # dL/dh2
        dz2 = dh2 * np.array([gelu_grad(v) for v in z2])
        g["W2"] += np.outer(dz2, h1)
        g["b2"] += dz2
        dh1 = p["W2"].T @ dz2
        dz1 = dh1 * np.array([gelu_grad(v) for v in z1])
        g["W1"] += np.outer(dz1, x)
        g["b1"] += dz1
    return pack(g), total


def adamw_step(theta, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
               eps: float = 1e-8, weight_decay: float = 0.0):
    """One AdamW step; returns (theta, m, v) as new float64 arrays."""
    theta = np.asarray(theta, dtype=np.float64)
    grad = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    theta = theta - lr * (m_hat / (np.sqrt(v_hat) + eps) + weight_decay * theta)
    return theta, m, v


def to_bf16_bits(a) -> np.ndarray:
    """bfloat16 bit patterns (uint16) of float32 values, round to nearest,
    ties to even: keep the top 16 bits of the float32 after adding
    0x7fff plus the lowest kept bit (finite inputs)."""
    bits = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def bf16_bits_to_f64(b) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


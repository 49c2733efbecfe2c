"""Seeded synthetic Pauli-string sets (the only module shared by the CUDA path
and the CPU oracle's tests; it holds none of the method's arithmetic).

The paper's molecular Hamiltonians (Sec. VI, dataset table) are not available,
so inputs are random Pauli strings with the shapes of its workloads: n strings
of q qubits, each character coded 0=I 1=X 2=Y 3=Z, row-major uint8 [n][q].

Laws:
  * ``uniform``: every position i.i.d. uniform over {I, X, Y, Z};
  * ``weighted``: every position non-identity with probability p, then X/Y/Z
    equiprobable -- low-weight, chemistry-like strings whose commuting
    fraction is about 1/2 (the paper's graphs are ~50% dense).
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed) & 0xFFFFFFFF, int(seed) >> 32, int(stream)]))


def pauli_uniform(n: int, q: int, seed: int, stream: int = 0) -> np.ndarray:
    """n strings of q characters, each uniform over {I, X, Y, Z}."""
    return _rng(seed, stream).integers(0, 4, size=(n, q), dtype=np.uint8)


def pauli_weighted(n: int, q: int, p: float, seed: int, stream: int = 0) -> np.ndarray:
    """n strings of q characters; non-identity w.p. p, then X/Y/Z uniform."""
    g = _rng(seed, stream)
    out = np.zeros((n, q), dtype=np.uint8)
    chunk = max(1, (1 << 24) // max(q, 1))
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        nz = g.random((e - s, q), dtype=np.float32) < np.float32(p)
        which = g.integers(1, 4, size=(e - s, q), dtype=np.uint8)
        out[s:e] = np.where(nz, which, 0).astype(np.uint8)
    return out


def batch_specs(count: int, seed: int, n_lo: int = 1000, n_hi: int = 50000,
                qs=(16, 24, 32, 48, 64), p_lo: float = 0.1, p_hi: float = 0.5):
    """Shapes of a batch of independent sets: n log-uniform in [n_lo, n_hi],
    q uniform over ``qs``, weight p uniform in [p_lo, p_hi]."""
    g = _rng(seed, 1 << 20)
    out = []
    for _ in range(count):
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        q = int(qs[int(g.integers(0, len(qs)))])
        p = float(g.uniform(p_lo, p_hi))
        out.append((n, q, p))
    return out


def batch_sets(count: int, seed: int, **kw):
    """List of (chars, n, q, p) for a batch drawn by ``batch_specs``."""
    sets = []
    for i, (n, q, p) in enumerate(batch_specs(count, seed, **kw)):
        sets.append((pauli_weighted(n, q, p, seed, stream=i + 1), n, q, p))
    return sets


def budget_bytes(n: int, g: np.random.Generator, lo: float = 9.0, hi: float = 15.0) -> float:
    """A memory budget for one instance's conflict structure: n * 2^u bytes,
    u uniform in [lo, hi] (from about 128 to 8192 int32 entries per vertex)."""
    return float(n) * 2.0 ** g.uniform(lo, hi)


def learned_specs(count: int, seed: int, n_lo: int = 1000, n_hi: int = 50000, qs=(16, 24, 32, 48, 64),
                  p_lo: float = 0.1, p_hi: float = 0.5, budget_lo: float = 9.0, budget_hi: float = 15.0):
    """Instances of the parameter-regressor data set: (n, q, p, budget_bytes,
    string seed, stream); shapes as ``batch_specs``, plus a budget."""
    g = _rng(seed, 1 << 21)
    out = []
    for i, (n, q, p) in enumerate(batch_specs(count, seed, n_lo=n_lo, n_hi=n_hi, qs=qs, p_lo=p_lo, p_hi=p_hi)):
        out.append((n, q, p, budget_bytes(n, g, budget_lo, budget_hi), seed, i + 1))
    return out


def mlp_init(seed: int, n_in: int = 5, n_hid: int = 64, n_out: int = 2) -> np.ndarray:
    """Initial weights of the n_in-n_hid-n_hid-n_out regressor as one float32
    vector W1 | b1 | W2 | b2 | W3 | b3 (row-major): weights normal with std
    sqrt(2 / fan_in), biases zero."""
    g = _rng(seed, 1 << 22)
    parts = []
    for rows, cols in ((n_hid, n_in), (n_hid, n_hid), (n_out, n_hid)):
        parts.append(g.normal(0.0, math.sqrt(2.0 / cols), size=rows * cols))
        parts.append(np.zeros(rows))
    return np.concatenate(parts).astype(np.float32)

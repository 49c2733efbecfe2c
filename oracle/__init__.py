"""CPU oracle for Picasso (arXiv 2401.06713) -- TEST INFRASTRUCTURE ONLY.

Plain C (``picasso_oracle.c``) behind ctypes.  Only ``tests/``, the smoke check
in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package.  It shares no code with the CUDA library: the Pauli predicate uses
the paper's 3-bit code (Sec. III-A), Philox4x32-10 and Floyd's sampling are
written out again from their published definitions.

Function map (paper passage each follows):
  philox4x32_10     Salmon et al., SC'11 (the counter-based generator)
  draw_list         Alg. 1 assign_rand_list_colors, Floyd's sampling
  priority          static Random order of Sec. III-B
  commute_chars     Sec. III-A, character comparison (anticommute iff odd count)
  encode3/commute3  Sec. III-A, inverse one-hot code + AND + popcount parity
  conflict_*        Alg. 1 construct_conflict_graph (color-major rows: per
                    list color, the commuting vertices holding it)
  conflict_edges    Sec. III-A's G_c with each edge once (commute and lists
                    meet)
  color_greedy      Sec. III-B static order, first available list color
  round_params      Table I / Sec. VI parameter rule
  run               Alg. 1, all rounds
  feature_counts    instance features of the Sec. V regressor (counts)
  features          the five regressor inputs from those counts
  mlp (module)      the Sec. V regressor as a 5-64-64-2 MLP, fp64 forward /
                    backward / AdamW (``oracle.mlp``)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "picasso_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TAG_LIST = 1
TAG_PRIO = 2

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", _SRC, "-o", _LIB, "-lm"]
        )
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_draw_u32.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_uint32]
        L.orc_draw_u32.restype = ctypes.c_uint32
        L.orc_priority.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64]
        L.orc_priority.restype = ctypes.c_uint32
        L.orc_draw_list.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int32, ctypes.c_int64, _i64p]
        L.orc_commute_chars.argtypes = [_u8p, _u8p, ctypes.c_int32]
        L.orc_commute_chars.restype = ctypes.c_int
        L.orc_words3.argtypes = [ctypes.c_int32]
        L.orc_words3.restype = ctypes.c_int32
        L.orc_encode3.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int32, _u32p]
        L.orc_commute3.argtypes = [_u32p, _u32p, ctypes.c_int32]
        L.orc_commute3.restype = ctypes.c_int
        L.orc_min_shared.argtypes = [_i64p, _i64p, ctypes.c_int32]
        L.orc_min_shared.restype = ctypes.c_int64
        L.orc_conflict_rows.argtypes = [ctypes.c_int64, _u32p, ctypes.c_int32, _i64p, ctypes.c_int32, _i64p,
                                        ctypes.c_int64, _i64p, _i64p, _i32p, ctypes.c_int32]
        L.orc_conflict_nnz.argtypes = [ctypes.c_int64, _u32p, ctypes.c_int32, _i64p, ctypes.c_int32, _i64p,
                                       ctypes.c_int32]
        L.orc_conflict_nnz.restype = ctypes.c_int64
        L.orc_conflict_fill.argtypes = [ctypes.c_int64, _u32p, ctypes.c_int32, _i64p, ctypes.c_int32, _i64p,
                                        _i64p, _i32p, ctypes.c_int32]
        L.orc_conflict_collect.argtypes = [ctypes.c_int64, _u32p, ctypes.c_int32, _i64p, ctypes.c_int32, _i64p,
                                           ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _i64p,
                                           ctypes.POINTER(_i32p)]
        L.orc_conflict_collect.restype = ctypes.c_int64
        L.orc_free.argtypes = [ctypes.c_void_p]
        L.orc_color_greedy.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, _i64p, _i64p,
                                       ctypes.c_int32, _i64p, _i32p, ctypes.c_int64, ctypes.c_int64, _i64p]
        L.orc_color_greedy.restype = ctypes.c_int64
        L.orc_draw_lists_many.argtypes = [ctypes.c_uint64, ctypes.c_int32, _i64p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_int64, _i64p]
        L.orc_priorities_many.argtypes = [ctypes.c_uint64, ctypes.c_int32, _i64p, ctypes.c_int64, _u32p]
        L.orc_round_params.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                       _i64p, _i32p]
        L.orc_run.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64,
                              ctypes.c_int64, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _i64p, _i64p]
        L.orc_run.restype = ctypes.c_int32
        L.orc_run_colorer.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64,
                                      ctypes.c_int64, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, _i64p, _i64p]
        L.orc_run_colorer.restype = ctypes.c_int32
        L.orc_color_dynamic.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, _i64p, _i64p,
                                        ctypes.c_int32, _i64p, _i32p, _i64p]
        L.orc_color_dynamic.restype = ctypes.c_int64
        L.orc_color_dynamic_par.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, _i64p, _i64p,
                                            ctypes.c_int32, _i64p, _i32p, _i64p, _i64p]
        L.orc_color_dynamic_par.restype = ctypes.c_int64
        L.orc_feature_counts.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64,
                                         _i64p]
        _lib = L
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def draw_u32(seed: int, rnd: int, gid: int, tag: int, i: int) -> int:
    return int(lib().orc_draw_u32(seed, rnd, gid, tag, i))


def priority(seed: int, rnd: int, gid: int) -> int:
    return int(lib().orc_priority(seed, rnd, gid))


def priorities(seed: int, rnd: int, gids) -> np.ndarray:
    gids = np.ascontiguousarray(np.asarray(list(gids) if not isinstance(gids, np.ndarray) else gids,
                                           dtype=np.int64))
    out = np.zeros(max(len(gids), 1), dtype=np.uint32)
    lib().orc_priorities_many(seed, rnd, _p(gids, _i64p), len(gids), _p(out, _u32p))
    return out[:len(gids)]


def draw_list(seed: int, rnd: int, gid: int, P: int, L: int, base: int = 0) -> np.ndarray:
    out = np.zeros(max(L, 1), dtype=np.int64)
    lib().orc_draw_list(seed, rnd, gid, P, L, base, _p(out, _i64p))
    return out[:L]


def draw_lists(seed: int, rnd: int, gids, P: int, L: int, base: int = 0) -> np.ndarray:
    gids = np.ascontiguousarray(np.asarray(gids, dtype=np.int64))
    out = np.zeros((max(len(gids), 1), L), dtype=np.int64)
    lib().orc_draw_lists_many(seed, rnd, _p(gids, _i64p), len(gids), P, L, base, _p(out, _i64p))
    return out[:len(gids)]


def commute_chars(a, b) -> bool:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint8))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.uint8))
    return bool(lib().orc_commute_chars(_p(a, _u8p), _p(b, _u8p), len(a)))


def encode3(chars: np.ndarray) -> np.ndarray:
    chars = np.ascontiguousarray(chars, dtype=np.uint8)
    n, q = chars.shape
    w3 = int(lib().orc_words3(q))
    enc = np.zeros((n, w3), dtype=np.uint32)
    lib().orc_encode3(_p(chars, _u8p), n, q, _p(enc, _u32p))
    return enc


def commute3(ea, eb) -> bool:
    ea = np.ascontiguousarray(ea, dtype=np.uint32)
    eb = np.ascontiguousarray(eb, dtype=np.uint32)
    return bool(lib().orc_commute3(_p(ea, _u32p), _p(eb, _u32p), len(ea)))


def min_shared(a, b) -> int:
    a = np.ascontiguousarray(a, dtype=np.int64)
    b = np.ascontiguousarray(b, dtype=np.int64)
    return int(lib().orc_min_shared(_p(a, _i64p), _p(b, _i64p), len(a)))


def round_params(n: int, num: int, den: int, alpha: float):
    P = ctypes.c_int64()
    L = ctypes.c_int32()
    lib().orc_round_params(n, num, den, alpha, ctypes.byref(P), ctypes.byref(L))
    return int(P.value), int(L.value)


def _collect(enc: np.ndarray, lists: np.ndarray, rows, edges: int, threads: int | None):
    enc = np.ascontiguousarray(enc, dtype=np.uint32)
    lists = np.ascontiguousarray(lists, dtype=np.int64)
    n, w3 = enc.shape
    L = lists.shape[1]
    if rows is None:
        m, rp = n, None
    else:
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        m, rp = len(rows), _p(rows, _i64p)
    off = np.zeros(m + 1, dtype=np.int64)
    colp = _i32p()
    nnz = lib().orc_conflict_collect(n, _p(enc, _u32p), w3, _p(lists, _i64p), L, rp, m, edges,
                                     threads or default_threads(), _p(off, _i64p), ctypes.byref(colp))
    col = np.ctypeslib.as_array(colp, shape=(max(nnz, 1),))[:nnz].copy()
    lib().orc_free(ctypes.cast(colp, ctypes.c_void_p))
    return off, col


def conflict_csr(enc: np.ndarray, lists: np.ndarray, threads: int | None = None):
    """Whole conflict CSR (off int64 [n+1], col int32) of one round, in the
    color-major layout (a neighbour once per shared color)."""
    return _collect(enc, lists, None, 0, threads)


def conflict_edges(enc: np.ndarray, lists: np.ndarray, threads: int | None = None):
    """The paper's G_c with each edge once: (off int64 [n+1], col int32), row
    u holding the partners v > u (ascending) that commute with u and share a
    list color with it."""
    return _collect(enc, lists, None, 1, threads)


def conflict_rows(enc: np.ndarray, lists: np.ndarray, rows, threads: int | None = None):
    """Selected rows: returns (lens int64 [m], list of int32 arrays)."""
    off, col = _collect(enc, lists, rows, 0, threads)
    m = len(off) - 1
    return np.diff(off), [col[off[i]:off[i + 1]].copy() for i in range(m)]


def color_greedy(seed: int, rnd: int, gids, lists, off, col, P: int, base: int) -> np.ndarray:
    gids = np.ascontiguousarray(np.asarray(gids, dtype=np.int64))
    lists = np.ascontiguousarray(lists, dtype=np.int64)
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = len(gids)
    L = lists.shape[1] if lists.ndim == 2 else 0
    out = np.zeros(max(n, 1), dtype=np.int64)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    lib().orc_color_greedy(seed, rnd, n, _p(gids, _i64p), _p(lists, _i64p), L, _p(off, _i64p), _p(col, _i32p),
                           P, base, _p(out, _i64p))
    return out[:n]


def color_dynamic(seed: int, rnd: int, gids, lists, off, col, parallel: bool = False):
    """Alg. 2 on the two-sided rows (off, col) of G_c: sequential (parallel
    False) or its parallel rule.  Returns (colors int64 [n] or -1, steps)."""
    gids = np.ascontiguousarray(np.asarray(gids, dtype=np.int64))
    lists = np.ascontiguousarray(lists, dtype=np.int64)
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = len(gids)
    L = lists.shape[1] if lists.ndim == 2 else 0
    out = np.zeros(max(n, 1), dtype=np.int64)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    steps = ctypes.c_int64(0)
    if parallel:
        lib().orc_color_dynamic_par(seed, rnd, n, _p(gids, _i64p), _p(lists, _i64p), L, _p(off, _i64p),
                                    _p(col, _i32p), _p(out, _i64p), ctypes.byref(steps))
    else:
        lib().orc_color_dynamic(seed, rnd, n, _p(gids, _i64p), _p(lists, _i64p), L, _p(off, _i64p),
                                _p(col, _i32p), _p(out, _i64p))
    return out[:n], int(steps.value)


def run(chars: np.ndarray, seed: int, num: int, den: int, alpha: float, max_rounds: int = 4096,
        threads: int | None = None, colorer: str = "static"):
    """Alg. 1 end to end.  Returns (color int64 [N], rounds, stats [rounds][6])
    with stats columns (n, P, L, base, nnz, colored).  colorer: "static"
    (Random order, first fit), "dynamic" (Alg. 2) or "dynamic_par" (Alg. 2's
    parallel rule)."""
    chars = np.ascontiguousarray(chars, dtype=np.uint8)
    N, q = chars.shape
    color = np.zeros(max(N, 1), dtype=np.int64)
    stats = np.zeros((max_rounds, 6), dtype=np.int64)
    which = {"static": 0, "dynamic": 1, "dynamic_par": 2}[colorer]
    r = lib().orc_run_colorer(_p(chars, _u8p), N, q, seed, num, den, alpha, max_rounds,
                              threads or default_threads(), which, _p(color, _i64p), _p(stats, _i64p))
    if r < 0:
        raise RuntimeError("oracle run hit max_rounds")
    return color[:N], int(r), stats[:r].copy()


def feature_counts(chars: np.ndarray, seed: int, samples: int) -> tuple[int, int]:
    """(non-identity characters, commuting pairs among the Philox-drawn sample)."""
    chars = np.ascontiguousarray(chars, dtype=np.uint8)
    n, q = chars.shape
    out = np.zeros(2, dtype=np.int64)
    lib().orc_feature_counts(_p(chars, _u8p), n, q, seed, samples, _p(out, _i64p))
    return int(out[0]), int(out[1])


def features(chars: np.ndarray, seed: int, samples: int, budget_bytes: float) -> np.ndarray:
    """The five regressor inputs (fp64): log2(ln n) - 3 (-3 for n = 1), q / 64,
    mean weight / q, commuting fraction of the sample (1 without samples),
    log2(budget / n) / 4 - 3.  Conflict entries per vertex grow like
    density * (alpha ln n)^2 / (P / n), so size and budget enter on log scales."""
    import math

    n, q = chars.shape
    w, c = feature_counts(chars, seed, samples)
    s = samples if n >= 2 else 0
    return np.array([math.log2(math.log(n)) - 3.0 if n > 1 else -3.0, q / 64.0, w / (n * q),
                     c / s if s > 0 else 1.0, (math.log2(budget_bytes) - math.log2(n)) / 4.0 - 3.0],
                    dtype=np.float64)

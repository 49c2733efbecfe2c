"""Strings of more than 64 qubits (W = ceil(q / 64) words per part) against
the CPU oracle, which works from the characters at any q.

Integer work, bit-exact: packed words, conflict CSRs of both forms and both
conflict strategies, round colorings, whole runs (static and dynamic order,
batches, chunks under a byte budget) and the regressor's feature counts."""
import numpy as np
import pytest
import torch

from paper_2401_06713_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2401_06713_b300 import build, picasso

    build.build()
    assert torch.cuda.is_available()
    return picasso


def _xz(pc, chars):
    return pc.pack(torch.from_numpy(np.ascontiguousarray(chars)).cuda())


@pytest.mark.parametrize("q", [65, 100, 128, 129, 200, 1024])
def test_pack_words_wide(pc, orc, q):
    n = 333
    chars = synth.pauli_uniform(n, q, seed=q)
    xz = _xz(pc, chars).cpu().numpy().view(np.uint64)
    W = (q + 63) // 64
    assert xz.shape == (n, 2 * W)
    for w in range(W):
        part = chars[:, 64 * w:64 * (w + 1)]
        bits = np.uint64(1) << np.arange(part.shape[1], dtype=np.uint64)
        x = (((part == 1) | (part == 2)).astype(np.uint64) * bits).sum(1, dtype=np.uint64)
        z = (((part == 3) | (part == 2)).astype(np.uint64) * bits).sum(1, dtype=np.uint64)
        assert np.array_equal(xz[:, w], x) and np.array_equal(xz[:, W + w], z), w
    enc = orc.encode3(chars)
    rng = np.random.default_rng(q)
    for _ in range(200):
        u, v = rng.integers(0, n, 2)
        acc = 0
        for w in range(W):
            acc ^= int((xz[u, w] & xz[v, W + w]) ^ (xz[u, W + w] & xz[v, w]))
        assert (bin(acc).count("1") % 2 == 0) == orc.commute3(enc[u], enc[v])


def test_limits(pc):
    codes = torch.zeros((4, 1025), dtype=torch.uint8, device="cuda")
    with pytest.raises(pc.PicassoError) as e:
        pc.pack(codes)
    assert e.value.status == pc.ERR_UNSUPPORTED


def _lower(off, col):
    n = len(off) - 1
    rows = [col[off[u]:off[u + 1]] for u in range(n)]
    rows = [r[r < u] for u, r in enumerate(rows)]
    lo = np.zeros(n + 1, dtype=np.int64)
    lo[1:] = np.cumsum([len(r) for r in rows])
    return lo, (np.concatenate(rows) if n else np.zeros(0, np.int32)).astype(np.int32)


@pytest.mark.parametrize("algo", ["allpairs", "bucket"])
@pytest.mark.parametrize("n,q,P,L", [(1500, 96, 150, 12), (700, 128, 60, 20), (300, 200, 40, 8),
                                     (120, 1024, 10, 5), (2000, 65, 250, 16), (40, 700, 3, 3)])
def test_conflict_wide(pc, orc, algo, n, q, P, L):
    chars = synth.pauli_weighted(n, q, 0.1, seed=n + q)
    seed = 5
    for form in ("full", "earlier"):
        with pc.Picasso(_xz(pc, chars), q, seed=seed, algo=algo, csr=form) as p:
            p.assign_lists(P, L, 0)
            prio = orc.priorities(seed, 1, range(n)).astype(np.int64)
            order = np.lexsort((np.arange(n), prio))
            assert np.array_equal(p.round_state()[0].cpu().numpy().astype(np.int64), order)
            enc = orc.encode3(chars)[order]
            lists = orc.draw_lists(seed, 1, order, P, L, 0)
            off_r, col_r = orc.conflict_csr(enc, lists)
            if form == "earlier":
                off_r, col_r = _lower(off_r, col_r)
            n_rows, nnz = p.build_conflicts()
            assert (n_rows, nnz) == (n, len(col_r))
            off, col = p.csr()
            assert np.array_equal(off.cpu().numpy(), off_r)
            assert np.array_equal(col.cpu().numpy(), col_r)
            assert p.stats()["conflict_algo_used"] == pc.ALGOS[algo]


@pytest.mark.parametrize("color", ["auto", "sweep"])
def test_round_coloring_wide(pc, orc, color):
    n, q, P, L, seed = 3000, 128, 375, 17, 11
    chars = synth.pauli_weighted(n, q, 0.12, seed=2)
    lists = orc.draw_lists(seed, 1, np.arange(n), P, L, 0)
    off_r, col_r = orc.conflict_csr(orc.encode3(chars), lists)
    ref = orc.color_greedy(seed, 1, np.arange(n), lists, off_r, col_r, P, 0)
    with pc.Picasso(_xz(pc, chars), q, seed=seed, algo="bucket", color=color) as p:
        p.assign_lists(P, L, 0)
        p.build_conflicts()
        k = p.color()
        assert k == int((ref >= 0).sum())
        assert np.array_equal(p.colors().cpu().numpy(), ref)


def _run_both(pc, orc, chars, seed, num, den, alpha, **kw):
    ref, rounds, stats = orc.run(chars, seed, num, den, alpha, colorer=kw.pop("colorer", "static"))
    with pc.Picasso(_xz(pc, chars), chars.shape[1], seed=seed, palette=(num, den), alpha=alpha, **kw) as p:
        got, r = p.run()
        st = p.stats()
    assert r == rounds and np.array_equal(got.cpu().numpy(), ref)
    assert st["colors_used"] == int(stats[:, 1].sum())
    # the small-round engine takes strings of at most two words per part
    assert st["small_rounds"] == 0 or chars.shape[1] <= 128
    return st


@pytest.mark.parametrize("n,q,pw,num,den,alpha,algo", [
    (4000, 128, 0.12, 1, 8, 2.0, "auto"),      # the q=64 workloads' weight per qubit, twice the qubits
    (4000, 128, 0.12, 1, 8, 2.0, "allpairs"),
    (3000, 96, 0.2, 1, 16, 1.5, "auto"),
    (1200, 300, 0.05, 1, 4, 3.0, "auto"),
    (500, 1024, 0.02, 1, 8, 2.0, "auto"),
])
def test_run_wide(pc, orc, n, q, pw, num, den, alpha, algo):
    st = _run_both(pc, orc, synth.pauli_weighted(n, q, pw, seed=q), 3, num, den, alpha, algo=algo)
    if q <= 128 and algo == "auto":
        assert st["small_rounds"] > 0  # every round in the engine (n <= 16384)


def test_run_wide_dynamic(pc, orc):
    _run_both(pc, orc, synth.pauli_weighted(2500, 160, 0.1, seed=4), 8, 1, 8, 2.0, color="dynamic",
              colorer="dynamic_par")


def test_run_wide_chunked(pc, orc):
    chars = synth.pauli_weighted(5000, 130, 0.1, seed=6)
    _, _, ostats = orc.run(chars, 6, 1, 8, 2.0)
    budget = (8 * (5000 + 1) + 4 * int(ostats[0, 4]) // 2) // 3
    st = _run_both(pc, orc, chars, 6, 1, 8, 2.0, byte_budget=budget, budget_mode="chunk")
    assert st["round_chunks"] >= 3


def test_batch_wide(pc, orc):
    specs = [(900, 80, 0.2), (1600, 70, 0.25), (40, 75, 0.5)]
    sets = [synth.pauli_weighted(n, q, p, seed=2, stream=i) for i, (n, q, p) in enumerate(specs)]
    offs = [0]
    for c in sets:
        offs.append(offs[-1] + len(c))
    pad = np.zeros((offs[-1], 80), dtype=np.uint8)
    for k, c in enumerate(sets):
        pad[offs[k]:offs[k + 1], :c.shape[1]] = c
    seeds = [31, 32, 33]
    with pc.Picasso(_xz(pc, pad), 80, set_offsets=offs, seeds=seeds) as p:
        got, _ = p.run()
        got = got.cpu().numpy()
        assert p.stats()["small_rounds"] > 0  # two words per part: the engine runs the rounds
    for k, c in enumerate(sets):
        ref, _, _ = orc.run(c, seeds[k], 1, 8, 2.0)
        assert np.array_equal(got[offs[k]:offs[k + 1]], ref), k


@pytest.mark.parametrize("q", [100, 256])
def test_features_wide(pc, orc, q):
    chars = synth.pauli_weighted(3000, q, 0.1, seed=q)
    counts, _ = pc.features(_xz(pc, chars), q, seed=9, budget_bytes=1e8, samples=20000)
    assert tuple(counts.cpu().numpy().tolist()) == orc.feature_counts(chars, 9, 20000)


@pytest.mark.parametrize("n", [1, 2, 33])
def test_run_wide_edge_sizes(pc, orc, n):
    for small in ("auto", "off"):
        _run_both(pc, orc, synth.pauli_uniform(n, 100, seed=n), 2, 1, 8, 2.0, small=small)

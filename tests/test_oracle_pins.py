"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test fixes one part of the oracle against an independent source:
  * Philox4x32-10: published known-answer vectors (tests/golden);
  * the Pauli predicate: 2x2 / Kronecker matrix products (Sec. III-A states the
    commutation rule; numpy's matrix algebra decides it independently), and the
    complete-set degree invariant of the 4^q Pauli group;
  * Floyd's list sampling: uniformity over all L-subsets (chi-square) and exact
    support;
  * the conflict graph: brute force over characters and Python sets, and the
    closed-form expected sizes (shared-color count L^2 / P per pair and the
    list-intersection probability);
  * the coloring: L = P reduces the round to plain greedy coloring in the
    priority order (networkx.greedy_color), P >> n L^2 gives no conflicts,
    P = L = 1 gives a greedy maximal independent set, plus validity of a whole
    run of Alg. 1.
"""
import itertools
import math
import os

import networkx as nx
import numpy as np
import pytest

from paper_2401_06713_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

PAULI = [
    np.eye(2, dtype=complex),
    np.array([[0, 1], [1, 0]], dtype=complex),
    np.array([[0, -1j], [1j, 0]], dtype=complex),
    np.array([[1, 0], [0, -1]], dtype=complex),
]


def _matrix(s):
    m = np.ones((1, 1), dtype=complex)
    for ch in s:
        m = np.kron(m, PAULI[ch])
    return m


def _commute_by_matrices(a, b):
    A, B = _matrix(a), _matrix(b)
    return np.allclose(A @ B, B @ A)


# ---------------------------------------------------------------- Philox
def test_philox_known_answers(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_draw_stream_layout(orc):
    # Draw i of (seed, round, gid, tag) is word i%4 of block i//4: the counter
    # (gid_lo, gid_hi, round, tag<<24 | block) and key (seed_lo, seed_hi).
    seed, rnd, gid, tag = 0x1234_5678_9ABC_DEF0, 7, (3 << 32) + 11, 1
    for i in range(9):
        blk = orc.philox4x32_10([gid & 0xFFFFFFFF, gid >> 32, rnd, (tag << 24) | (i // 4)],
                                [seed & 0xFFFFFFFF, seed >> 32])
        assert orc.draw_u32(seed, rnd, gid, tag, i) == int(blk[i % 4])


# ---------------------------------------------------------------- predicate
def test_pauli_truth_table(orc):
    for a in range(4):
        for b in range(4):
            truth = _commute_by_matrices([a], [b])
            assert orc.commute_chars([a], [b]) == truth
            e = orc.encode3(np.array([[a], [b]], dtype=np.uint8))
            assert orc.commute3(e[0], e[1]) == truth


def test_pauli_strings_against_kronecker(orc):
    rng = np.random.default_rng(1)
    for q in (1, 2, 3, 4, 5):
        for _ in range(60):
            a = rng.integers(0, 4, q).astype(np.uint8)
            b = rng.integers(0, 4, q).astype(np.uint8)
            truth = _commute_by_matrices(a, b)
            assert orc.commute_chars(a, b) == truth
            e = orc.encode3(np.stack([a, b]))
            assert orc.commute3(e[0], e[1]) == truth


def test_encoding_word_boundaries(orc):
    # q spanning several 10-character words: commute3 == character rule.
    rng = np.random.default_rng(2)
    for q in (9, 10, 11, 20, 21, 48, 64, 65):
        s = rng.integers(0, 4, size=(40, q)).astype(np.uint8)
        e = orc.encode3(s)
        for i in range(40):
            for j in range(40):
                assert orc.commute3(e[i], e[j]) == orc.commute_chars(s[i], s[j])


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_complete_pauli_group_degree(orc, q):
    # Every non-identity string commutes with exactly half of the 4^q strings
    # (itself and I included); I commutes with all of them.
    allp = np.array(list(itertools.product(range(4), repeat=q)), dtype=np.uint8)
    e = orc.encode3(allp)
    for i in range(len(allp)):
        cnt = sum(orc.commute3(e[i], e[j]) for j in range(len(allp)))
        assert cnt == (4 ** q if i == 0 else 4 ** q // 2)


# ---------------------------------------------------------------- lists
def test_lists_distinct_sorted_in_range(orc):
    for (P, L) in [(1, 1), (5, 5), (250, 16), (62500, 21), (7, 3)]:
        for gid in range(50):
            lst = orc.draw_list(3, 2, gid, P, L, base=100)
            assert len(lst) == L
            assert np.all(np.diff(lst) > 0)
            assert lst[0] >= 100 and lst[-1] < 100 + P


def test_floyd_uniform_over_subsets(orc):
    from scipy.stats import chisquare

    P, L, N = 6, 3, 30000
    subsets = {s: 0 for s in itertools.combinations(range(P), L)}
    for gid in range(N):
        subsets[tuple(int(x) for x in orc.draw_list(11, 1, gid, P, L))] += 1
    counts = np.array(list(subsets.values()))
    assert counts.min() > 0
    assert chisquare(counts).pvalue > 1e-4


def test_floyd_marginals_large_palette(orc):
    # Each color is in a list with probability L/P.
    P, L, N = 40, 5, 20000
    hits = np.zeros(P)
    for gid in range(N):
        hits[orc.draw_list(5, 3, gid, P, L)] += 1
    expect = N * L / P
    assert np.all(np.abs(hits - expect) < 6 * math.sqrt(expect))


def test_round_params_workloads(orc):
    assert orc.round_params(2000, 1, 8, 2.0) == (250, 16)
    assert orc.round_params(100_000, 1, 8, 2.0) == (12500, 24)
    assert orc.round_params(1_000_000, 1, 16, 1.5) == (62500, 21)
    assert orc.round_params(1, 1, 8, 2.0) == (1, 1)
    assert orc.round_params(3, 1, 8, 2.0) == (1, 1)  # L capped by P
    assert orc.round_params(100, 3, 100, 30.0) == (3, 3)


# ---------------------------------------------------------------- conflict graph
def _brute_rows(chars, lists):
    """Row u: for each color of u's list in list order, the other vertices that
    commute with u (character rule) and hold that color, ascending."""
    n = len(chars)
    rows = []
    for u in range(n):
        row = []
        for c in lists[u].tolist():
            for v in range(n):
                if v == u or c not in set(lists[v].tolist()):
                    continue
                cnt = sum(1 for a, b in zip(chars[u], chars[v]) if a and b and a != b)
                if cnt % 2 == 0:
                    row.append(v)
        rows.append(row)
    return rows


@pytest.mark.parametrize("n,q,P,L", [(1, 5, 3, 2), (2, 3, 2, 1), (37, 6, 9, 3), (64, 20, 12, 4), (50, 3, 5, 5)])
def test_conflict_csr_brute_force(orc, n, q, P, L):
    chars = synth.pauli_uniform(n, q, seed=n * 7 + q)
    lists = orc.draw_lists(4, 1, np.arange(n), P, L)
    off, col = orc.conflict_csr(orc.encode3(chars), lists)
    rows = _brute_rows(chars, lists)
    assert off[0] == 0 and len(off) == n + 1
    for u in range(n):
        assert col[off[u]:off[u + 1]].tolist() == rows[u]


def test_conflict_rows_match_csr(orc):
    chars = synth.pauli_weighted(300, 48, 0.25, seed=3)
    lists = orc.draw_lists(9, 1, np.arange(300), 40, 6)
    enc = orc.encode3(chars)
    off, col = orc.conflict_csr(enc, lists)
    sample = [0, 17, 150, 299]
    lens, rows = orc.conflict_rows(enc, lists, sample)
    for i, u in enumerate(sample):
        assert lens[i] == off[u + 1] - off[u]
        assert rows[i].tolist() == col[off[u]:off[u + 1]].tolist()


def test_conflict_symmetric(orc):
    # (u, v) at color c iff (v, u) at color c; a pair appears once per shared color
    chars = synth.pauli_uniform(400, 20, seed=5)
    lists = orc.draw_lists(0, 1, np.arange(400), 50, 16)
    off, col = orc.conflict_csr(orc.encode3(chars), lists)
    triples = set()
    for u in range(400):
        seg = col[off[u]:off[u + 1]].tolist()
        per_color = [[] for _ in range(16)]
        k, at = 0, 0
        # runs are in list order; split the row by membership
        for v in seg:
            while lists[u][k] not in set(lists[v].tolist()) or (per_color[k] and per_color[k][-1] >= v):
                k += 1
            per_color[k].append(v)
        for k in range(16):
            for v in per_color[k]:
                triples.add((u, v, int(lists[u][k])))
    assert all((v, u, c) in triples for (u, v, c) in triples)
    assert len(triples) == len(col)


def test_conflict_count_closed_form(orc):
    # Two uniform L-subsets of a P-palette share L^2 / P colors on average
    # (each of u's L colors lies in v's list w.p. L/P), so the expected number
    # of (pair, shared color) entries is 2 * (#commuting pairs) * L^2 / P, and
    # the expected number of distinct conflict pairs is (#commuting pairs) *
    # (1 - C(P-L, L) / C(P, L)) (Sec. III-C: an edge is kept iff lists meet).
    n, q, P, L = 2000, 20, 250, 16
    chars = synth.pauli_uniform(n, q, seed=0)
    enc = orc.encode3(chars)
    # commuting pairs counted by the character rule on 3-bit words via numpy
    x = ((chars == 1) | (chars == 2)).astype(np.int64)
    z = ((chars == 3) | (chars == 2)).astype(np.int64)
    anti = (x @ z.T + z @ x.T) % 2
    n_comm = (int((anti == 0).sum()) - n) // 2
    p_meet = 1.0 - math.comb(P - L, L) / math.comb(P, L)
    for seed in range(3):
        lists = orc.draw_lists(seed, 1, np.arange(n), P, L)
        off, col = orc.conflict_csr(enc, lists)
        entries = len(col) // 2
        mean = n_comm * L * L / P
        assert abs(entries - mean) < 0.03 * mean, (entries, mean)
        distinct = sum(len(set(col[off[u]:off[u + 1]].tolist())) for u in range(n)) // 2
        mean_d = n_comm * p_meet
        assert abs(distinct - mean_d) < 0.03 * mean_d, (distinct, mean_d)


def _brute_edges(chars, lists):
    """G_c with each edge once: pairs u < v that commute (character rule) and
    whose lists share at least one color (Python sets)."""
    n = len(chars)
    sets = [set(l.tolist()) for l in lists]
    out = []
    for u in range(n):
        for v in range(u + 1, n):
            cnt = sum(1 for a, b in zip(chars[u], chars[v]) if a and b and a != b)
            if cnt % 2 == 0 and sets[u] & sets[v]:
                out.append((u, v))
    return out


@pytest.mark.parametrize("n,q,P,L", [(1, 5, 3, 2), (2, 3, 2, 1), (37, 6, 9, 3), (64, 20, 12, 4), (50, 3, 5, 5),
                                     (90, 8, 40, 2)])
def test_conflict_edges_brute_force(orc, n, q, P, L):
    chars = synth.pauli_uniform(n, q, seed=n * 5 + q)
    lists = orc.draw_lists(6, 1, np.arange(n), P, L)
    off, col = orc.conflict_edges(orc.encode3(chars), lists)
    got = [(u, int(v)) for u in range(n) for v in col[off[u]:off[u + 1]]]
    assert got == _brute_edges(chars, lists)


def test_conflict_edges_are_the_distinct_pairs_of_the_runs(orc):
    # the color-major rows list a pair once per shared color; their distinct
    # pairs are exactly the edge set
    chars = synth.pauli_weighted(500, 24, 0.3, seed=2)
    lists = orc.draw_lists(3, 1, np.arange(500), 60, 9)
    enc = orc.encode3(chars)
    off, col = orc.conflict_csr(enc, lists)
    eo, ec = orc.conflict_edges(enc, lists)
    runs = {(min(u, int(v)), max(u, int(v))) for u in range(500) for v in col[off[u]:off[u + 1]]}
    edges = {(u, int(v)) for u in range(500) for v in ec[eo[u]:eo[u + 1]]}
    assert runs == edges and len(edges) == len(ec)


def test_conflict_edges_closed_form(orc):
    # E|E_c| = (#commuting pairs) * (1 - C(P-L, L) / C(P, L)) on the n = 2,000
    # uniform workload (Sec. III-C: a commuting pair is kept iff its lists meet)
    n, q, P, L = 2000, 20, 250, 16
    chars = synth.pauli_uniform(n, q, seed=0)
    x = ((chars == 1) | (chars == 2)).astype(np.int64)
    z = ((chars == 3) | (chars == 2)).astype(np.int64)
    n_comm = (int((((x @ z.T + z @ x.T) % 2) == 0).sum()) - n) // 2
    mean = n_comm * (1.0 - math.comb(P - L, L) / math.comb(P, L))
    enc = orc.encode3(chars)
    for seed in range(3):
        _, col = orc.conflict_edges(enc, orc.draw_lists(seed, 1, np.arange(n), P, L))
        assert abs(len(col) - mean) < 0.03 * mean, (len(col), mean)


# ---------------------------------------------------------------- coloring
def test_full_palette_is_plain_greedy(orc):
    # L = P: every list is the whole palette, so the conflict graph is G' and
    # round 1 is sequential greedy coloring of G' in priority order.
    n, q = 120, 6
    chars = synth.pauli_uniform(n, q, seed=8)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    for u in range(n):
        for v in range(u + 1, n):
            if orc.commute_chars(chars[u], chars[v]):
                G.add_edge(u, v)
    P = max(d for _, d in G.degree()) + 1
    gids = np.arange(n)
    lists = orc.draw_lists(2, 1, gids, P, P)
    off, col = orc.conflict_csr(orc.encode3(chars), lists)
    color = orc.color_greedy(2, 1, gids, lists, off, col, P, 0)
    prio = orc.priorities(2, 1, gids).astype(np.uint64)
    order = sorted(range(n), key=lambda v: (int(prio[v]), v))
    ref = nx.greedy_color(G, strategy=lambda g, c: iter(order))
    assert all(int(color[v]) == ref[v] for v in range(n))


def test_no_conflicts_one_round(orc):
    n = 50
    chars = synth.pauli_uniform(n, 10, seed=1)
    color, rounds, stats = orc.run(chars, 0, 10**7, 1, 1.0)  # P = 10^7 n, L = ceil(ln n) = 4
    assert rounds == 1 and stats[0][4] == 0
    lists = orc.draw_lists(0, 1, np.arange(n), stats[0][1], int(stats[0][2]))
    assert np.array_equal(color, lists[:, 0])


def test_single_color_round_is_greedy_mis(orc):
    # P = L = 1: the round colors a maximal independent set of G', greedy in
    # priority order.
    n = 80
    chars = synth.pauli_uniform(n, 6, seed=4)
    gids = np.arange(n)
    lists = orc.draw_lists(3, 1, gids, 1, 1)
    off, col = orc.conflict_csr(orc.encode3(chars), lists)
    color = orc.color_greedy(3, 1, gids, lists, off, col, 1, 0)
    chosen = set(np.nonzero(color >= 0)[0].tolist())
    prio = orc.priorities(3, 1, gids).astype(np.uint64)
    order = sorted(range(n), key=lambda v: (int(prio[v]), v))
    mis = []
    for v in order:
        if all(not orc.commute_chars(chars[v], chars[u]) for u in mis):
            mis.append(v)
    assert chosen == set(mis)


def _check_valid_run(orc, chars, seed, num, den, alpha):
    color, rounds, stats = orc.run(chars, seed, num, den, alpha)
    n = len(chars)
    assert np.all(color >= 0)
    x = ((chars == 1) | (chars == 2)).astype(np.int64)
    z = ((chars == 3) | (chars == 2)).astype(np.int64)
    comm = ((x @ z.T + z @ x.T) % 2) == 0
    np.fill_diagonal(comm, False)
    same = color[:, None] == color[None, :]
    assert not np.any(comm & same)  # each color class is a clique of G
    # every color comes from the vertex's list in the round it was colored
    gids = np.arange(n)
    remaining = gids
    base = 0
    for r in range(rounds):
        P, L = int(stats[r][1]), int(stats[r][2])
        lists = orc.draw_lists(seed, r + 1, remaining, P, L, base)
        c = color[remaining]
        inround = (c >= base) & (c < base + P)
        for i in np.nonzero(inround)[0]:
            assert c[i] in lists[i]
        remaining = remaining[~inround]
        base += P
    assert len(remaining) == 0
    assert len(np.unique(color)) <= base
    return color, rounds, stats


def test_run_valid_workload_small(orc):
    chars = synth.pauli_uniform(2000, 20, seed=0)
    color, rounds, stats = _check_valid_run(orc, chars, 0, 1, 8, 2.0)
    assert stats[0][0] == 2000 and stats[0][1] == 250 and stats[0][2] == 16
    assert 1 <= rounds < 30


def test_run_valid_weighted(orc):
    chars = synth.pauli_weighted(700, 48, 0.25, seed=2)
    _check_valid_run(orc, chars, 5, 1, 16, 1.5)


# ------------------------------------------------------------ Alg. 2 (dynamic)
def _dyn_case(orc, n, q, P, L, seed, chars=None):
    if chars is None:
        chars = synth.pauli_uniform(n, q, seed=seed)
    gids = np.arange(n)
    lists = orc.draw_lists(seed, 1, gids, P, L)
    off, col = orc.conflict_csr(orc.encode3(chars), lists)
    return chars, gids, lists, off, col


@pytest.mark.parametrize("parallel", [False, True])
def test_dynamic_single_color_is_greedy_mis(orc, parallel):
    # P = L = 1: every list has one color, so the lowest bucket is always the
    # whole active set and both forms of Alg. 2 reduce to the maximal
    # independent set of G', greedy in priority order (the parallel rule is
    # the local-minimum iteration, whose fixed point is that same set)
    n = 90
    chars, gids, lists, off, col = _dyn_case(orc, n, 6, 1, 1, 7)
    color, _ = orc.color_dynamic(7, 1, gids, lists, off, col, parallel=parallel)
    chosen = set(np.nonzero(color >= 0)[0].tolist())
    prio = orc.priorities(7, 1, gids).astype(np.uint64)
    mis = []
    for v in sorted(range(n), key=lambda v: (int(prio[v]), v)):
        if all(not orc.commute_chars(chars[v], chars[u]) for u in mis):
            mis.append(v)
    assert chosen == set(mis)


@pytest.mark.parametrize("parallel", [False, True])
def test_dynamic_without_conflicts_takes_the_drawn_color(orc, parallel):
    # no pair commutes (each string anticommutes with every other: the
    # anticommuting set {X I.., Z I.., Y I..} extended by singles), so G_c has
    # no edge and every vertex takes the entry floor(x L / 2^32) of its list,
    # x = word 0 of its Philox stream with tag 4
    chars = np.array([[1, 0], [3, 0], [2, 0]], dtype=np.uint8)
    n = 3
    gids = np.arange(n) + 40
    P, L = 50, 7
    lists = orc.draw_lists(11, 2, gids, P, L)
    off, col = orc.conflict_csr(orc.encode3(chars), lists)
    assert off[-1] == 0
    color, _ = orc.color_dynamic(11, 2, gids, lists, off, col, parallel=parallel)
    for v in range(n):
        x = orc.draw_u32(11, 2, int(gids[v]), 4, 0)
        assert color[v] == lists[v][(x * L) >> 32]


@pytest.mark.parametrize("parallel", [False, True])
def test_dynamic_complete_graph_full_palette(orc, parallel):
    # identical strings all commute: G' is complete.  With L = P every list is
    # the whole palette, each coloring removes one color from every other
    # list, so exactly min(n, P) vertices are colored, all with distinct colors
    for n, P in ((12, 5), (6, 9)):
        chars = np.zeros((n, 4), dtype=np.uint8)
        gids = np.arange(n)
        lists = orc.draw_lists(2, 1, gids, P, P)
        off, col = orc.conflict_csr(orc.encode3(chars), lists)
        color, _ = orc.color_dynamic(2, 1, gids, lists, off, col, parallel=parallel)
        got = color[color >= 0]
        assert len(got) == min(n, P) and len(set(got.tolist())) == len(got)


@pytest.mark.parametrize("parallel", [False, True])
def test_dynamic_valid_and_blocked(orc, parallel):
    # a proper list coloring of G_c, and a vertex is left uncolored only when
    # every color of its list went to a conflict neighbour
    n, P, L = 400, 30, 5
    chars, gids, lists, off, col = _dyn_case(orc, n, 8, P, L, 5)
    color, steps = orc.color_dynamic(5, 1, gids, lists, off, col, parallel=parallel)
    assert (steps > 0) == parallel
    for v in range(n):
        nb = col[off[v]:off[v + 1]]
        taken = set(int(color[u]) for u in nb if color[u] >= 0)
        if color[v] >= 0:
            assert color[v] in lists[v] and color[v] not in taken
        else:
            assert set(lists[v].tolist()) <= taken


def test_dynamic_colors_more_than_static(orc):
    # Sec. III-B: the dynamic order (most constrained first) leaves fewer
    # vertices uncolored than the static Random order on the same round
    n, P, L = 3000, 375, 16
    chars, gids, lists, off, col = _dyn_case(orc, n, 24, P, L, 1)
    static = orc.color_greedy(1, 1, gids, lists, off, col, P, 0)
    dyn, _ = orc.color_dynamic(1, 1, gids, lists, off, col)
    par, _ = orc.color_dynamic(1, 1, gids, lists, off, col, parallel=True)
    s, d, p = int((static >= 0).sum()), int((dyn >= 0).sum()), int((par >= 0).sum())
    assert d > s and p > s

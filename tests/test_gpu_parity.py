"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work throughout, so every comparison is bit-exact: Philox draws,
packed words, lists, priorities, conflict CSR (row offsets, color-major
columns, run offsets), the round's coloring and whole runs of Alg. 1.  At the full workload sizes the oracle checks sampled rows exactly
and the whole coloring through properties that hold at any size.
"""
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


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


# ------------------------------------------------------------------ generators
def test_philox_draws(pc, orc):
    for (seed, rnd, gid, tag) in [(0, 1, 0, 1), (0xDEADBEEF12345678, 7, 123456, 2), (5, 3, (1 << 33) + 9, 1)]:
        got = _u32(pc.philox_draws(seed, rnd, gid, tag, 0, 64))
        ref = [orc.draw_u32(seed, rnd, gid, tag, i) for i in range(64)]
        assert got.tolist() == ref
    got = _u32(pc.philox_draws(9, 2, 77, 1, 1000, 8))
    assert got.tolist() == [orc.draw_u32(9, 2, 77, 1, 1000 + i) for i in range(8)]


@pytest.mark.parametrize("q", [20, 64])
def test_pack_other_bytes(pc, q):
    # bytes outside 0..3 are no Pauli code: both packing kernels (q = 64 takes
    # the 16-byte one, q = 20 the byte one) give them neither bit
    chars = np.random.default_rng(5).integers(0, 256, (513, q), dtype=np.uint8)
    xz = _xz(pc, chars).cpu().numpy().view(np.uint64)
    bits = np.uint64(1) << np.arange(q, dtype=np.uint64)
    x = (((chars == 1) | (chars == 2)).astype(np.uint64) * bits).sum(1, dtype=np.uint64)
    z = (((chars == 3) | (chars == 2)).astype(np.uint64) * bits).sum(1, dtype=np.uint64)
    assert np.array_equal(xz[:, 0], x) and np.array_equal(xz[:, 1], z)


@pytest.mark.parametrize("q", [1, 13, 16, 20, 32, 48, 64])
def test_pack_words(pc, orc, q):
    chars = synth.pauli_uniform(777, q, seed=q)
    xz = _xz(pc, chars).cpu().numpy().view(np.uint64)
    bits = np.uint64(1) << np.arange(q, dtype=np.uint64)
    x = (((chars == 1) | (chars == 2)).astype(np.uint64) * bits).sum(1, dtype=np.uint64)
    z = (((chars == 3) | (chars == 2)).astype(np.uint64) * bits).sum(1, dtype=np.uint64)
    assert np.array_equal(xz[:, 0], x) and np.array_equal(xz[:, 1], z)
    # the packed commutation test agrees with the oracle's 3-bit predicate
    enc = orc.encode3(chars)
    rng = np.random.default_rng(q)
    for _ in range(300):
        u, v = rng.integers(0, 777, 2)
        par = bin(int((xz[u, 0] & xz[v, 1]) ^ (xz[u, 1] & xz[v, 0]))).count("1") % 2
        assert (par == 0) == orc.commute3(enc[u], enc[v])


@pytest.mark.parametrize("n,P,L", [(2000, 250, 16), (5000, 7, 7), (300, 1000, 100), (150, 400, 300), (3, 1, 1)])
def test_lists_and_priorities(pc, orc, n, P, L):
    chars = synth.pauli_uniform(n, 8, seed=1)
    with pc.Picasso(_xz(pc, chars), 8, seed=42) as p:
        p.assign_lists(P, L, 17)
        gid, lists, prio = p.round_state()
        gid = gid.cpu().numpy().astype(np.int64)
        lists = lists.cpu().numpy().astype(np.int64)
        ref = orc.draw_lists(42, 1, np.arange(n), P, L, 0)
        ref_prio = orc.priorities(42, 1, range(n)).astype(np.int64)
        # round-local id t is the t-th vertex of the coloring order
        assert np.array_equal(np.sort(gid), np.arange(n))
        assert np.array_equal(gid, np.lexsort((np.arange(n), ref_prio)))
        assert np.array_equal(lists, ref[gid])
        assert np.array_equal(_u32(prio).astype(np.int64), ref_prio[gid])


# ------------------------------------------------------------------ conflict graph
def _ranked(p, orc, chars, seed, P, L):
    """Oracle inputs in the round's coloring order: the oracle's own priorities
    give the order, checked against the context's."""
    n = len(chars)
    prio = orc.priorities(seed, 1, range(n)).astype(np.int64)
    order = np.lexsort((np.arange(n), prio))
    gid = p.round_state()[0].cpu().numpy().astype(np.int64)
    assert np.array_equal(gid, order)
    enc = orc.encode3(chars)[order]
    lists = orc.draw_lists(seed, 1, order, P, L, 0)
    return order, enc, lists


def _lower(off, col):
    """Rows restricted to smaller partners (the EARLIER form of the CSR)."""
    n = len(off) - 1
    rows = [col[off[u]:off[u + 1]] for u in range(n)]
    rows = [r[r < u] for u, r in enumerate(rows)]
    lo = np.zeros(n + 1, dtype=np.int64)
    lo[1:] = np.cumsum([len(r) for r in rows])
    return lo, (np.concatenate(rows) if n else np.zeros(0, np.int32)).astype(np.int32)


def _check_build(pc, orc, chars, seed, P, L, algo):
    n = len(chars)
    for form in ("full", "earlier"):
        with pc.Picasso(_xz(pc, chars), chars.shape[1], seed=seed, algo=algo, csr=form) as p:
            p.assign_lists(P, L, 0)
            _, enc, lists = _ranked(p, orc, chars, seed, P, L)
            off_r, col_r = orc.conflict_csr(enc, lists)
            if form == "earlier":
                off_r, col_r = _lower(off_r, col_r)
            n_rows, nnz = p.build_conflicts()
            assert (n_rows, nnz) == (n, len(col_r))
            off, col = p.csr()
            assert np.array_equal(off.cpu().numpy(), off_r)
            assert np.array_equal(col.cpu().numpy(), col_r)
            runoff = p.runs().cpu().numpy()
            # run k of row u holds exactly the commuting neighbours that hold c_k
            for u in range(n):
                assert runoff[u * L] == off_r[u]
                if u < 150:
                    for k in range(L):
                        seg = col_r[runoff[u * L + k]:runoff[u * L + k + 1]]
                        assert all(lists[u][k] in lists[v] for v in seg)
                        assert np.all(np.diff(seg) > 0)
            assert runoff[-1] == len(col_r)
            st = p.stats()
            assert st["conflict_algo_used"] == pc.ALGOS[algo] or algo == "auto"


@pytest.mark.parametrize("algo", ["allpairs", "bucket"])
def test_conflict_workload_small(pc, orc, algo):
    # n=2000 strings on q=20 qubits, uniform I/X/Y/Z, P=n/8, L=ceil(2 ln n)
    _check_build(pc, orc, synth.pauli_uniform(2000, 20, seed=0), 0, 250, 16, algo)


@pytest.mark.parametrize("algo", ["allpairs", "bucket"])
@pytest.mark.parametrize("n,q,P,L", [(1, 5, 3, 2), (2, 3, 2, 1), (33, 64, 5, 3), (1000, 48, 40, 6),
                                     (777, 20, 97, 21), (2000, 64, 30, 30)])
def test_conflict_shapes(pc, orc, algo, n, q, P, L):
    _check_build(pc, orc, synth.pauli_weighted(n, q, 0.3, seed=n + q), 3, P, L, algo)


def test_bucket_cap_reported(pc):
    # every vertex holds all P colors: 2500 members per bucket exceed the
    # bucket join's cap, which says so; AUTO then takes the all-pairs path
    chars = synth.pauli_weighted(2500, 64, 0.3, seed=1)
    with pc.Picasso(_xz(pc, chars), 64, seed=3, algo="bucket") as p:
        p.assign_lists(30, 30, 0)
        with pytest.raises(pc.PicassoError) as e:
            p.build_conflicts()
        assert e.value.status == pc.ERR_UNSUPPORTED
    with pc.Picasso(_xz(pc, chars), 64, seed=3, algo="auto") as p:
        p.assign_lists(30, 30, 0)
        p.build_conflicts()
        assert p.stats()["conflict_algo_used"] == pc.ALGOS["allpairs"]


def test_conflict_identity_and_duplicates(pc, orc):
    chars = synth.pauli_weighted(600, 24, 0.2, seed=9)
    chars[:50] = 0           # identity strings commute with everything
    chars[50:100] = chars[100]  # duplicated strings commute with each other
    for algo in ("allpairs", "bucket"):
        _check_build(pc, orc, chars, 1, 60, 8, algo)


def test_conflict_weighted_mid(pc, orc):
    # the weighted law at n=6000, q=48 (P=n/8, alpha=2): bucket path, exact
    n = 6000
    P, L = orc.round_params(n, 1, 8, 2.0)
    _check_build(pc, orc, synth.pauli_weighted(n, 48, 0.25, seed=4), 7, P, L, "auto")


@pytest.mark.parametrize("P,lo,hi", [(500, 440, 480), (450, 500, 512)])
def test_conflict_bits_large_buckets(pc, orc, P, lo, hi):
    # the bit pass of the build at the bucket sizes of the n = 1M workload (mean
    # n L / P = 408) and up to its limit of 512 members (mean 453, largest
    # 511): n = 12,000 strings of the weighted law, L = 17; whole CSRs of
    # both forms (EARLIER through the bit pass, FULL through the two-pass
    # build) element by element against the oracle
    n, L, seed = 12000, 17, 7
    chars = synth.pauli_weighted(n, 64, 0.25, seed=21)
    _check_build(pc, orc, chars, seed, P, L, "bucket")
    with pc.Picasso(_xz(pc, chars), 64, seed=seed) as p:
        p.assign_lists(P, L, 0)
        _, nnz = p.build_conflicts()
        st = p.stats()
        assert lo <= st["max_bucket"] <= hi
        # the bit pass (the per-round default for buckets of at most 512
        # members) counts 28 bytes per list entry and 4 per word of the
        # buckets' lower blocks: 32 nwb (nwb + 1) / 2 words, nwb = ceil(s / 32)
        _, lists, _ = p.round_state()
        sizes = np.bincount(lists.cpu().numpy().ravel(), minlength=P).astype(np.int64)
        nwb = (sizes + 31) // 32
        words = int((16 * nwb * (nwb + 1)).sum())
        assert st["emit_launches"] == 1 and st["emit_bytes"] == 4 * words + 28 * n * L


@pytest.mark.parametrize("P,palette,alpha", [(450, (3, 80), 1.8)])
@pytest.mark.parametrize("small", ["off", "auto"])
def test_run_bits_large_buckets(pc, orc, P, palette, alpha, small):
    # whole runs whose every per-round build has buckets of about 450 members
    n = 12000
    assert orc.round_params(n, *palette, alpha) == (P, 17)
    _run_both(pc, orc, synth.pauli_weighted(n, 64, 0.25, seed=21), 7, *palette, alpha, small=small)


def _pair_keys(off, col):
    """Distinct unordered pairs {u, v} of a CSR, as sorted keys min * n + max."""
    n = len(off) - 1
    u = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    v = col.astype(np.int64)
    return np.unique(np.minimum(u, v) * n + np.maximum(u, v))


@pytest.mark.parametrize("case", ["n2000_q20", "n12000_q64_large_buckets"])
@pytest.mark.parametrize("form", ["earlier", "full"])
def test_conflict_edges_deduplicated(pc, orc, case, form):
    # the paper's G_c has each edge once (Sec. III-A: u, v adjacent iff they
    # commute and their lists meet); the CSR lists a pair once per shared
    # color, so its distinct pairs must be exactly the oracle's edge set
    if case == "n2000_q20":
        chars, q, seed, P, L = synth.pauli_uniform(2000, 20, seed=0), 20, 0, 250, 16
    else:
        chars, q, seed, P, L = synth.pauli_weighted(12000, 64, 0.25, seed=21), 64, 7, 500, 17
    n = len(chars)
    with pc.Picasso(_xz(pc, chars), q, seed=seed, csr=form) as p:
        p.assign_lists(P, L, 0)
        p.build_conflicts()
        off, col = p.csr()
        _, enc, lists = _ranked(p, orc, chars, seed, P, L)
        got = _pair_keys(off.cpu().numpy(), col.cpu().numpy())
    eo, ec = orc.conflict_edges(enc, lists)
    ref = np.repeat(np.arange(n, dtype=np.int64), np.diff(eo)) * n + ec.astype(np.int64)
    assert np.all(np.diff(ref) > 0)  # the oracle's rows are ascending, rows in order
    assert np.array_equal(got, ref)


def test_budget_rejects_before_allocation(pc):
    chars = synth.pauli_uniform(2000, 20, seed=0)
    with pc.Picasso(_xz(pc, chars), 20, seed=0, byte_budget=1000) as p:
        p.assign_lists(250, 16, 0)
        with pytest.raises(pc.PicassoError) as e:
            p.build_conflicts()
        assert e.value.status == pc.ERR_BUDGET
        # the context stays usable: lift nothing, just re-run with a new one
    with pc.Picasso(_xz(pc, chars), 20, seed=0) as p:
        p.assign_lists(250, 16, 0)
        assert p.build_conflicts()[1] > 0


# ------------------------------------------------------------------ coloring
@pytest.mark.parametrize("algo,color", [("allpairs", "auto"), ("bucket", "auto"), ("bucket", "sweep")])
def test_round_coloring_exact(pc, orc, algo, color):
    n, q, P, L, seed = 3000, 48, 375, 17, 11
    chars = synth.pauli_weighted(n, q, 0.25, seed=2)
    enc = orc.encode3(chars)
    lists = orc.draw_lists(seed, 1, np.arange(n), P, L, 0)
    off_r, col_r = orc.conflict_csr(enc, lists)
    ref = orc.color_greedy(seed, 1, np.arange(n), lists, off_r, col_r, P, 0)
    with pc.Picasso(_xz(pc, chars), q, seed=seed, algo=algo, color=color) as p:
        p.assign_lists(P, L, 0)
        p.build_conflicts()
        k = p.color()
        assert p.stats()["ordered_fallbacks"] == 0
        got = p.colors().cpu().numpy()
        assert k == int((ref >= 0).sum())
        assert np.array_equal(got, ref)


def _run_both(pc, orc, chars, seed, num, den, alpha, algo="auto", color="auto", small="auto"):
    ref, rounds, stats = orc.run(chars, seed, num, den, alpha)
    with pc.Picasso(_xz(pc, chars), chars.shape[1], seed=seed, palette=(num, den), alpha=alpha, algo=algo,
                    color=color, small=small) as p:
        got, r = p.run()
        got = got.cpu().numpy()
        assert r == rounds
        assert np.array_equal(got, ref)
        assert p.stats()["colors_used"] == int(stats[:, 1].sum())
    return ref


@pytest.mark.parametrize("color", ["auto", "sweep"])
def test_run_workload_small(pc, orc, color):
    # n=2000, q=20 uniform, P=n/8, alpha=2, seed 0: every round, every color
    _run_both(pc, orc, synth.pauli_uniform(2000, 20, seed=0), 0, 1, 8, 2.0, color=color)


@pytest.mark.parametrize("algo", ["allpairs", "bucket"])
def test_run_weighted(pc, orc, algo):
    _run_both(pc, orc, synth.pauli_weighted(4000, 48, 0.25, seed=1), 5, 1, 8, 2.0, algo)


@pytest.mark.parametrize("color,small", [("auto", "auto"), ("auto", "off"), ("sweep", "auto")])
def test_run_throughput_law_small(pc, orc, color, small):
    # the n=1M law (q=64, p=0.25, P=n/16, alpha=1.5) at a size the oracle
    # runs; "auto" runs every round in the small-round engine, "off" per round
    _run_both(pc, orc, synth.pauli_weighted(5000, 64, 0.25, seed=3), 0, 1, 16, 1.5, color=color, small=small)


@pytest.mark.parametrize("small", ["auto", "off"])
@pytest.mark.parametrize("n", [1, 2, 31, 257])
def test_run_edge_sizes(pc, orc, n, small):
    _run_both(pc, orc, synth.pauli_uniform(n, 6, seed=n), 2, 1, 8, 2.0, small=small)


def test_color_host_entry(pc, orc):
    # Alg. 1 from host buffers to host buffers (picasso_color_host): the
    # oracle's colors and rounds, from pinned and from pageable memory
    chars = synth.pauli_weighted(3000, 40, 0.3, seed=8)
    ref, rounds, _ = orc.run(chars, 5, 1, 8, 2.0)
    colors, r = pc.color_host(torch.from_numpy(chars).pin_memory(), 40, seed=5, palette=(1, 8), alpha=2.0)
    assert r == rounds and np.array_equal(colors.numpy(), ref)
    colors2, r2 = pc.color_host(torch.from_numpy(chars), 40, seed=5, palette=(1, 8), alpha=2.0)
    assert r2 == rounds and np.array_equal(colors2.numpy(), ref)
    with pytest.raises(pc.PicassoError) as e:
        pc.color_host(torch.from_numpy(chars[:0]), 40)
    assert e.value.status == pc.ERR_INVALID_ARG


def test_run_all_identity(pc, orc):
    # G' is complete: each round colors exactly min(P, ...) vertices
    chars = np.zeros((300, 10), dtype=np.uint8)
    _run_both(pc, orc, chars, 1, 1, 8, 2.0)


def test_run_all_commuting_bucket_path(pc, orc):
    # Z/I strings all commute, so every pair of a bucket is an edge: every bit
    # of the bit layout's rows is set (the densest runs the coloring reads);
    # per round the CSR is checked against the oracle through the canonical
    # form
    g = np.random.default_rng(12)
    chars = (g.integers(0, 2, size=(4000, 16)) * 3).astype(np.uint8)  # 0 = I, 3 = Z
    _run_both(pc, orc, chars, 3, 1, 8, 2.0, small="off")
    P, L = orc.round_params(4000, 1, 8, 2.0)
    _check_build(pc, orc, chars, 3, P, L, "auto")


def test_run_aggressive_small(pc, orc):
    # the paper's aggressive mode (P = 3%, alpha = 30) on a small set
    _run_both(pc, orc, synth.pauli_weighted(1500, 24, 0.3, seed=8), 4, 3, 100, 30.0)


# ------------------------------------------------------------------ full sizes
def _enc_np(orc, chars):
    return orc.encode3(chars)


def _anticommute_pairs(enc, a, b):
    x = np.bitwise_and(enc[a], enc[b])
    return (np.bitwise_count(x).sum(axis=1) % 2) == 1


def _check_cliques(enc, colors):
    """Every color class is a clique of G (mutually anticommuting)."""
    order = np.argsort(colors, kind="stable")
    cs = colors[order]
    n = len(cs)
    d = 1
    while True:
        same = cs[d:] == cs[:-d] if d < n else np.zeros(0, bool)
        if not same.any():
            break
        a = order[:-d][same]
        b = order[d:][same]
        assert _anticommute_pairs(enc, a, b).all()
        d += 1


def _sampled_rows(col, off, rows):
    """Rows `rows` of a device CSR, gathered on the device and copied once."""
    lens = off[rows + 1] - off[rows]
    starts = np.repeat(off[rows] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    idx = torch.from_numpy(starts + np.arange(lens.sum(), dtype=np.int64)).cuda()
    flat = col[idx].cpu().numpy()
    return np.split(flat, np.cumsum(lens)[:-1])


def _full_size(pc, orc, n, q, p_w, num, den, alpha, seed, samples):
    chars = synth.pauli_weighted(n, q, p_w, seed=seed)
    enc = _enc_np(orc, chars)
    P, L = orc.round_params(n, num, den, alpha)
    rng = np.random.default_rng(seed + 1)
    rows = np.sort(rng.choice(n, samples, replace=False))
    with pc.Picasso(_xz(pc, chars), q, seed=seed, palette=(num, den), alpha=alpha) as p:
        P2, L2, b = p.round_params()
        assert (P2, L2, b) == (P, L, 0)
        p.assign_lists(P, L, 0)
        p.build_conflicts()
        off, col = p.csr()
        off = off.cpu().numpy()
        # the oracle draws every priority and list itself; round-local ids
        # are ranks in the coloring order
        order, enc_r, lists_r = _ranked(p, orc, chars, seed, P, L)
        _, glists, _ = p.round_state()
        assert np.array_equal(glists.cpu().numpy().astype(np.int64), lists_r)
        lens, ref_rows = orc.conflict_rows(enc_r, lists_r, rows)
        got_rows = _sampled_rows(col, off, rows)
        del col
        for i, u in enumerate(rows):
            assert np.array_equal(got_rows[i], ref_rows[i][ref_rows[i] < u])  # the EARLIER form
        p.color()
        c1 = p.colors().cpu().numpy()
        # first fit in coloring order at every sampled vertex
        for i, u in enumerate(rows):
            earlier = got_rows[i]
            cn = c1[order[earlier]]
            taken = np.unique(cn[cn >= 0])
            free = lists_r[u][~np.isin(lists_r[u], taken)]
            want = int(free[0]) if len(free) else -1
            assert int(c1[order[u]]) == want
        p.carry()
        colors, rounds = p.run()
        colors = colors.cpu().numpy()
    assert (colors >= 0).all()
    _check_cliques(enc, colors)
    return colors, rounds


def test_full_size_n100k(pc, orc):
    # n=100,000, q=48, p=0.25, P=n/8, alpha=2
    _full_size(pc, orc, 100_000, 48, 0.25, 1, 8, 2.0, 0, 120)


def test_full_size_n1m(pc, orc):
    # n=1,000,000, q=64, p=0.25, P=n/16, alpha=1.5 (the throughput workload):
    # the exact round-1 conflict rows of a seeded 20,000-vertex sample
    _full_size(pc, orc, 1_000_000, 64, 0.25, 1, 16, 1.5, 0, 20_000)


@pytest.mark.slow
def test_run_n100k_whole(pc, orc):
    # n=100,000, q=48, p=0.25, P=n/8, alpha=2: every round and every color
    # of the GPU run against the oracle's whole run
    _run_both(pc, orc, synth.pauli_weighted(100_000, 48, 0.25, seed=0), 0, 1, 8, 2.0)


def test_full_size_wide_n200k(pc, orc):
    # n=200,000 strings of 128 qubits (two words per part, the table pass),
    # p=0.125, P=n/16, alpha=1.5
    _full_size(pc, orc, 200_000, 128, 0.125, 1, 16, 1.5, 3, 40)

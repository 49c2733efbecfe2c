"""Batched form: many independent sets in one context colored together.

Each set of a batch must be colored exactly as the oracle colors it alone
(same seed, same parameters), whatever the other sets are."""
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


def _batch(sets):
    """Sets back to back, every set padded with identity to the widest q
    (identity positions never change a commutation)."""
    q = max(q for _, q in sets)
    offs = [0]
    for c, _ in sets:
        offs.append(offs[-1] + len(c))
    padded = np.zeros((offs[-1], q), dtype=np.uint8)
    for k, (c, _) in enumerate(sets):
        padded[offs[k]:offs[k + 1], :c.shape[1]] = c
    return padded, offs, q


def _run_batch(pc, sets, seeds, palette=(1, 8), alpha=2.0, algo="auto", color="auto", small="auto", stats=False):
    padded, offs, q = _batch(sets)
    xz = pc.pack(torch.from_numpy(padded).cuda())
    with pc.Picasso(xz, q, palette=palette, alpha=alpha, algo=algo, color=color, set_offsets=offs,
                    seeds=seeds, small=small) as p:
        colors, rounds = p.run()
        if stats:
            st = p.stats()
            st["set_stats"] = p.set_stats()
            return colors.cpu().numpy(), offs, rounds, st
        return colors.cpu().numpy(), offs, rounds


@pytest.mark.parametrize("small", ["auto", "off"])
def test_batch_matches_oracle_per_set(pc, orc, small):
    # "auto": the whole run in the small-round engine (the union has under
    # 16384 vertices); "off": every round through the per-round path
    specs = [(700, 16, 0.3), (1, 24, 0.2), (2500, 64, 0.25), (1200, 32, 0.45), (33, 48, 0.1), (2048, 20, 0.5)]
    sets = [(synth.pauli_weighted(n, q, p, seed=11, stream=i), q) for i, (n, q, p) in enumerate(specs)]
    seeds = [100 + i for i in range(len(sets))]
    colors, offs, rounds, st = _run_batch(pc, sets, seeds, small=small, stats=True)
    used, peak, left = st["set_stats"]
    for k, (c, q) in enumerate(sets):
        ref, r, ostats = orc.run(c, seeds[k], 1, 8, 2.0)
        assert np.array_equal(colors[offs[k]:offs[k + 1]], ref), k
        assert r <= rounds
        assert used[k] == int(ostats[:, 1].sum()) and left[k] == 0, k
        # the largest conflict CSR of the set in one round, EARLIER form:
        # 8 (n_l + 1) + 4 nnz_l / 2 of the oracle's two-sided rows
        assert peak[k] == max(8 * (int(m) + 1) + 4 * (int(z) // 2) for m, z in ostats[:, [0, 4]]), k
    assert (st["small_rounds"] == rounds) if small == "auto" else (st["small_rounds"] == 0)


def test_batch_engine_hands_over_and_matches_per_round(pc):
    # union above 16384 at first: the per-round path runs the first rounds,
    # the engine the rest; everything equals the per-round-only run
    specs = synth.batch_specs(10, seed=4, n_lo=1000, n_hi=20000)
    sets = [(synth.pauli_weighted(n, q, p, seed=4, stream=i + 1), q) for i, (n, q, p) in enumerate(specs)]
    seeds = [50 + i for i in range(len(sets))]
    a, offs, ra, sa = _run_batch(pc, sets, seeds, small="auto", stats=True)
    b, _, rb, sb = _run_batch(pc, sets, seeds, small="off", stats=True)
    assert sum(n for n, _, _ in specs) > 16384
    assert ra == rb and np.array_equal(a, b)
    assert sa["set_stats"] == sb["set_stats"]
    assert sa["nnz_total"] == sb["nnz_total"] and sa["logical_pairs"] == sb["logical_pairs"]
    assert 0 < sa["small_rounds"] < ra and sb["small_rounds"] == 0


def test_batch_engine_empty_and_single_sets(pc, orc):
    # an empty set between others and sets of one string
    c0 = synth.pauli_weighted(300, 24, 0.3, seed=2)
    c2 = synth.pauli_weighted(500, 24, 0.3, seed=3)
    c3 = synth.pauli_weighted(1, 24, 0.3, seed=4)
    padded = np.concatenate([c0, c2, c3])
    offs = [0, 300, 300, 800, 801]
    seeds = [5, 6, 7, 8]
    xz = pc.pack(torch.from_numpy(padded).cuda())
    with pc.Picasso(xz, 24, set_offsets=offs, seeds=seeds) as p:
        colors, _ = p.run()
        colors = colors.cpu().numpy()
        used, _, left = p.set_stats()
        assert p.stats()["small_rounds"] > 0
    for k, c in ((0, c0), (2, c2), (3, c3)):
        ref, _, _ = orc.run(c, seeds[k], 1, 8, 2.0)
        assert np.array_equal(colors[offs[k]:offs[k + 1]], ref), k
    assert used[1] == 0 and left == [0, 0, 0, 0]


@pytest.mark.parametrize("algo,color", [("allpairs", "auto"), ("bucket", "sweep")])
def test_batch_paths(pc, orc, algo, color):
    specs = [(500, 16, 0.3), (900, 40, 0.25), (300, 64, 0.5)]
    sets = [(synth.pauli_weighted(n, q, p, seed=5, stream=i), q) for i, (n, q, p) in enumerate(specs)]
    seeds = [7, 8, 9]
    colors, offs, _ = _run_batch(pc, sets, seeds, algo=algo, color=color)
    for k, (c, q) in enumerate(sets):
        ref, _, _ = orc.run(c, seeds[k], 1, 8, 2.0)
        assert np.array_equal(colors[offs[k]:offs[k + 1]], ref), k


def test_batch_equals_single_runs_larger(pc):
    # the batch law (n log-uniform, q in {16..64}, p in [0.1, 0.5]) on 12 sets:
    # batch colors equal the per-set runs of the single-set entry points
    specs = synth.batch_specs(12, seed=3, n_lo=1000, n_hi=30000)
    sets = [(synth.pauli_weighted(n, q, p, seed=3, stream=i + 1), q) for i, (n, q, p) in enumerate(specs)]
    seeds = [1000 + i for i in range(len(sets))]
    colors, offs, _ = _run_batch(pc, sets, seeds)
    for k, (c, q) in enumerate(sets):
        xz = pc.pack(torch.from_numpy(c).cuda())
        with pc.Picasso(xz, q, seed=seeds[k]) as p:
            single, _ = p.run()
        assert np.array_equal(colors[offs[k]:offs[k + 1]], single.cpu().numpy()), k


# Launch schedules (picasso_schedule): the engine's grid, the rounds it gives
# to one thread-block cluster and to one block, the blocks per SM of the bit
# pass and of the mask coloring.  None of them may change a color.
_SCHEDULES = [
    {},
    {"engine_blocks_per_sm": 1},
    {"cluster_max_n": -1},
    {"cluster_max_n": 512, "cluster_blocks": 8},
    {"cluster_max_n": 8192, "cluster_blocks": 2},
    {"bits_blocks_per_sm": 2, "color_blocks_per_sm": 3},
    {"bits_blocks_per_sm": 1, "color_blocks_per_sm": 1, "engine_blocks_per_sm": 1},
    {"engine_max_n": 4096},
    {"engine_max_n": 64, "cluster_max_n": 16},
    {"block_max_n": -1},
    {"block_max_n": 2048, "cluster_max_n": 1024},
    {"block_max_n": 16384},
    {"block_max_n": 40, "cluster_max_n": -1},
]


def _mixed_sets():
    # a batch whose first rounds go through the per-round path (more than
    # 16,384 strings), the bit pass and the mask coloring, then the engine's
    # grid and cluster launches
    specs = [(9000, 64, 0.25), (300, 16, 0.4), (6000, 48, 0.2), (2200, 32, 0.35), (1, 24, 0.3)]
    return [(synth.pauli_weighted(n, q, p, seed=17, stream=i), q) for i, (n, q, p) in enumerate(specs)]


@pytest.mark.parametrize("sched", _SCHEDULES)
def test_schedules_keep_colors(pc, orc, sched):
    sets = _mixed_sets()
    seeds = [40 + k for k in range(len(sets))]
    padded, offs, q = _batch(sets)
    xz = pc.pack(torch.from_numpy(padded).cuda())
    with pc.Picasso(xz, q, set_offsets=offs, seeds=seeds, schedule=sched) as p:
        colors, _ = p.run()
        colors = colors.cpu().numpy()
        st = p.stats()
    assert st["small_rounds"] > 0 and st["pairs_launches"] > 0
    for k, (c, _) in enumerate(sets):
        ref, _, _ = orc.run(c, seeds[k], 1, 8, 2.0)
        assert np.array_equal(colors[offs[k]:offs[k + 1]], ref), (sched, k)


def test_autotune_picks_a_valid_schedule(pc, orc):
    sets = _mixed_sets()
    seeds = [40 + k for k in range(len(sets))]
    padded, offs, q = _batch(sets)
    xz = pc.pack(torch.from_numpy(padded).cuda())
    best, best_ms, start_ms = pc.autotune(xz, q, set_offsets=offs, seeds=seeds, reps=1)
    assert set(best) == {"engine_blocks_per_sm", "cluster_max_n", "cluster_blocks", "bits_blocks_per_sm",
                         "color_blocks_per_sm", "engine_max_n", "block_max_n"}
    assert best["engine_max_n"] in (0, 16384, 8192, 4096)
    assert best["engine_blocks_per_sm"] in (0, 1, 2) and best["cluster_max_n"] in (0, -1, 512, 2048, 8192)
    assert best["cluster_blocks"] in (0, 8, 16) and best["bits_blocks_per_sm"] in (0, 2, 3, 4)
    assert best["color_blocks_per_sm"] in (0, 3, 4, 6) and best["block_max_n"] in (0, -1, 64, 256, 1024)
    # a candidate replaces the start only if it is at least 1 % faster
    assert 0 < best_ms <= start_ms
    with pc.Picasso(xz, q, set_offsets=offs, seeds=seeds, schedule=best) as p:
        colors = p.run()[0].cpu().numpy()
    for k, (c, _) in enumerate(sets):
        ref, _, _ = orc.run(c, seeds[k], 1, 8, 2.0)
        assert np.array_equal(colors[offs[k]:offs[k + 1]], ref), k


@pytest.mark.parametrize("bad", [{"engine_blocks_per_sm": 3}, {"cluster_max_n": -2}, {"cluster_max_n": 16385},
                                 {"cluster_blocks": 6}, {"bits_blocks_per_sm": 5}, {"color_blocks_per_sm": 9},
                                 {"engine_max_n": -1}, {"engine_max_n": 16385}, {"block_max_n": -2},
                                 {"block_max_n": 16385}])
def test_schedule_validated(pc, bad):
    chars = synth.pauli_uniform(50, 10, seed=2)
    xz = pc.pack(torch.from_numpy(chars).cuda())
    with pytest.raises(pc.PicassoError) as e:
        pc.Picasso(xz, 10, schedule=bad)
    assert e.value.status == pc.ERR_INVALID_ARG

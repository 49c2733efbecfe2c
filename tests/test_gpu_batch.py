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


def _run_batch(pc, sets, seeds, palette=(1, 8), alpha=2.0, algo="auto", color="auto"):
    padded, offs, q = _batch(sets)
    xz = pc.pack(torch.from_numpy(padded).cuda())
    with pc.Picasso(xz, q, palette=palette, alpha=alpha, algo=algo, color=color, set_offsets=offs,
                    seeds=seeds) as p:
        colors, rounds = p.run()
        return colors.cpu().numpy(), offs, rounds


def test_batch_matches_oracle_per_set(pc, orc):
    specs = [(700, 16, 0.3), (1, 24, 0.2), (2500, 64, 0.25), (1200, 32, 0.45), (33, 48, 0.1), (2048, 20, 0.5)]
    sets = [(synth.pauli_weighted(n, q, p, seed=11, stream=i), q) for i, (n, q, p) in enumerate(specs)]
    seeds = [100 + i for i in range(len(sets))]
    colors, offs, rounds = _run_batch(pc, sets, seeds)
    for k, (c, q) in enumerate(sets):
        ref, r, _ = orc.run(c, seeds[k], 1, 8, 2.0)
        assert np.array_equal(colors[offs[k]:offs[k + 1]], ref), k
        assert r <= rounds


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
